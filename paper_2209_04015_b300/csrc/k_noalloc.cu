// afq_exchange_energy_static: the exchange energy for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own pool or fixed arena (a raw cudaMalloc would bypass its
// accounting and can fail under its budget), or a latency-critical loop that must
// not hit the implicit device synchronisation of cudaMalloc / cudaFree.  This entry
// point computes the same per-walker exchange energy as the context path, but the
// exchange kernel's per-group partial sums live in the file-scope array below, so
// nothing is allocated: the caller passes only its inputs and its output.
//
// The array (AFQ_STATIC_EXCHANGE_SLOTS complex doubles, 4 MiB) is held by every GPU
// that loads the library until the process exits.  Every call shares it and it
// keeps the last call's contents; each call writes every slot it later reads (one
// slot per walker, spin and Cholesky group), so nothing has to be cleared first.
// Calls that overlap on the GPU (two streams, or two host threads) race on it.
#include <cstdio>
#include <mutex>

#include "afq_internal.cuh"

cudaError_t launch_exchange_fp64_raw(int M, int X, int na, int nb, int W, const double* Lt,
                                     const double2* thetaT, double2* ekp, cudaStream_t stream);

namespace {

__device__ __align__(256) double2 g_exchange_scratch[AFQ_STATIC_EXCHANGE_SLOTS];

constexpr int kMaxDevices = 64;
double2* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, looked up once per
// device (the array's name in host code is only a host-side stand-in).
cudaError_t scratch_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_exchange_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// ek_z = sum over the walker's 2 x ngroups slots (read straight from the array).
__global__ void k_exchange_static_reduce(int W, int slots_per_walker, double2* __restrict__ ek) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= W) return;
  double2 s = cmk(0.0, 0.0);
  for (int e = 0; e < slots_per_walker; ++e)
    s = cadd(s, g_exchange_scratch[(long)z * slots_per_walker + e]);
  ek[z] = s;
}

}  // namespace

extern "C" int afq_exchange_energy_static(int M, int X, int na, int nb, int W,
                                          const double* Lt_dev, const double* thetaT_dev,
                                          double* ek_dev, void* cuda_stream) {
  if (!Lt_dev || !thetaT_dev || !ek_dev || M < 1 || M > AFQ_MMAX || X < 1 || W < 1 || na < 0 ||
      nb < 0 || na > AFQ_NMAX || nb > AFQ_NMAX || na + nb < 1) {
    std::fprintf(stderr, "afq_exchange_energy_static: bad pointer or size\n");
    return AFQ_ERR_ARG;
  }
  const int G = exchange_group_size(na > nb ? na : nb);
  const long slots = (long)W * 2 * ((X + G - 1) / G);
  if (slots > AFQ_STATIC_EXCHANGE_SLOTS) {
    std::fprintf(stderr,
                 "afq_exchange_energy_static: needs %ld partial-sum slots (W x 2 x ceil(X/%d)) "
                 "but the static scratch holds %d; use afq_local_energy for this size\n",
                 slots, G, AFQ_STATIC_EXCHANGE_SLOTS);
    return AFQ_ERR_ARG;
  }
  double2* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "afq_exchange_energy_static: cudaGetSymbolAddress: %s\n",
                 cudaGetErrorString(e));
    return AFQ_ERR_CUDA;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  e = launch_exchange_fp64_raw(M, X, na, nb, W, Lt_dev,
                               reinterpret_cast<const double2*>(thetaT_dev), scratch, stream);
  if (e == cudaSuccess) {
    k_exchange_static_reduce<<<(W + 127) / 128, 128, 0, stream>>>(
        W, (int)(slots / W), reinterpret_cast<double2*>(ek_dev));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    std::fprintf(stderr, "afq_exchange_energy_static: launch: %s\n", cudaGetErrorString(e));
    return AFQ_ERR_CUDA;
  }
  return AFQ_OK;
}
