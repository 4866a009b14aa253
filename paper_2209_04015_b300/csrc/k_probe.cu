// Throughput probe of the FP64 pipe, measured beside the FP64 kernels' roofline (a
// measurement helper; the method itself has no counterpart).
//
// Every thread runs kChains independent fused multiply-add chains, the grid holds 8
// CTAs of 256 threads per SM (64 warps, far more independent FMAs in flight than the
// pipe's latency needs), and the chains' values feed a store that the compiler cannot
// drop.  Timed with CUDA events on the caller's stream, best of five launches after
// three untimed ones.
#include <cstdio>

#include "afq_internal.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kThreadsProbe = 256;

// written only if the chains' sum were -1, which cannot happen (every chain stays near
// 1 for multipliers just below 1 and c > 0); the store keeps the loop from being removed
__device__ double g_probe_sink[1];

__global__ void __launch_bounds__(kThreadsProbe) k_fp64_fma_loop(int iters, double m, double c) {
  double a[kChains], f[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    f[k] = m - 1e-12 * k;  // a multiplier per chain: no operand is shared between chains
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], f[k], c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) g_probe_sink[0] = s;
}

}  // namespace

extern "C" int afq_fp64_fma_rate(double* tflops, void* cuda_stream) {
  if (!tflops) return AFQ_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return AFQ_ERR_CUDA;
  const int blocks = sms * 8, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return AFQ_ERR_CUDA;
  }
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  // three untimed launches bring the clocks up, then the best of five timed ones
  for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    k_fp64_fma_loop<<<blocks, kThreadsProbe, 0, st>>>(iters, 0.999999999, 1e-9);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess && rep >= 3 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        ms > 0.f && ms < best)
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || best >= 1e29f) {
    std::fprintf(stderr, "afq_fp64_fma_rate: %s\n", cudaGetErrorString(e));
    return AFQ_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreadsProbe;
  *tflops = flops / (best * 1e-3) / 1e12;
  return AFQ_OK;
}
