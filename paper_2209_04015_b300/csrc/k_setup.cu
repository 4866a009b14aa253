// Trial / Hamiltonian set-up kernels of libafqmc (run once per afq_init_trial).
//
// The hot path never calls these; they build the trial-dependent intermediates of
// Sec. "One-body Green's function and force bias" (half-rotated Cholesky vectors)
// and the mean-field one-body operator h'' that the propagator needs.
#include "afq_internal.cuh"

namespace {

constexpr int GT = 32;  // output tile edge
constexpr int GK = 32;  // k chunk

// C[b] = alpha * A[b] B[b] + beta * C[b] for arbitrary element strides, FP64.
// blockIdx.z = b * ksplit + ks; split-K partials go to C + (b * ksplit + ks) * scb
// (then beta must be 0).
__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int k, double alpha,
                                               const double* __restrict__ A, long sam, long sak,
                                               long sab, const double* __restrict__ B, long sbk,
                                               long sbn, long sbb, double beta, double* C,
                                               long scm, long scn, long scb, int ksplit) {
  __shared__ double As[GT][GK + 1];
  __shared__ double Bs[GK][GT + 1];
  const int b = blockIdx.z / ksplit, ks = blockIdx.z % ksplit;
  const int kc = (k + ksplit - 1) / ksplit;
  const int kbeg = ks * kc, kend = min(k, kbeg + kc);
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;  // ty in 0..7
  A += b * sab;
  B += b * sbb;
  C += (long)blockIdx.z * scb;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
      int r = e / GK, kk = e % GK;
      int gi = i0 + r, gk = k0 + kk;
      As[r][kk] = (gi < m && gk < kend) ? A[gi * sam + gk * sak] : 0.0;
      int kr = e / GT, cc = e % GT;
      int gk2 = k0 + kr, gj = j0 + cc;
      Bs[kr][cc] = (gj < n && gk2 < kend) ? B[gk2 * sbk + gj * sbn] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      double bv = Bs[kk][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(As[ty + 8 * r][kk], bv, acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gi = i0 + ty + 8 * r, gj = j0 + tx;
    if (gi < m && gj < n) {
      double* cp = C + gi * scm + gj * scn;
      *cp = beta == 0.0 ? alpha * acc[r] : alpha * acc[r] + beta * *cp;
    }
  }
}

__global__ void k_pack_L(int X, int M, int Mp, const double* __restrict__ L,
                         const int2* __restrict__ tpq, double* __restrict__ Lpk) {
  long total = (long)X * Mp;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int g = (int)(e / Mp), t = (int)(e % Mp);
    int2 pq = tpq[t];
    Lpk[e] = L[(long)g * M * M + (long)pq.x * M + pq.y];
  }
}

template <int NT>
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  __syncthreads();
  return s;  // valid in thread 0
}

// vbar_g = sum_j sum_p L~_g,jp Psi^T_jp  (the trial's <v_g>, both spins)
__global__ void __launch_bounds__(256) k_vbar(int NM, const double* __restrict__ Lt,
                                              const double* __restrict__ psiT,
                                              double* __restrict__ vbar) {
  __shared__ double red[8];
  const int g = blockIdx.x;
  double s = 0.0;
  for (int e = threadIdx.x; e < NM; e += 256) s += Lt[(long)g * NM + e] * psiT[e];
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) vbar[g] = s;
}

// h''_pq = h1_pq - 1/2 sym(sum_g L_g L_g)_pq + sum_g vbar_g sym(L_g)_pq, exactly symmetric.
__global__ void k_hpp(int M, int X, const double* __restrict__ h1,
                      const double* __restrict__ s2part, int ksplit,
                      const double* __restrict__ L, const double* __restrict__ vbar,
                      double* __restrict__ hpp) {
  long MM = (long)M * M;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < MM;
       e += (long)gridDim.x * blockDim.x) {
    int p = (int)(e / M), q = (int)(e % M);
    long et = (long)q * M + p;
    double s2a = 0.0, s2b = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) {
      s2a += s2part[ks * MM + e];
      s2b += s2part[ks * MM + et];
    }
    double mf = 0.0;
    for (int g = 0; g < X; ++g) mf += vbar[g] * 0.5 * (L[g * MM + e] + L[g * MM + et]);
    hpp[e] = 0.5 * (h1[e] + h1[et]) - 0.25 * (s2a + s2b) + mf;
  }
}

// y = a x + b y; with b == 0 the old y is not read (it may be uninitialised memory,
// and 0 * NaN would poison the result)
__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, double* y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    y[e] = b == 0.0 ? a * x[e] : a * x[e] + b * y[e];
}

__global__ void k_identity(int M, double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += gridDim.x * blockDim.x)
    out[e] = (e / M == e % M) ? 1.0 : 0.0;
}

int grid_for(long n, int threads) {
  long g = (n + threads - 1) / threads;
  return (int)(g < 148 * 32 ? (g < 1 ? 1 : g) : 148 * 32);
}

}  // namespace

int launch_dgemm(afq_ctx* ctx, int m, int n, int k, double alpha, const double* A, long sam,
                 long sak, long sab, const double* B, long sbk, long sbn, long sbb, double beta,
                 double* C, long scm, long scn, long scb, int batch, int ksplit) {
  if (m <= 0 || n <= 0) return AFQ_OK;
  if (ksplit < 1) ksplit = 1;
  dim3 grid((n + GT - 1) / GT, (m + GT - 1) / GT, batch * ksplit);
  if (grid.z > 65535) return afq_fail(ctx, AFQ_ERR_ARG, "dgemm: batch*ksplit too large");
  k_dgemm<<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, sam, sak, sab, B, sbk, sbn, sbb,
                                         beta, C, scm, scn, scb, ksplit);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_pack_L(afq_ctx* ctx) {
  long total = (long)ctx->X * ctx->Mp;
  k_pack_L<<<grid_for(total, 256), 256, 0, ctx->stream>>>(ctx->X, ctx->M, ctx->Mp, ctx->L,
                                                          ctx->tpq, ctx->Lpk);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_vbar(afq_ctx* ctx) {
  k_vbar<<<ctx->X, 256, 0, ctx->stream>>>(ctx->N * ctx->M, ctx->Lt, ctx->psiT, ctx->vbar);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_hpp(afq_ctx* ctx, const double* s2part, int ksplit) {
  long MM = (long)ctx->M * ctx->M;
  k_hpp<<<grid_for(MM, 256), 256, 0, ctx->stream>>>(ctx->M, ctx->X, ctx->h1, s2part, ksplit,
                                                    ctx->L, ctx->vbar, ctx->hpp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_axpby(afq_ctx* ctx, int n, double a, const double* x, double b, double* y) {
  k_axpby<<<grid_for(n, 256), 256, 0, ctx->stream>>>(n, a, x, b, y);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_set_identity(afq_ctx* ctx, int M, double* out) {
  k_identity<<<grid_for((long)M * M, 256), 256, 0, ctx->stream>>>(M, out);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
