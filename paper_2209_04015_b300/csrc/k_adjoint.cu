// Adjoint of the mixed local energy (FP64): gradients of Loss = sum_z Re(conj(g_z)
// E_L,z) with respect to h1, the Cholesky vectors L_g and the walkers Phi.
//
// The paper leaves automatic differentiation to future work (Sec. "Customized
// mixed estimators"); these are the closed forms of its local energy
// (Sec. "Local energy"), theta = Phi (Psi^T Phi)^-1, G^s = Psi_s theta_s^T:
//   dLoss/dh1  = Re sum_z conj(g_z) G_z = Psi Re(Theta),  Theta_s = sum_z conj(g_z) theta_s,z^T
//   dLoss/dL_g = Re sum_s Psi_s F_g,s,
//                F_g,s = sum_z conj(g_z) (c_zg theta_s,z^T - T_zg,s^T theta_s,z^T),
//                T_zg,s = L~_g,s theta_s,z
//   dLoss/dPhi_s = g conj((I - Psi_s theta_s^T) Gbar_s S_s^-T),
//                Gbar_s = h~_s^T + (sum_g c_g L~_g,s)^T - (sum_g T_g,s L~_g,s)^T
// Like the forward exchange, T is rebuilt per (walker, g) in shared memory and never
// stored.  Accumulators live in registers: n_s M <= 8192 per spin.
#include "afq_internal.cuh"

namespace {

constexpr int BT = 256;
constexpr int MAXE = 32;  // accumulator elements per thread: n M <= BT * MAXE

__device__ __forceinline__ double2 cfma_r(double a, double2 b, double2 acc) {
  return cmk(fma(a, b.x, acc.x), fma(a, b.y, acc.y));
}

// ---------------------------------------------------------------------------
// Gbar^T_z[j][p] for one (walker, spin): loops over every g.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BT) k_bwd_gbar(int M, int N, int na, int nb, int X,
                                                 const double* __restrict__ Lt,
                                                 const double* __restrict__ ht,
                                                 const double2* __restrict__ thetaT,
                                                 const double2* __restrict__ c,
                                                 double2* __restrict__ gbarT) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int z = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) return;
  const int nM = n * M;
  double2* th = reinterpret_cast<double2*>(smraw);  // n x M
  double2* T = th + nM;                             // n x n
  double* Lg = reinterpret_cast<double*>(T + n * n);  // n x M
  for (int e = tid; e < nM; e += BT) th[e] = thetaT[((long)z * N + off) * M + e];
  double2 acc[MAXE];
#pragma unroll
  for (int k = 0; k < MAXE; ++k) acc[k] = cmk(0.0, 0.0);
  __syncthreads();
  for (int g = 0; g < X; ++g) {
    for (int e = tid; e < nM; e += BT) Lg[e] = Lt[((long)g * N + off) * M + e];
    __syncthreads();
    // T_ij = sum_p L~_ip theta_pj = sum_p Lg[i][p] th[j][p]
    for (int e = tid; e < n * n; e += BT) {
      const int i = e / n, j = e % n;
      double2 t = cmk(0.0, 0.0);
      for (int p = 0; p < M; ++p) t = cfma_r(Lg[i * M + p], th[j * M + p], t);
      T[i * n + j] = t;
    }
    __syncthreads();
    const double2 cg = c[(long)z * X + g];
#pragma unroll
    for (int k = 0; k < MAXE; ++k) {
      const int e = tid + k * BT;
      if (e < nM) {
        const int j = e / M, p = e % M;
        double2 a = acc[k];
        const double l = Lg[j * M + p];
        a = cmk(fma(cg.x, l, a.x), fma(cg.y, l, a.y));
        for (int i = 0; i < n; ++i) {
          const double2 tji = T[j * n + i];
          const double li = Lg[i * M + p];
          a = cmk(fma(-tji.x, li, a.x), fma(-tji.y, li, a.y));
        }
        acc[k] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < MAXE; ++k) {
    const int e = tid + k * BT;
    if (e < nM) {
      const double h = ht[(long)off * M + e];
      gbarT[((long)z * N + off) * M + e] = cmk(acc[k].x + h, acc[k].y);
    }
  }
}

// ---------------------------------------------------------------------------
// dLoss/dPhi for one (walker, spin): S = Psi^T Phi and its inverse (Gauss-Jordan,
// partial pivoting), W1 = theta^T Gbar, Y = Gbar - Psi W1, dE/dPhi = Y S^-T.
// ---------------------------------------------------------------------------
// MODE 0: out = g conj(d) (dLoss/dRe Phi + i dLoss/dIm Phi); MODE 1: out = conj(g) d
// (the holomorphic cotangent); MODE 2: out += d (accumulate; gE unused).  d = Y S^-T.
template <int MODE>
__global__ void __launch_bounds__(BT) k_bwd_dphi(int M, int N, int na, int nb,
                                                 const double* __restrict__ psiT,
                                                 const double2* __restrict__ phi,
                                                 const double2* __restrict__ thetaT,
                                                 const double2* __restrict__ gbarT,
                                                 const double2* __restrict__ gE,
                                                 double2* __restrict__ dphi) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_piv;
  const int z = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) return;
  const int n2 = 2 * n;
  double2* aug = reinterpret_cast<double2*>(smraw);  // n x 2n -> [I | S^-1]
  double2* W1 = aug + n * n2;                        // n x n
  double2* fac = W1 + n * n;                         // n
  const double2* phz = phi + (long)z * M * N;
  const double2* thz = thetaT + ((long)z * N + off) * M;
  const double2* gbz = gbarT + ((long)z * N + off) * M;
  for (int e = tid; e < n * n; e += BT) {
    const int i = e / n, j = e % n;
    double2 sv = cmk(0.0, 0.0), wv = cmk(0.0, 0.0);
    for (int p = 0; p < M; ++p) {
      sv = cfma_r(psiT[(long)(off + i) * M + p], phz[(long)p * N + off + j], sv);
      wv = cfma(thz[(long)i * M + p], gbz[(long)j * M + p], wv);
    }
    aug[i * n2 + j] = sv;
    aug[i * n2 + n + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
    W1[i * n + j] = wv;
  }
  __syncthreads();
  for (int kc = 0; kc < n; ++kc) {
    if (tid < 32) {
      double best = -1.0;
      int bi = kc;
      for (int r = kc + tid; r < n; r += 32) {
        const double v = cabs2(aug[r * n2 + kc]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != kc)
      for (int cc = tid; cc < n2; cc += BT) {
        const double2 t = aug[kc * n2 + cc];
        aug[kc * n2 + cc] = aug[piv * n2 + cc];
        aug[piv * n2 + cc] = t;
      }
    __syncthreads();
    double2 pv = aug[kc * n2 + kc];
    if (!(cabs2(pv) >= 1e-300)) pv = cmk(1.0, 0.0);
    const double2 inv = cdiv(cmk(1.0, 0.0), pv);
    for (int r = tid; r < n; r += BT) fac[r] = aug[r * n2 + kc];
    __syncthreads();
    for (int cc = tid; cc < n2; cc += BT) aug[kc * n2 + cc] = cmul(aug[kc * n2 + cc], inv);
    __syncthreads();
    for (int e = tid; e < n * n2; e += BT) {
      const int r = e / n2, cc = e % n2;
      if (r != kc) aug[e] = cfms(fac[r], aug[kc * n2 + cc], aug[e]);
    }
    __syncthreads();
  }
  const double2 g = MODE == 2 ? cmk(1.0, 0.0) : gE[z];
  for (int e = tid; e < M * n; e += BT) {
    const int p = e / n, k = e % n;
    double2 d = cmk(0.0, 0.0);
    for (int j = 0; j < n; ++j) {
      double2 y = gbz[(long)j * M + p];
      for (int i = 0; i < n; ++i) {
        const double2 wv = W1[i * n + j];
        const double ps = psiT[(long)(off + i) * M + p];
        y = cmk(fma(-wv.x, ps, y.x), fma(-wv.y, ps, y.y));
      }
      d = cfma(y, aug[k * n2 + n + j], d);  // (S^-1)_kj
    }
    double2* o = dphi + (long)z * M * N + (long)p * N + off + k;
    if (MODE == 0) *o = cmul(g, cconj(d));
    else if (MODE == 1) *o = cmul(cconj(g), d);
    else *o = cadd(*o, d);
  }
}

// Theta_jp = sum_z conj(g_z) theta^T_z[j][p], real part only (dh1 = Psi Re Theta).
__global__ void k_bwd_theta_sum(int W, long NM, const double2* __restrict__ thetaT,
                                const double2* __restrict__ gE, double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NM;
       e += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < W; ++z) {
      const double2 t = thetaT[(long)z * NM + e];
      const double2 g = gE[z];
      acc += g.x * t.x + g.y * t.y;  // Re(conj(g) t)
    }
    out[e] = acc;
  }
}

// Re F_g,s[j][p] for one (g, spin), added to F: loops over every walker.
__global__ void __launch_bounds__(BT) k_bwd_lfac(int M, int N, int na, int nb, int X, int W,
                                                 const double* __restrict__ Lt,
                                                 const double2* __restrict__ thetaT,
                                                 const double2* __restrict__ c,
                                                 const double2* __restrict__ gE,
                                                 double* __restrict__ F) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int g = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) return;
  const int nM = n * M;
  double2* th = reinterpret_cast<double2*>(smraw);    // n x M
  double2* T = th + nM;                               // n x n
  double* Lg = reinterpret_cast<double*>(T + n * n);  // n x M
  for (int e = tid; e < nM; e += BT) Lg[e] = Lt[((long)g * N + off) * M + e];
  double2 acc[MAXE];
#pragma unroll
  for (int k = 0; k < MAXE; ++k) acc[k] = cmk(0.0, 0.0);
  for (int z = 0; z < W; ++z) {
    __syncthreads();
    for (int e = tid; e < nM; e += BT) th[e] = thetaT[((long)z * N + off) * M + e];
    __syncthreads();
    for (int e = tid; e < n * n; e += BT) {
      const int i = e / n, j = e % n;
      double2 t = cmk(0.0, 0.0);
      for (int p = 0; p < M; ++p) t = cfma_r(Lg[i * M + p], th[j * M + p], t);
      T[i * n + j] = t;
    }
    __syncthreads();
    const double2 wg = cconj(gE[z]);
    const double2 wc = cmul(wg, c[(long)z * X + g]);
#pragma unroll
    for (int k = 0; k < MAXE; ++k) {
      const int e = tid + k * BT;
      if (e < nM) {
        const int j = e / M, p = e % M;
        double2 v = cmul(wc, th[j * M + p]);
        double2 u = cmk(0.0, 0.0);
        for (int i = 0; i < n; ++i) u = cfma(T[i * n + j], th[i * M + p], u);
        v = csub(v, cmul(wg, u));
        acc[k] = cadd(acc[k], v);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MAXE; ++k) {
    const int e = tid + k * BT;
    if (e < nM) F[((long)g * N + off) * M + e] += acc[k].x;
  }
}

size_t bwd_smem(int n, int M) { return (size_t)n * M * 24 + (size_t)n * n * 16 + 16; }
size_t dphi_smem(int n) { return (size_t)n * 2 * n * 16 + (size_t)n * n * 16 + (size_t)n * 16; }

int configure_bwd(afq_ctx* ctx, size_t smem, size_t sm2) {
  static size_t configured = 0, configured2 = 0;
  if (smem > configured) {
    AFQ_CUDA(ctx, cudaFuncSetAttribute(k_bwd_gbar, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AFQ_CUDA(ctx, cudaFuncSetAttribute(k_bwd_lfac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  if (sm2 > configured2) {
    AFQ_CUDA(ctx, cudaFuncSetAttribute(k_bwd_dphi<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    AFQ_CUDA(ctx, cudaFuncSetAttribute(k_bwd_dphi<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    AFQ_CUDA(ctx, cudaFuncSetAttribute(k_bwd_dphi<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
    configured2 = sm2;
  }
  return AFQ_OK;
}

int launch_bwd_dphi(afq_ctx* ctx, WalkerSet& t, const double2* gbarT, const double2* gE,
                    double2* out, int mode) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  const size_t sm2 = dphi_smem(nmax);
  const dim3 grid(t.W, 2);
  if (mode == 0)
    k_bwd_dphi<0><<<grid, BT, sm2, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb, ctx->psiT,
                                                  t.phi, t.thetaT, gbarT, gE, out);
  else if (mode == 1)
    k_bwd_dphi<1><<<grid, BT, sm2, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb, ctx->psiT,
                                                  t.phi, t.thetaT, gbarT, gE, out);
  else
    k_bwd_dphi<2><<<grid, BT, sm2, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb, ctx->psiT,
                                                  t.phi, t.thetaT, gbarT, gE, out);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

}  // namespace

int adjoint_energy_core(afq_ctx* ctx, WalkerSet& t, const double2* gE, double* dh1, double* F,
                        double2* out, int mode) {
  const int M = ctx->M, N = ctx->N, X = ctx->X, W = t.W;
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  if ((long)nmax * M > (long)BT * MAXE)
    return afq_fail(ctx, AFQ_ERR_ARG, "local-energy backward needs max(na, nb) * M <= 8192");
  const size_t smem = bwd_smem(nmax, M);
  if (smem > 220 * 1024) return afq_fail(ctx, AFQ_ERR_ARG, "local-energy backward: shared memory");
  AFQ_TRY(configure_bwd(ctx, smem, dphi_smem(nmax)));
  double2* buf = nullptr;  // Gbar^T (W x N x M complex), then Theta (N x M reals)
  if (cudaMalloc((void**)&buf, (size_t)W * N * M * sizeof(double2)) != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_NOMEM, "local-energy backward workspace");
  int rc = AFQ_OK;
  if (out) {
    k_bwd_gbar<<<dim3(W, 2), BT, smem, ctx->stream>>>(M, N, ctx->na, ctx->nb, X, ctx->Lt, ctx->ht,
                                                      t.thetaT, t.c, buf);
    ctx->launches++;
    rc = launch_bwd_dphi(ctx, t, buf, gE, out, mode);
    if (rc == AFQ_OK && cudaGetLastError() != cudaSuccess)
      rc = afq_fail(ctx, AFQ_ERR_CUDA, "backward dPhi launch");
  }
  if (dh1 && rc == AFQ_OK) {
    double* theta_sum = reinterpret_cast<double*>(buf);  // N x M reals (after the dPhi kernels)
    const long NM = (long)N * M;
    k_bwd_theta_sum<<<(int)((NM + 255) / 256), 256, 0, ctx->stream>>>(W, NM, t.thetaT, gE,
                                                                      theta_sum);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) rc = afq_fail(ctx, AFQ_ERR_CUDA, "backward dh1 launch");
    // dh1 = Psi (M x N) Re(Theta) (N x M); Psi(p, j) = psiT[j M + p]
    if (rc == AFQ_OK)
      rc = launch_dgemm(ctx, M, M, N, 1.0, ctx->psiT, 1, M, 0, theta_sum, M, 1, 0, 0.0, dh1, M, 1, 0,
                        1, 1);
  }
  if (F && rc == AFQ_OK) {
    k_bwd_lfac<<<dim3(X, 2), BT, smem, ctx->stream>>>(M, N, ctx->na, ctx->nb, X, W, ctx->Lt,
                                                      t.thetaT, t.c, gE, F);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) rc = afq_fail(ctx, AFQ_ERR_CUDA, "k_bwd_lfac");
  }
  // the workspace is released only after the kernels that read it are done
  cudaStreamSynchronize(ctx->stream);
  cudaFree(buf);
  return rc;
}

// lambda_in += (I - Psi theta^T) lambda_theta S^-T for every walker (lamT: W x N x M,
// the cotangent of theta stored transposed like thetaT).
int launch_bwd_theta(afq_ctx* ctx, WalkerSet& t, const double2* lamT, double2* lam) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  AFQ_TRY(configure_bwd(ctx, bwd_smem(nmax, ctx->M), dphi_smem(nmax)));
  return launch_bwd_dphi(ctx, t, lamT, nullptr, lam, 2);
}

// Gradients of sum_z Re(conj(g_z) E_L,z) at the current walkers; any output may be
// NULL.  gE: W complex, dh1: M x M, dL: X x M x M, dphi: W x M x N complex (device).
int adjoint_local_energy(afq_ctx* ctx, const double2* gE, double* dh1, double* dL, double2* dphi) {
  const int M = ctx->M, N = ctx->N, X = ctx->X, W = ctx->ws.W;
  // theta and c of the current walkers, recomputed in FP64 into private buffers so
  // that the context's own state (and a split-precision trajectory) is untouched
  WalkerSet t;
  t.W = W;
  t.phi = ctx->ws.phi;
  double* F = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&t.thetaT, (size_t)W * N * M * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&t.det, (size_t)W * 2 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&t.e1, (size_t)W * 2 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&t.c, (size_t)W * X * sizeof(double2)) != cudaSuccess ||
      (dL && cudaMalloc((void**)&F, (size_t)X * N * M * sizeof(double)) != cudaSuccess))
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "local-energy backward workspace");
  if (rc == AFQ_OK) rc = launch_overlap_theta(ctx, t);
  if (rc == AFQ_OK) rc = launch_force_bias_fp64(ctx, t);
  if (rc == AFQ_OK && F &&
      cudaMemsetAsync(F, 0, (size_t)X * N * M * sizeof(double), ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "backward dL workspace");
  if (rc == AFQ_OK) rc = adjoint_energy_core(ctx, t, gE, dh1, F, dphi, 0);
  // dL_g = Psi (M x N) F_g (N x M), batched over g
  if (rc == AFQ_OK && dL)
    rc = launch_dgemm(ctx, M, M, N, 1.0, ctx->psiT, 1, M, 0, F, M, 1, (long)N * M, 0.0, dL, M, 1,
                      (long)M * M, X, 1);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(t.thetaT);
  cudaFree(t.det);
  cudaFree(t.e1);
  cudaFree(t.c);
  if (F) cudaFree(F);
  return rc;
}
