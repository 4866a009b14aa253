// Adjoint of the mixed local energy (FP64): gradients of Loss = sum_z Re(conj(g_z)
// E_L,z) with respect to h1, the Cholesky vectors L_g and the walkers Phi.
//
// The paper leaves automatic differentiation to future work (Sec. "Customized
// mixed estimators"); these are the closed forms of its local energy
// (Sec. "Local energy"), theta = Phi (Psi^T Phi)^-1, G^s = Psi_s theta_s^T,
// w_z = conj(g_z):
//   dLoss/dh1  = Re sum_z w_z G_z = Psi Re(Theta),  Theta_s = sum_z w_z theta_s,z^T
//   dLoss/dL_g = Re sum_s Psi_s F_g,s,
//                F_g,s = sum_z w_z (c_zg theta_s,z^T - T_zg,s^T theta_s,z^T),
//                T_zg,s = L~_g,s theta_s,z
//   dLoss/dPhi_s = g conj((I - Psi_s theta_s^T) Gbar_s S_s^-T),
//                Gbar_s = h~_s^T + (sum_g c_g L~_g,s)^T - (sum_g T_g,s L~_g,s)^T
// The two terms with T are contracted without forming T (index pairs (j,p) run over
// the n_s x M entries of theta^T, row-major):
//   (sum_g T_zg L~_g)^T[(j,p)] = sum_(i,q) V[(j,p),(i,q)] theta^T_z[(i,q)],
//        V[(j,p),(i,q)] = sum_g L~_g[j][q] L~_g[i][p]   (symmetric; trial-fixed, cached)
//   (sum_z w_z T_zg^T theta_z^T)[(j,p)] = sum_(i,q) L~_g[(i,q)] Y[(i,q),(j,p)],
//        Y[(i,q),(j,p)] = sum_z w_z theta^T_z[j][q] theta^T_z[i][p]   (symmetric)
// so both become FP64 GEMMs of (n_s M)^2 size: W (n_s M)^2 and X (n_s M)^2
// multiply-adds instead of W X n_s^2 M per pass over T.
#include "afq_internal.cuh"

namespace {

constexpr int BT = 256;

__device__ __forceinline__ double2 cfma_r(double a, double2 b, double2 acc) {
  return cmk(fma(a, b.x, acc.x), fma(a, b.y, acc.y));
}

// Gbar^T_z[e] = h~[e] for every walker (both spins; e < N M), the first term of Gbar
__global__ void k_bwd_gbar_init(long W, long NM, const double* __restrict__ ht,
                                double2* __restrict__ gbarT) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < W * NM;
       e += (long)gridDim.x * blockDim.x)
    gbarT[e] = cmk(ht[e % NM], 0.0);
}

// out[z n + e] = conj(g_z) in[z n + e]: the walker-weighted operands of dL
__global__ void k_bwd_weight(long W, long n, const double2* __restrict__ gE,
                             const double2* __restrict__ in, double2* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < W * n;
       e += (long)gridDim.x * blockDim.x)
    out[e] = cmul(cconj(gE[e / n]), in[e]);
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
  // Gauss-Jordan with partial pivoting, three barriers per pivot (as in the forward
  // overlap kernel): pivot and reciprocal in warp 0; swap, scaling and the column
  // factors in one phase; updates of the unreduced columns, warps over rows
  __shared__ double2 s_inv, s_old;
  const int wid = tid >> 5, lane = tid & 31;
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
      if (tid == 0) {
        double2 pv = aug[bi * n2 + kc];
        if (!(cabs2(pv) >= 1e-300)) pv = cmk(1.0, 0.0);
        s_inv = cdiv(cmk(1.0, 0.0), pv);
        s_old = aug[kc * n2 + kc];
        s_piv = bi;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    const double2 inv = s_inv;
    for (int r = tid; r < n; r += BT)
      if (r != kc) fac[r] = r == piv ? s_old : aug[r * n2 + kc];
    for (int c = kc + tid; c < n2; c += BT) {
      const double2 top = aug[piv * n2 + c];
      if (piv != kc) aug[piv * n2 + c] = aug[kc * n2 + c];
      aug[kc * n2 + c] = cmul(top, inv);
    }
    __syncthreads();
    for (int r = wid; r < n; r += BT / 32) {
      if (r == kc) continue;
      const double2 f = fac[r];
      for (int c = kc + 1 + lane; c < n2; c += 32)
        aug[r * n2 + c] = cfms(f, aug[kc * n2 + c], aug[r * n2 + c]);
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

// Y[(i,q),(j,p)] = Y[(j,p),(i,q)] for the blocks i < j (Y: n M x n M, blocks M x M)
__global__ void k_mirror_blocks(int n, int M, double* __restrict__ Y) {
  const long nM = (long)n * M, total = nM * nM;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long r = e / nM, c = e % nM;
    if (r / M < c / M) Y[e] = Y[c * nM + r];
  }
}

int bwd_grid(long n, int threads) {
  const long g = (n + threads - 1) / threads;
  return (int)(g < 148 * 16 ? (g < 1 ? 1 : g) : 148 * 16);
}

// counts one launch and reports a launch error without returning early (the caller
// still frees its workspaces)
int launched(afq_ctx* ctx) {
  ctx->launches++;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AFQ_OK
                          : afq_fail(ctx, AFQ_ERR_CUDA, std::string("kernel launch: ") +
                                                            cudaGetErrorString(e));
}

size_t dphi_smem(int n) { return (size_t)n * 2 * n * 16 + (size_t)n * n * 16 + (size_t)n * 16; }

int configure_bwd(afq_ctx* ctx, size_t sm2) {
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_bwd_dphi<0>, sm2));
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_bwd_dphi<1>, sm2));
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_bwd_dphi<2>, sm2));
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
  const long NM = (long)N * M;
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  if (nmax > 64)
    return afq_fail(ctx, AFQ_ERR_ARG, "local-energy backward needs max(na, nb) <= 64");
  AFQ_TRY(configure_bwd(ctx, dphi_smem(nmax)));
  if (out) AFQ_TRY(build_exchange_v(ctx));
  const long nmM = (long)nmax * M;
  // buf: Gbar^T (W x N x M complex), then Theta (N x M reals); for dL also
  // u = conj(g) theta^T (W x N x M complex), q = conj(g) c (W x X complex) and
  // Y (n_s M x n_s M, one spin at a time)
  double2 *buf = nullptr, *u = nullptr, *q = nullptr;
  double* Y = nullptr;
  int rc = AFQ_OK;
  if ((out || dh1) && cudaMalloc((void**)&buf, (size_t)W * NM * sizeof(double2)) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "local-energy backward workspace");
  if (rc == AFQ_OK && F &&
      (cudaMalloc((void**)&u, (size_t)W * NM * sizeof(double2)) != cudaSuccess ||
       cudaMalloc((void**)&q, (size_t)W * X * sizeof(double2)) != cudaSuccess ||
       cudaMalloc((void**)&Y, (size_t)nmM * nmM * sizeof(double)) != cudaSuccess))
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "local-energy backward dL workspace");
  const double* th = reinterpret_cast<const double*>(t.thetaT);
  if (rc == AFQ_OK && out) {
    double* gb = reinterpret_cast<double*>(buf);
    k_bwd_gbar_init<<<bwd_grid((long)W * NM, 256), 256, 0, ctx->stream>>>(W, NM, ctx->ht, buf);
    rc = launched(ctx);
    for (int s = 0; s < 2 && rc == AFQ_OK; ++s) {
      const int n = s ? ctx->nb : ctx->na, off = s ? ctx->na : 0;
      if (n == 0) continue;
      const long nM = (long)n * M, o2 = 2L * off * M;
      const double* V = ctx->Vx + (s ? (long)ctx->na * M * ctx->na * M : 0);
      // Gbar^T += sum_g c_zg L~_g (re and im rows as a batch of two)
      rc = launch_dgemm(ctx, W, (int)nM, X, 1.0, reinterpret_cast<const double*>(t.c), 2L * X, 2,
                        1, ctx->Lt + (long)off * M, NM, 1, 0, 1.0, gb + o2, 2 * NM, 2, 1, 2, 1);
      // Gbar^T -= theta^T V
      if (rc == AFQ_OK)
        rc = launch_dgemm(ctx, W, (int)nM, (int)nM, -1.0, th + o2, 2 * NM, 2, 1, V, nM, 1, 0, 1.0,
                          gb + o2, 2 * NM, 2, 1, 2, 1);
    }
    if (rc == AFQ_OK) rc = launch_bwd_dphi(ctx, t, buf, gE, out, mode);
  }
  if (dh1 && rc == AFQ_OK) {
    double* theta_sum = reinterpret_cast<double*>(buf);  // N x M reals (after the dPhi kernels)
    k_bwd_theta_sum<<<(int)((NM + 255) / 256), 256, 0, ctx->stream>>>(W, NM, t.thetaT, gE,
                                                                      theta_sum);
    rc = launched(ctx);
    // dh1 = Psi (M x N) Re(Theta) (N x M); Psi(p, j) = psiT[j M + p]
    if (rc == AFQ_OK)
      rc = launch_dgemm(ctx, M, M, N, 1.0, ctx->psiT, 1, M, 0, theta_sum, M, 1, 0, 0.0, dh1, M, 1,
                        0, 1, 1);
  }
  if (F && rc == AFQ_OK) {
    k_bwd_weight<<<bwd_grid((long)W * NM, 256), 256, 0, ctx->stream>>>(W, NM, gE, t.thetaT, u);
    k_bwd_weight<<<bwd_grid((long)W * X, 256), 256, 0, ctx->stream>>>(W, X, gE, t.c, q);
    ctx->launches++;
    rc = launched(ctx);
    const double* ur = reinterpret_cast<const double*>(u);
    const double* qr = reinterpret_cast<const double*>(q);
    for (int s = 0; s < 2 && rc == AFQ_OK; ++s) {
      const int n = s ? ctx->nb : ctx->na, off = s ? ctx->na : 0;
      if (n == 0) continue;
      const long nM = (long)n * M, o2 = 2L * off * M;
      double* Fs = F + (long)off * M;
      // F += Re sum_z q_zg theta^T_z
      rc = launch_dgemm(ctx, X, (int)nM, W, 1.0, qr, 2, 2L * X, 0, th + o2, 2 * NM, 2, 0, 1.0, Fs,
                        NM, 1, 0, 1, 1);
      if (rc == AFQ_OK)
        rc = launch_dgemm(ctx, X, (int)nM, W, -1.0, qr + 1, 2, 2L * X, 0, th + o2 + 1, 2 * NM, 2,
                          0, 1.0, Fs, NM, 1, 0, 1, 1);
      // Y: for each j, the blocks (q, p) of the i >= j: Re sum_z u_z[j][q] theta_z[i][p];
      // Y is symmetric, so the blocks i < j are the transposes of blocks (j, i)
      for (int j = 0; j < n && rc == AFQ_OK; ++j)
        for (int ri = 0; ri < 2 && rc == AFQ_OK; ++ri)
          rc = launch_dgemm(ctx, M, M, W, ri ? -1.0 : 1.0, ur + 2L * (off + j) * M + ri, 2, 2 * NM,
                            0, th + o2 + ri + 2L * j * M, 2 * NM, 2, 2L * M, ri ? 1.0 : 0.0,
                            Y + (long)j * M + (long)j * M * nM, nM, 1, (long)M * nM, n - j, 1);
      if (rc == AFQ_OK && n > 1) {
        k_mirror_blocks<<<bwd_grid((long)n * n * M * M, 256), 256, 0, ctx->stream>>>(n, M, Y);
        rc = launched(ctx);
      }
      // F -= L~ Y
      if (rc == AFQ_OK)
        rc = launch_dgemm(ctx, X, (int)nM, (int)nM, -1.0, ctx->Lt + (long)off * M, NM, 1, 0, Y,
                          nM, 1, 0, 1.0, Fs, NM, 1, 0, 1, 1);
    }
  }
  if (rc == AFQ_OK && cudaGetLastError() != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "local-energy backward launch");
  // the workspaces are released only after the kernels that read them are done
  cudaStreamSynchronize(ctx->stream);
  if (buf) cudaFree(buf);
  if (u) cudaFree(u);
  if (q) cudaFree(q);
  if (Y) cudaFree(Y);
  return rc;
}

// lambda_in += (I - Psi theta^T) lambda_theta S^-T for every walker (lamT: W x N x M,
// the cotangent of theta stored transposed like thetaT).
int launch_bwd_theta(afq_ctx* ctx, WalkerSet& t, const double2* lamT, double2* lam) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  if (nmax > 64) return afq_fail(ctx, AFQ_ERR_ARG, "adjoint needs max(na, nb) <= 64");
  AFQ_TRY(configure_bwd(ctx, dphi_smem(nmax)));
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
