// Adjoint of a K-step phaseless chain (FP64).
//
// The paper leaves automatic differentiation to future work (Sec. "Customized mixed
// estimators").  The objective is Loss = sum_z Re(conj(g_z) E_L(Phi_z^K)) after K
// steps of Sec. "Review of AFQMC" with the fields xi held fixed; the force bias is
// differentiated through, the weights are not part of the objective.  Cotangents
// are carried as holomorphic duals lam = conj(dLoss/dRe Phi + i dLoss/dIm Phi), so
// every adjoint is a plain transpose; real parameters take Re at the end.
//
// One step, per walker (B(y) Phi = P T_n(A) P Phi):
//   t_0 = P Phi, t_k = A t_{k-1} / k, Phi2 = sum_k t_k, Phi' = P Phi2
//   lam2 = P lam', mu_n = lam2, mu_{k-1} = lam2 + A mu_k / k, lam1 = mu_0, lam = P lam1
//   Pbar += Re(lam' Phi2^T + lam1 Phi^T)
//   Abar = sum_k mu_k t_{k-1}^T / k; A = i sqrt(dt) sum_g y_g L_g:
//     Q_g = <Abar, L_g>, ybar = i sqrt(dt) Q, Lbar_g += Re(i sqrt(dt) sum_z y_zg Abar_z)
//   y = xi - xbar, xbar = -i sqrt(dt) (c - vbar): cbar = -dt Q, vbar_bar += dt Re sum_z Q
//   c_g = sum_s tr(L~_g,s theta_s): theta_bar = sum_g cbar_g L~_g^T,
//     F_g += Re sum_z cbar_zg theta_z^T (dL_g = Psi F_g at the end)
//   theta = Phi S^-1: lam += (I - Psi theta^T) theta_bar S^-T
// QR (a gauge: the objective is invariant under Phi -> Phi C): lam_pre = lam_post R^-T
// with R = Q^H Phi_pre.  P = exp(B), B = -dt h''/2: hbar'' = -dt/2 L_exp(B, Pbar),
// the Frechet adjoint taken as the upper-right block of exp([[B, Pbar], [0, B]])
// (Van Loan 1978; Higham, Functions of Matrices, 2008, Sec. 3.2).  Then
// h'' = h1 - 1/2 sum L_g L_g + sum vbar_g L_g and vbar_g = sum_s tr(Psi_s^T L_g Psi_s)
// give dh1 and the rest of dL_g.  Gradients in h1 and L_g are symmetrised.
#include <cmath>
#include <vector>

#include "afq_internal.cuh"

namespace {

constexpr int ZT = 32, ZK = 16;

// C_b = alpha (A_b B_b + D_b) + beta C_b for complex matrices with arbitrary element
// strides; D may be NULL.  blockIdx.z = batch index.  Each complex multiply-add is
// Gauss's three real products: with the tile sums a+ = Re a + Im a, b+ = Re b + Im b
// formed once per staged element, Re = sum Re a Re b - sum Im a Im b and
// Im = sum a+ b+ - (both sums): 3 FMAs instead of 4 on B300's 2-lane FP64 pipe.
__global__ void __launch_bounds__(256) k_zgemm(int m, int n, int k, double alpha,
                                               const double2* __restrict__ A, long sam, long sak,
                                               long sab, const double2* __restrict__ B, long sbk,
                                               long sbn, long sbb, const double2* __restrict__ D,
                                               long sdm, long sdn, long sdb, double beta,
                                               double2* C, long scm, long scn, long scb) {
  __shared__ double2 As[ZT][ZK + 1];
  __shared__ double2 Bs[ZK][ZT + 1];
  __shared__ double Ap[ZT][ZK + 1];
  __shared__ double Bp[ZK][ZT + 1];
  const long b = blockIdx.z;
  const int i0 = blockIdx.y * ZT, j0 = blockIdx.x * ZT;
  const int tx = threadIdx.x % ZT, ty = threadIdx.x / ZT;  // ty in 0..7
  A += b * sab;
  B += b * sbb;
  C += b * scb;
  if (D) D += b * sdb;
  const bool a_rowmajor = sak == 1 || sam != 1;  // consecutive threads walk k (else rows)
  const bool b_colfast = sbn == 1 || sbk != 1;   // consecutive threads walk columns (else k)
  double p1[4], p2[4], p3[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) p1[r] = p2[r] = p3[r] = 0.0;
  for (int k0 = 0; k0 < k; k0 += ZK) {
    for (int e = threadIdx.x; e < ZT * ZK; e += 256) {
      const int r = a_rowmajor ? e / ZK : e % ZT, kk = a_rowmajor ? e % ZK : e / ZT;
      const int gi = i0 + r, gk = k0 + kk;
      const double2 av = (gi < m && gk < k) ? A[gi * sam + gk * sak] : cmk(0.0, 0.0);
      As[r][kk] = av;
      Ap[r][kk] = av.x + av.y;
      const int kr = b_colfast ? e / ZT : e % ZK, cc = b_colfast ? e % ZT : e / ZK;
      const int gk2 = k0 + kr, gj = j0 + cc;
      const double2 bv = (gj < n && gk2 < k) ? B[gk2 * sbk + gj * sbn] : cmk(0.0, 0.0);
      Bs[kr][cc] = bv;
      Bp[kr][cc] = bv.x + bv.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < ZK; ++kk) {
      const double2 bv = Bs[kk][tx];
      const double bp = Bp[kk][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double2 av = As[ty + 8 * r][kk];
        p1[r] = fma(av.x, bv.x, p1[r]);
        p2[r] = fma(av.y, bv.y, p2[r]);
        p3[r] = fma(Ap[ty + 8 * r][kk], bp, p3[r]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 8 * r, gj = j0 + tx;
    if (gi < m && gj < n) {
      double2 v = cmk(p1[r] - p2[r], p3[r] - p1[r] - p2[r]);
      if (D) v = cadd(v, D[gi * sdm + gj * sdn]);
      v = cscale(v, alpha);
      double2* cp = C + gi * scm + gj * scn;
      if (beta != 0.0) v = cadd(v, cscale(*cp, beta));
      *cp = v;
    }
  }
}

__global__ void __launch_bounds__(256) k_re_outer(int W, int M, int N, int zchunk,
                                                  const double2* __restrict__ Xm,
                                                  const double2* __restrict__ Ym,
                                                  double* __restrict__ part) {
  __shared__ double2 Xs[ZT][ZK + 1];
  __shared__ double2 Ys[ZT][ZK + 1];
  const int zs = blockIdx.z;
  const int z0 = zs * zchunk, z1 = min(W, z0 + zchunk);
  const int p0 = blockIdx.y * ZT, q0 = blockIdx.x * ZT;
  const int tx = threadIdx.x % ZT, ty = threadIdx.x / ZT;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long kt = (long)(z1 > z0 ? z1 - z0 : 0) * N;
  for (long k0 = 0; k0 < kt; k0 += ZK) {
    for (int e = threadIdx.x; e < ZT * ZK; e += 256) {
      const int r = e / ZK, kk = e % ZK;
      const long gk = k0 + kk;
      double2 xv = cmk(0.0, 0.0), yv = cmk(0.0, 0.0);
      if (gk < kt) {
        const long z = z0 + gk / N, j = gk % N;
        if (p0 + r < M) xv = Xm[(z * M + p0 + r) * N + j];
        if (q0 + r < M) yv = Ym[(z * M + q0 + r) * N + j];
      }
      Xs[r][kk] = xv;
      Ys[r][kk] = yv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < ZK; ++kk) {
      const double2 yv = Ys[tx][kk];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double2 xv = Xs[ty + 8 * r][kk];
        acc[r] = fma(xv.x, yv.x, fma(-xv.y, yv.y, acc[r]));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + ty + 8 * r, q = q0 + tx;
    if (p < M && q < M) part[((long)zs * M + p) * M + q] = acc[r];
  }
}

__global__ void k_add_parts(long n, int nparts, const double* __restrict__ part,
                            double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    double s = out[e];
    for (int k = 0; k < nparts; ++k) s += part[(long)k * n + e];
    out[e] = s;
  }
}

// Abar'' [z][t] = Abar_pq + Abar_qp (p < q) or Abar_pp, t = packed index of (p, q)
__global__ void k_pack_sym(int W, int M, int Mp, const int2* __restrict__ tpq,
                           const double2* __restrict__ Abar, double2* __restrict__ out) {
  const long n = (long)W * Mp;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const long z = e / Mp;
    const int2 pq = tpq[e % Mp];
    const double2* a = Abar + z * M * M;
    double2 v = a[(long)pq.x * M + pq.y];
    if (pq.x != pq.y) v = cadd(v, a[(long)pq.y * M + pq.x]);
    out[e] = v;
  }
}

// lv[g] += alpha sum_z Re Q[z][g]
__global__ void k_colsum_re(int W, int X, double alpha, const double2* __restrict__ Q,
                            double* __restrict__ lv) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= X) return;
  double s = 0.0;
  for (int z = 0; z < W; ++z) s += Q[(long)z * X + g].x;
  lv[g] += alpha * s;
}

// Phi2 = sum_{k=0..nb-1} T[:, :, k N : (k+1) N]   (T rows hold nb blocks of N)
__global__ void k_sum_blocks(long WM, int N, int nb, const double2* __restrict__ T,
                             double2* __restrict__ out) {
  const long n = WM * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const long row = e / N;
    const int j = (int)(e % N);
    const double2* t = T + row * (long)nb * N + j;
    double2 s = cmk(0.0, 0.0);
    for (int k = 0; k < nb; ++k) s = cadd(s, t[(long)k * N]);
    out[e] = s;
  }
}

// dst row r (stride ld) = a * src row r (stride N), r over W M rows
__global__ void k_scale_rows(long WM, int N, double a, const double2* __restrict__ src,
                             double2* __restrict__ dst, long ld) {
  const long n = WM * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const long row = e / N;
    const int j = (int)(e % N);
    dst[row * ld + j] = cscale(src[e], a);
  }
}

__global__ void k_conj(long n, const double2* __restrict__ src, double2* __restrict__ dst) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    dst[e] = cconj(src[e]);
}

// lam <- lam R^-T per (walker, spin) with R = Q^H Phi_pre upper triangular: the
// cotangent of the walkers before the QR, from that of its output Q.
__global__ void __launch_bounds__(256) k_bwd_qr(int M, int N, int na, int nb,
                                                const double2* __restrict__ Qm,
                                                const double2* __restrict__ pre,
                                                double2* __restrict__ lam) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* R = reinterpret_cast<double2*>(smraw);  // n x n
  const int z = blockIdx.x, s = blockIdx.y;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) return;
  const double2* Qz = Qm + (long)z * M * N;
  const double2* Pz = pre + (long)z * M * N;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double2 v = cmk(0.0, 0.0);
    if (i <= j)
      for (int p = 0; p < M; ++p)
        v = cfma_conj(Qz[(long)p * N + off + i], Pz[(long)p * N + off + j], v);
    R[e] = v;
  }
  __syncthreads();
  double2* Lz = lam + (long)z * M * N;
  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    double2* row = Lz + (long)p * N + off;
    for (int j = n - 1; j >= 0; --j) {
      double2 v = row[j];
      for (int k = j + 1; k < n; ++k) v = cfms(R[j * n + k], row[k], v);
      row[j] = cdiv(v, R[j * n + j]);
    }
  }
}

// Z = [[B, E / s], [0, B]] (2M x 2M) for the Frechet adjoint of exp
__global__ void k_block_frechet(int M, const double* __restrict__ B, const double* __restrict__ E,
                                double inv_s, double* __restrict__ Z) {
  const long n = 4L * M * M;
  const int M2 = 2 * M;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M2), j = (int)(e % M2);
    double v = 0.0;
    if (i < M && j < M) v = B[(long)i * M + j];
    else if (i >= M && j >= M) v = B[(long)(i - M) * M + (j - M)];
    else if (i < M) v = E[(long)i * M + (j - M)] * inv_s;
    Z[e] = v;
  }
}

// out = s * upper-right block of expZ, scaled by a
__global__ void k_block_extract(int M, const double* __restrict__ expZ, double a,
                                double* __restrict__ out) {
  const long n = (long)M * M;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e % M);
    out[e] = a * expZ[(long)i * 2 * M + M + j];
  }
}

// dL_g,pq = sym(D_g)_pq + vbar_g sym(hb)_pq + lv_g Pt_pq + unpack(Lpk_bar)_g,pq
// (the packed part holds Abar_pq + Abar_qp off the diagonal: halved here)
__global__ void k_dl_assemble(int X, int M, int Mp, const double* __restrict__ D,
                              const double* __restrict__ hb, const double* __restrict__ vbar,
                              const double* __restrict__ lv, const double* __restrict__ Pt,
                              const double* __restrict__ Lpkb, double* __restrict__ out) {
  const long MM = (long)M * M, n = (long)X * MM;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const int g = (int)(e / MM);
    const int p = (int)((e % MM) / M), q = (int)(e % M);
    const double* Dg = D + (long)g * MM;
    const int a = p < q ? p : q, b = p < q ? q : p;
    const long t = (long)a * M - (long)a * (a - 1) / 2 + (b - a);
    const double pk = Lpkb[(long)g * Mp + t] * (p == q ? 1.0 : 0.5);
    out[e] = 0.5 * (Dg[(long)p * M + q] + Dg[(long)q * M + p]) +
             vbar[g] * 0.5 * (hb[(long)p * M + q] + hb[(long)q * M + p]) + lv[g] * Pt[(long)p * M + q] +
             pk;
  }
}

// out = sym(a + b); b may be NULL
__global__ void k_sym_sum(int M, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ out) {
  const long n = (long)M * M;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const int p = (int)(e / M), q = (int)(e % M);
    const long et = (long)q * M + p;
    out[e] = 0.5 * (a[e] + a[et] + (b ? b[e] + b[et] : 0.0));
  }
}

// q[(z X + g) 2 + ri] = sum_ks part[((ri ksplit + ks) W + z) X + g]  (fixed order)
__global__ void k_q_reduce(long WX, int ksplit, const double* __restrict__ part,
                           double* __restrict__ q) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < 2 * WX;
       e += (long)gridDim.x * blockDim.x) {
    const int ri = (int)(e / WX);
    const long zg = e % WX;
    double s = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) s += part[((long)ri * ksplit + ks) * WX + zg];
    q[2 * zg + ri] = s;
  }
}

// lv_g += <L_g, a> over the M x M entries (one block per g, fixed-order reduction)
__global__ void __launch_bounds__(256) k_dot_rows(long MM, const double* __restrict__ L,
                                                  const double* __restrict__ a,
                                                  double* __restrict__ lv) {
  __shared__ double red[8];
  const int g = blockIdx.x;
  double v = 0.0;
  for (long e = threadIdx.x; e < MM; e += 256) v = fma(L[(long)g * MM + e], a[e], v);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    lv[g] += t;
  }
}

int grid_of(long n) {
  long g = (n + 255) / 256;
  if (g > 148 * 32) g = 148 * 32;
  return (int)(g < 1 ? 1 : g);
}

int launch_zgemm(afq_ctx* ctx, int m, int n, int k, double alpha, const double2* A, long sam,
                 long sak, long sab, const double2* B, long sbk, long sbn, long sbb,
                 const double2* D, long sdm, long sdn, long sdb, double beta, double2* C, long scm,
                 long scn, long scb, int batch) {
  if (m <= 0 || n <= 0) return AFQ_OK;
  if (batch > 65535) return afq_fail(ctx, AFQ_ERR_ARG, "zgemm: batch too large");
  dim3 grid((n + ZT - 1) / ZT, (m + ZT - 1) / ZT, batch);
  k_zgemm<<<grid, 256, 0, ctx->stream>>>(m, n, k, alpha, A, sam, sak, sab, B, sbk, sbn, sbb, D,
                                         sdm, sdn, sdb, beta, C, scm, scn, scb);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// Device workspace of one chain backward.
struct ChainWork {
  double2 *lam = nullptr, *lam2 = nullptr, *mu0 = nullptr, *phi2 = nullptr;
  double2 *T = nullptr, *U = nullptr, *Abar = nullptr, *Apk = nullptr, *Q = nullptr;
  double2 *lamT = nullptr, *seg = nullptr;
  double2 *A = nullptr, *xbar = nullptr, *y = nullptr, *cfb = nullptr, *cmf = nullptr;
  double *Ppart = nullptr, *Pbar = nullptr, *F = nullptr, *Lpkb = nullptr, *lv = nullptr;
  double *dh1E = nullptr, *hb = nullptr, *Pt = nullptr, *Z = nullptr, *D = nullptr;
  double *qpart = nullptr, *hs = nullptr;
  WalkerSet ws;
  std::vector<void*> owned;
};

template <class T>
int walloc(afq_ctx* ctx, ChainWork& w, T** p, size_t n) {
  if (n == 0) n = 1;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    return afq_fail(ctx, AFQ_ERR_NOMEM, "chain backward workspace");
  }
  w.owned.push_back(*p);
  return AFQ_OK;
}

constexpr int ZSPLIT = 32;  // walker chunks of the Pbar partial sums

// Pbar += Re sum_z X_z Y_z^T
int add_re_outer(afq_ctx* ctx, ChainWork& w, const double2* Xm, const double2* Ym) {
  const int M = ctx->M, N = ctx->N, W = ctx->chain.W;
  const int zchunk = (W + ZSPLIT - 1) / ZSPLIT;
  const int parts = (W + zchunk - 1) / zchunk;
  dim3 grid((M + ZT - 1) / ZT, (M + ZT - 1) / ZT, parts);
  k_re_outer<<<grid, 256, 0, ctx->stream>>>(W, M, N, zchunk, Xm, Ym, w.Ppart);
  AFQ_LAUNCHED(ctx);
  const long MM = (long)M * M;
  k_add_parts<<<grid_of(MM), 256, 0, ctx->stream>>>(MM, parts, w.Ppart, w.Pbar);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

constexpr int QSPLIT = 4;  // K split of the Q = <Abar, L_g> contraction (load balance)

// The step's operands live in per-step slots of the segment: i sqrt(dt) V (ctx->A),
// the shifted fields y and the Taylor tape t_0 .. t_n.
void point_step(afq_ctx* ctx, ChainWork& w, int i) {
  const long W = ctx->chain.W, MM = (long)ctx->M * ctx->M;
  ctx->A = w.A + i * W * MM;
  ctx->y = w.y + i * W * ctx->X;
}
double2* tape_of(afq_ctx* ctx, ChainWork& w, int i) {
  return w.T + (long)i * (ctx->p.taylor_order + 1) * ctx->chain.W * ctx->M * ctx->N;
}

// Recompute step i of a segment from phi_in (fields xi) into phi_out, keeping its
// operands for the backward: t_0 = P phi_in (real P on re/im interleaved rows),
// t_k = A t_{k-1} / k, phi_out = P sum_k t_k.
int forward_tape(afq_ctx* ctx, ChainWork& w, int i, double2* phi_in, const double* xi,
                 double2* phi_out) {
  const int M = ctx->M, N = ctx->N, W = ctx->chain.W, n = ctx->p.taylor_order;
  const long MN = (long)M * N, WMN = (long)W * MN, MM = (long)M * M, RT = (long)(n + 1) * N;
  double2* T = tape_of(ctx, w, i);
  point_step(ctx, w, i);
  ctx->ws.phi = phi_in;
  AFQ_TRY(launch_overlap_theta(ctx, ctx->ws));
  AFQ_TRY(launch_force_bias_fp64(ctx, ctx->ws));
  AFQ_TRY(launch_fields(ctx, xi));
  AFQ_TRY(launch_vhs_fp64(ctx));
  AFQ_TRY(launch_dgemm(ctx, M, 2 * N, M, 1.0, ctx->P, M, 1, 0, reinterpret_cast<double*>(phi_in),
                       2 * N, 1, 2 * MN, 0.0, reinterpret_cast<double*>(T), 2 * RT, 1, 2 * M * RT,
                       W, 1));
  for (int k = 1; k <= n; ++k)
    AFQ_TRY(launch_zgemm(ctx, M, N, M, 1.0 / k, ctx->A, M, 1, MM, T + (long)(k - 1) * N, RT, 1,
                         M * RT, nullptr, 0, 0, 0, 0.0, T + (long)k * N, RT, 1, M * RT, W));
  k_sum_blocks<<<grid_of(WMN), 256, 0, ctx->stream>>>((long)W * M, N, n + 1, T, w.phi2);
  AFQ_LAUNCHED(ctx);
  AFQ_TRY(launch_dgemm(ctx, M, 2 * N, M, 1.0, ctx->P, M, 1, 0, reinterpret_cast<double*>(w.phi2),
                       2 * N, 1, 2 * MN, 0.0, reinterpret_cast<double*>(phi_out), 2 * N, 1, 2 * MN,
                       W, 1));
  return AFQ_OK;
}

// Backward of step i of a segment at walkers phi_in (its operands kept by
// forward_tape): lam (cotangent of the step's output before any QR) becomes the
// cotangent of phi_in; Pbar, F, Lpkb and lv accumulate.
int step_backward(afq_ctx* ctx, ChainWork& w, double2* phi_in, int i) {
  const int M = ctx->M, N = ctx->N, X = ctx->X, W = ctx->chain.W, Mp = ctx->Mp;
  const int n = ctx->p.taylor_order;
  const long MN = (long)M * N, WMN = (long)W * MN, MM = (long)M * M, NM = (long)N * M;
  const long RT = (long)(n + 1) * N, RU = (long)n * N;
  const double dt = ctx->p.dt, sdt = std::sqrt(dt);
  double2* T = tape_of(ctx, w, i);
  point_step(ctx, w, i);
  ctx->ws.phi = phi_in;
  AFQ_TRY(launch_overlap_theta(ctx, ctx->ws));  // theta at phi_in
  k_sum_blocks<<<grid_of(WMN), 256, 0, ctx->stream>>>((long)W * M, N, n + 1, T, w.phi2);
  AFQ_LAUNCHED(ctx);
  // outer P: lam2 = P lam, Pbar += Re lam Phi2^T
  AFQ_TRY(launch_dgemm(ctx, M, 2 * N, M, 1.0, ctx->P, M, 1, 0, reinterpret_cast<double*>(w.lam),
                       2 * N, 1, 2 * MN, 0.0, reinterpret_cast<double*>(w.lam2), 2 * N, 1, 2 * MN,
                       W, 1));
  AFQ_TRY(add_re_outer(ctx, w, w.lam, w.phi2));
  // Taylor: U block k-1 = mu_k / k; mu_n = lam2; mu_{k-1} = lam2 + A U_k
  k_scale_rows<<<grid_of(WMN), 256, 0, ctx->stream>>>((long)W * M, N, 1.0 / n, w.lam2,
                                                      w.U + (long)(n - 1) * N, RU);
  AFQ_LAUNCHED(ctx);
  for (int k = n; k >= 1; --k) {
    const double2* Uk = w.U + (long)(k - 1) * N;
    if (k > 1)
      AFQ_TRY(launch_zgemm(ctx, M, N, M, 1.0 / (k - 1), ctx->A, M, 1, MM, Uk, RU, 1, M * RU, w.lam2,
                           N, 1, MN, 0.0, w.U + (long)(k - 2) * N, RU, 1, M * RU, W));
    else
      AFQ_TRY(launch_zgemm(ctx, M, N, M, 1.0, ctx->A, M, 1, MM, Uk, RU, 1, M * RU, w.lam2, N, 1,
                           MN, 0.0, w.mu0, N, 1, MN, W));
  }
  // Abar = [mu_1/1 .. mu_n/n] [t_0 .. t_{n-1}]^T
  AFQ_TRY(launch_zgemm(ctx, M, M, n * N, 1.0, w.U, RU, 1, M * RU, T, 1, RT, M * RT, nullptr, 0, 0,
                       0, 0.0, w.Abar, M, 1, MM, W));
  // inner P: lam = P mu0, Pbar += Re mu0 phi_in^T
  AFQ_TRY(add_re_outer(ctx, w, w.mu0, phi_in));
  AFQ_TRY(launch_dgemm(ctx, M, 2 * N, M, 1.0, ctx->P, M, 1, 0, reinterpret_cast<double*>(w.mu0),
                       2 * N, 1, 2 * MN, 0.0, reinterpret_cast<double*>(w.lam), 2 * N, 1, 2 * MN,
                       W, 1));
  // VHS: Q_zg = <Abar_z, L_g> over packed symmetric pairs; re and im as a batch of two,
  // the packed dimension split QSPLIT ways (partials summed in a fixed order)
  k_pack_sym<<<grid_of((long)W * Mp), 256, 0, ctx->stream>>>(W, M, Mp, ctx->tpq, w.Abar, w.Apk);
  AFQ_LAUNCHED(ctx);
  const double* apk = reinterpret_cast<const double*>(w.Apk);
  double* q = reinterpret_cast<double*>(w.Q);
  const long WX = (long)W * X;
  AFQ_TRY(launch_dgemm(ctx, W, X, Mp, 1.0, apk, 2L * Mp, 2, 1, ctx->Lpk, 1, Mp, 0, 0.0, w.qpart, X,
                       1, WX, 2, QSPLIT));
  k_q_reduce<<<grid_of(2 * WX), 256, 0, ctx->stream>>>(WX, QSPLIT, w.qpart, q);
  AFQ_LAUNCHED(ctx);
  // Lbar (packed) += Re(i sqrt(dt) sum_z y_zg Abar''_z) = -sqrt(dt) (y_i Abar''_r + y_r Abar''_i)
  const double* yv = reinterpret_cast<const double*>(ctx->y);
  AFQ_TRY(launch_dgemm(ctx, X, Mp, W, -sdt, yv + 1, 2, 2L * X, 0, apk, 2L * Mp, 2, 0, 1.0, w.Lpkb,
                       Mp, 1, 0, 1, 1));
  AFQ_TRY(launch_dgemm(ctx, X, Mp, W, -sdt, yv, 2, 2L * X, 0, apk + 1, 2L * Mp, 2, 0, 1.0, w.Lpkb,
                       Mp, 1, 0, 1, 1));
  // force bias: cbar = -dt Q, vbar_bar += dt Re sum_z Q
  k_colsum_re<<<(X + 255) / 256, 256, 0, ctx->stream>>>(W, X, dt, w.Q, w.lv);
  AFQ_LAUNCHED(ctx);
  // theta_bar^T = sum_g cbar_g L~_g (W x N x M complex)
  double* lt = reinterpret_cast<double*>(w.lamT);
  for (int ri = 0; ri < 2; ++ri)
    AFQ_TRY(launch_dgemm(ctx, W, (int)NM, X, -dt, q + ri, 2L * X, 2, 0, ctx->Lt, NM, 1, 0, 0.0,
                         lt + ri, 2 * NM, 2, 0, 1, 1));
  // F_g += Re sum_z cbar_zg theta_z^T = -dt (Q_r theta_r - Q_i theta_i)
  const double* th = reinterpret_cast<const double*>(ctx->ws.thetaT);
  AFQ_TRY(launch_dgemm(ctx, X, (int)NM, W, -dt, q, 2, 2L * X, 0, th, 2 * NM, 2, 0, 1.0, w.F, NM, 1,
                       0, 1, 1));
  AFQ_TRY(launch_dgemm(ctx, X, (int)NM, W, dt, q + 1, 2, 2L * X, 0, th + 1, 2 * NM, 2, 0, 1.0, w.F,
                       NM, 1, 0, 1, 1));
  // theta = Phi S^-1
  AFQ_TRY(launch_bwd_theta(ctx, ctx->ws, w.lamT, w.lam));
  return AFQ_OK;
}

// hbar'' = -dt/2 L_exp(B, Pbar), B = -dt h''/2 (symmetric)
int exp_adjoint(afq_ctx* ctx, ChainWork& w) {
  const int M = ctx->M;
  const long MM = (long)M * M;
  std::vector<double> hpp(MM), pb(MM);
  AFQ_CUDA(ctx, cudaMemcpyAsync(hpp.data(), ctx->hpp, MM * 8, cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_CUDA(ctx, cudaMemcpyAsync(pb.data(), w.Pbar, MM * 8, cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double nb = 0.0, ne = 0.0;
  for (int q = 0; q < M; ++q) {
    double sb = 0.0, se = 0.0;
    for (int p = 0; p < M; ++p) {
      sb += std::fabs(hpp[(size_t)p * M + q]);
      se += std::fabs(pb[(size_t)p * M + q]);
    }
    nb = std::fmax(nb, sb);
    ne = std::fmax(ne, se);
  }
  nb *= 0.5 * ctx->p.dt;
  if (!std::isfinite(nb) || !std::isfinite(ne)) return afq_fail(ctx, AFQ_ERR_NAN, "P adjoint not finite");
  if (ne == 0.0) {
    AFQ_CUDA(ctx, cudaMemsetAsync(w.hb, 0, MM * 8, ctx->stream));
    return AFQ_OK;
  }
  const double s = ne / 0.5;  // the Frechet block enters with 1-norm 0.5
  double* B = w.Z + 8 * MM;   // -dt/2 h''
  AFQ_TRY(launch_axpby(ctx, (int)MM, -0.5 * ctx->p.dt, ctx->hpp, 0.0, B));
  k_block_frechet<<<grid_of(4 * MM), 256, 0, ctx->stream>>>(M, B, w.Pbar, 1.0 / s, w.Z);
  AFQ_LAUNCHED(ctx);
  double* E = w.Z + 4 * MM;
  AFQ_TRY(expm_taylor(ctx, w.Z, 1.0, 2 * M, nb + 0.5, E));
  k_block_extract<<<grid_of(MM), 256, 0, ctx->stream>>>(M, E, -0.5 * ctx->p.dt * s, w.hb);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int run_backward(afq_ctx* ctx, ChainWork& w, const double2* gE, double* dh1, double* dL,
                 double2* dphi0) {
  ChainTape& tp = ctx->chain;
  const int M = ctx->M, N = ctx->N, X = ctx->X, W = tp.W, Mp = ctx->Mp;
  const long MN = (long)M * N, WMN = (long)W * MN, MM = (long)M * M, NM = (long)N * M;
  const long WX = (long)W * X;
  AFQ_CUDA(ctx, cudaMemsetAsync(w.Pbar, 0, MM * 8, ctx->stream));
  AFQ_CUDA(ctx, cudaMemsetAsync(w.F, 0, (size_t)X * NM * 8, ctx->stream));
  AFQ_CUDA(ctx, cudaMemsetAsync(w.Lpkb, 0, (size_t)X * Mp * 8, ctx->stream));
  AFQ_CUDA(ctx, cudaMemsetAsync(w.lv, 0, (size_t)X * 8, ctx->stream));
  // the energy at Phi^K (the context's walkers): dh1, F and lam = conj(g) dE/dPhi
  AFQ_TRY(launch_overlap_theta(ctx, ctx->ws));
  AFQ_TRY(launch_force_bias_fp64(ctx, ctx->ws));
  AFQ_TRY(adjoint_energy_core(ctx, ctx->ws, gE, w.dh1E, w.F, w.lam, 1));
  for (int si = (int)tp.segs.size() - 1; si >= 0; --si) {
    const ChainSeg sg = tp.segs[si];
    // recompute the segment's walkers from its checkpoint
    AFQ_CUDA(ctx, cudaMemcpyAsync(w.seg, tp.ckpt + (long)sg.ck_in * WMN, WMN * 16,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    for (int i = 0; i < sg.len; ++i) {
      double2* cur = w.seg + (long)i * WMN;
      AFQ_TRY(forward_tape(ctx, w, i, cur, tp.fields + (long)(sg.start + i) * WX, cur + WMN));
    }
    if (sg.qr_end) {
      const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
      const size_t sm = (size_t)nmax * nmax * 16;
      AFQ_CUDA(ctx, raise_smem_limit((const void*)k_bwd_qr, sm));
      k_bwd_qr<<<dim3(W, 2), 256, sm, ctx->stream>>>(M, N, ctx->na, ctx->nb,
                                                     tp.ckpt + (long)sg.ck_out * WMN,
                                                     w.seg + (long)sg.len * WMN, w.lam);
      AFQ_LAUNCHED(ctx);
    }
    for (int i = sg.len - 1; i >= 0; --i)
      AFQ_TRY(step_backward(ctx, w, w.seg + (long)i * WMN, i));
  }
  // parameters
  AFQ_TRY(exp_adjoint(ctx, w));
  if (dphi0) {
    k_conj<<<grid_of(WMN), 256, 0, ctx->stream>>>(WMN, w.lam, dphi0);
    AFQ_LAUNCHED(ctx);
  }
  if (dh1) {
    k_sym_sum<<<grid_of(MM), 256, 0, ctx->stream>>>(M, w.hb, w.dh1E, dh1);
    AFQ_LAUNCHED(ctx);
  }
  if (dL) {
    // hs = sym(hbar''); with L_g symmetric, <hbar'', L_g> = <hs, L_g> and
    // sym(hbar'' L_g + L_g hbar'') = sym(2 hs L_g)
    k_sym_sum<<<grid_of(MM), 256, 0, ctx->stream>>>(M, w.hb, nullptr, w.hs);
    AFQ_LAUNCHED(ctx);
    // lv_g += <hs, L_g>
    k_dot_rows<<<X, 256, 0, ctx->stream>>>(MM, ctx->L, w.hs, w.lv);
    AFQ_LAUNCHED(ctx);
    // Pt = Psi Psi^T
    AFQ_TRY(launch_dgemm(ctx, M, M, N, 1.0, ctx->psiT, 1, M, 0, ctx->psiT, M, 1, 0, 0.0, w.Pt, M, 1,
                         0, 1, 1));
    // D_g = Psi F_g - hs L_g (symmetrised by the assembly)
    AFQ_TRY(launch_dgemm(ctx, M, M, N, 1.0, ctx->psiT, 1, M, 0, w.F, M, 1, NM, 0.0, w.D, M, 1, MM,
                         X, 1));
    AFQ_TRY(launch_dgemm(ctx, M, M, M, -1.0, w.hs, M, 1, 0, ctx->L, M, 1, MM, 1.0, w.D, M, 1, MM, X,
                         1));
    k_dl_assemble<<<grid_of((long)X * MM), 256, 0, ctx->stream>>>(X, M, Mp, w.D, w.hs, ctx->vbar,
                                                                  w.lv, w.Pt, w.Lpkb, dL);
    AFQ_LAUNCHED(ctx);
  }
  return AFQ_OK;
}

}  // namespace

void chain_free(afq_ctx* ctx) {
  ChainTape& t = ctx->chain;
  if (t.fields) cudaFree(t.fields);
  if (t.ckpt) cudaFree(t.ckpt);
  t = ChainTape();
}

int expm_taylor(afq_ctx* ctx, const double* src, double scale, int n, double norm1, double* out) {
  const size_t nn = (size_t)n * n;
  int sq = 0;
  while (norm1 / std::ldexp(1.0, sq) > 0.5) ++sq;
  double *Bm = nullptr, *E = nullptr, *T = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&Bm, nn * 8) != cudaSuccess || cudaMalloc((void**)&E, nn * 8) != cudaSuccess ||
      cudaMalloc((void**)&T, nn * 8) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "expm workspace");
  if (rc == AFQ_OK) rc = launch_axpby(ctx, (int)nn, scale / std::ldexp(1.0, sq), src, 0.0, Bm);
  if (rc == AFQ_OK) rc = launch_set_identity(ctx, n, E);
  for (int k = 18; k >= 1 && rc == AFQ_OK; --k) {
    rc = launch_set_identity(ctx, n, T);
    if (rc == AFQ_OK) rc = launch_dgemm(ctx, n, n, n, 1.0 / k, Bm, n, 1, 0, E, n, 1, 0, 1.0, T, n, 1, 0, 1, 1);
    std::swap(E, T);
  }
  for (int k = 0; k < sq && rc == AFQ_OK; ++k) {
    rc = launch_dgemm(ctx, n, n, n, 1.0, E, n, 1, 0, E, n, 1, 0, 0.0, T, n, 1, 0, 1, 1);
    std::swap(E, T);
  }
  if (rc == AFQ_OK &&
      cudaMemcpyAsync(out, E, nn * 8, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "expm copy");
  cudaStreamSynchronize(ctx->stream);
  if (Bm) cudaFree(Bm);
  if (E) cudaFree(E);
  if (T) cudaFree(T);
  return rc;
}

// Gradients of sum_z Re(conj(g_z) E_L(Phi_z^K)) for the chain on the tape: dh1 and dL
// symmetrised, dphi0 = dLoss/dRe Phi^0 + i dLoss/dIm Phi^0.  Device pointers; any
// output may be NULL.  The context's walkers, fields and force bias are untouched.
int chain_backward(afq_ctx* ctx, const double2* gE, double* dh1, double* dL, double2* dphi0) {
  ChainTape& tp = ctx->chain;
  if (!tp.valid) return afq_fail(ctx, AFQ_ERR_STATE, "afq_chain_forward first");
  if (ctx->step != tp.s0 + (uint64_t)tp.K || ctx->ws.W != tp.W)
    return afq_fail(ctx, AFQ_ERR_STATE, "the walkers changed since afq_chain_forward");
  const int M = ctx->M, N = ctx->N, X = ctx->X, W = tp.W, Mp = ctx->Mp;
  const int n = ctx->p.taylor_order;
  const size_t MN = (size_t)M * N, WMN = (size_t)W * MN, MM = (size_t)M * M;
  ChainWork w;
  int rc = AFQ_OK;
  auto A = [&](auto** p, size_t cnt) {
    if (rc == AFQ_OK) rc = walloc(ctx, w, p, cnt);
  };
  A(&w.lam, WMN);
  A(&w.lam2, WMN);
  A(&w.mu0, WMN);
  A(&w.phi2, WMN);
  const size_t cap = (size_t)tp.seg_cap;  // per-step operands of the longest segment
  A(&w.T, cap * WMN * (n + 1));
  A(&w.U, WMN * n);
  A(&w.Abar, (size_t)W * MM);
  A(&w.Apk, (size_t)W * Mp);
  A(&w.Q, (size_t)W * X);
  A(&w.lamT, WMN);
  A(&w.seg, WMN * (tp.seg_cap + 1));
  A(&w.A, cap * W * MM);
  A(&w.xbar, (size_t)W * X);
  A(&w.y, cap * W * X);
  A(&w.cfb, (size_t)W);
  A(&w.cmf, (size_t)W);
  A(&w.Ppart, (size_t)ZSPLIT * MM);
  A(&w.Pbar, MM);
  A(&w.F, (size_t)X * N * M);
  A(&w.Lpkb, (size_t)X * Mp);
  A(&w.lv, (size_t)X);
  A(&w.dh1E, MM);
  A(&w.hb, MM);
  A(&w.Pt, MM);
  A(&w.Z, 9 * MM);
  A(&w.qpart, (size_t)2 * QSPLIT * W * X);
  A(&w.hs, MM);
  if (dL) A(&w.D, (size_t)X * MM);
  w.ws.W = W;
  A(&w.ws.thetaT, WMN);
  A(&w.ws.det, (size_t)W * 2);
  A(&w.ws.e1, (size_t)W * 2);
  A(&w.ws.c, (size_t)W * X);
  if (rc == AFQ_OK) {
    // swap in private per-step buffers so the context's state survives the backward
    WalkerSet saved = ctx->ws;
    double2 *sA = ctx->A, *sx = ctx->xbar, *sy = ctx->y, *sf = ctx->cfb, *sm = ctx->cmf;
    w.ws.phi = saved.phi;  // Phi^K for the energy term
    ctx->ws = w.ws;
    ctx->A = w.A;
    ctx->xbar = w.xbar;
    ctx->y = w.y;
    ctx->cfb = w.cfb;
    ctx->cmf = w.cmf;
    rc = run_backward(ctx, w, gE, dh1, dL, dphi0);
    cudaStreamSynchronize(ctx->stream);
    ctx->ws = saved;
    ctx->A = sA;
    ctx->xbar = sx;
    ctx->y = sy;
    ctx->cfb = sf;
    ctx->cmf = sm;
  }
  cudaStreamSynchronize(ctx->stream);
  for (void* p : w.owned) cudaFree(p);
  return rc;
}
