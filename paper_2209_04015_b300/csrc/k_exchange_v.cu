// Exchange energy from the stored half-rotated two-electron tensor (FP64).
//
// Sec. "Local energy" writes the exchange term of a single determinant as
//   E_K,z = -1/2 sum_s sum_g tr(T_zg,s T_zg,s),   T_zg,s = L~_g,s theta_s,z
// and evaluates it by forming and consuming T per (walker, g): 2 X n^2 M
// multiply-adds per walker and spin.  Summing over g first gives the same number
// from a trial-fixed tensor (the paper cites this family of local-energy algorithms
// among the ones it implements):
//   sum_g tr(T_zg T_zg) = x_z^T V x_z,   x_z = theta^T_z flattened over (j, p),
//   V[(j,p),(i,q)] = sum_g L~_g[j][q] L~_g[i][p]   (real, symmetric, (n M)^2 per spin)
// which costs (n M)^2 multiply-adds per walker and spin when only the blocks on and
// above the diagonal of V are read (x^T V x = sum_I x_I^T (V_II x_I + 2 sum_J>I V_IJ x_J)).
// That is M / (2 X) of the direct count: 8x fewer at M = 100, X = 400.
//
// Work split: V is cut into 32 x 32 blocks; block row I needs the nbk - I blocks
// J >= I, so rows I and nbk - 1 - I are paired (nbk + 1 blocks per pair) and each
// pair's list of blocks is cut into S chunks of C blocks.  One CTA takes one chunk for
// 32 walkers (lane = walker, warp = 4 rows of the block) and writes -1/2 of its
// partial x_I^T y_I into its own exchange slot; the energy assembly adds the slots in
// a fixed order, so the result does not depend on scheduling.
#include "afq_internal.cuh"

namespace {

constexpr int VB = 32;   // edge of one block of V
constexpr int VT = 256;  // threads per CTA: 8 warps x 4 rows, one walker per lane
constexpr int kCtaTarget = 16 * 148;  // CTAs per launch (both spins): short CTAs, small tail
constexpr int kMaxChunks = 32;        // chunks per pair of block rows

struct ExSpin {
  const double* V;  // K x K, row-major
  long offe;        // first entry of the spin's rows in a walker's theta^T (off * M)
  int K, nbk, npairs, S, C;
};

__device__ __forceinline__ void load_v(const ExSpin& sp, int I, int J, double (*Vs)[VB + 1]) {
  for (int e = threadIdx.x; e < VB * VB; e += VT) {
    const int r = e / VB, k = e % VB, row = I * VB + r, col = J * VB + k;
    Vs[r][k] = (row < sp.K && col < sp.K) ? sp.V[(long)row * sp.K + col] : 0.0;
  }
}

// Xs[k][walker] = x_{z0 + walker}[J * 32 + k]
__device__ __forceinline__ void load_x(const ExSpin& sp, const double2* __restrict__ thetaT,
                                       long NM, int W, int z0, int J, double2 (*Xs)[VB + 1]) {
  for (int e = threadIdx.x; e < VB * VB; e += VT) {
    const int zl = e / VB, k = e % VB, z = z0 + zl, col = J * VB + k;
    Xs[k][zl] = (z < W && col < sp.K) ? thetaT[(long)z * NM + sp.offe + col] : cmk(0.0, 0.0);
  }
}

// acc[r] += sum_k V_IJ[wp + 8 r][k] x_J[k]   (x complex, V real)
__device__ __forceinline__ void block_fma(const double (*Vs)[VB + 1], const double2 (*Xs)[VB + 1],
                                          int wp, int lane, double2* acc) {
#pragma unroll 8
  for (int k = 0; k < VB; ++k) {
    const double2 x = Xs[k][lane];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double v = Vs[wp + 8 * r][k];
      acc[r].x = fma(v, x.x, acc[r].x);
      acc[r].y = fma(v, x.y, acc[r].y);
    }
  }
}

__global__ void __launch_bounds__(VT) k_exchange_v(int W, long NM, int ex_groups, ExSpin sa,
                                                   ExSpin sb, const double2* __restrict__ thetaT,
                                                   double2* __restrict__ ekp) {
  __shared__ double Vs[VB][VB + 1];
  __shared__ double2 Xs[VB][VB + 1];
  __shared__ double2 red[VT / 32][VB];
  const int spin = blockIdx.z;
  const ExSpin sp = spin ? sb : sa;
  if (sp.K == 0 || (int)blockIdx.x >= sp.npairs * sp.S) return;  // uniform per CTA
  const int p = blockIdx.x / sp.S, s = blockIdx.x % sp.S;
  const int z0 = blockIdx.y * VB;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int I1 = p, I2 = sp.nbk - 1 - p;
  const int len1 = sp.nbk - I1, len2 = I2 > I1 ? sp.nbk - I2 : 0;
  const int beg = s * sp.C, end = min(beg + sp.C, len1 + len2);
  double2 part = cmk(0.0, 0.0);
  for (int seg = 0; seg < 2; ++seg) {
    // positions pos in [lo, hi) of row I's list stand for the blocks J = I + pos
    const int I = seg ? I2 : I1;
    const int lo = seg ? max(beg, len1) - len1 : beg;
    const int hi = seg ? end - len1 : min(end, len1);
    if (hi <= lo) continue;
    double2 acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = cmk(0.0, 0.0);
    for (int pos = max(lo, 1); pos < hi; ++pos) {  // blocks above the diagonal
      __syncthreads();
      load_v(sp, I, I + pos, Vs);
      load_x(sp, thetaT, NM, W, z0, I + pos, Xs);
      __syncthreads();
      block_fma(Vs, Xs, wp, lane, acc);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = cscale(acc[r], 2.0);
    __syncthreads();
    load_x(sp, thetaT, NM, W, z0, I, Xs);  // x_I: the diagonal block's operand and the dot
    if (lo == 0) load_v(sp, I, I, Vs);
    __syncthreads();
    if (lo == 0) block_fma(Vs, Xs, wp, lane, acc);
#pragma unroll
    for (int r = 0; r < 4; ++r) part = cfma(Xs[wp + 8 * r][lane], acc[r], part);
  }
  red[wp][lane] = part;
  __syncthreads();
  if (wp == 0) {
    double2 t = red[0][lane];
#pragma unroll
    for (int w = 1; w < VT / 32; ++w) t = cadd(t, red[w][lane]);
    const int z = z0 + lane;
    if (z < W) ekp[((long)z * 2 + spin) * ex_groups + blockIdx.x] = cscale(t, -0.5);
  }
}

ExSpin spin_geometry(const afq_ctx* ctx, int spin) {
  ExSpin sp{};
  const int n = spin ? ctx->nb : ctx->na;
  const long Ka = (long)ctx->na * ctx->M;
  sp.K = n * ctx->M;
  sp.V = ctx->Vx ? ctx->Vx + (spin ? Ka * Ka : 0) : nullptr;
  sp.offe = spin ? Ka : 0;
  sp.nbk = (sp.K + VB - 1) / VB;
  sp.npairs = (sp.nbk + 1) / 2;
  return sp;
}

}  // namespace

// Largest number of exchange slots one walker and spin can take:
// npairs * min(nbk + 1, kMaxChunks).
int exchange_v_slots(const afq_ctx* ctx) {
  int slots = 0;
  for (int s = 0; s < 2; ++s) {
    const ExSpin sp = spin_geometry(ctx, s);
    const int smax = sp.nbk + 1 < kMaxChunks ? sp.nbk + 1 : kMaxChunks;
    if (sp.npairs * smax > slots) slots = sp.npairs * smax;
  }
  return slots;
}

// V_s[(j,p),(i,q)] = sum_g L~_g,s[j][q] L~_g,s[i][p] for both spins, once per trial:
// for each j one GEMM batched over i gives the M x M block (p, q) = A_i^T A_j, with
// A_i the X x M matrix L~_g,s[i][.] over g.
int build_exchange_v(afq_ctx* ctx) {
  if (ctx->Vx) return AFQ_OK;
  const int M = ctx->M, N = ctx->N, X = ctx->X;
  const long NM = (long)N * M;
  const long nMa = (long)ctx->na * M, nMb = (long)ctx->nb * M;
  if (cudaMalloc((void**)&ctx->Vx, (size_t)(nMa * nMa + nMb * nMb) * sizeof(double)) !=
      cudaSuccess) {
    ctx->Vx = nullptr;
    cudaGetLastError();
    return afq_fail(ctx, AFQ_ERR_NOMEM, "half-rotated exchange tensor");
  }
  for (int s = 0; s < 2; ++s) {
    const int n = s ? ctx->nb : ctx->na, off = s ? ctx->na : 0;
    const long nM = (long)n * M;
    double* V = ctx->Vx + (s ? nMa * nMa : 0);
    for (int j = 0; j < n; ++j)
      AFQ_TRY(launch_dgemm(ctx, M, M, X, 1.0, ctx->Lt + (long)off * M, 1, NM, M,
                           ctx->Lt + (long)(off + j) * M, NM, 1, 0, 0.0, V + j * M * nM, nM, 1,
                           M, n, 1));
  }
  return AFQ_OK;
}

int launch_exchange_v(afq_ctx* ctx, WalkerSet& s) {
  if (!ctx->Vx) return afq_fail(ctx, AFQ_ERR_STATE, "half-rotated exchange tensor not built");
  const int nzb = (s.W + VB - 1) / VB;
  ExSpin sp[2];
  int items = 0;
  for (int spin = 0; spin < 2; ++spin) {
    ExSpin& e = sp[spin];
    e = spin_geometry(ctx, spin);
    if (e.K == 0) {
      e.S = e.C = 1;
      continue;
    }
    const int L = e.nbk + 1;  // blocks per pair of block rows
    int S = (kCtaTarget + 2 * e.npairs * nzb - 1) / (2 * e.npairs * nzb);
    const int scap = ctx->ex_groups / e.npairs;
    if (S > L) S = L;
    if (S > scap) S = scap;
    if (S < 1) S = 1;
    e.C = (L + S - 1) / S;
    e.S = (L + e.C - 1) / e.C;
    if (e.npairs * e.S > ctx->ex_groups)
      return afq_fail(ctx, AFQ_ERR_STATE, "exchange chunks exceed slots");
    if (e.npairs * e.S > items) items = e.npairs * e.S;
  }
  if (items == 0) return AFQ_OK;
  k_exchange_v<<<dim3(items, nzb, 2), VT, 0, ctx->stream>>>(s.W, (long)ctx->N * ctx->M,
                                                           ctx->ex_groups, sp[0], sp[1], s.thetaT,
                                                           s.ekp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
