// The overlap matrices S_z,s = Psi_s^T Phi_z,s (Sec. "Overlap") of a split-precision
// walker set on the tensor cores, to FP64 quality.
//
// Overlaps, determinants and inverses stay FP64 in split precision; here only the
// product S, which the overlap kernel otherwise forms with the FP64 pipe (half of
// that kernel's time at 290 orbitals), runs as one GEMM on 7 exact digits per operand:
// every row of Psi^T (one per orbital of the trial) and every row (z, j) of Phi^T is
// scaled by a power of two and cut into 7 balanced 8-bit digits (55 bits, more than
// FP64's 53), and the 28 digit products with s + t <= 6 accumulate in 7 TMEM diagonals
// (tc_engine.cuh's exact-diagonal form).  The leading diagonal's sum is bounded by
// 128^2 M < 2^24 for M <= 1024, so it is exact in FP32; the lower diagonals are
// random-sign sums 2^-8 and more below it.  The epilogue recombines the diagonals in
// two int64 halves (d <= 3 and d >= 4, each below 2^53) and adds them in FP64 once,
// so S carries FP64-level rounding, and writes the two diagonal spin blocks per walker.
//
// GEMM: A = Phi^T digits (128-row tiles of the rows (z, re/im, j), K = p), B = Psi^T
// digits (N rows, alpha then beta, in 64-column tiles), D[(z, re/im, j)][i] = S^T;
// the off-diagonal spin blocks are computed and dropped.  The B digit slots lie one
// after another in shared memory, so A digit s times B digits 0 .. 6 - s is one MMA of
// (7 - s) 64 columns (split at 256) into accumulators s .. 6: 10 MMAs per 16-wide K
// step instead of the 28 digit pairs, each reading its A digit once.
#include "tc_engine.cuh"

using namespace tce;

namespace {

constexpr int kOvDigits = 7;
constexpr int kOvBN = 64;  // columns i per tile: 7 accumulators x 64 fit the 512 TMEM columns

// Real rows of K doubles (row pitch ld; rows from rows1 on come from in2) -> S digit
// planes of rows x Kp with one exponent per row (one warp per row).
__global__ void k_slice_rows7(const double* __restrict__ in, const double* __restrict__ in2,
                              long rows1, long ld, long rows, int K, int Kp, int S,
                              __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = rows * Kp;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const double* row = r < rows1 ? in + r * ld : in2 + (r - rows1) * ld;
    int m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, exp_field(row[k]));
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    if (lane == 0) eout[r] = e;
    for (int k = lane; k < Kp; k += 32) {
      float q[kOvDigits];
      exact_digits_f<kOvDigits>(k < K ? row[k] : 0.0, e, S, q);
#pragma unroll
      for (int s = 0; s < kOvDigits; ++s)
        if (s < S) out[s * plane + r * Kp + k] = digit_bf16(q[s]);
    }
  }
}

// Phi (W x M x N complex) -> S digit planes [s][z][re/im][j][Kp] of Phi^T, one exponent
// per complex row (z, j) shared by its real and imaginary parts.  A block takes kPhiJG
// consecutive columns j of one walker: its threads copy those columns of every row p
// (kPhiJG complex, contiguous in Phi) into shared memory once, then warp w cuts column
// j0 + w.  (Read straight from Phi, a column strides N complex per element, so each 16
// bytes cost a 32-byte sector, and it was read twice: for the maximum, for the digits.)
constexpr int kPhiJG = 8;
constexpr int kPhiJGP = kPhiJG + 1;  // tile pitch: a warp's column reads are conflict-free
__global__ void __launch_bounds__(32 * kPhiJG) k_slice_phiT7(const double2* __restrict__ phi,
                                                             int W, int M, int N, int Kp, int S,
                                                             __nv_bfloat16* __restrict__ out,
                                                             int* __restrict__ eout) {
  extern __shared__ __align__(16) unsigned char phraw[];
  double2* tile = reinterpret_cast<double2*>(phraw);  // [p][jj], kPhiJGP apart
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ngrp = (N + kPhiJG - 1) / kPhiJG;
  const long plane = 2L * W * N * Kp, items = (long)W * ngrp;
  for (long it = blockIdx.x; it < items; it += gridDim.x) {  // block-uniform
    const long z = it / ngrp;
    const int j0 = (int)(it - z * ngrp) * kPhiJG;
    const double2* pz = phi + z * (long)M * N + j0;
    __syncthreads();  // the previous item's column reads are done
    for (int e = threadIdx.x; e < M * kPhiJG; e += 32 * kPhiJG) {
      const int p = e / kPhiJG, jj = e - p * kPhiJG;
      tile[p * kPhiJGP + jj] = j0 + jj < N ? pz[(long)p * N + jj] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int j = j0 + w;
    if (j >= N) continue;
    int m = 0;
    for (int p = lane; p < M; p += 32) {
      const double2 v = tile[p * kPhiJGP + w];
      m = max(m, max(exp_field(v.x), exp_field(v.y)));
    }
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    if (lane == 0) eout[z * N + j] = e;
    __nv_bfloat16* ore = out + ((2 * z) * N + j) * (long)Kp;
    __nv_bfloat16* oim = ore + (long)N * Kp;
    for (int p = lane; p < Kp; p += 32) {
      const double2 v = p < M ? tile[p * kPhiJGP + w] : make_double2(0.0, 0.0);
      float qr[kOvDigits], qi[kOvDigits];
      exact_digits_f<kOvDigits>(v.x, e, S, qr);
      exact_digits_f<kOvDigits>(v.y, e, S, qi);
#pragma unroll
      for (int s = 0; s < kOvDigits; ++s)
        if (s < S) {
          ore[s * plane + p] = digit_bf16(qr[s]);
          oim[s * plane + p] = digit_bf16(qi[s]);
        }
    }
  }
}

// value = 2^scale_exp sum_d acc_d 256^-d for 7 diagonals, as two int64 halves
// (d <= 3 and d >= 4, each exact in FP64) added once in FP64.
__device__ __forceinline__ double combine7(const float (&acc)[kOvDigits], int scale_exp) {
  long long hi = 0, lo = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) hi += (long long)__float2int_rn(acc[d]) * (1LL << (8 * (3 - d)));
#pragma unroll
  for (int d = 4; d < kOvDigits; ++d)
    lo += (long long)__float2int_rn(acc[d]) * (1LL << (8 * (6 - d)));
  double h = 0.0, l = 0.0;
  if (hi != 0)
    h = __longlong_as_double(__double_as_longlong(__ll2double_rn(hi)) +
                             ((long long)(scale_exp - 24) << 52));
  if (lo != 0)
    l = __longlong_as_double(__double_as_longlong(__ll2double_rn(lo)) +
                             ((long long)(scale_exp - 48) << 52));
  return h + l;
}

struct OvP {
  struct Args {
    TcCommon c;
    int N, na, nb, nmax;
    long rows_a;        // 2 W N rows (z, re/im, j) of Phi^T
    const int* ea;      // row exponents of Psi^T
    const int* eb;      // exponents of Phi^T per complex row (z, j)
    double2* S;         // W x 2 x nmax x nmax
    double2* H;         // W x 2 x nmax x nmax: h~ Phi (B rows N .. 2N - 1), or unused
  };
  struct Tile {
    int r0, n0, kb0, kb1;
  };
  static constexpr int kUA = 1, kUB = 1;
  template <int SS>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    issue_split<SS>(a.c, tmem, sa, sb, bslot, first);
  }
  // column tiles fastest: the S and H tiles of a row tile run side by side, so the
  // second reads the Phi^T digits from L2
  static __device__ Tile tile(const Args& a) {
    return Tile{(int)blockIdx.y * 128, (int)blockIdx.x * kOvBN, 0, a.c.nkb};
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.r0, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.n0, s, bar);
  }
  template <int SS>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const long row = (long)t.r0 + warp * 32 + lane;  // row of Phi^T: (z, re/im, j)
    const bool valid = row < a.rows_a;
    const int N = a.N;
    const long zp = valid ? row / N : 0;
    const int j = valid ? (int)(row - zp * N) : 0, part = (int)(zp & 1);
    const long z = zp >> 1;
    const int sj = j < a.na ? 0 : 1, oj = sj ? a.na : 0;
    const int ej = valid ? a.eb[z * N + j] : 0;
    double* dst = reinterpret_cast<double*>(a.S + (z * 2 + sj) * (long)a.nmax * a.nmax) + part;
    double* hdst = a.H ? reinterpret_cast<double*>(a.H + (z * 2 + sj) * (long)a.nmax * a.nmax) + part
                       : nullptr;
    for (int c0 = 0; c0 < a.c.BN; c0 += 16) {
      float f[kOvDigits][16];
#pragma unroll
      for (int d = 0; d < kOvDigits; ++d) tmem_row16(tmem + (uint32_t)(d * a.c.BN), warp, c0, f[d]);
      if (!valid) continue;
#pragma unroll
      for (int ii = 0; ii < 16; ++ii) {
        const int ib = t.n0 + c0 + ii;  // B row: orbital i of Psi^T, or of h~ from N on
        const int i = ib < N ? ib : ib - N;
        if (ib >= (a.H ? 2 * N : N) || (i < a.na ? 0 : 1) != sj) continue;
        float acc[kOvDigits];
#pragma unroll
        for (int d = 0; d < kOvDigits; ++d) acc[d] = f[d][ii];
        double* out = ib < N ? dst : hdst;
        out[2 * ((long)(i - oj) * a.nmax + (j - oj))] = combine7(acc, a.ea[ib] + ej - 14);
      }
    }
  }
};

int warp_grid7(long rows) {
  long g = (rows + 7) / 8;
  return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

}  // namespace

// Once per trial: the 7 digits of Psi^T and of h~ (N x M each, rows alpha then beta)
// and their map.
int overlap_tc_init_trial(afq_ctx* ctx) {
  const int N = ctx->N, M = ctx->M, Mpad = ctx->Mpad;
  if (ctx->ov_psi_sl) cudaFree(ctx->ov_psi_sl);
  if (ctx->ov_ea) cudaFree(ctx->ov_ea);
  ctx->ov_psi_sl = nullptr;
  ctx->ov_ea = nullptr;
  // B rows: Psi^T (N), then h~ = Psi^T h1 (N), so that one GEMM also gives h~ Phi, from
  // which E1 = tr(S^-1 h~ Phi) follows when theta itself is formed at 4 digits
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_psi_sl, (size_t)kOvDigits * 2 * N * Mpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_ea, (size_t)2 * N * sizeof(int)));
  k_slice_rows7<<<warp_grid7(2 * N), 256, 0, ctx->stream>>>(ctx->psiT, ctx->ht, N, M, 2 * N, M,
                                                             Mpad, kOvDigits, ctx->ov_psi_sl,
                                                             ctx->ov_ea);
  AFQ_LAUNCHED(ctx);
  const uint64_t da[3] = {(uint64_t)Mpad, (uint64_t)(2 * N), (uint64_t)kOvDigits};
  const uint32_t ba[3] = {kBK, (uint32_t)kOvBN, 1};
  if (!make_tmap(&ctx->tm_ov_a, ctx->ov_psi_sl, 3, da, ba))
    return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (overlap) failed");
  return AFQ_OK;
}

// Per walker set: Phi^T's digit planes, their exponents, the S buffer and the map.
int overlap_tc_init_walkers(afq_ctx* ctx) {
  const int N = ctx->N, W = ctx->ws.W, Mpad = ctx->Mpad;
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  for (void* p : {(void*)ctx->ov_phi_sl, (void*)ctx->ov_eb, (void*)ctx->ov_S, (void*)ctx->ov_H})
    if (p) cudaFree(p);
  ctx->ov_phi_sl = nullptr;
  ctx->ov_eb = nullptr;
  ctx->ov_S = nullptr;
  ctx->ov_H = nullptr;
  const long rows = 2L * W * N;
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_phi_sl, (size_t)kOvDigits * rows * Mpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_eb, (size_t)W * N * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_S, (size_t)W * 2 * nmax * nmax * sizeof(double2)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->ov_H, (size_t)W * 2 * nmax * nmax * sizeof(double2)));
  const uint64_t db[3] = {(uint64_t)Mpad, (uint64_t)rows, (uint64_t)kOvDigits};
  const uint32_t bb[3] = {kBK, 128, 1};
  if (!make_tmap(&ctx->tm_ov_b, ctx->ov_phi_sl, 3, db, bb))
    return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (overlap) failed");
  return theta_tc_init_walkers(ctx);
}

void overlap_tc_free(afq_ctx* ctx) {
  theta_tc_free(ctx);
  for (void* p : {(void*)ctx->ov_psi_sl, (void*)ctx->ov_ea, (void*)ctx->ov_phi_sl,
                  (void*)ctx->ov_eb, (void*)ctx->ov_S, (void*)ctx->ov_H})
    if (p) cudaFree(p);
  ctx->ov_H = nullptr;
  ctx->ov_psi_sl = nullptr;
  ctx->ov_ea = nullptr;
  ctx->ov_phi_sl = nullptr;
  ctx->ov_eb = nullptr;
  ctx->ov_S = nullptr;
}

// S_z,s = Psi_s^T Phi_z,s for the walker set (its digits, then the GEMM) into ctx->ov_S,
// and with the tensor-core theta also H_z,s = h~_s Phi_z,s into ctx->ov_H.
int launch_overlap_s_tc(afq_ctx* ctx, WalkerSet& s) {
  const int N = ctx->N, M = ctx->M, Mpad = ctx->Mpad, W = s.W;
  {
    const size_t smem = (size_t)M * kPhiJGP * sizeof(double2);
    AFQ_CUDA(ctx, raise_smem_limit((const void*)k_slice_phiT7, smem));
    const long items = (long)W * ((N + kPhiJG - 1) / kPhiJG);
    const int grid = (int)(items < 1 ? 1 : items < 148 * 16 ? items : 148 * 16);
    k_slice_phiT7<<<grid, 32 * kPhiJG, smem, ctx->stream>>>(s.phi, W, M, N, Mpad, kOvDigits,
                                                            ctx->ov_phi_sl, ctx->ov_eb);
  }
  AFQ_LAUNCHED(ctx);
  OvP::Args a{};
  a.c.nkb = Mpad / kBK;
  a.c.BN = kOvBN;
  a.c.tx_bytes = (uint32_t)kOvDigits * (kBK * 128 * 2 + kBK * kOvBN * 2);
  a.c.tmem_cols = tmem_cols_for(kOvDigits * kOvBN);
  a.c.err = ctx->flags + 2;
  a.c.per_pair = ctx->p.prop_kernel == 2;
  a.N = N;
  a.na = ctx->na;
  a.nb = ctx->nb;
  a.nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  a.rows_a = 2L * W * N;
  a.ea = ctx->ov_ea;
  a.eb = ctx->ov_eb;
  a.S = ctx->ov_S;
  const bool with_h = ctx->th_sinv != nullptr && &s == &ctx->ws;  // E1 = tr(S^-1 H)
  a.H = with_h ? ctx->ov_H : nullptr;
  size_t smem = 0;
  plan_smem(kOvDigits, 1, 1, kOvBN, 0, &a.c.stages, &smem);
  if (a.c.stages < 1 || smem > kSmemLimit)
    return afq_fail(ctx, AFQ_ERR_ARG, "overlap tile does not fit in shared memory");
  const int brows = with_h ? 2 * N : N;
  dim3 grid((unsigned)((brows + kOvBN - 1) / kOvBN), (unsigned)((a.rows_a + 127) / 128));
  cudaError_t e = launch_tc<kOvDigits, OvP>(grid, smem, ctx->stream, ctx->tm_ov_b, ctx->tm_ov_a, a);
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("overlap tc: ") + cudaGetErrorString(e));
  return AFQ_OK;
}
