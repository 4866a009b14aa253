// Split-precision tensor-core contractions of the walker's Green's-function
// intermediates (precision AFQ_SPLIT_BF16): the force bias / Coulomb vector of
// Eq. rfb and the exchange term of Sec. "Local energy", plus a plain GEMM entry
// point that exercises the same engine (tc_engine.cuh).
#include <cstdio>

#include "tc_engine.cuh"

using namespace tce;

namespace {

// ---------------------------------------------------------------------------
// Policy: plain GEMM C (m x n, FP64) = A (m x K) B (n x K)^T from slice planes
// [s][rows][Kp] (3D tensor maps {Kp, rows, S}).
// ---------------------------------------------------------------------------
struct GemmP {
  struct Args {
    TcCommon c;
    int m, n;
    double* C;
    long ldc;
  };
  static constexpr int kUA = 1, kUB = 1;
  template <int S>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    issue_pairs<S>(tmem, sa, sb, bslot, 0, 0, tc::idesc_bf16(128, a.c.BN), first);
  }
  struct Tile {
    int m0, n0, kb0, kb1;
  };
  static __device__ Tile tile(const Args& a) {
    return Tile{(int)blockIdx.y * 128, (int)blockIdx.x * a.c.BN, 0, a.c.nkb};
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.m0, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.n0, s, bar);
  }
  template <int S>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const int row = t.m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < a.c.BN; c0 += 16) {
      float v[16];
      tmem_row16(tmem, warp, c0, v);
      if (row < a.m)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = t.n0 + c0 + j;
          if (col < a.n) a.C[(long)row * a.ldc + col] = v[j];
        }
    }
  }
};

// ---------------------------------------------------------------------------
// Policy: force bias / Coulomb vector, split over K.  Rows g of L~ (K = N Mpad),
// columns (z, re/im) of theta, both as exact integer digits (a power-of-two scale per
// row g and per column); every digit order accumulates in its own TMEM region, where
// the integer sums are exact in FP32, so the result carries only the digits' own
// rounding (the tensor core's FP32 accumulation of float slices is biased and its
// error grew with K).  Partial sums part[ks][col][g] in FP64 (g contiguous).
// ---------------------------------------------------------------------------
struct FbP {
  struct Args {
    TcCommon c;
    int X, W2, kbper;
    const int* ea;  // row exponents of L~ (X)
    const int* eb;  // exponents of theta per column (z, re/im) (W2)
    double* part;
  };
  static constexpr int kUA = 1, kUB = 1;
  template <int S>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    issue_split<S>(a.c, tmem, sa, sb, bslot, first);
  }
  struct Tile {
    int g0, n0, ks, kb0, kb1;
  };
  static __device__ Tile tile(const Args& a) {
    const int ks = blockIdx.z;
    const int kb0 = ks * a.kbper;
    const int kb1 = min(a.c.nkb, kb0 + a.kbper);
    return Tile{(int)blockIdx.y * 128, (int)blockIdx.x * a.c.BN, ks, kb0, kb1};
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.g0, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.n0, s, bar);
  }
  template <int S>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const int g = t.g0 + warp * 32 + lane;
    const bool valid = g < a.X;
    const int eg = valid ? a.ea[g] : 0;
    double* out = a.part + (long)t.ks * a.W2 * a.X;
    for (int c0 = 0; c0 < a.c.BN; c0 += 16) {
      float f[S][16];
#pragma unroll
      for (int d = 0; d < S; ++d) tmem_row16(tmem + (uint32_t)(d * a.c.BN), warp, c0, f[d]);
      if (!valid) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = t.n0 + c0 + j;
        if (col >= a.W2) continue;
        float acc[S];
#pragma unroll
        for (int d = 0; d < S; ++d) acc[d] = f[d][j];
        out[(long)col * a.X + g] = combine_exact<S>(acc, eg + a.eb[col] - 14);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// slicing kernels: FP64 -> S bfloat16 planes
// ---------------------------------------------------------------------------
// in: rows x K (row pitch ld); out: S planes of rows x Kp, zero for k >= K
__global__ void k_slice_real(const double* __restrict__ in, long ld, long rows, int K, int Kp,
                             int S, __nv_bfloat16* __restrict__ out) {
  const long total = rows * Kp, plane = rows * Kp;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long r = e / Kp;
    const int k = (int)(e % Kp);
    split_bf16(k < K ? in[r * ld + k] : 0.0, S, out + e, plane);
  }
}

// Rows of K doubles (row pitch ld) -> S planes of scaled digits (split_scaled) of
// rows x Kp, zero for k >= K, with one exponent per row (one warp per row); for the
// direct exchange, which takes at most 4 digits
__global__ void k_slice_rows_scaled(const double* __restrict__ in, long ld, long rows, int K,
                                    int Kp, int S, __nv_bfloat16* __restrict__ out) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = rows * Kp;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const double* row = in + r * ld;
    int m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, exp_field(row[k]));
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    for (int k = lane; k < Kp; k += 32)
      split_scaled<kFastSlices>(k < K ? row[k] : 0.0, e, S, out + r * Kp + k, plane);
  }
}

// thetaT W x N x M complex -> S planes of scaled digits [z][re/im][j][Mpad], with the
// exponents eb of the exact digits (one per walker and re/im)
__global__ void k_slice_theta_scaled(const double2* __restrict__ thetaT, int W, int N, int M,
                                     int Mpad, int S, const int* __restrict__ eb,
                                     __nv_bfloat16* __restrict__ out) {
  const long NMp = (long)N * Mpad, total = (long)W * NMp, plane = 2 * total;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long z = e / NMp, r = e % NMp;
    const int j = (int)(r / Mpad), p = (int)(r % Mpad);
    const double2 v = p < M ? thetaT[(z * N + j) * M + p] : make_double2(0.0, 0.0);
    __nv_bfloat16* o = out + (2 * z) * NMp + r;
    split_scaled<kFastSlices>(v.x, eb[2 * z], S, o, plane);
    split_scaled<kFastSlices>(v.y, eb[2 * z + 1], S, o + NMp, plane);
  }
}

// c_zg = sum_ks part[ks][2z + re/im][g] in FP64 (fixed order)
__global__ void k_fb_reduce(int X, int W, int ksplit, const double* __restrict__ part,
                            double2* __restrict__ c) {
  const long total = (long)W * X;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int z = (int)(e / X), g = (int)(e % X);
    double re = 0.0, im = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) {
      re += part[((long)ks * 2 * W + 2 * z) * X + g];
      im += part[((long)ks * 2 * W + 2 * z + 1) * X + g];
    }
    c[e] = make_double2(re, im);
  }
}

__device__ __forceinline__ int warp_max_e(int v) { return __reduce_max_sync(0xffffffffu, v); }

// L~ (X rows of N x M) -> integer digit planes [s][g][N Mpad] with one exponent per g
// (one warp per row; zero padding)
__global__ void k_slice_lt_exact(const double* __restrict__ Lt, int X, int N, int M, int Mpad,
                                 int S, __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long NM = (long)N * M, NMp = (long)N * Mpad, plane = (long)X * NMp;
  for (long g = (long)blockIdx.x * warps + (threadIdx.x >> 5); g < X;
       g += (long)gridDim.x * warps) {
    const double* row = Lt + g * NM;
    int m = 0;
    for (long e = lane; e < NM; e += 32) m = max(m, exp_field(row[e]));
    const int ex = row_exponent_field(warp_max_e(m));
    if (lane == 0) eout[g] = ex;
    for (long e = lane; e < NMp; e += 32) {
      const int j = (int)(e / Mpad), p = (int)(e % Mpad);
      split_exact(p < M ? row[(long)j * M + p] : 0.0, ex, S, out + g * NMp + e, plane);
    }
  }
}

// Exponents of theta^T per (z, re/im) over both spins: one block per walker, the
// walker's N x M complex values read once, coalesced.
__global__ void __launch_bounds__(256) k_theta_exponents(const double2* __restrict__ thetaT,
                                                         long NM, int* __restrict__ eb) {
  __shared__ int red[2][8];
  const long z = blockIdx.x;
  const double2* th = thetaT + z * NM;
  int mr = 0, mi = 0;
  for (long e = threadIdx.x; e < NM; e += 256) {
    const double2 v = th[e];
    mr = max(mr, exp_field(v.x));
    mi = max(mi, exp_field(v.y));
  }
  mr = warp_max_e(mr);
  mi = warp_max_e(mi);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mr;
    red[1][threadIdx.x >> 5] = mi;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    int m = 0;
    for (int w = 0; w < 8; ++w) m = max(m, red[threadIdx.x][w]);
    eb[2 * z + threadIdx.x] = row_exponent_field(m);
  }
}

// theta^T (W x N x M complex) -> integer digit planes [s][z][re/im][N Mpad] with the
// exponents above (zero padding); one thread per pair of consecutive elements
// (z, j, p, p + 1 < Mpad; Mpad is even), written as bfloat16 pairs; D >= S
template <int D>
__global__ void k_slice_theta_exact(const double2* __restrict__ thetaT, int W, int N, int M,
                                    int Mpad, int S, const int* __restrict__ eb,
                                    __nv_bfloat16* __restrict__ out) {
  const long NMp = (long)N * Mpad, total = (long)W * NMp, plane = 2 * total;
  for (long e2 = blockIdx.x * (long)blockDim.x + threadIdx.x; e2 < total / 2;
       e2 += (long)gridDim.x * blockDim.x) {
    const long e = 2 * e2, z = e / NMp, r = e % NMp;
    const int j = (int)(r / Mpad), p = (int)(r % Mpad);
    const double2* src = thetaT + (z * N + j) * M + p;
    const double2 v0 = p < M ? src[0] : make_double2(0.0, 0.0);
    const double2 v1 = p + 1 < M ? src[1] : make_double2(0.0, 0.0);
    const int er = eb[2 * z], ei = eb[2 * z + 1];
    float a0[D], a1[D], b0[D], b1[D];
    exact_digits_f<D>(v0.x, er, S, a0);
    exact_digits_f<D>(v1.x, er, S, a1);
    exact_digits_f<D>(v0.y, ei, S, b0);
    exact_digits_f<D>(v1.y, ei, S, b1);
    __nv_bfloat16* o = out + (2 * z) * NMp + r;
#pragma unroll
    for (int s = 0; s < D; ++s)
      if (s < S) {
        *reinterpret_cast<__nv_bfloat162*>(o + s * plane) = digit_bf16x2(a0[s], a1[s]);
        *reinterpret_cast<__nv_bfloat162*>(o + NMp + s * plane) = digit_bf16x2(b0[s], b1[s]);
      }
  }
}

constexpr int kFbKbExact = 32;  // K blocks per force-bias split beyond 4 digits

int warp_grid_rows(long rows) {
  const long b = (rows + 7) / 8;  // 8 warps per 256-thread block
  return (int)(b < 1 ? 1 : (b > 148 * 64 ? 148 * 64 : b));
}

}  // namespace

// ===========================================================================
// context integration
// ===========================================================================
// Walkers per exchange tile for one spin: the MMA width and the theta tensor map.
bool set_exchange_zb(afq_ctx* ctx, int spin, int zb) {
  const int n = spin ? ctx->nb : ctx->na;
  ctx->ex_zb[spin] = zb;
  ctx->ex_BN[spin] = round_up(2 * n * zb, 16);
  const uint64_t db[4] = {(uint64_t)ctx->Mpad, (uint64_t)ctx->N, (uint64_t)(2 * ctx->ws.W),
                          (uint64_t)ctx->S};
  const uint32_t bb[4] = {kBK, (uint32_t)n, (uint32_t)(2 * zb), 1};
  return make_tmap(&ctx->tm_ex_b[spin], ctx->th_sl, 4, db, bb);
}

// Tile of the direct exchange for n electrons: G Cholesky indices of n rows each (128
// rows), zb walkers of 2n columns; the head and tail accumulators of two tiles in
// flight take 4 BN-wide regions of the 512 TMEM columns, so BN <= 128.
int mixed_exchange_tiles(int n, int* G, int* zb, int* BN) {
  if (n <= 0) return 0;
  *G = 128 / n;
  *zb = 128 / (2 * n);
  if (*zb < 1) *zb = 1;
  *BN = round_up(2 * n * *zb, 16);
  while (*BN > 128 && *zb > 1) {
    *zb -= 1;
    *BN = round_up(2 * n * *zb, 16);
  }
  return 1;
}

void mixed_free(afq_ctx* ctx) {
  mixed_prop_free(ctx);
  overlap_tc_free(ctx);
  if (ctx->Lt_sl) cudaFree(ctx->Lt_sl);
  if (ctx->th_sl) cudaFree(ctx->th_sl);
  if (ctx->fb_part) cudaFree(ctx->fb_part);
  for (void* p : {(void*)ctx->Vsl, (void*)ctx->exv_ea, (void*)ctx->exv_th, (void*)ctx->exv_eb,
                  (void*)ctx->exv_y, (void*)ctx->Lt_ex, (void*)ctx->e_fb})
    if (p) cudaFree(p);
  ctx->Lt_sl = nullptr;
  ctx->th_sl = nullptr;
  ctx->fb_part = nullptr;
  ctx->Lt_ex = nullptr;
  ctx->e_fb = nullptr;
  ctx->Vsl = nullptr;
  ctx->exv_ea = nullptr;
  ctx->exv_th = nullptr;
  ctx->exv_eb = nullptr;
  ctx->exv_y = nullptr;
}

// Slices L~ once per trial: integer digits with one exponent per g for the force bias,
// and scaled digits with one exponent per row (g, j) for the direct exchange when it
// is the chosen exchange; S planes of [g][j][Mpad] each.
int mixed_init_trial(afq_ctx* ctx) {
  const int S = ctx->S, X = ctx->X, N = ctx->N, M = ctx->M;
  ctx->Mpad = round_up(M, kBK);
  const size_t plane = (size_t)X * N * ctx->Mpad;
  for (void* p : {(void*)ctx->Lt_sl, (void*)ctx->Lt_ex, (void*)ctx->e_fb})
    if (p) cudaFree(p);
  ctx->Lt_sl = nullptr;
  ctx->Lt_ex = nullptr;
  ctx->e_fb = nullptr;
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->Lt_ex, plane * S * sizeof(__nv_bfloat16)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_fb, (size_t)X * sizeof(int)));
  k_slice_lt_exact<<<warp_grid_rows(X), 256, 0, ctx->stream>>>(ctx->Lt, X, N, M, ctx->Mpad, S,
                                                               ctx->Lt_ex, ctx->e_fb);
  AFQ_LAUNCHED(ctx);
  AFQ_TRY(overlap_tc_init_trial(ctx));
  if (!ctx->ex_stored) {
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->Lt_sl, plane * S * sizeof(__nv_bfloat16)));
    k_slice_rows_scaled<<<warp_grid_rows((long)X * N), 256, 0, ctx->stream>>>(
        ctx->Lt, M, (long)X * N, M, ctx->Mpad, S, ctx->Lt_sl);
    AFQ_LAUNCHED(ctx);
  }
  return AFQ_OK;
}

// Per walker set: theta slices, force-bias partials and all tensor maps.
int mixed_init_walkers(afq_ctx* ctx) {
  const int S = ctx->S, X = ctx->X, N = ctx->N, W = ctx->ws.W, Mp = ctx->Mpad;
  for (void* p : {(void*)ctx->th_sl, (void*)ctx->fb_part, (void*)ctx->exv_th, (void*)ctx->exv_eb})
    if (p) cudaFree(p);
  ctx->th_sl = nullptr;
  ctx->fb_part = nullptr;
  ctx->exv_th = nullptr;
  ctx->exv_eb = nullptr;
  const int W2 = 2 * W;
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->exv_th, (size_t)S * W2 * N * Mp * sizeof(__nv_bfloat16)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->exv_eb, (size_t)W2 * sizeof(int)));
  if (!ctx->Vsl)  // scaled digits of theta for the direct exchange
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_sl,
                             (size_t)S * W * 2 * N * Mp * sizeof(__nv_bfloat16)));
  // force bias: rows g (X), columns (z, re/im) (2W), K = N Mpad; S digit accumulators
  // of BN columns fit the 512 TMEM columns
  ctx->fb_BN = pick_bn(W2, S, 256);
  const int nkb = N * Mp / kBK;
  const int tiles = ((X + 127) / 128) * ((W2 + ctx->fb_BN - 1) / ctx->fb_BN);
  int ks = (296 + tiles - 1) / tiles;
  // beyond 4 digits (FP64 quality) each split covers at most 32 K blocks, K = 1024: the
  // leading digit products' sum, at most 128^2 K = 2^24, stays exact in FP32
  if (S > 4 && ks < (nkb + kFbKbExact - 1) / kFbKbExact) ks = (nkb + kFbKbExact - 1) / kFbKbExact;
  if (ks > nkb) ks = nkb;
  if (ks < 1) ks = 1;
  ctx->fb_kbper = (nkb + ks - 1) / ks;
  ctx->fb_ksplit = (nkb + ctx->fb_kbper - 1) / ctx->fb_kbper;
  ctx->fb_ksplit_cap = 4 * ctx->fb_ksplit;  // the autotuner may deepen the split
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->fb_part,
                           (size_t)ctx->fb_ksplit_cap * W2 * X * sizeof(double)));
  {
    const uint64_t da[3] = {(uint64_t)N * Mp, (uint64_t)X, (uint64_t)S};
    const uint32_t ba[3] = {kBK, 128, 1};
    const uint64_t db[3] = {(uint64_t)N * Mp, (uint64_t)W2, (uint64_t)S};
    const uint32_t bb[3] = {kBK, (uint32_t)ctx->fb_BN, 1};
    if (!make_tmap(&ctx->tm_fb_a, ctx->Lt_ex, 3, da, ba) ||
        !make_tmap(&ctx->tm_fb_b, ctx->exv_th, 3, db, bb))
      return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (force bias) failed");
  }
  // direct exchange: per spin
  for (int s = 0; s < 2 && !ctx->Vsl; ++s) {
    const int n = s ? ctx->nb : ctx->na;
    if (!mixed_exchange_tiles(n, &ctx->ex_G[s], &ctx->ex_zb[s], &ctx->ex_BN[s])) continue;
    const uint64_t da[4] = {(uint64_t)Mp, (uint64_t)N, (uint64_t)X, (uint64_t)S};
    const uint32_t ba[4] = {kBK, (uint32_t)n, (uint32_t)ctx->ex_G[s], 1};
    if (!make_tmap(&ctx->tm_ex_a[s], ctx->Lt_sl, 4, da, ba) || !set_exchange_zb(ctx, s, ctx->ex_zb[s]))
      return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (exchange) failed");
  }
  if (ctx->Vsl) AFQ_TRY(mixed_exchange_v_walkers(ctx));
  AFQ_TRY(overlap_tc_init_walkers(ctx));
  return AFQ_OK;
}

// Tunable tiles of the split-precision energy contractions: walkers per exchange
// tile (per spin) and the split-K depth of the force bias, timed on the walkers.
int mixed_autotune(afq_ctx* ctx) {
  WalkerSet& s = ctx->ws;
  auto timeit = [&](auto&& f) {
    if (f() != AFQ_OK) return 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, ctx->stream);
    int rc = AFQ_OK;
    for (int r = 0; r < 3 && rc == AFQ_OK; ++r) rc = f();
    cudaEventRecord(b, ctx->stream);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc == AFQ_OK ? ms / 3 : 1e30f;
  };
  for (int spin = 0; spin < 2 && !ctx->Vsl; ++spin) {  // direct exchange only
    const int n = spin ? ctx->nb : ctx->na;
    if (n == 0) continue;
    const int zbmax = ctx->ex_zb[spin];
    int best_zb = zbmax;
    float best = 1e30f;
    for (int zb : {zbmax, zbmax * 3 / 4, zbmax / 2, zbmax / 3, zbmax / 4}) {
      if (zb < 1 || (zb != zbmax && zb == best_zb)) continue;
      if (!set_exchange_zb(ctx, spin, zb)) return afq_fail(ctx, AFQ_ERR_CUDA, "exchange map");
      const float ms = timeit([&] { return launch_exchange_tc(ctx, s); });
      if (ms < best) {
        best = ms;
        best_zb = zb;
      }
    }
    if (!set_exchange_zb(ctx, spin, best_zb)) return afq_fail(ctx, AFQ_ERR_CUDA, "exchange map");
  }
  // force bias split-K: K blocks per CTA, within the partial-sum buffer's ksplit bound
  const int nkb = ctx->N * ctx->Mpad / kBK;
  const int kb0 = ctx->fb_kbper, cap = ctx->fb_ksplit_cap;
  int best_kb = kb0;
  float best = 1e30f;
  for (int kb : {kb0, kb0 * 2, kb0 * 4, (kb0 + 1) / 2, (kb0 + 3) / 4}) {
    if (kb < 1 || kb > nkb || (ctx->S > 4 && kb > kFbKbExact)) continue;
    const int ks = (nkb + kb - 1) / kb;
    if (ks > cap) continue;
    ctx->fb_kbper = kb;
    ctx->fb_ksplit = ks;
    const float ms = timeit([&] { return launch_force_bias_tc(ctx, s); });
    if (ms < best) {
      best = ms;
      best_kb = kb;
    }
  }
  ctx->fb_kbper = best_kb;
  ctx->fb_ksplit = (nkb + best_kb - 1) / best_kb;
  return AFQ_OK;
}

// theta's integer digits (force bias, stored exchange) and, for the direct exchange,
// its scaled digits (the same exponents)
int launch_slice_theta(afq_ctx* ctx, WalkerSet& s) {
  k_theta_exponents<<<s.W, 256, 0, ctx->stream>>>(s.thetaT, (long)ctx->N * ctx->M, ctx->exv_eb);
  AFQ_LAUNCHED(ctx);
  (ctx->S <= kFastSlices ? k_slice_theta_exact<kFastSlices> : k_slice_theta_exact<kMaxSlices>)
      <<<grid1d((long)s.W * ctx->N * ctx->Mpad / 2), 256, 0, ctx->stream>>>(
          s.thetaT, s.W, ctx->N, ctx->M, ctx->Mpad, ctx->S, ctx->exv_eb, ctx->exv_th);
  AFQ_LAUNCHED(ctx);
  if (ctx->th_sl) {
    const long total = (long)s.W * ctx->N * ctx->Mpad;
    k_slice_theta_scaled<<<grid1d(total), 256, 0, ctx->stream>>>(
        s.thetaT, s.W, ctx->N, ctx->M, ctx->Mpad, ctx->S, ctx->exv_eb, ctx->th_sl);
    AFQ_LAUNCHED(ctx);
  }
  return AFQ_OK;
}

int launch_force_bias_tc(afq_ctx* ctx, WalkerSet& s) {
  FbP::Args a{};
  a.c.nkb = ctx->N * ctx->Mpad / kBK;
  a.c.BN = ctx->fb_BN;
  a.c.tx_bytes = (uint32_t)ctx->S * (kBK * 128 * 2 + kBK * ctx->fb_BN * 2);
  a.c.tmem_cols = tmem_cols_for(ctx->S * ctx->fb_BN);
  a.c.err = ctx->flags + 2;
  a.c.per_pair = ctx->p.prop_kernel == 2;
  a.X = ctx->X;
  a.W2 = 2 * s.W;
  a.kbper = ctx->fb_kbper;
  a.ea = ctx->e_fb;
  a.eb = ctx->exv_eb;
  a.part = ctx->fb_part;
  size_t smem = 0;
  plan_smem(ctx->S, 1, 1, a.c.BN, 0, &a.c.stages, &smem);
  dim3 grid((a.W2 + a.c.BN - 1) / a.c.BN, (ctx->X + 127) / 128, ctx->fb_ksplit);
  cudaError_t e = launch_tc_s<FbP>(ctx->S, grid, smem, ctx->stream, ctx->tm_fb_a, ctx->tm_fb_b, a);
  ctx->launches++;
  if (e != cudaSuccess) return afq_fail(ctx, AFQ_ERR_CUDA, std::string("force bias tc: ") + cudaGetErrorString(e));
  k_fb_reduce<<<grid1d((long)s.W * ctx->X), 256, 0, ctx->stream>>>(ctx->X, s.W, ctx->fb_ksplit,
                                                                   ctx->fb_part, s.c);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// ===========================================================================
// Library GEMM on the same engine (C ABI)
// ===========================================================================
extern "C" int afq_gemm_split_bf16(int m, int n, int k, int slices, const double* A_dev,
                                   const double* B_dev, double* C_dev, void* cuda_stream) {
  if (m < 1 || n < 1 || k < 1 || slices < 1 || slices > 4 || !A_dev || !B_dev || !C_dev)
    return AFQ_ERR_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int Kp = round_up(k, kBK);
  const int BN = n >= 256 ? 256 : round_up(n, 16);
  __nv_bfloat16 *As = nullptr, *Bs = nullptr;
  int* err = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&As, (size_t)slices * m * Kp * 2) != cudaSuccess ||
      cudaMalloc((void**)&Bs, (size_t)slices * n * Kp * 2) != cudaSuccess ||
      cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess)
    rc = AFQ_ERR_NOMEM;
  CUtensorMap ta, tb;
  if (rc == AFQ_OK) {
    k_slice_real<<<grid1d((long)m * Kp), 256, 0, stream>>>(A_dev, k, m, k, Kp, slices, As);
    k_slice_real<<<grid1d((long)n * Kp), 256, 0, stream>>>(B_dev, k, n, k, Kp, slices, Bs);
    const uint64_t da[3] = {(uint64_t)Kp, (uint64_t)m, (uint64_t)slices};
    const uint32_t ba[3] = {kBK, 128, 1};
    const uint64_t db[3] = {(uint64_t)Kp, (uint64_t)n, (uint64_t)slices};
    const uint32_t bb[3] = {kBK, (uint32_t)BN, 1};
    if (!make_tmap(&ta, As, 3, da, ba) || !make_tmap(&tb, Bs, 3, db, bb)) rc = AFQ_ERR_CUDA;
  }
  if (rc == AFQ_OK) {
    GemmP::Args a{};
    a.c.nkb = Kp / kBK;
    a.c.BN = BN;
    a.c.tx_bytes = (uint32_t)slices * (kBK * 128 * 2 + kBK * BN * 2);
    a.c.tmem_cols = tmem_cols_for(BN);
    a.c.err = err;
    size_t smem = 0;
    plan_smem(slices, 1, 1, BN, 0, &a.c.stages, &smem);
    a.m = m;
    a.n = n;
    a.C = C_dev;
    a.ldc = n;
    dim3 grid((n + BN - 1) / BN, (m + 127) / 128);
    if (launch_tc_s<GemmP>(slices, grid, smem, stream, ta, tb, a) != cudaSuccess)
      rc = AFQ_ERR_CUDA;
  }
  int herr = 0;
  if (cudaStreamSynchronize(stream) != cudaSuccess) rc = AFQ_ERR_CUDA;
  if (err && cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && herr)
    rc = AFQ_ERR_CUDA;
  cudaFree(As);
  cudaFree(Bs);
  cudaFree(err);
  return rc;
}
