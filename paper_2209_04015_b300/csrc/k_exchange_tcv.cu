// Split-precision exchange from the stored half-rotated tensor (AFQ_SPLIT_BF16 with
// the stored exchange): E_K = -1/2 sum_s x_s^T V_s x_s (Sec. "Local energy" summed
// over g first; see k_exchange_v.cu for the identity), x_s = theta^T_s per walker.
//
// y = V' x runs on the tensor cores as one GEMM per spin (the k_tc_split engine):
// rows of V' (128 per tile) against the walkers' theta (columns (z, re/im)).
// V' holds V in the padded (j, p) layout with its blocks above the 128 x 128
// diagonal doubled and those below unused, so row tile I reads only the K blocks
// from its own diagonal on: x^T V x = sum_I x_I^T (V_II x_I + 2 sum_{J>I} V_IJ x_J),
// half the products of a full GEMM.
//
// K = n Mpad is long (8320 at 290 orbitals and 26 electrons), and the tensor core's
// FP32 accumulation is biased: measured on float slices its error grew with K to
// 3e-5 of E_K.  Both operands are therefore cut into exact integer digits (8 bits
// each, a power-of-two scale per row of V' and per (walker, re/im) of theta),
// every digit order accumulates in its own TMEM region, and the integer sums stay
// exact in FP32 (they stay far below 2^24 for these magnitudes); the epilogue
// recombines them in FP64 and a small FP64 kernel forms x^T y per walker.
#include "tc_engine.cuh"

using namespace tce;

namespace {

// Both spins in one GEMM: A stacks the rows of V'_alpha (padded to whole 128-row
// tiles, Ra rows) and of V'_beta, pitch C = max(Ka, Kb); a row tile knows its spin.
struct ExVGeom {
  int Ka, Kb, Ra, C, nrt_a, nrt_b, kb_off_b;  // kb_off_b: beta's first K block in theta
};

struct ExVP {
  struct Args {
    TcCommon c;
    ExVGeom g;
    int W2;
    const int* ea;  // row exponents of the stacked V' (Ra + Kb)
    const int* eb;  // exponents of theta per column (z, re/im) (W2)
    double* y;      // y^T per spin: alpha W2 x Ka, then beta W2 x Kb
  };
  static constexpr int kUA = 1, kUB = 1;
  template <int S>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    issue_split<S>(a.c, tmem, sa, sb, bslot, first);
  }
  struct Tile {
    int r0, n0, kb0, kb1;  // r0: first row in the stacked V'; K blocks from the diagonal
    int spin, rl0, K, kb_off;
  };
  static __device__ Tile tile(const Args& a) {
    const int I = blockIdx.y;
    const bool b = I >= a.g.nrt_a;
    const int Il = b ? I - a.g.nrt_a : I;
    const int K = b ? a.g.Kb : a.g.Ka;
    Tile t;
    t.spin = b ? 1 : 0;
    t.rl0 = Il * 128;
    t.r0 = (b ? a.g.Ra : 0) + t.rl0;
    t.n0 = (int)blockIdx.x * a.c.BN;
    t.kb0 = Il * (128 / kBK);
    t.kb1 = K / kBK;
    t.K = K;
    t.kb_off = b ? a.g.kb_off_b : 0;
    return t;
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.r0, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, (t.kb_off + kb) * kBK, t.n0, s, bar);
  }
  template <int S>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const int rl = t.rl0 + warp * 32 + lane;  // row within the spin
    const bool valid = rl < t.K;
    const int er = valid ? a.ea[t.r0 + warp * 32 + lane] : 0;
    double* y = a.y + (t.spin ? (long)a.W2 * a.g.Ka : 0);
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
        y[(long)col * t.K + rl] = combine_exact<S>(acc, er + a.eb[col] - 14);
      }
    }
  }
};

__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

// Entry (r, k) of V'_s (Kp x Kp, Kp = n Mpad) from V_s (K x K over (j, p), K = n M):
// w V[(j,p)][(i,q)] with r = j Mpad + p, k = i Mpad + q, zero on the padding,
// w = 2 above the 128 x 128 diagonal blocks, 1 on them, 0 below.
__device__ __forceinline__ double v_prime(const double* __restrict__ V, int M, int Mpad, long K,
                                          long r, long k) {
  const int j = (int)(r / Mpad), p = (int)(r % Mpad), i = (int)(k / Mpad), q = (int)(k % Mpad);
  const long tr = r / 128, tk = k / 128;
  if (p >= M || q >= M || tk < tr) return 0.0;
  const double v = V[((long)j * M + p) * K + (long)i * M + q];
  return tk > tr ? 2.0 * v : v;
}

// One warp per row of the stacked V' (Ra + Kb rows, pitch C): the row exponent, then
// the S integer digit planes (zero beyond the spin's K and on alpha's padding rows).
__global__ void k_slice_v_exact(const double* __restrict__ Va, const double* __restrict__ Vb,
                                int na, int nb, int M, int Mpad, ExVGeom g, int S,
                                __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const long R = (long)g.Ra + g.Kb, C = g.C, plane = R * C;
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < R;
       r += (long)gridDim.x * warps) {
    const bool b = r >= g.Ra;
    const long rl = b ? r - g.Ra : r;
    const long Kp = b ? g.Kb : g.Ka, K = (long)(b ? nb : na) * M;
    const double* V = b ? Vb : Va;
    const bool live = rl < Kp;
    int m = 0;
    for (long k = lane; k < Kp && live; k += 32)
      m = max(m, exp_field(v_prime(V, M, Mpad, K, rl, k)));
    const int e = row_exponent_field(warp_max(m));
    if (lane == 0) eout[r] = e;
    for (long k = lane; k < C; k += 32)
      split_exact(live && k < Kp ? v_prime(V, M, Mpad, K, rl, k) : 0.0, e, S, out + r * C + k,
                  plane);
  }
}

// ekp[z][spin][0] = -1/2 sum_rows x[row] y[row] (complex, FP64), x = theta^T_s,z;
// blockIdx.y = spin
__global__ void __launch_bounds__(256) k_exv_dot(int Ka, int Kb, int na, int nb, int M, int Mpad,
                                                 long NM, int W2, const double* __restrict__ y,
                                                 const double2* __restrict__ thetaT,
                                                 int ex_groups, double2* __restrict__ ekp) {
  __shared__ double2 red[8];
  const int z = blockIdx.x, spin = blockIdx.y;
  const int Kp = spin ? Kb : Ka;
  if ((spin ? nb : na) == 0) return;
  const long offM = (long)(spin ? na : 0) * M;
  const double* yr = y + (spin ? (long)W2 * Ka : 0) + (long)(2 * z) * Kp;
  const double* yi = yr + Kp;
  double2 acc = make_double2(0.0, 0.0);
  // four consecutive elements of one row per thread (Mpad is a multiple of 32), their
  // loads issued together ahead of the multiply-adds
  for (int r0 = 4 * threadIdx.x; r0 < Kp; r0 += 4 * 256) {
    const int j = r0 / Mpad, p0 = r0 - j * Mpad;
    const double2* th = thetaT + (long)z * NM + offM + (long)j * M + p0;
    double2 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = p0 + u < M ? th[u] : make_double2(0.0, 0.0);
    const double2 a01 = *reinterpret_cast<const double2*>(yr + r0);
    const double2 a23 = *reinterpret_cast<const double2*>(yr + r0 + 2);
    const double2 b01 = *reinterpret_cast<const double2*>(yi + r0);
    const double2 b23 = *reinterpret_cast<const double2*>(yi + r0 + 2);
    const double av[4] = {a01.x, a01.y, a23.x, a23.y}, bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc.x = fma(x[u].x, av[u], fma(-x[u].y, bv[u], acc.x));
      acc.y = fma(x[u].x, bv[u], fma(x[u].y, av[u], acc.y));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = red[0];
    for (int w = 1; w < 8; ++w) t = make_double2(t.x + red[w].x, t.y + red[w].y);
    ekp[((long)z * 2 + spin) * ex_groups] = make_double2(-0.5 * t.x, -0.5 * t.y);
  }
}

ExVGeom geometry(const afq_ctx* ctx, int Mpad) {
  ExVGeom g{};
  g.Ka = ctx->na * Mpad;
  g.Kb = ctx->nb * Mpad;
  g.Ra = round_up(g.Ka, 128);
  g.C = g.Ka > g.Kb ? g.Ka : g.Kb;
  g.nrt_a = g.Ra / 128;
  g.nrt_b = (g.Kb + 127) / 128;
  g.kb_off_b = ctx->na * Mpad / kBK;
  return g;
}

int warp_blocks(long rows) {
  const long b = (rows + 7) / 8;  // 8 warps per 256-thread block
  return (int)(b < 1 ? 1 : (b > 148 * 64 ? 148 * 64 : b));
}

}  // namespace

// Bytes of the digit planes of the stacked V' (S planes) and their row exponents.
double exchange_tcv_bytes(const afq_ctx* ctx, int Mpad) {
  const ExVGeom g = geometry(ctx, Mpad);
  const double rows = (double)g.Ra + g.Kb;
  return 2.0 * ctx->S * rows * g.C + 4.0 * rows;
}

// Once per trial (after mixed_init_trial set Mpad and after the FP64 V was built):
// the digit planes of the stacked V', their row exponents and tensor map.
int mixed_exchange_v_init(afq_ctx* ctx) {
  if (!ctx->Vx) return afq_fail(ctx, AFQ_ERR_STATE, "stored exchange: V not built");
  const int S = ctx->S;
  const ExVGeom g = geometry(ctx, ctx->Mpad);
  const long R = (long)g.Ra + g.Kb;
  if (ctx->Vsl) cudaFree(ctx->Vsl);
  if (ctx->exv_ea) cudaFree(ctx->exv_ea);
  ctx->Vsl = nullptr;
  ctx->exv_ea = nullptr;
  if (cudaMalloc((void**)&ctx->Vsl, (size_t)S * R * g.C * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->exv_ea, (size_t)R * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return afq_fail(ctx, AFQ_ERR_NOMEM, "stored exchange: digit planes of V");
  }
  const long nMa = (long)ctx->na * ctx->M;
  k_slice_v_exact<<<warp_blocks(R), 256, 0, ctx->stream>>>(
      ctx->Vx, ctx->Vx + nMa * nMa, ctx->na, ctx->nb, ctx->M, ctx->Mpad, g, S, ctx->Vsl,
      ctx->exv_ea);
  AFQ_LAUNCHED(ctx);
  const uint64_t da[3] = {(uint64_t)g.C, (uint64_t)R, (uint64_t)S};
  const uint32_t ba[3] = {kBK, 128, 1};
  if (!make_tmap(&ctx->tm_exv_a[0], ctx->Vsl, 3, da, ba))
    return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (stored exchange)");
  return AFQ_OK;
}

// Per walker set (after the theta digit planes exist): y, the column tile and the
// B-operand map.  The column tile is the widest that fits the S accumulators in TMEM
// with little padding (pick_bn) and still gives about two CTAs per SM, but not below
// 64 (narrower MMAs waste the tensor core on re-reading A).
int mixed_exchange_v_walkers(afq_ctx* ctx) {
  if (ctx->exv_y) cudaFree(ctx->exv_y);
  ctx->exv_y = nullptr;
  const int W2 = 2 * ctx->ws.W;
  const ExVGeom g = geometry(ctx, ctx->Mpad);
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->exv_y, (size_t)W2 * (g.Ka + g.Kb) * sizeof(double)));
  const int rows = g.nrt_a + g.nrt_b;
  int BN = pick_bn(W2, ctx->S, 256);
  while (BN > 64 && rows * ((W2 + BN - 1) / BN) < 2 * 148) BN -= 16;
  ctx->exv_BN = BN;
  const uint64_t db[3] = {(uint64_t)ctx->N * ctx->Mpad, (uint64_t)W2, (uint64_t)ctx->S};
  const uint32_t bb[3] = {kBK, (uint32_t)ctx->exv_BN, 1};
  if (!make_tmap(&ctx->tm_exv_b, ctx->exv_th, 3, db, bb))
    return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (stored exchange theta)");
  return AFQ_OK;
}

// Needs theta's digit planes of the current walkers (launch_slice_theta).
int launch_exchange_tcv(afq_ctx* ctx, WalkerSet& s) {
  const int W2 = 2 * s.W;
  ExVP::Args a{};
  a.g = geometry(ctx, ctx->Mpad);
  a.c.nkb = a.g.C / kBK;
  a.c.BN = ctx->exv_BN;
  a.c.tx_bytes = (uint32_t)ctx->S * (kBK * 128 * 2 + kBK * ctx->exv_BN * 2);
  a.c.tmem_cols = tmem_cols_for(ctx->S * ctx->exv_BN);
  a.c.err = ctx->flags + 2;
  a.c.per_pair = ctx->p.prop_kernel == 2;
  a.W2 = W2;
  a.ea = ctx->exv_ea;
  a.eb = ctx->exv_eb;
  a.y = ctx->exv_y;
  size_t smem = 0;
  plan_smem(ctx->S, 1, 1, a.c.BN, 0, &a.c.stages, &smem);
  if (a.c.stages < 1 || a.c.tmem_cols > 512)
    return afq_fail(ctx, AFQ_ERR_ARG, "stored exchange tile does not fit");
  dim3 grid((W2 + a.c.BN - 1) / a.c.BN, a.g.nrt_a + a.g.nrt_b);
  cudaError_t e = launch_tc_s<ExVP>(ctx->S, grid, smem, ctx->stream, ctx->tm_exv_a[0],
                                    ctx->tm_exv_b, a);
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("stored exchange tc: ") + cudaGetErrorString(e));
  k_exv_dot<<<dim3(s.W, 2), 256, 0, ctx->stream>>>(a.g.Ka, a.g.Kb, ctx->na, ctx->nb, ctx->M,
                                                   ctx->Mpad, (long)ctx->N * ctx->M, W2,
                                                   ctx->exv_y, s.thetaT, ctx->ex_groups, s.ekp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
