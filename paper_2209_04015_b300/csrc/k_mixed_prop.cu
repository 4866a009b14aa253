// Split-precision tensor-core propagation (precision AFQ_SPLIT_BF16): the VHS build
// A_z = i sqrt(dt) sum_g y_zg L_g and Phi_z <- P T_n(A_z) P Phi_z (Eq. Bx and the
// walker update of Sec. "Review of AFQMC") on the engine of tc_engine.cuh, in its
// exact-diagonal form.
//
// Every operand row is scaled by a power of two and cut into S integer-valued
// bfloat16 digits (|q| <= 128); the slice products of one diagonal s + t = d go to
// their own TMEM accumulator, where the FP32 sums are integers and therefore exact,
// and the epilogue recombines the diagonals in FP64.  The only error left is the
// truncation of the digits (about 2^-(8S-1) of each row's largest element), so the
// walker keeps near-FP64 accuracy step after step; an FP32-accumulated split loses
// ~1e-7 per step to the long sums of the VHS (K = X) and the Taylor terms.  Digits,
// row scales and the recombination run on the integer pipe (tc_engine.cuh): B300's
// FP64 pipe would otherwise dominate these memory-bound passes.
//
// VHS: D[(p,q)][(z, re/im)] = sum_g L_g,pq y_zg, A operand the Cholesky tensor over
// its packed upper triangle (rows (p <= q), K = g: half the MMAs of the dense form);
// the epilogue writes V_z in FP64 to both triangles (the factor i sqrt(dt) of
// A_z is applied with 1/k in the Taylor epilogue).
// Taylor terms and one-body halves: per walker, 128-row tile of p and 64-column
// tile of j, Re and Im accumulators of A T (A M x M, T M x N as K-major T^T rows
// j), four MMA streams per slice pair with the negate-A bit for -Im A Im T.  The
// identity parts stay in FP64: P Phi = Phi + (P - I) Phi, and each Taylor term is
// added to an FP64 accumulator.
#include "tc_engine.cuh"

using namespace tce;

namespace {

constexpr int kPropBN = 64;  // columns j per tile of the propagation GEMMs

// ---------------------------------------------------------------------------
// VHS policy
// ---------------------------------------------------------------------------
struct VhsP {
  struct Args {
    TcCommon c;
    int M, W, Mp;
    const int2* tpq;  // packed row t -> (p, q), p <= q
    const int* ea;    // row exponents of L^T, per packed (p, q)
    const int* eb;    // row exponents of y, per (z, re/im)
    double2* V;       // W x M x M: V_z = sum_g y_zg L_g, FP64, both triangles
  };
  struct Tile {
    int r0, n0, kb0, kb1;
  };
  static constexpr int kUA = 1, kUB = 1;
  template <int S>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    issue_diagonals<S>(tmem, (uint32_t)a.c.BN, sa, sb, bslot, 0, 0, tc::idesc_bf16(128, a.c.BN),
                       first);
  }
  static __device__ Tile tile(const Args& a) {
    return Tile{(int)blockIdx.y * 128, (int)blockIdx.x * a.c.BN, 0, a.c.nkb};
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.r0, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t, int,
                                int s, int kb, uint64_t* bar) {
    tc::tma_load_3d(dst, tm, kb * kBK, t.n0, s, bar);
  }
  template <int S>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const long MM = (long)a.M * a.M;
    const long row = (long)t.r0 + warp * 32 + lane;
    const bool valid = row < a.Mp;
    const int er = valid ? a.ea[row] : 0;
    const int2 pq = valid ? a.tpq[row] : make_int2(0, 0);
    const long e_pq = (long)pq.x * a.M + pq.y, e_qp = (long)pq.y * a.M + pq.x;
    for (int c0 = 0; c0 < a.c.BN; c0 += 16) {
      float f[S][16];
#pragma unroll
      for (int d = 0; d < S; ++d) tmem_row16(tmem + (uint32_t)(d * a.c.BN), warp, c0, f[d]);
      if (!valid) continue;
#pragma unroll
      for (int jj = 0; jj < 16; jj += 2) {
        const int col = t.n0 + c0 + jj, z = col >> 1;
        if (z >= a.W) continue;
        float ar[S], ai[S];
#pragma unroll
        for (int d = 0; d < S; ++d) {
          ar[d] = f[d][jj];
          ai[d] = f[d][jj + 1];
        }
        const double2 v = make_double2(combine_exact<S>(ar, er + a.eb[col] - 14),
                                       combine_exact<S>(ai, er + a.eb[col + 1] - 14));
        a.V[(long)z * MM + e_pq] = v;
        if (e_qp != e_pq) a.V[(long)z * MM + e_qp] = v;
      }
    }
  }
};

// ---------------------------------------------------------------------------
// Complex (or real-A) times complex policy
// ---------------------------------------------------------------------------
enum { kModeFirst = 0, kModeTerm = 1, kModeLast = 2 };

template <bool REAL>
struct CplxP {
  struct Args {
    TcCommon c;
    int M, N, W, mode, acc_out;
    double coef;            // term k: sqrt(dt) / k (A = i sqrt(dt) V)
    const int* ea;          // row exponents of A: P - I per p, or V_z per (z, p)
    const int* eb;          // row exponents of T^T per (z, j)
    const double2* phi_in;  // mode first: Phi (W x M x N)
    double2* accT;          // W x N x M FP64 accumulator of P T_n(A) P Phi, transposed
    double2* phi_out;       // mode last: Phi (W x M x N)
    double2* tout;          // W x N x M FP64: the next operand (sliced by the next kernel)
  };
  struct Tile {
    int p0, z, n0, kb0, kb1;
  };
  static constexpr int kUA = REAL ? 1 : 2, kUB = 2;
  template <int S>
  static __device__ void issue(const Args& a, uint32_t tmem, uint32_t sa, uint32_t sb,
                               uint32_t bslot, bool first) {
    const int BN = a.c.BN;
    const uint32_t id = tc::idesc_bf16(128, BN), idn = tc::idesc_bf16(128, BN, true);
    const uint32_t acc_re = tmem, acc_im = tmem + (uint32_t)(S * BN);
    issue_diagonals<S>(acc_re, BN, sa, sb, bslot, 0, 0, id, first);     // Re A Re T
    issue_diagonals<S>(acc_im, BN, sa, sb, bslot, 0, 1, id, first);     // Re A Im T
    if (!REAL) {
      issue_diagonals<S>(acc_re, BN, sa, sb, bslot, 1, 1, idn, false);  // -Im A Im T
      issue_diagonals<S>(acc_im, BN, sa, sb, bslot, 1, 0, id, false);   // Im A Re T
    }
  }
  static __device__ Tile tile(const Args& a) {
    return Tile{(int)blockIdx.x * 128, (int)blockIdx.y, (int)blockIdx.z * kPropBN, 0, a.c.nkb};
  }
  static __device__ void load_a(const CUtensorMap* tm, void* dst, const Args&, const Tile& t,
                                int u, int s, int kb, uint64_t* bar) {
    if (REAL)
      tc::tma_load_3d(dst, tm, kb * kBK, t.p0, s, bar);
    else
      tc::tma_load_4d(dst, tm, kb * kBK, t.p0, 2 * t.z + u, s, bar);
  }
  static __device__ void load_b(const CUtensorMap* tm, void* dst, const Args&, const Tile& t,
                                int u, int s, int kb, uint64_t* bar) {
    tc::tma_load_4d(dst, tm, kb * kBK, t.n0, 2 * t.z + u, s, bar);
  }
  template <int S>
  static __device__ void epilogue(const Args& a, const Tile& t, uint32_t tmem, uint8_t*, int warp,
                                  int lane) {
    const int p = t.p0 + warp * 32 + lane, z = t.z, N = a.N, BN = a.c.BN;
    const bool valid = p < a.M;
    const int ep = valid ? (REAL ? a.ea[p] : a.ea[(long)z * a.M + p]) : 0;
    for (int c0 = 0; c0 < BN && t.n0 + c0 < N; c0 += 16) {
      float fr[S][16], fi[S][16];
#pragma unroll
      for (int d = 0; d < S; ++d) {
        tmem_row16(tmem + (uint32_t)(d * BN), warp, c0, fr[d]);
        tmem_row16(tmem + (uint32_t)((S + d) * BN), warp, c0, fi[d]);
      }
      if (!valid) continue;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = t.n0 + c0 + jj;
        if (j >= N) continue;
        const int sc = ep + a.eb[(long)z * N + j] - 14;
        float ar[S], ai[S];
#pragma unroll
        for (int d = 0; d < S; ++d) {
          ar[d] = fr[d][jj];
          ai[d] = fi[d][jj];
        }
        const double dr = combine_exact<S>(ar, sc), di = combine_exact<S>(ai, sc);
        const long ia = ((long)z * N + j) * a.M + p;    // [z][j][p]
        const long iphi = ((long)z * a.M + p) * N + j;  // [z][p][j]
        if (a.mode == kModeFirst) {
          const double2 f = a.phi_in[iphi];
          const double2 out = make_double2(dr + f.x, di + f.y);
          a.accT[ia] = out;
          a.tout[ia] = out;
        } else if (a.mode == kModeTerm) {
          // T_k = i sqrt(dt) V T_{k-1} / k = c (-Im(V T), Re(V T)), c = sqrt(dt) / k
          const double2 out = make_double2(-a.coef * di, a.coef * dr);
          const double2 acc = a.accT[ia];
          const double2 sum = make_double2(acc.x + out.x, acc.y + out.y);
          a.accT[ia] = sum;
          a.tout[ia] = a.acc_out ? sum : out;
        } else {
          const double2 acc = a.accT[ia];
          a.phi_out[iphi] = make_double2(dr + acc.x, di + acc.y);
        }
      }
    }
  }
};

// ---------------------------------------------------------------------------
// slicing kernels (one warp per row: row maximum, then integer digits)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_max_int(int v) { return __reduce_max_sync(0xffffffffu, v); }

// y (W x X complex) -> rows (z, re/im) of K = X, padded to Xpad
__global__ void k_slice_y(const double2* __restrict__ y, int W, int X, int Xpad, int S,
                          __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = 2L * W * Xpad;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < 2L * W;
       r += (long)gridDim.x * warps) {
    const long z = r >> 1;
    const int part = (int)(r & 1);
    const double* row = reinterpret_cast<const double*>(y + z * X) + part;
    int m = 0;
    for (int g = lane; g < X; g += 32) m = max(m, exp_field(row[2 * g]));
    const int e = row_exponent_field(warp_max_int(m));
    if (lane == 0) eout[r] = e;
    for (int g = lane; g < Xpad; g += 32)
      split_exact(g < X ? row[2 * g] : 0.0, e, S, out + r * Xpad + g, plane);
  }
}

// complex rows (z, i), i < R, K elements each -> planes [s][z][re/im][i][Kp]; one
// exponent per complex row, shared by its real and imaginary parts
__global__ void k_slice_cplx(const double2* __restrict__ in, long rows, int R, int K, int Kp, int S,
                             __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = 2L * rows * Kp;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const double2* row = in + r * K;
    int m = 0;
    for (int k = lane; k < K; k += 32) m = max(m, max(exp_field(row[k].x), exp_field(row[k].y)));
    const int e = row_exponent_field(warp_max_int(m));
    if (lane == 0) eout[r] = e;
    const long z = r / R, i = r % R;
    __nv_bfloat16* ore = out + ((z * 2) * R + i) * Kp;
    __nv_bfloat16* oim = ore + (long)R * Kp;
    for (int k = lane; k < Kp; k += 32) {
      const double2 v = k < K ? row[k] : make_double2(0.0, 0.0);
      split_exact(v.x, e, S, ore + k, plane);
      split_exact(v.y, e, S, oim + k, plane);
    }
  }
}

// Phi (W x M x N) -> W x N x M (transposed copy, FP64)
__global__ void k_transpose_phi(const double2* __restrict__ phi, int W, int M, int N,
                                double2* __restrict__ out) {
  const long total = (long)W * N * M;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int p = (int)(e % M);
    const long zj = e / M;
    const int j = (int)(zj % N);
    const long z = zj / N;
    out[e] = phi[(z * M + p) * N + j];
  }
}

// exponent of each (p, q) row of L^T: max over g of |L_g,pq|
// Row exponents of L^T over the packed upper triangle (rows t -> (p, q), p <= q).
__global__ void k_lt_exponents(const double* __restrict__ L, int X, int M, long Mp,
                               const int2* __restrict__ tpq, int* __restrict__ e) {
  const long MM = (long)M * M;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < Mp;
       r += (long)gridDim.x * blockDim.x) {
    const int2 pq = tpq[r];
    const long o = (long)pq.x * M + pq.y;
    int m = 0;
    for (int g = 0; g < X; ++g) m = max(m, exp_field(L[(long)g * MM + o]));
    e[r] = row_exponent_field(m);
  }
}

// L (X x M x M) -> planes [t][Xpad] of integer digits over the packed upper triangle
// (t -> (p, q), p <= q): 32 x 32 tile transpose
__global__ void k_slice_LT(const double* __restrict__ L, int X, int M, long Mp, int Xpad, int S,
                           const int2* __restrict__ tpq, const int* __restrict__ e,
                           __nv_bfloat16* __restrict__ out) {
  __shared__ double tileb[32][33];
  const long MM = (long)M * M;
  const long r0 = (long)blockIdx.x * 32;
  const int g0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const long r = r0 + tx;
  const int2 pq = r < Mp ? tpq[r] : make_int2(0, 0);
  for (int k = ty; k < 32; k += 8) {
    const int g = g0 + k;
    tileb[k][tx] = (g < X && r < Mp) ? L[(long)g * MM + (long)pq.x * M + pq.y] : 0.0;
  }
  __syncthreads();
  const long plane = Mp * Xpad;
  for (int k = ty; k < 32; k += 8) {
    const long rr = r0 + k;
    const int g = g0 + tx;
    if (rr < Mp && g < Xpad) split_exact(tileb[tx][k], e[rr], S, out + rr * Xpad + g, plane);
  }
}

// P - I -> rows p of K = M, padded to Mpad (one warp per row)
__global__ void k_slice_pm(const double* __restrict__ P, int M, int Mpad, int S,
                           __nv_bfloat16* __restrict__ out, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < M; p += gridDim.x * warps) {
    int m = 0;
    for (int q = lane; q < M; q += 32) m = max(m, exp_field(P[(long)p * M + q] - (p == q ? 1.0 : 0.0)));
    const int e = row_exponent_field(warp_max_int(m));
    if (lane == 0) eout[p] = e;
    for (int q = lane; q < Mpad; q += 32) {
      const double v = q < M ? P[(long)p * M + q] - (p == q ? 1.0 : 0.0) : 0.0;
      split_exact(v, e, S, out + (long)p * Mpad + q, (long)M * Mpad);
    }
  }
}

int warp_grid(long rows) {
  long g = (rows + 7) / 8;
  return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

}  // namespace

// ===========================================================================
// context integration
// ===========================================================================
void mixed_prop_free(afq_ctx* ctx) {
  for (auto** p : {&ctx->LT_sl, &ctx->Pm_sl, &ctx->y_sl, &ctx->A_sl, &ctx->T_sl[0], &ctx->T_sl[1]})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  for (auto** p : {&ctx->e_lt, &ctx->e_pm, &ctx->e_y, &ctx->e_a, &ctx->e_t[0], &ctx->e_t[1]})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  if (ctx->accT) cudaFree(ctx->accT);
  if (ctx->tout) cudaFree(ctx->tout);
  ctx->accT = nullptr;
  ctx->tout = nullptr;
}

// Once per trial: digits of L^T (the VHS operand) and of P - I, with row exponents.
int mixed_prop_init_trial(afq_ctx* ctx) {
  const int S = ctx->Sp, M = ctx->M, X = ctx->X;
  ctx->Xpad = round_up(X, kBK);
  const long Mp = ctx->Mp;  // packed upper-triangle rows of L^T
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->LT_sl, (size_t)S * Mp * ctx->Xpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->Pm_sl, (size_t)S * M * ctx->Mpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_lt, (size_t)Mp * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_pm, (size_t)M * sizeof(int)));
  k_lt_exponents<<<grid1d(Mp), 256, 0, ctx->stream>>>(ctx->L, X, M, Mp, ctx->tpq, ctx->e_lt);
  AFQ_LAUNCHED(ctx);
  dim3 g((unsigned)((Mp + 31) / 32), (unsigned)((ctx->Xpad + 31) / 32));
  k_slice_LT<<<g, dim3(32, 8), 0, ctx->stream>>>(ctx->L, X, M, Mp, ctx->Xpad, S, ctx->tpq,
                                                 ctx->e_lt, ctx->LT_sl);
  AFQ_LAUNCHED(ctx);
  k_slice_pm<<<warp_grid(M), 256, 0, ctx->stream>>>(ctx->P, M, ctx->Mpad, S, ctx->Pm_sl, ctx->e_pm);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// Per walker set: operand buffers and tensor maps of the propagation.
int mixed_prop_init_walkers(afq_ctx* ctx) {
  const int S = ctx->Sp, M = ctx->M, N = ctx->N, W = ctx->ws.W, Mp = ctx->Mpad;
  for (auto** p : {&ctx->y_sl, &ctx->A_sl, &ctx->T_sl[0], &ctx->T_sl[1]})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  for (auto** p : {&ctx->e_y, &ctx->e_a, &ctx->e_t[0], &ctx->e_t[1]})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  if (ctx->accT) cudaFree(ctx->accT);
  if (ctx->tout) cudaFree(ctx->tout);
  ctx->accT = nullptr;
  ctx->tout = nullptr;
  const size_t tbytes = (size_t)S * 2 * W * N * Mp * 2;
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->y_sl, (size_t)S * 2 * W * ctx->Xpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->A_sl, (size_t)S * 2 * W * M * Mp * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->T_sl[0], tbytes));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->T_sl[1], tbytes));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->accT, (size_t)W * N * M * sizeof(double2)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->tout, (size_t)W * N * M * sizeof(double2)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_y, (size_t)2 * W * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_a, (size_t)W * M * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_t[0], (size_t)W * N * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_t[1], (size_t)W * N * sizeof(int)));
  ctx->vhs_BN = 2 * W >= 128 ? 128 : round_up(2 * W, 16);
  ctx->prop_BN = N >= kPropBN ? kPropBN : round_up(N, 16);
  if (S * ctx->vhs_BN > 512 || 2 * S * ctx->prop_BN > 512)
    return afq_fail(ctx, AFQ_ERR_ARG, "split propagation: too many slices for TMEM");
  const uint32_t brows = (uint32_t)(N >= kPropBN ? kPropBN : N);
  bool ok = true;
  {
    const uint64_t da[3] = {(uint64_t)ctx->Xpad, (uint64_t)ctx->Mp, (uint64_t)S};
    const uint32_t ba[3] = {kBK, 128, 1};
    const uint64_t db[3] = {(uint64_t)ctx->Xpad, (uint64_t)(2 * W), (uint64_t)S};
    const uint32_t bb[3] = {kBK, (uint32_t)ctx->vhs_BN, 1};
    ok = ok && make_tmap(&ctx->tm_vhs_a, ctx->LT_sl, 3, da, ba) &&
         make_tmap(&ctx->tm_vhs_b, ctx->y_sl, 3, db, bb);
  }
  {
    const uint64_t dp[3] = {(uint64_t)Mp, (uint64_t)M, (uint64_t)S};
    const uint32_t bp[3] = {kBK, 128, 1};
    const uint64_t daz[4] = {(uint64_t)Mp, (uint64_t)M, (uint64_t)(2 * W), (uint64_t)S};
    const uint32_t baz[4] = {kBK, 128, 1, 1};
    const uint64_t dt[4] = {(uint64_t)Mp, (uint64_t)N, (uint64_t)(2 * W), (uint64_t)S};
    const uint32_t bt[4] = {kBK, brows, 1, 1};
    ok = ok && make_tmap(&ctx->tm_pm, ctx->Pm_sl, 3, dp, bp) &&
         make_tmap(&ctx->tm_az, ctx->A_sl, 4, daz, baz) &&
         make_tmap(&ctx->tm_t[0], ctx->T_sl[0], 4, dt, bt) &&
         make_tmap(&ctx->tm_t[1], ctx->T_sl[1], 4, dt, bt);
  }
  if (!ok) return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (propagation) failed");
  return AFQ_OK;
}

// V_z = sum_g y_zg L_g for every walker (FP64 into ctx->A), then its digits; the
// factor i sqrt(dt) of A_z = i sqrt(dt) V_z is applied by the Taylor epilogue.
int launch_vhs_tc(afq_ctx* ctx) {
  const int W = ctx->ws.W, M = ctx->M, S = ctx->Sp;
  k_slice_y<<<warp_grid(2L * W), 256, 0, ctx->stream>>>(ctx->y, W, ctx->X, ctx->Xpad, S,
                                                       ctx->y_sl, ctx->e_y);
  AFQ_LAUNCHED(ctx);
  VhsP::Args a{};
  a.c.nkb = ctx->Xpad / kBK;
  a.c.BN = ctx->vhs_BN;
  a.c.tx_bytes = (uint32_t)S * (kBK * 128 * 2 + kBK * a.c.BN * 2);
  a.c.tmem_cols = tmem_cols_for(S * a.c.BN);
  a.c.err = ctx->flags + 2;
  a.M = M;
  a.W = W;
  a.Mp = ctx->Mp;
  a.tpq = ctx->tpq;
  a.ea = ctx->e_lt;
  a.eb = ctx->e_y;
  a.V = ctx->A;
  size_t smem = 0;
  plan_smem(S, 1, 1, a.c.BN, 0, &a.c.stages, &smem);
  dim3 grid((2 * W + a.c.BN - 1) / a.c.BN, (unsigned)(((long)ctx->Mp + 127) / 128));
  cudaError_t e = launch_tc_s<VhsP>(S, grid, smem, ctx->stream, ctx->tm_vhs_a, ctx->tm_vhs_b, a);
  ctx->launches++;
  if (e != cudaSuccess) return afq_fail(ctx, AFQ_ERR_CUDA, std::string("vhs tc: ") + cudaGetErrorString(e));
  k_slice_cplx<<<warp_grid((long)W * M), 256, 0, ctx->stream>>>(ctx->A, (long)W * M, M, M,
                                                               ctx->Mpad, S, ctx->A_sl, ctx->e_a);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

namespace {
template <bool REAL>
int launch_cplx(afq_ctx* ctx, const CUtensorMap& ta, const CUtensorMap& tb, const int* ea,
                const int* eb, int mode, double coef, int acc_out) {
  using P = CplxP<REAL>;
  typename P::Args a{};
  const int N = ctx->N, S = ctx->Sp;
  const int brows = N >= kPropBN ? kPropBN : N;
  a.c.nkb = ctx->Mpad / kBK;
  a.c.BN = ctx->prop_BN;
  a.c.tx_bytes = (uint32_t)S * (P::kUA * kBK * 128 * 2 + 2 * kBK * brows * 2);
  a.c.tmem_cols = tmem_cols_for(2 * S * a.c.BN);
  a.c.err = ctx->flags + 2;
  a.M = ctx->M;
  a.N = N;
  a.W = ctx->ws.W;
  a.mode = mode;
  a.acc_out = acc_out;
  a.coef = coef;
  a.ea = ea;
  a.eb = eb;
  a.phi_in = ctx->ws.phi;
  a.accT = ctx->accT;
  a.phi_out = ctx->ws.phi;
  a.tout = ctx->tout;
  size_t smem = 0;
  plan_smem(S, P::kUA, P::kUB, a.c.BN, 0, &a.c.stages, &smem);
  dim3 grid((ctx->M + 127) / 128, ctx->ws.W, (N + kPropBN - 1) / kPropBN);
  cudaError_t e = launch_tc_s<P>(S, grid, smem, ctx->stream, ta, tb, a);
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("propagate tc: ") + cudaGetErrorString(e));
  return AFQ_OK;
}

// digits of tout (W x N x M) into Taylor operand buffer b
int slice_tout(afq_ctx* ctx, int b) {
  const int W = ctx->ws.W, N = ctx->N, M = ctx->M;
  k_slice_cplx<<<warp_grid((long)W * N), 256, 0, ctx->stream>>>(ctx->tout, (long)W * N, N, M,
                                                               ctx->Mpad, ctx->Sp, ctx->T_sl[b],
                                                               ctx->e_t[b]);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
}  // namespace

// Phi <- P T_n(A) P Phi for every walker, A from the last launch_vhs_tc.
int launch_propagate_tc(afq_ctx* ctx) {
  const int W = ctx->ws.W;
  k_transpose_phi<<<grid1d((long)W * ctx->N * ctx->M), 256, 0, ctx->stream>>>(
      ctx->ws.phi, W, ctx->M, ctx->N, ctx->tout);
  AFQ_LAUNCHED(ctx);
  int cur = 0, rc;
  if ((rc = slice_tout(ctx, cur)) != AFQ_OK) return rc;
  // T_0 = P Phi = Phi + (P - I) Phi
  rc = launch_cplx<true>(ctx, ctx->tm_pm, ctx->tm_t[cur], ctx->e_pm, ctx->e_t[cur], kModeFirst,
                         1.0, 0);
  if (rc != AFQ_OK) return rc;
  cur = 1 - cur;
  if ((rc = slice_tout(ctx, cur)) != AFQ_OK) return rc;
  const int n = ctx->p.taylor_order;
  for (int k = 1; k <= n; ++k) {
    rc = launch_cplx<false>(ctx, ctx->tm_az, ctx->tm_t[cur], ctx->e_a, ctx->e_t[cur], kModeTerm,
                            sqrt(ctx->p.dt) / k, k == n);
    if (rc != AFQ_OK) return rc;
    cur = 1 - cur;
    if ((rc = slice_tout(ctx, cur)) != AFQ_OK) return rc;
  }
  // Phi = P acc = acc + (P - I) acc
  return launch_cplx<true>(ctx, ctx->tm_pm, ctx->tm_t[cur], ctx->e_pm, ctx->e_t[cur], kModeLast,
                           1.0, 0);
}
