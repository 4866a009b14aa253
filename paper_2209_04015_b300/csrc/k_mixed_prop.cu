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
// diagonal of P stays in FP64: P Phi = diag(P) Phi + O Phi with O the off-diagonal
// part of P, so the digits of O carry its own row scale (the off-diagonal elements
// are ~100x smaller than the diagonal ones, which would otherwise set the scale), and
// each Taylor term is added to an FP64 accumulator.
#include <cmath>
#include <vector>

#include "tc_engine.cuh"

using namespace tce;

namespace {

constexpr int kPropRows = 64;  // walker columns j per propagation tile (x2: re and im)

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
    issue_split<S>(a.c, tmem, sa, sb, bslot, first);
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
// Taylor terms and one-body halves: a persistent kernel per GEMM pass
// ---------------------------------------------------------------------------
// Tile: rows p (128) x columns (re | im, j) (2 brows, brows a multiple of 16), for one
// walker.  With B = [Re T; Im T] (one operand tile, K = q) the complex product
// D = A T is, per K block,
//   D[:, re|im] += Re A B                   (N = 2 brows)
//   D[:, re]    += -Im A (Im T rows of B)   (N = brows, negate-A)
//   D[:, im]    +=  Im A (Re T rows of B)   (N = brows)
// (real A = O, the off-diagonal part of P: the first product only).  Exact digit
// diagonals accumulate in S TMEM regions of BN columns; each epilogue thread
// recombines a real column and its imaginary partner brows columns later and writes
// whole complex FP64 values.
// Column-concatenated form (CAT, up to 4 digits): the B digit slots t = 0 .. S - 1
// lie one after another in shared memory, so A digit s times the first S - s slots
// is ONE MMA of N = (S - s) BN columns whose column block t lands in accumulator s + t
// (the accumulators are BN columns apart): S MMAs per K block and A unit instead of
// S (S + 1) / 2, each reading its A digit from shared memory once.  The complex
// product takes a second B region [-Im T; Re T] per slot (the negated digits come from
// the slicing pass), so that Im A times it adds [-Im A Im T | Im A Re T] in the same
// two MMAs per digit.  The sums per accumulator are the same exact integer sums, so
// the results are bit-identical to the per-pair form.
// Roles: warp 0 TMA, warp 1 MMA (and TMEM), warps 2-9 epilogue (two per TMEM lane
// quarter, splitting the column chunks); the producer runs ahead across tiles while
// the epilogue drains TMEM.
enum { kModeFirst = 0, kModeTerm = 1, kModeLast = 2, kModeTheta = 3 };
// kModeTheta: the same kernel forms theta = Phi S^-1 per unit u = (z, spin) (A = the
// digits of the unit's Phi rows over its K = n columns, B = those of S^-1; N = nmax)
// and writes theta^T into tout at the unit's rows of the W x (na + nb) x M layout
constexpr int kPropWarps = 10;
constexpr int kAccAhead = 4;  // FP64 Taylor sums loaded ahead of the last pass's stores
constexpr int kPropEpi = 8;

struct PropArgs {
  int M, N, W, mode, brows, BN, nkb, stages, npt, njt, ntiles;
  int nbuf;               // TMEM accumulator sets (2 when 2 S BN <= 512: the epilogue of
                          // one tile overlaps the MMAs of the next)
  int split;              // column-concatenated complex pass: each K block takes two ring
                          // stages, [Re A digits | Re T; Im T] then [Im A digits | -Im T; Re T]
  uint32_t tx_bytes, tmem_cols;
  const int* ea;          // row exponents of A: O (P off the diagonal) per p, or V_z per (z, p)
  const double* pdiag;    // M: diagonal of P (mode last adds diag(P) acc in FP64)
  const int* eb;          // row exponents of T^T per (z, j)
  double2* accT;          // W x N x M FP64 accumulator of P T_n(A) P Phi, transposed
  double2* phi_out;       // mode last: Phi (W x M x N)
  double2* tout;          // W x N x M FP64: the next operand (sliced by the next kernel)
  int* err;
  int na, nb, Ntot;       // kModeTheta: electrons per spin and their sum
};

// kModeTheta's output element: theta^T at the unit's rows
__device__ __forceinline__ void prop_store_theta(const PropArgs& a, int z, int j, int p, double dr,
                                                 double di) {
  const int sg = z & 1;
  if (j < (sg ? a.nb : a.na))
    a.tout[((long)(z >> 1) * a.Ntot + sg * a.na + j) * a.M + p] = make_double2(dr, di);
}

// The exact digit diagonals of a kModeTheta element (K <= 64, at most 4 digits: every
// diagonal sum is an integer of magnitude at most (d + 1) 64 128^2 <= 2^22, and their
// weighted int64 sum is below 2^47) recombined without the
// FP64 pipe: float -> int by the 1.5 2^23 shift, int64 -> double by normalising the bits.
template <int S>
__device__ __forceinline__ double combine_theta(const float (&acc)[S], int scale_exp) {
  long long t = 0;
#pragma unroll
  for (int d = 0; d < S; ++d)
    t += (long long)(__float_as_int(__fadd_rn(acc[d], 12582912.0f)) - 0x4B400000) *
         (1LL << (8 * (S - 1 - d)));
  if (t == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)t & 0x8000000000000000ull;
  const unsigned long long m = (unsigned long long)(t < 0 ? -t : t);
  const int msb = 63 - __clzll((long long)m);  // <= 52
  const unsigned long long bits = sgn |
      ((unsigned long long)(msb + 1023 + scale_exp - 8 * (S - 1)) << 52) |
      ((m << (52 - msb)) & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// TMEM load of CW (16 or 8) consecutive columns of this warp's lanes.
template <int CW>
__device__ __forceinline__ void prop_tmem_ld(uint32_t taddr, float (&v)[CW]) {
  if constexpr (CW == 16) {
    tc::tmem_ld16(taddr, v);
  } else {
    uint32_t r[8];
    tc::tmem_ld8_nowait(taddr, r);
    tc::tmem_wait_ld();
    tc::tmem_regs_ready8(r);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
  }
}

__device__ __forceinline__ void prop_epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kPropEpi * 32) : "memory");
}

// Epilogue of one group of CW columns (c0 .. c0 + CW - 1) of this thread's row p (the
// form the kernel takes beyond 4 digits): real parts first (digits -> FP64), then
// their imaginary partners, then the pass's output.
template <int S, int CW, bool THETA>
__device__ __forceinline__ void prop_epi_group(const PropArgs& a, uint32_t trow, int BN, int brows,
                                               int c0, int z, int j0, int p, bool valid, int ep) {
  const int M = a.M, N = a.N;
  float f[S][CW];
  double dre[CW];
#pragma unroll
  for (int d = 0; d < S; ++d) prop_tmem_ld<CW>(trow + (uint32_t)(d * BN + c0), f[d]);
#pragma unroll
  for (int jj = 0; jj < CW; ++jj) {
    const int j = j0 + c0 + jj;
    float ar[S];
#pragma unroll
    for (int d = 0; d < S; ++d) ar[d] = f[d][jj];
    dre[jj] = (valid && j < N) ? combine_exact<S>(ar, ep + a.eb[(long)z * N + j] - 14) : 0.0;
  }
#pragma unroll
  for (int d = 0; d < S; ++d) prop_tmem_ld<CW>(trow + (uint32_t)(d * BN + brows + c0), f[d]);
  if (!valid) return;
  const double pd = a.mode == kModeLast ? a.pdiag[p] : 0.0;
#pragma unroll
  for (int h = 0; h < CW; h += kAccAhead) {
    double2 accv[kAccAhead];  // the last pass's Taylor sums, loaded ahead of the stores
    if (a.mode == kModeLast) {
#pragma unroll
      for (int jj = 0; jj < kAccAhead; ++jj) {
        const int j = j0 + c0 + h + jj;
        accv[jj] = j < N ? a.accT[((long)z * N + j) * M + p] : make_double2(0.0, 0.0);
      }
    }
#pragma unroll
    for (int jj = 0; jj < kAccAhead; ++jj) {
      const int j = j0 + c0 + h + jj;
      if (j >= N) continue;
      float ai[S];
#pragma unroll
      for (int d = 0; d < S; ++d) ai[d] = f[d][h + jj];
      const double dr = dre[h + jj], di = combine_exact<S>(ai, ep + a.eb[(long)z * N + j] - 14);
      if constexpr (THETA) {  // (theta runs at most 4 digits: the inline epilogue)
        continue;
      }
      const long ia = ((long)z * N + j) * M + p;    // [z][j][p]
      if (a.mode == kModeFirst) {
        // O Phi; the slicing pass adds diag(P) Phi (FP64) and cuts u_0 = P Phi
        a.accT[ia] = make_double2(dr, di);
      } else if (a.mode == kModeTerm) {
        // u_k = V u_{k-1}: the unscaled power; the slicing pass adds i^k g_k u_k to the
        // FP64 Taylor sum
        a.tout[ia] = make_double2(dr, di);
      } else {
        a.phi_out[((long)z * M + p) * N + j] =
            make_double2(fma(pd, accv[jj].x, dr), fma(pd, accv[jj].y, di));
      }
    }
  }
}

// Column-concatenated MMAs of one A unit (S digit slots of 128 rows at a0) against one
// B region (S slots of BN rows at b0): A digit s times B slots t0 .. t0 + nt - 1 is one
// MMA of nt BN columns (N <= 256) into accumulators s + t0 .. (BN columns apart).
template <int S>
__device__ __forceinline__ void prop_issue_cat(uint32_t acc, int BN, uint32_t a0, uint32_t b0,
                                               uint32_t bslot, bool first) {
  if constexpr (S <= 4) {  // S BN <= 256 (BN <= 64): one MMA per A digit
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const uint32_t idn = tc::idesc_bf16(128, (S - s) * BN);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(acc + (uint32_t)(s * BN), tc::sdesc_k64(a0 + s * kASlot + ks * 32),
                     tc::sdesc_k64(b0 + ks * 32), idn, !(first && s == 0 && ks == 0));
    }
  } else {
    const int tmax = 256 / BN;
#pragma unroll
    for (int s = 0; s < S; ++s)
      for (int t0 = 0; t0 < S - s; t0 += tmax) {
        const int nt = S - s - t0 < tmax ? S - s - t0 : tmax;
        const uint32_t idn = tc::idesc_bf16(128, nt * BN);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          tc::mma_bf16(acc + (uint32_t)((s + t0) * BN), tc::sdesc_k64(a0 + s * kASlot + ks * 32),
                       tc::sdesc_k64(b0 + (uint32_t)t0 * bslot + ks * 32), idn,
                       !(first && s == 0 && ks == 0));
      }
  }
}

template <int S, bool REAL, bool CAT, bool THETA = false>
__global__ void __launch_bounds__(32 * kPropWarps, 1)
    k_prop_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmBn, const __grid_constant__ PropArgs a) {
  constexpr int kUA = REAL ? 1 : 2;
  constexpr int kUB = (CAT && !REAL) ? 2 : 1;  // B regions per digit: [Re; Im] (+ [-Im; Re])
  static_assert(!CAT || S <= kMaxSlices, "digits");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t tfull[2];
  __shared__ __align__(8) uint64_t tempty[2];
  __shared__ __align__(8) uint64_t fin;
  __shared__ uint32_t tmem_base;
  __shared__ int skip;
  __shared__ int ep_ok[2];  // per tile parity: with two accumulator sets the lead
                            // epilogue thread can reach the next tile before every
                            // warp has read this tile's flag
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = a.stages, BN = a.BN, brows = a.brows;
  const uint32_t bslot = (uint32_t)BN * 64u;
  const int nh = (kUB == 2 && a.split) ? 2 : 1;  // ring stages per K block
  const uint32_t stage_bytes = nh == 2 ? S * (kASlot + bslot) : S * (kUA * kASlot + kUB * bslot);
  int* err = a.err;
  if (threadIdx.x == 0) skip = *(const volatile int*)err;
  __syncthreads();
  if (skip) return;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], kPropEpi);
    }
    tc::mbar_init(&fin, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
    if (kUB == 2) tc::prefetch_tmap(&tmBn);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int per_z = a.njt * a.npt;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
        const int z = tile / per_z, r = tile - z * per_z;
        const int p0 = (r % a.npt) * 128, j0 = (r / a.npt) * brows;
        for (int hb = 0; hb < nh * a.nkb; ++hb, ++it) {
          const int kb = hb / nh, h = hb - kb * nh;
          const int st = it % nst;
          if (it >= nst && !tc::mbar_wait(&empty[st], ((it / nst) - 1) & 1, err)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[st], a.tx_bytes);
          uint8_t* sa = smem + st * stage_bytes;
          if (nh == 2) {  // h = 0: Re A and [Re T; Im T]; h = 1: Im A and [-Im T; Re T]
            uint8_t* sb = sa + S * kASlot;
#pragma unroll
            for (int s = 0; s < S; ++s) {
              tc::tma_load_4d(sa + s * kASlot, &tmA, kb * kBK, p0, 2 * z + h, s, &full[st]);
              if (h == 0)
                tc::tma_load_4d(sb + s * bslot, &tmB, kb * kBK, j0, 2 * z, s, &full[st]);
              else
                tc::tma_load_4d(sb + s * bslot, &tmBn, kb * kBK, j0, z, s, &full[st]);
              tc::tma_load_4d(sb + s * bslot + brows * 64, &tmB, kb * kBK, j0, 2 * z + 1 - h, s,
                              &full[st]);
            }
            continue;
          }
          uint8_t* sb = sa + S * kUA * kASlot;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (REAL) {
              tc::tma_load_3d(sa + s * kASlot, &tmA, kb * kBK, p0, s, &full[st]);
            } else {
              tc::tma_load_4d(sa + s * kASlot, &tmA, kb * kBK, p0, 2 * z, s, &full[st]);
              tc::tma_load_4d(sa + (S + s) * kASlot, &tmA, kb * kBK, p0, 2 * z + 1, s, &full[st]);
            }
            tc::tma_load_4d(sb + s * bslot, &tmB, kb * kBK, j0, 2 * z, s, &full[st]);
            tc::tma_load_4d(sb + s * bslot + brows * 64, &tmB, kb * kBK, j0, 2 * z + 1, s,
                            &full[st]);
            if (kUB == 2) {  // the second region: [-Im T; Re T]
              uint8_t* sb2 = sb + S * bslot;
              tc::tma_load_4d(sb2 + s * bslot, &tmBn, kb * kBK, j0, z, s, &full[st]);
              tc::tma_load_4d(sb2 + s * bslot + brows * 64, &tmB, kb * kBK, j0, 2 * z, s,
                              &full[st]);
            }
          }
        }
      }
      for (int i = it > nst ? it - nst : 0; i < it; ++i)
        tc::mbar_wait(&full[i % nst], (i / nst) & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id_full = tc::idesc_bf16(128, BN);
      const uint32_t id_half = tc::idesc_bf16(128, brows), id_half_neg = tc::idesc_bf16(128, brows, true);
      int it = 0, lt = 0;
      bool ok = true;
      const int nbuf = a.nbuf;
      for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++lt) {
        const int buf = lt % nbuf, use = lt / nbuf;  // use-th fill of accumulator set buf
        if (use >= 1 && !tc::mbar_wait(&tempty[buf], (use - 1) & 1, err)) {
          atomicExch(err, 1);
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(buf * S * BN);
        for (int hb = 0; hb < nh * a.nkb; ++hb, ++it) {
          const int kb = hb / nh, h = hb - kb * nh;
          const int st = it % nst;
          if (!tc::mbar_wait(&full[st], (it / nst) & 1, err)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
          if (nh == 2) {
            // one A unit against one B region per stage: Re A [Re T; Im T] adds
            // [Re A Re T | Re A Im T], Im A [-Im T; Re T] adds [-Im A Im T | Im A Re T]
            if constexpr (CAT) prop_issue_cat<S>(acc, BN, sa, sa + S * kASlot, bslot, kb == 0 && h == 0);
            tc::mma_commit(&empty[st]);
            continue;
          }
          const uint32_t sb = sa + S * kUA * kASlot;
          if constexpr (CAT) {
            prop_issue_cat<S>(acc, BN, sa, sb, bslot, kb == 0);
            if (!REAL) prop_issue_cat<S>(acc, BN, sa + S * kASlot, sb + S * bslot, bslot, false);
          } else {
            issue_diagonals<S>(acc, (uint32_t)BN, sa, sb, bslot, 0, 0, id_full, kb == 0);
            if (!REAL) {
              issue_diagonals<S>(acc, (uint32_t)BN, sa, sb + (uint32_t)brows * 64u, bslot, 1, 0,
                                 id_half_neg, false);
              issue_diagonals<S>(acc + (uint32_t)brows, (uint32_t)BN, sa, sb, bslot, 1, 0,
                                 id_half, false);
            }
          }
          tc::mma_commit(&empty[st]);
        }
        if (ok) tc::mma_commit(&tfull[buf]);
      }
      tc::mma_commit(&fin);
    }
  } else {
    const int q = warp - 2, lq = warp & 3, part = q >> 2;  // two warps per lane quarter
    const int M = a.M, N = a.N;
    int lt = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++lt) {
      const int buf = lt % a.nbuf;
      if (q == 0 && lane == 0) {
        ep_ok[lt & 1] = tc::mbar_wait(&tfull[buf], (lt / a.nbuf) & 1, err) ? 1 : 0;
        if (!ep_ok[lt & 1]) atomicExch(err, 1);
      }
      prop_epi_sync();
      if (!ep_ok[lt & 1]) break;
      tc::fence_after_sync();
      const int z = tile / per_z, r = tile - z * per_z;
      const int p0 = (r % a.npt) * 128, j0 = (r / a.npt) * brows;
      const int p = p0 + 32 * lq + lane;
      const bool valid = p < M;
      const int ep = valid ? (REAL ? a.ea[p] : a.ea[(long)z * M + p]) : 0;
      const uint32_t trow = tmem + (uint32_t)(buf * S * BN) + ((uint32_t)(32 * lq) << 16);
      for (int c0 = 16 * part; c0 < brows; c0 += 32) {
        if constexpr (S > 4) {
          // more digits than registers for 16 columns at once: two groups of 8
          prop_epi_group<S, 8, THETA>(a, trow, BN, brows, c0, z, j0, p, valid, ep);
          prop_epi_group<S, 8, THETA>(a, trow, BN, brows, c0 + 8, z, j0, p, valid, ep);
        } else {
          // real parts of 16 columns first (digits -> FP64), then their imaginary partners.
          // In the last pass the FP64 Taylor sums are loaded into registers kAccAhead
          // columns ahead of the stores: the compiler cannot move a load across a store through
          // another pointer, and one DRAM latency per column serialised the epilogue.
          float f[S][16];
          double dre[16];
#pragma unroll
          for (int d = 0; d < S; ++d) tc::tmem_ld16(trow + (uint32_t)(d * BN + c0), f[d]);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = j0 + c0 + jj;
            float ar[S];
#pragma unroll
            for (int d = 0; d < S; ++d) ar[d] = f[d][jj];
            if constexpr (THETA)
              dre[jj] = (valid && j < N) ? combine_theta<S>(ar, ep + a.eb[(long)z * N + j] - 14) : 0.0;
            else
              dre[jj] = (valid && j < N) ? combine_exact<S>(ar, ep + a.eb[(long)z * N + j] - 14) : 0.0;
          }
#pragma unroll
          for (int d = 0; d < S; ++d) tc::tmem_ld16(trow + (uint32_t)(d * BN + brows + c0), f[d]);
          if (!valid) continue;
          const double pd = a.mode == kModeLast ? a.pdiag[p] : 0.0;
#pragma unroll
          for (int h = 0; h < 16; h += kAccAhead) {
            double2 accv[kAccAhead];
            if (a.mode == kModeLast) {
#pragma unroll
              for (int jj = 0; jj < kAccAhead; ++jj) {
                const int j = j0 + c0 + h + jj;
                accv[jj] = j < N ? a.accT[((long)z * N + j) * M + p] : make_double2(0.0, 0.0);
              }
            }
#pragma unroll
            for (int jj = 0; jj < kAccAhead; ++jj) {
              const int j = j0 + c0 + h + jj;
              if (j >= N) continue;
              float ai[S];
#pragma unroll
              for (int d = 0; d < S; ++d) ai[d] = f[d][h + jj];
              const double dr = dre[h + jj];
              const double di = THETA ? combine_theta<S>(ai, ep + a.eb[(long)z * N + j] - 14)
                                      : combine_exact<S>(ai, ep + a.eb[(long)z * N + j] - 14);
              if constexpr (THETA) {
                prop_store_theta(a, z, j, p, dr, di);
                continue;
              }
              const long ia = ((long)z * N + j) * M + p;  // [z][j][p]
              if (a.mode == kModeFirst) {
                // O Phi; the slicing pass adds diag(P) Phi (FP64) and cuts u_0 = P Phi
                a.accT[ia] = make_double2(dr, di);
              } else if (a.mode == kModeTerm) {
                // u_k = V u_{k-1}: the unscaled power; the slicing pass adds i^k g_k u_k
                // to the FP64 Taylor sum
                a.tout[ia] = make_double2(dr, di);
              } else {
                a.phi_out[((long)z * M + p) * N + j] =
                    make_double2(fma(pd, accv[jj].x, dr), fma(pd, accv[jj].y, di));
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      if (lane == 0) tc::mbar_arrive(&tempty[buf]);
    }
  }
  __syncthreads();
  if (warp == 1) {
    static const int zero = 0;
    tc::mbar_wait(&fin, 0, &zero);
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// slicing kernels (one warp per row: row maximum, then integer digits)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_max_int(int v) { return __reduce_max_sync(0xffffffffu, v); }

// y (W x X complex) -> rows (z, re/im) of K = X, padded to Xpad (D >= S: digit loop bound)
template <int D>
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
      split_exact<D>(g < X ? row[2 * g] : 0.0, e, S, out + r * Xpad + g, plane);
  }
}

// complex rows (z, i), i < R, K elements each -> planes [s][z][re/im][i][Kp]; one
// exponent per complex row, shared by its real and imaginary parts
template <int D>
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
      split_exact<D>(v.x, e, S, ore + k, plane);
      split_exact<D>(v.y, e, S, oim + k, plane);
    }
  }
}

int warp_grid(long rows);

// One-pass form of k_slice_cplx for rows of K <= 64 NP: each lane holds NP pairs of
// consecutive elements in registers (one read of the row), the warp takes the row
// exponent, and every digit plane is written as bfloat16 pairs (128-byte warp stores).
template <int NP, int D>
__global__ void __launch_bounds__(256, (NP <= 6 && D <= kFastSlices) ? 3 : 2) k_slice_cplx1(const double2* __restrict__ in, long rows,
                                                     int R, int K, int Kp, int S,
                                                     __nv_bfloat16* __restrict__ out,
                                                     int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = 2L * rows * Kp;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const double2* row = in + r * K;
    double2 v[NP][2];
    int m = 0;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      const int k = 2 * lane + 64 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        v[t][h] = k + h < K ? row[k + h] : make_double2(0.0, 0.0);
        m = max(m, max(exp_field(v[t][h].x), exp_field(v[t][h].y)));
      }
    }
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    if (lane == 0) eout[r] = e;
    const long z = r / R, i = r % R;
    __nv_bfloat16* ore = out + ((z * 2) * R + i) * Kp;
    __nv_bfloat16* oim = ore + (long)R * Kp;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      const int k = 2 * lane + 64 * t;
      if (k >= Kp) continue;
      float q0[D], q1[D];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        exact_digits_f<D>(part ? v[t][0].y : v[t][0].x, e, S, q0);
        exact_digits_f<D>(part ? v[t][1].y : v[t][1].x, e, S, q1);
        __nv_bfloat16* o = (part ? oim : ore) + k;
#pragma unroll
        for (int s = 0; s < D; ++s)
          if (s < S) *reinterpret_cast<__nv_bfloat162*>(o + s * plane) = digit_bf16x2(q0[s], q1[s]);
      }
    }
  }
}

// Taylor step of the split propagation, one pass over u_k (W x N x M, rows (z, j)):
// acc += i^k g_k u_k (FP64), then the digits of u_k for the next term -- or, after
// the last term (last != 0), the digits of the finished sum acc for the second
// one-body half.  kmod = k mod 4 selects the rotation i^k; kscale (M values, or NULL)
// scales element p of every row first (the diagonal of P in the first call).
template <int NP, int D>
__global__ void __launch_bounds__(256, (NP <= 6 && D <= kFastSlices) ? 3 : 2) k_taylor_slice(const double2* __restrict__ in,
                                                      double2* __restrict__ acc, long rows,
                                                      int R, int K, int Kp, int S, double gk,
                                                      int kmod, int last,
                                                      const double* __restrict__ kscale,
                                                      __nv_bfloat16* __restrict__ out,
                                                      __nv_bfloat16* __restrict__ nout,
                                                      int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long plane = 2L * rows * Kp, nplane = rows * Kp;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const double2* row = in + r * K;
    double2* arow = acc + r * K;
    double2 v[NP][2];
    int m = 0;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      const int k = 2 * lane + 64 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        double2 u = make_double2(0.0, 0.0);
        if (k + h < K) {
          u = row[k + h];
          // i^k u: multiply by i kmod times
          double2 w = u;
          if (kmod == 1) w = make_double2(-u.y, u.x);
          else if (kmod == 2) w = make_double2(-u.x, -u.y);
          else if (kmod == 3) w = make_double2(u.y, -u.x);
          if (kscale) {
            const double sc = kscale[k + h];
            w.x *= sc;
            w.y *= sc;
          }
          double2 a = arow[k + h];
          a.x = fma(gk, w.x, a.x);
          a.y = fma(gk, w.y, a.y);
          arow[k + h] = a;
          if (last) u = a;
        }
        v[t][h] = u;
        m = max(m, max(exp_field(u.x), exp_field(u.y)));
      }
    }
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    if (lane == 0) eout[r] = e;
    const long z = r / R, i = r % R;
    __nv_bfloat16* ore = out + ((z * 2) * R + i) * Kp;
    __nv_bfloat16* oim = ore + (long)R * Kp;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      const int k = 2 * lane + 64 * t;
      if (k >= Kp) continue;
      float q0[D], q1[D];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        exact_digits_f<D>(part ? v[t][0].y : v[t][0].x, e, S, q0);
        exact_digits_f<D>(part ? v[t][1].y : v[t][1].x, e, S, q1);
        __nv_bfloat16* o = (part ? oim : ore) + k;
#pragma unroll
        for (int s = 0; s < D; ++s)
          if (s < S) *reinterpret_cast<__nv_bfloat162*>(o + s * plane) = digit_bf16x2(q0[s], q1[s]);
        if (part && nout) {  // -Im digits [s][z][j][Kp] for the column-concatenated GEMM
          __nv_bfloat16* on = nout + r * Kp + k;
#pragma unroll
          for (int s = 0; s < D; ++s)
            if (s < S)
              *reinterpret_cast<__nv_bfloat162*>(on + s * nplane) = digit_bf16x2(-q0[s], -q1[s]);
        }
      }
    }
  }
}

// acc += i^k g_k u_k elementwise (the long-row form of k_taylor_slice's update; rows
// of K elements, element p scaled by kscale[p] when kscale is not NULL)
__global__ void k_taylor_acc(const double2* __restrict__ u, double2* __restrict__ acc, long n,
                             int K, double gk, int kmod, const double* __restrict__ kscale) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const double2 x = u[e];
    double2 w = x;
    if (kmod == 1) w = make_double2(-x.y, x.x);
    else if (kmod == 2) w = make_double2(-x.x, -x.y);
    else if (kmod == 3) w = make_double2(x.y, -x.x);
    if (kscale) {
      const double sc = kscale[e % K];
      w.x *= sc;
      w.y *= sc;
    }
    double2 a = acc[e];
    a.x = fma(gk, w.x, a.x);
    a.y = fma(gk, w.y, a.y);
    acc[e] = a;
  }
}

// Operands of theta = Phi S^-1 on the tensor cores, per unit u = (z, spin).
// A: row (u, p) holds Phi[z][p][off + k] over the spin's n columns k, zero-padded to
// Kt; one exponent per row shared by the real and imaginary parts; planes
// [s][u][re/im][p][Kt].  Each half-warp takes a row, two consecutive k per lane (Kt of
// 32 or 64), so every digit plane is written as 64-byte bfloat16-pair runs.
template <int D>
__global__ void k_slice_phi_theta(const double2* __restrict__ phi, int W, int M, int N, int na,
                                  int nb, int Kt, int S, __nv_bfloat16* __restrict__ out,
                                  int* __restrict__ eout) {
  const int lane = threadIdx.x & 31, hl = lane & 15;
  const unsigned hmask = (lane < 16) ? 0x0000FFFFu : 0xFFFF0000u;
  const long rows = 2L * W * M, plane = 2L * rows * Kt;
  const long hw0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const long nhw = ((long)gridDim.x * blockDim.x) >> 4;
  for (long r = hw0; r - (hw0 & 1) < rows; r += nhw) {  // both halves of a warp iterate alike
    const bool live = r < rows;
    const long rr = live ? r : rows - 1;
    const long u = rr / M;
    const int p = (int)(rr - u * M), sg = (int)(u & 1);
    const int n = sg ? nb : na, off = sg ? na : 0;
    const double2* row = phi + ((u >> 1) * M + p) * (long)N + off;
    double2 v[2][2];
    int m = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * hl + 32 * t + h;
        v[t][h] = k < n ? row[k] : make_double2(0.0, 0.0);
        m = max(m, max(exp_field(v[t][h].x), exp_field(v[t][h].y)));
      }
    const int e = row_exponent_field(__reduce_max_sync(hmask, m));
    if (live && hl == 0) eout[rr] = e;
    __nv_bfloat16* ore = out + ((u * 2) * M + p) * (long)Kt;
    __nv_bfloat16* oim = ore + (long)M * Kt;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int k = 2 * hl + 32 * t;
      if (!live || k >= Kt) continue;
      float r0[D], r1[D], i0[D], i1[D];
      exact_digits_f<D>(v[t][0].x, e, S, r0);
      exact_digits_f<D>(v[t][1].x, e, S, r1);
      exact_digits_f<D>(v[t][0].y, e, S, i0);
      exact_digits_f<D>(v[t][1].y, e, S, i1);
#pragma unroll
      for (int s = 0; s < D; ++s)
        if (s < S) {
          *reinterpret_cast<__nv_bfloat162*>(ore + s * plane + k) = digit_bf16x2(r0[s], r1[s]);
          *reinterpret_cast<__nv_bfloat162*>(oim + s * plane + k) = digit_bf16x2(i0[s], i1[s]);
        }
    }
  }
}

// B: row (u, j) holds S^-1[k][j] over k < n (the unit's spin; S^-1 is u's nmax x nmax
// block of sinv, [k][j]), zero-padded to Kt, rows j >= n zero; one exponent per row;
// planes [s][u][re/im][j][Kt] and the negated imaginary digits [s][u][j][Kt] (the
// second B region of the column-concatenated complex GEMM).
template <int D>
__global__ void k_slice_sinv(const double2* __restrict__ sinv, int W, int nmax, int na, int nb,
                             int Kt, int S, __nv_bfloat16* __restrict__ out,
                             __nv_bfloat16* __restrict__ nout, int* __restrict__ eout) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const long rows = 2L * W * nmax, plane = 2L * rows * Kt, nplane = rows * Kt;
  for (long r = (long)blockIdx.x * warps + (threadIdx.x >> 5); r < rows;
       r += (long)gridDim.x * warps) {
    const long u = r / nmax;
    const int j = (int)(r - u * nmax), n = (u & 1) ? nb : na;
    const double2* blk = sinv + u * (long)nmax * nmax;
    double2 v[2];
    int m = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      v[h] = k < n && j < n ? blk[(long)k * nmax + j] : make_double2(0.0, 0.0);
      m = max(m, max(exp_field(v[h].x), exp_field(v[h].y)));
    }
    const int e = row_exponent_field(__reduce_max_sync(0xffffffffu, m));
    if (lane == 0) eout[r] = e;
    __nv_bfloat16* ore = out + ((u * 2) * nmax + j) * (long)Kt;
    __nv_bfloat16* oim = ore + (long)nmax * Kt;
    __nv_bfloat16* onm = nout + r * Kt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      if (k >= Kt) continue;
      float qr[D], qi[D];
      exact_digits_f<D>(v[h].x, e, S, qr);
      exact_digits_f<D>(v[h].y, e, S, qi);
#pragma unroll
      for (int s = 0; s < D; ++s)
        if (s < S) {
          ore[s * plane + k] = digit_bf16(qr[s]);
          oim[s * plane + k] = digit_bf16(qi[s]);
          onm[s * nplane + k] = digit_bf16(-qi[s]);
        }
    }
  }
}

// Digits of complex rows (z, i) of K elements into planes [s][z][re/im][i][Kp]: the
// one-pass kernel for K <= 1024, else the two-pass one.
template <int D>
void slice_rows_d(const double2* in, long rows, int R, int K, int Kp, int S,
                  __nv_bfloat16* out, int* eout, cudaStream_t st) {
  const int g = warp_grid(rows);
  if (Kp <= 128)
    k_slice_cplx1<2, D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
  else if (Kp <= 256)
    k_slice_cplx1<4, D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
  else if (Kp <= 320)  // the row in as few registers as it needs: more warps per SM
    k_slice_cplx1<5, D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
  else if (Kp <= 384)
    k_slice_cplx1<6, D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
  else if (Kp <= 512)
    k_slice_cplx1<8, D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
  else
    k_slice_cplx<D><<<g, 256, 0, st>>>(in, rows, R, K, Kp, S, out, eout);
}

void slice_rows(const double2* in, long rows, int R, int K, int Kp, int S,
                __nv_bfloat16* out, int* eout, cudaStream_t st) {
  if (S <= kFastSlices)
    slice_rows_d<kFastSlices>(in, rows, R, K, Kp, S, out, eout, st);
  else
    slice_rows_d<kMaxSlices>(in, rows, R, K, Kp, S, out, eout, st);
}

// out[z] = in[z]^T for W complex R x C matrices (FP64; Phi -> Phi^T), through
// 32 x 32 shared-memory tiles so that reads and writes are both coalesced.
__global__ void __launch_bounds__(256) k_transpose_cplx(const double2* __restrict__ in, int W,
                                                        int R, int C, double2* __restrict__ out) {
  __shared__ double2 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int z = blockIdx.z; z < W; z += gridDim.z) {
    const double2* src = in + (long)z * R * C;
    double2* dst = out + (long)z * R * C;
    for (int k = ty; k < 32; k += 8)
      if (r0 + k < R && c0 + tx < C) t[k][tx] = src[(long)(r0 + k) * C + c0 + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8)
      if (c0 + k < C && r0 + tx < R) dst[(long)(c0 + k) * R + r0 + tx] = t[tx][k];
    __syncthreads();
  }
}

void transpose_cplx(const double2* in, int W, int R, int C, double2* out, cudaStream_t st) {
  const dim3 grid((C + 31) / 32, (R + 31) / 32, W < 65535 ? W : 65535);
  k_transpose_cplx<<<grid, dim3(32, 8), 0, st>>>(in, W, R, C, out);
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

// P -> its diagonal (FP64, pdiag) and the digits of its off-diagonal part O as rows p
// of K = M, padded to Mpad, with O's own row exponents (one warp per row)
__global__ void k_slice_poff(const double* __restrict__ P, int M, int Mpad, int S,
                             __nv_bfloat16* __restrict__ out, int* __restrict__ eout,
                             double* __restrict__ pdiag) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < M; p += gridDim.x * warps) {
    int m = 0;
    for (int q = lane; q < M; q += 32)
      if (q != p) m = max(m, exp_field(P[(long)p * M + q]));
    const int e = row_exponent_field(warp_max_int(m));
    if (lane == 0) {
      eout[p] = e;
      pdiag[p] = P[(long)p * M + p];
    }
    for (int q = lane; q < Mpad; q += 32) {
      const double v = (q < M && q != p) ? P[(long)p * M + q] : 0.0;
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
  for (auto** p : {&ctx->LT_sl, &ctx->Pm_sl, &ctx->y_sl, &ctx->A_sl, &ctx->T_sl[0], &ctx->T_sl[1],
                   &ctx->T_neg[0], &ctx->T_neg[1]})
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
  if (ctx->pdiag) cudaFree(ctx->pdiag);
  ctx->accT = nullptr;
  ctx->tout = nullptr;
  ctx->pdiag = nullptr;
}

// Once per trial: digits of L^T (the VHS operand) and of the off-diagonal part of P,
// with row exponents, and the diagonal of P.
// Digits per pass.  A Taylor power u_k = V u_{k-1} enters the sum scaled by
// g_k = dt^(k/2) / k!, so with x = sqrt(dt) |V|_2 the term is at most x^k / k! of Phi,
// and cutting both its operands to S exact digits costs about 2^-(8S-1) of the term.
// Each power gets the fewest digits that keep this below 2^-(8 Sp - 1) of Phi (the
// level of the leading term with Sp digits: 2^-31 with 4, 2^-55 with 7); the P passes
// keep all Sp.  |V|_2 is estimated at
// set-up by power iteration on V = sum_g y_g L_g for four seeded N(0,1) field draws,
// times 1.5 for the force-bias shift and the spread over walkers (a term whose x is
// twice the estimate still stays near 2^-30).
int prop_digit_schedule(afq_ctx* ctx) {
  const int M = ctx->M, X = ctx->X, n = ctx->p.taylor_order, Sp = ctx->Sp;
  const long MM = (long)M * M;
  constexpr int kDraws = 4;
  std::vector<double> y((size_t)kDraws * X), V((size_t)kDraws * MM);
  uint64_t st = 0x9E3779B97F4A7C15ull;  // splitmix64 stream, Box-Muller pairs
  auto uni = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (size_t i = 0; i < y.size(); i += 2) {
    const double r = std::sqrt(-2.0 * std::log(uni())), t = 6.283185307179586 * uni();
    y[i] = r * std::cos(t);
    if (i + 1 < y.size()) y[i + 1] = r * std::sin(t);
  }
  double *dy = nullptr, *dv = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&dy, y.size() * 8) != cudaSuccess ||
      cudaMalloc((void**)&dv, V.size() * 8) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "propagation digit schedule");
  if (rc == AFQ_OK && cudaMemcpyAsync(dy, y.data(), y.size() * 8, cudaMemcpyHostToDevice,
                                      ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "propagation digit schedule");
  // V_d = sum_g y_dg L_g: (kDraws x X) (X x M^2)
  if (rc == AFQ_OK)
    rc = launch_dgemm(ctx, kDraws, (int)MM, X, 1.0, dy, X, 1, 0, ctx->L, MM, 1, 0, 0.0, dv, MM, 1,
                      0, 1, 1);
  if (rc == AFQ_OK && (cudaMemcpyAsync(V.data(), dv, V.size() * 8, cudaMemcpyDeviceToHost,
                                       ctx->stream) != cudaSuccess ||
                       cudaStreamSynchronize(ctx->stream) != cudaSuccess))
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "propagation digit schedule");
  if (dy) cudaFree(dy);
  if (dv) cudaFree(dv);
  if (rc != AFQ_OK) return rc;
  double rho = 0.0;
  std::vector<double> v(M), w(M);
  for (int d = 0; d < kDraws; ++d) {
    const double* A = V.data() + (size_t)d * MM;
    for (int p = 0; p < M; ++p) v[p] = 1.0 + 0.01 * p;
    double lam = 0.0;
    for (int it = 0; it < 100; ++it) {
      double nv = 0.0;
      for (int p = 0; p < M; ++p) nv += v[p] * v[p];
      nv = std::sqrt(nv);
      if (!(nv > 0.0)) break;
      for (int p = 0; p < M; ++p) v[p] /= nv;
      for (int p = 0; p < M; ++p) {
        double s = 0.0;
        for (int q = 0; q < M; ++q) s += 0.5 * (A[(size_t)p * M + q] + A[(size_t)q * M + p]) * v[q];
        w[p] = s;
      }
      double r = 0.0;
      for (int p = 0; p < M; ++p) r += v[p] * w[p];
      lam = std::fabs(r);
      v.swap(w);
    }
    rho = std::fmax(rho, lam);
  }
  const double x = 1.5 * std::sqrt(ctx->p.dt) * rho;
  ctx->prop_x = x;
  if (n + 2 > (int)(sizeof(ctx->prop_digits) / sizeof(int)))
    return afq_fail(ctx, AFQ_ERR_ARG, "Taylor order too high for the split propagation");
  ctx->prop_digits[0] = ctx->prop_digits[n + 1] = Sp;
  double term = 1.0;
  for (int k = 1; k <= n; ++k) {
    term *= x / k;
    int S = Sp;
    if (std::isfinite(term) && term > 0.0) {
      S = (int)std::ceil((8.0 * Sp + std::log2(term)) / 8.0);
      if (S < 1) S = 1;
      if (S > Sp) S = Sp;
    }
    ctx->prop_digits[k] = S;
  }
  return AFQ_OK;
}

int mixed_prop_init_trial(afq_ctx* ctx) {
  const int S = ctx->Sp, M = ctx->M, X = ctx->X;
  ctx->Xpad = round_up(X, kBK);
  const long Mp = ctx->Mp;  // packed upper-triangle rows of L^T
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->LT_sl, (size_t)S * Mp * ctx->Xpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->Pm_sl, (size_t)S * M * ctx->Mpad * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_lt, (size_t)Mp * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_pm, (size_t)M * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->pdiag, (size_t)M * sizeof(double)));
  k_lt_exponents<<<grid1d(Mp), 256, 0, ctx->stream>>>(ctx->L, X, M, Mp, ctx->tpq, ctx->e_lt);
  AFQ_LAUNCHED(ctx);
  dim3 g((unsigned)((Mp + 31) / 32), (unsigned)((ctx->Xpad + 31) / 32));
  k_slice_LT<<<g, dim3(32, 8), 0, ctx->stream>>>(ctx->L, X, M, Mp, ctx->Xpad, S, ctx->tpq,
                                                 ctx->e_lt, ctx->LT_sl);
  AFQ_LAUNCHED(ctx);
  k_slice_poff<<<warp_grid(M), 256, 0, ctx->stream>>>(ctx->P, M, ctx->Mpad, S, ctx->Pm_sl,
                                                      ctx->e_pm, ctx->pdiag);
  AFQ_LAUNCHED(ctx);
  return prop_digit_schedule(ctx);
}

// Per walker set: operand buffers and tensor maps of the propagation.
int mixed_prop_init_walkers(afq_ctx* ctx) {
  const int S = ctx->Sp, M = ctx->M, N = ctx->N, W = ctx->ws.W, Mp = ctx->Mpad;
  for (auto** p : {&ctx->y_sl, &ctx->A_sl, &ctx->T_sl[0], &ctx->T_sl[1], &ctx->T_neg[0],
                   &ctx->T_neg[1]})
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
  // -Im digits of the operands (column-concatenated complex GEMMs)
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->T_neg[0], tbytes / 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->T_neg[1], tbytes / 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->accT, (size_t)W * N * M * sizeof(double2)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->tout, (size_t)W * N * M * sizeof(double2)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_y, (size_t)2 * W * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_a, (size_t)W * M * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_t[0], (size_t)W * N * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->e_t[1], (size_t)W * N * sizeof(int)));
  // tiles whose S digit accumulators fit the 512 TMEM columns: the VHS's BN <= 512 / S,
  // the propagation's 2 x prop_rows <= 512 / S (64 walker columns up to 4 digits)
  const int vhs_cap = (512 / S) / 16 * 16, rows_cap = (256 / S) / 16 * 16;
  ctx->vhs_BN = 2 * W >= vhs_cap ? (vhs_cap < 128 ? vhs_cap : 128) : round_up(2 * W, 16);
  ctx->prop_rows = N >= kPropRows ? kPropRows : round_up(N, 16);
  if (ctx->prop_rows > rows_cap) ctx->prop_rows = rows_cap;
  if (S * ctx->vhs_BN > 512 || 2 * S * ctx->prop_rows > 512)
    return afq_fail(ctx, AFQ_ERR_ARG, "split propagation: too many slices for TMEM");
  const uint32_t brows = (uint32_t)ctx->prop_rows;
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
    // the real P passes read A = O from L2 (one matrix for all walkers), so they
    // take half-width column tiles whose accumulators fit twice in TMEM (the epilogue
    // of one tile overlaps the MMAs of the next)
    ctx->prop_rows_real = ctx->prop_rows > 32 ? 32 : ctx->prop_rows;
    const uint32_t btr[4] = {kBK, (uint32_t)ctx->prop_rows_real, 1, 1};
    const uint64_t dtn[4] = {(uint64_t)Mp, (uint64_t)N, (uint64_t)W, (uint64_t)S};
    ctx->prop_rows_fused = fused_prop_rows(N);
    const uint32_t btf[4] = {kBK, (uint32_t)ctx->prop_rows_fused, 1, 1};
    ok = ok && make_tmap(&ctx->tm_pm, ctx->Pm_sl, 3, dp, bp) &&
         make_tmap(&ctx->tm_az, ctx->A_sl, 4, daz, baz) &&
         make_tmap(&ctx->tm_t[0], ctx->T_sl[0], 4, dt, bt) &&
         make_tmap(&ctx->tm_t[1], ctx->T_sl[1], 4, dt, bt) &&
         make_tmap(&ctx->tm_t_real[0], ctx->T_sl[0], 4, dt, btr) &&
         make_tmap(&ctx->tm_t_real[1], ctx->T_sl[1], 4, dt, btr) &&
         make_tmap(&ctx->tm_t_fused[0], ctx->T_sl[0], 4, dt, btf) &&
         make_tmap(&ctx->tm_t_fused[1], ctx->T_sl[1], 4, dt, btf);
    if (ctx->T_neg[0])
      ok = ok && make_tmap(&ctx->tm_tneg[0], ctx->T_neg[0], 4, dtn, btr) &&
           make_tmap(&ctx->tm_tneg[1], ctx->T_neg[1], 4, dtn, btr);
    else
      ctx->tm_tneg[0] = ctx->tm_tneg[1] = ctx->tm_t_real[0];  // unused
  }
  if (!ok) return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (propagation) failed");
  return AFQ_OK;
}

// V_z = sum_g y_zg L_g for every walker (FP64 into ctx->A), then its digits; the
// factor i sqrt(dt) of A_z = i sqrt(dt) V_z is applied by the Taylor epilogue.
int launch_vhs_tc(afq_ctx* ctx) {
  const int W = ctx->ws.W, M = ctx->M, S = ctx->Sp;
  if (S <= kFastSlices)
    k_slice_y<kFastSlices><<<warp_grid(2L * W), 256, 0, ctx->stream>>>(ctx->y, W, ctx->X,
                                                                      ctx->Xpad, S, ctx->y_sl,
                                                                      ctx->e_y);
  else
    k_slice_y<kMaxSlices><<<warp_grid(2L * W), 256, 0, ctx->stream>>>(ctx->y, W, ctx->X,
                                                                     ctx->Xpad, S, ctx->y_sl,
                                                                     ctx->e_y);
  AFQ_LAUNCHED(ctx);
  VhsP::Args a{};
  a.c.nkb = ctx->Xpad / kBK;
  a.c.BN = ctx->vhs_BN;
  a.c.tx_bytes = (uint32_t)S * (kBK * 128 * 2 + kBK * a.c.BN * 2);
  a.c.tmem_cols = tmem_cols_for(S * a.c.BN);
  a.c.err = ctx->flags + 2;
  a.c.per_pair = ctx->p.prop_kernel == 2;
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
  slice_rows(ctx->A, (long)W * M, M, M, ctx->Mpad, S, ctx->A_sl, ctx->e_a, ctx->stream);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

namespace {
int sm_count_prop() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int S, bool REAL, bool CAT, bool THETA = false>
cudaError_t launch_prop_s(int grid, size_t smem, cudaStream_t stream, const CUtensorMap& ta,
                          const CUtensorMap& tb, const CUtensorMap& tbn, const PropArgs& a) {
  cudaError_t e = raise_smem_limit((const void*)k_prop_tc<S, REAL, CAT, THETA>, smem);
  if (e != cudaSuccess) return e;
  k_prop_tc<S, REAL, CAT, THETA><<<grid, 32 * kPropWarps, smem, stream>>>(ta, tb, tbn, a);
  return cudaGetLastError();
}

// Whether a pass of S digits takes the column-concatenated form (the default per-pass
// kernel, whose S accumulators of prop_rows_real-wide tiles fit TMEM; complex passes
// also need the negated digits, written by the one-pass slicing kernel for rows up to
// 512).  Complex passes of 1 or 2 digits keep
// the per-pair form on 64-column tiles: their two accumulator sets fit there already,
// and 32-column tiles would read the A digits twice (measured slower: 133 -> 183 us
// per 2-digit pass at 290 orbitals; 3 digits 304 -> 238 us, 4 digits 400 -> 390 us).
bool prop_cat(const afq_ctx* ctx, int S, bool real) {
  return ctx->p.prop_kernel == 0 && 2 * S * ctx->prop_rows_real <= 512 &&
         (real || (S >= 3 && ctx->Mpad <= 512 && ctx->T_neg[0] != nullptr));
}

// One GEMM pass of the propagation (mode first / term / last) on operand buffer b.
template <bool REAL>
int launch_prop(afq_ctx* ctx, const CUtensorMap& ta, int b, const int* ea, int mode, int S) {
  PropArgs a{};
  const int N = ctx->N;
  a.M = ctx->M;
  a.N = N;
  a.W = ctx->ws.W;
  a.mode = mode;
  const bool cat = prop_cat(ctx, S, REAL);
  a.brows = REAL || cat ? ctx->prop_rows_real : ctx->prop_rows;
  a.BN = 2 * a.brows;
  a.nkb = ctx->Mpad / kBK;
  a.npt = (ctx->M + 127) / 128;
  a.njt = (N + a.brows - 1) / a.brows;
  a.ntiles = a.W * a.njt * a.npt;
  const int kUA = REAL ? 1 : 2, kUB = cat && !REAL ? 2 : 1;
  // a complex pass in the concatenated form whose K block fills less than two ring
  // stages takes two stages per K block (one A unit and one B region each): twice the
  // ring depth for the same bytes (measured at 290 orbitals with 7 digits: propagation
  // 8.64 -> 7.36 ms; at 4 digits, where two whole stages fit, 3.04 -> 3.09 ms, so not there)
  const size_t whole = (size_t)S * (kUA * (size_t)kASlot + (size_t)kUB * a.BN * 64);
  a.split = kUB == 2 && (kSmemLimit - 2048 - 1024) / whole < 2 ? 1 : 0;
  a.tx_bytes = a.split ? (uint32_t)S * (kBK * 128 * 2 + 2 * kBK * a.brows * 2)
                       : (uint32_t)S * (kUA * kBK * 128 * 2 + kUB * 2 * kBK * a.brows * 2);
  a.nbuf = 2 * S * a.BN <= 512 ? 2 : 1;
  a.tmem_cols = tmem_cols_for(a.nbuf * S * a.BN);
  a.ea = ea;
  a.eb = ctx->e_t[b];
  a.accT = ctx->accT;
  a.pdiag = ctx->pdiag;
  a.tout = ctx->tout;
  a.phi_out = ctx->ws.phi;
  a.err = ctx->flags + 2;
  const size_t stage = a.split ? (size_t)S * ((size_t)kASlot + (size_t)a.BN * 64)
                               : (size_t)S * (kUA * (size_t)kASlot + (size_t)kUB * a.BN * 64);
  int nst = (int)((kSmemLimit - 2048 - 1024) / stage);
  if (nst > kMaxStages) nst = kMaxStages;
  if (nst < 1 || S * a.BN > 512) return afq_fail(ctx, AFQ_ERR_ARG, "propagation tile does not fit");
  a.stages = nst;
  const size_t smem = stage * nst + 1024;
  const int grid = a.ntiles < sm_count_prop() ? a.ntiles : sm_count_prop();
  const CUtensorMap& tb = REAL || cat ? ctx->tm_t_real[b] : ctx->tm_t[b];
  const CUtensorMap& tbn = ctx->tm_tneg[b];
  cudaError_t e = cudaErrorInvalidValue;
  if (cat) {
    switch (S) {
      case 1: e = launch_prop_s<1, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 2: e = launch_prop_s<2, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 3: e = launch_prop_s<3, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 4: e = launch_prop_s<4, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 5: e = launch_prop_s<5, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 6: e = launch_prop_s<6, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 7: e = launch_prop_s<7, REAL, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
    }
  } else {
    switch (S) {
      case 1: e = launch_prop_s<1, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 2: e = launch_prop_s<2, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 3: e = launch_prop_s<3, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 4: e = launch_prop_s<4, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 5: e = launch_prop_s<5, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 6: e = launch_prop_s<6, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 7: e = launch_prop_s<7, REAL, false>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
    }
  }
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("propagate tc: ") + cudaGetErrorString(e));
  return AFQ_OK;
}

// acc += i^k g_k u_k and the digits of u_k (or of acc after the last term) into
// operand buffer b; rows longer than 512 take the two-kernel form
int taylor_slice(afq_ctx* ctx, int b, double gk, int kmod, int last, int S,
                 const double* kscale = nullptr, bool neg = false) {
  __nv_bfloat16* nout = neg ? ctx->T_neg[b] : nullptr;
  const int W = ctx->ws.W, N = ctx->N, M = ctx->M, Kp = ctx->Mpad;
  const long rows = (long)W * N;
  const int g = warp_grid(rows);
  const bool fast = S <= kFastSlices;
  if (Kp <= 128)
    (fast ? k_taylor_slice<2, kFastSlices> : k_taylor_slice<2, kMaxSlices>)<<<g, 256, 0, ctx->stream>>>(
        ctx->tout, ctx->accT, rows, N, M, Kp, S, gk, kmod, last, kscale, ctx->T_sl[b], nout, ctx->e_t[b]);
  else if (Kp <= 256)
    (fast ? k_taylor_slice<4, kFastSlices> : k_taylor_slice<4, kMaxSlices>)<<<g, 256, 0, ctx->stream>>>(
        ctx->tout, ctx->accT, rows, N, M, Kp, S, gk, kmod, last, kscale, ctx->T_sl[b], nout, ctx->e_t[b]);
  else if (Kp <= 320)  // the row in as few registers as it needs: more warps per SM
    (fast ? k_taylor_slice<5, kFastSlices> : k_taylor_slice<5, kMaxSlices>)<<<g, 256, 0, ctx->stream>>>(
        ctx->tout, ctx->accT, rows, N, M, Kp, S, gk, kmod, last, kscale, ctx->T_sl[b], nout, ctx->e_t[b]);
  else if (Kp <= 384)
    (fast ? k_taylor_slice<6, kFastSlices> : k_taylor_slice<6, kMaxSlices>)<<<g, 256, 0, ctx->stream>>>(
        ctx->tout, ctx->accT, rows, N, M, Kp, S, gk, kmod, last, kscale, ctx->T_sl[b], nout, ctx->e_t[b]);
  else if (Kp <= 512)
    (fast ? k_taylor_slice<8, kFastSlices> : k_taylor_slice<8, kMaxSlices>)<<<g, 256, 0, ctx->stream>>>(
        ctx->tout, ctx->accT, rows, N, M, Kp, S, gk, kmod, last, kscale, ctx->T_sl[b], nout, ctx->e_t[b]);
  else {
    k_taylor_acc<<<grid1d(rows * M), 256, 0, ctx->stream>>>(ctx->tout, ctx->accT, rows * M, M,
                                                            gk, kmod, kscale);
    AFQ_LAUNCHED(ctx);
    slice_rows(last ? ctx->accT : ctx->tout, rows, N, M, Kp, S, ctx->T_sl[b], ctx->e_t[b],
               ctx->stream);
  }
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// S digits of tout (W x N x M) into Taylor operand buffer b
int slice_tout(afq_ctx* ctx, int b, int S) {
  const int W = ctx->ws.W, N = ctx->N, M = ctx->M;
  slice_rows(ctx->tout, (long)W * N, N, M, ctx->Mpad, S, ctx->T_sl[b], ctx->e_t[b],
             ctx->stream);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
}  // namespace

// Phi <- P T_n(A) P Phi for every walker, A from the last launch_vhs_tc.  With
// A = i sqrt(dt) V the Taylor terms are t_k = i^k g_k u_k, g_k = dt^(k/2) / k!, and
// u_k = V u_{k-1} (u_0 = P Phi) runs on the tensor cores unscaled; the FP64 sum of the
// t_k is kept by the slicing passes.  With prop_kernel = 1 the cluster kernel of
// k_prop_fused.cu runs every pass in one launch instead (the same arithmetic).
int launch_propagate_tc(afq_ctx* ctx) {
  if (ctx->p.prop_kernel == 1) {
    const int rc = launch_propagate_fused(ctx);
    if (rc != -1) return rc;
  }
  const int W = ctx->ws.W;
  transpose_cplx(ctx->ws.phi, W, ctx->M, ctx->N, ctx->tout, ctx->stream);  // Phi^T
  AFQ_LAUNCHED(ctx);
  int cur = 0, rc;
  const int n = ctx->p.taylor_order;
  const int* dg = ctx->prop_digits;  // digits of each pass (prop_digit_schedule)
  if ((rc = slice_tout(ctx, cur, dg[0])) != AFQ_OK) return rc;
  // u_0 = P Phi = diag(P) Phi + O Phi, also the first term of the sum: the GEMM writes
  // O Phi into the sum, the slicing pass adds diag(P) Phi^T (Phi^T in tout) and cuts u_0
  rc = launch_prop<true>(ctx, ctx->tm_pm, cur, ctx->e_pm, kModeFirst, dg[0]);
  if (rc != AFQ_OK) return rc;
  cur = 1 - cur;
  // u_0 (or, with no Taylor terms, the sum for the last pass); a complex pass of the
  // column-concatenated form after it also takes the negated imaginary digits
  if ((rc = taylor_slice(ctx, cur, 1.0, 0, 1, dg[n >= 1 ? 1 : n + 1], ctx->pdiag,
                         n >= 1 && prop_cat(ctx, dg[1], false))) != AFQ_OK)
    return rc;
  double gk = 1.0;
  for (int k = 1; k <= n; ++k) {
    rc = launch_prop<false>(ctx, ctx->tm_az, cur, ctx->e_a, kModeTerm, dg[k]);
    if (rc != AFQ_OK) return rc;
    cur = 1 - cur;
    gk *= sqrt(ctx->p.dt) / k;
    if ((rc = taylor_slice(ctx, cur, gk, k & 3, k == n, dg[k + 1], nullptr,
                           k < n && prop_cat(ctx, dg[k + 1], false))) != AFQ_OK)
      return rc;
  }
  // Phi = P acc = diag(P) acc + O acc (written in place: a Phi^T output with a tiled
  // transpose after it measured 35 us slower per step at 290 orbitals)
  return launch_prop<true>(ctx, ctx->tm_pm, cur, ctx->e_pm, kModeLast, dg[n + 1]);
}

// ---------------------------------------------------------------------------
// theta = Phi S^-1 on the tensor cores (split-precision walker ensembles)
// ---------------------------------------------------------------------------
// theta_s = Phi_s S_s^-1 (Eq. halfgf) per unit u = (z, spin) is a complex product of
// Phi's M x n rows and the n x n inverse: the propagation kernel's form with K = n
// (one or two K blocks) and N = nmax columns, on exact digits of both operands (as
// many as the force bias and the exchange take; up to 4).  The double-float form on
// the FP32 pipe cost ~0.5 ms at 290 orbitals and 640 walkers.

void theta_tc_free(afq_ctx* ctx) {
  for (void* p : {(void*)ctx->th_a_sl, (void*)ctx->th_b_sl, (void*)ctx->th_bn_sl,
                  (void*)ctx->th_ea, (void*)ctx->th_eb, (void*)ctx->th_sinv})
    if (p) cudaFree(p);
  ctx->th_a_sl = ctx->th_b_sl = ctx->th_bn_sl = nullptr;
  ctx->th_ea = ctx->th_eb = nullptr;
  ctx->th_sinv = nullptr;
}

int theta_tc_init_walkers(afq_ctx* ctx) {
  theta_tc_free(ctx);
  const int W = ctx->ws.W, M = ctx->M;
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  const int hi = ctx->S > ctx->Sp ? ctx->S : ctx->Sp;
  // beyond 4 digits (FP64 quality) the double-float theta stays: the epilogue's int64
  // recombination of 5 to 7 digit orders takes two FP64 conversions per element and
  // one TMEM accumulator set, which measured slower at 290 orbitals (0.41 ms)
  if (nmax < 1 || nmax > 64 || hi > kFastSlices) return AFQ_OK;
  ctx->th_S = hi;
  ctx->th_K = round_up(nmax, kBK);
  ctx->th_brows = nmax >= 32 ? 32 : round_up(nmax, 16);
  const int S = ctx->th_S, Kt = ctx->th_K, brows = ctx->th_brows;
  const long units = 2L * W;
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_a_sl, (size_t)S * 2 * units * M * Kt * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_b_sl, (size_t)S * 2 * units * nmax * Kt * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_bn_sl, (size_t)S * units * nmax * Kt * 2));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_ea, (size_t)units * M * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_eb, (size_t)units * nmax * sizeof(int)));
  AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->th_sinv, (size_t)units * nmax * nmax * sizeof(double2)));
  const uint64_t da[4] = {(uint64_t)Kt, (uint64_t)M, (uint64_t)(2 * units), (uint64_t)S};
  const uint32_t ba[4] = {kBK, 128, 1, 1};
  const uint64_t db[4] = {(uint64_t)Kt, (uint64_t)nmax, (uint64_t)(2 * units), (uint64_t)S};
  const uint64_t dbn[4] = {(uint64_t)Kt, (uint64_t)nmax, (uint64_t)units, (uint64_t)S};
  const uint32_t bb[4] = {kBK, (uint32_t)brows, 1, 1};
  if (!make_tmap(&ctx->tm_tha, ctx->th_a_sl, 4, da, ba) ||
      !make_tmap(&ctx->tm_thb, ctx->th_b_sl, 4, db, bb) ||
      !make_tmap(&ctx->tm_thbn, ctx->th_bn_sl, 4, dbn, bb))
    return afq_fail(ctx, AFQ_ERR_CUDA, "cuTensorMapEncodeTiled (theta) failed");
  return AFQ_OK;
}

int launch_theta_tc(afq_ctx* ctx, WalkerSet& s) {
  const int W = s.W, M = ctx->M, N = ctx->N, na = ctx->na, nb = ctx->nb;
  const int nmax = na > nb ? na : nb, S = ctx->th_S, Kt = ctx->th_K;
  const long units = 2L * W;
  if (S < 1 || W != ctx->ws.W) return afq_fail(ctx, AFQ_ERR_STATE, "theta operands not set up");
  // the digits of S^-1 (B) and of Phi (A)
  if (S <= kFastSlices) {
    k_slice_sinv<kFastSlices><<<warp_grid(units * nmax), 256, 0, ctx->stream>>>(
        ctx->th_sinv, W, nmax, na, nb, Kt, S, ctx->th_b_sl, ctx->th_bn_sl, ctx->th_eb);
    AFQ_LAUNCHED(ctx);
    k_slice_phi_theta<kFastSlices><<<warp_grid(units * M), 256, 0, ctx->stream>>>(
        s.phi, W, M, N, na, nb, Kt, S, ctx->th_a_sl, ctx->th_ea);
  } else {
    k_slice_sinv<kMaxSlices><<<warp_grid(units * nmax), 256, 0, ctx->stream>>>(
        ctx->th_sinv, W, nmax, na, nb, Kt, S, ctx->th_b_sl, ctx->th_bn_sl, ctx->th_eb);
    AFQ_LAUNCHED(ctx);
    k_slice_phi_theta<kMaxSlices><<<warp_grid(units * M), 256, 0, ctx->stream>>>(
        s.phi, W, M, N, na, nb, Kt, S, ctx->th_a_sl, ctx->th_ea);
  }
  AFQ_LAUNCHED(ctx);
  PropArgs a{};
  a.M = M;
  a.N = nmax;
  a.W = (int)units;
  a.mode = kModeTheta;
  const bool cat = ctx->p.prop_kernel != 2 && 2 * S * ctx->th_brows <= 512;
  a.brows = ctx->th_brows;
  a.BN = 2 * a.brows;
  a.nkb = Kt / kBK;
  a.npt = (M + 127) / 128;
  a.njt = (nmax + a.brows - 1) / a.brows;
  a.ntiles = a.W * a.njt * a.npt;
  const int kUA = 2, kUB = cat ? 2 : 1;
  const size_t whole = (size_t)S * (kUA * (size_t)kASlot + (size_t)kUB * a.BN * 64);
  a.split = kUB == 2 && (kSmemLimit - 2048 - 1024) / whole < 2 ? 1 : 0;
  a.tx_bytes = a.split ? (uint32_t)S * (kBK * 128 * 2 + 2 * kBK * a.brows * 2)
                       : (uint32_t)S * (kUA * kBK * 128 * 2 + kUB * 2 * kBK * a.brows * 2);
  a.nbuf = 2 * S * a.BN <= 512 ? 2 : 1;
  a.tmem_cols = tmem_cols_for(a.nbuf * S * a.BN);
  a.ea = ctx->th_ea;
  a.eb = ctx->th_eb;
  a.tout = s.thetaT;
  a.err = ctx->flags + 2;
  a.na = na;
  a.nb = nb;
  a.Ntot = N;
  const size_t stage = a.split ? (size_t)S * ((size_t)kASlot + (size_t)a.BN * 64)
                               : (size_t)S * (kUA * (size_t)kASlot + (size_t)kUB * a.BN * 64);
  int nst = (int)((kSmemLimit - 2048 - 1024) / stage);
  if (nst > kMaxStages) nst = kMaxStages;
  if (nst < 1 || S * a.BN > 512) return afq_fail(ctx, AFQ_ERR_ARG, "theta tile does not fit");
  a.stages = nst;
  const size_t smem = stage * nst + 1024;
  const int grid = a.ntiles < sm_count_prop() ? a.ntiles : sm_count_prop();
  cudaError_t e = cudaErrorInvalidValue;
  const CUtensorMap &ta = ctx->tm_tha, &tb = ctx->tm_thb, &tbn = ctx->tm_thbn;
  if (cat) {
    switch (S) {
      case 1: e = launch_prop_s<1, false, true, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 2: e = launch_prop_s<2, false, true, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 3: e = launch_prop_s<3, false, true, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 4: e = launch_prop_s<4, false, true, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
    }
  } else {
    switch (S) {
      case 1: e = launch_prop_s<1, false, false, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 2: e = launch_prop_s<2, false, false, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 3: e = launch_prop_s<3, false, false, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
      case 4: e = launch_prop_s<4, false, false, true>(grid, smem, ctx->stream, ta, tb, tbn, a); break;
    }
  }
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("theta tc: ") + cudaGetErrorString(e));
  return AFQ_OK;
}
