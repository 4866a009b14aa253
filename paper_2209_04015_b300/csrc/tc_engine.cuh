// The split-precision tensor-core GEMM engine of libafqmc (sm_103a).
//
// Each FP64 operand x is split into S bfloat16 slices, x ~ x_0 + x_1 + ... + x_{S-1}
// (x_0 = bf16(x), x_k = bf16 of the remainder), and a product A B^T becomes the sum
// of the slice products A_s B_t^T with s + t <= S - 1, issued as tcgen05.mma (BF16 in,
// FP32 accumulate in TMEM), smallest terms first.
//
// k_tc_split is one kernel template for every contraction; a policy P supplies the
// tile coordinates, the TMA loads of its operand units, the MMAs of one stage and
// the epilogue.  A stage holds all S slices of P::kUA A units (128 rows x 32 K,
// 8 KB each) and P::kUB B units (BN rows x 32 K) of one K block, 64-byte swizzled.
// Roles in a 128-thread CTA: thread 0 issues the TMA loads into a ring of stages,
// thread 32 issues the MMAs and commits each stage back to the producer, and all
// four warps (one per 32 TMEM lanes) run the epilogue out of TMEM.  Every wait is
// bounded in time and by a grid-wide error flag, so a broken pipeline ends the
// kernel with an error instead of hanging.
#pragma once

#include <cudaTypedefs.h>

#include <string>

#include "afq_internal.cuh"
#include "tc_sm103.cuh"

namespace tce {

constexpr int kThreads = 128;
constexpr int kBK = 32;           // K elements per block: one 64-byte row
constexpr int kASlot = 128 * 64;  // bytes of one 128-row A unit of one K block
constexpr int kMaxStages = 4;
constexpr int kMaxSlices = 7;  // 7 exact 8-bit digits: 55 bits, FP64 quality
constexpr int kFastSlices = 4;  // digit loop bound of the per-step slicing kernels when S <= 4
constexpr size_t kSmemLimit = 227 * 1024;

struct TcCommon {
  int nkb;            // K blocks of a full K range
  int BN;             // MMA N (multiple of 16, <= 256)
  uint32_t tx_bytes;  // bytes the TMA loads of one stage deliver
  uint32_t tmem_cols;
  int stages;         // ring depth, 1..kMaxStages
  int* err;           // grid-wide error flag: set to 1 when a pipeline wait gives up
  int per_pair;       // 1: one MMA per digit pair (issue_diagonals), else issue_split's
                      // column-concatenated form; the two give the same bits
};

// Slice pairs (s, t) with s + t <= S - 1, from the smallest contributions up.
template <int S>
__device__ __forceinline__ void slice_pair(int k, int& s, int& t) {
  int idx = 0;
#pragma unroll
  for (int d = S - 1; d >= 0; --d)
#pragma unroll
    for (int ss = d; ss >= 0; --ss) {
      if (idx == k) {
        s = ss;
        t = d - ss;
      }
      ++idx;
    }
}

// Shared-memory byte address of A unit u, slice s (and the same for B).
__device__ __forceinline__ uint32_t a_unit(uint32_t sa, int S, int u, int s) {
  return sa + (uint32_t)(u * S + s) * kASlot;
}
__device__ __forceinline__ uint32_t b_unit(uint32_t sb, uint32_t bslot, int S, int u, int s) {
  return sb + (uint32_t)(u * S + s) * bslot;
}

// The MMAs of one stage for one A unit and one B unit into one accumulator.
template <int S>
__device__ __forceinline__ void issue_pairs(uint32_t acc, uint32_t sa, uint32_t sb, uint32_t bslot,
                                            int ua, int ub, uint32_t idesc, bool first) {
#pragma unroll
  for (int k = 0; k < S * (S + 1) / 2; ++k) {
    int s = 0, t = 0;
    slice_pair<S>(k, s, t);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
      tc::mma_bf16(acc, tc::sdesc_k64(a_unit(sa, S, ua, s) + ks * 32),
                   tc::sdesc_k64(b_unit(sb, bslot, S, ub, t) + ks * 32), idesc,
                   !(first && k == 0 && ks == 0));
  }
}

// Head-and-tail form for scaled digits (split_scaled): the leading pair (0, 0) goes to
// accumulator acc_head (exact), every other pair with s + t <= S - 1 to acc_tail.
template <int S>
__device__ __forceinline__ void issue_head_tail(uint32_t acc_head, uint32_t acc_tail, uint32_t sa,
                                                uint32_t sb, uint32_t bslot, uint32_t idesc,
                                                bool first) {
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
    tc::mma_bf16(acc_head, tc::sdesc_k64(a_unit(sa, S, 0, 0) + ks * 32),
                 tc::sdesc_k64(b_unit(sb, bslot, S, 0, 0) + ks * 32), idesc, !(first && ks == 0));
  bool lead = true;
#pragma unroll
  for (int d = 1; d < S; ++d)
#pragma unroll
    for (int s = 0; s <= d; ++s)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        tc::mma_bf16(acc_tail, tc::sdesc_k64(a_unit(sa, S, 0, s) + ks * 32),
                     tc::sdesc_k64(b_unit(sb, bslot, S, 0, d - s) + ks * 32), idesc,
                     !(first && lead));
        lead = false;
      }
}

// Exact-diagonal form: pair (s, d - s) goes to accumulator d (acc0 + d * stride
// columns).  With integer slices (split_exact) every accumulator holds a sum of
// integer products, exact in FP32 while its magnitude stays below 2^24 (balanced
// random-sign digits keep typical sums far below; a larger sum is rounded like any
// FP32 sum of that diagonal), and the diagonals are combined in FP64 afterwards.
template <int S>
__device__ __forceinline__ void issue_diagonals(uint32_t acc0, uint32_t stride, uint32_t sa,
                                                uint32_t sb, uint32_t bslot, int ua, int ub,
                                                uint32_t idesc, bool first) {
#pragma unroll
  for (int d = 0; d < S; ++d)
#pragma unroll
    for (int s = 0; s <= d; ++s)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(acc0 + (uint32_t)d * stride, tc::sdesc_k64(a_unit(sa, S, ua, s) + ks * 32),
                     tc::sdesc_k64(b_unit(sb, bslot, S, ub, d - s) + ks * 32), idesc,
                     !(first && s == 0 && ks == 0));
}

// Column-concatenated form of the exact-diagonal issue (one A unit, one B unit whose S
// digit slots of BN rows lie one after another, accumulators BN columns apart): A digit
// s times B digits t0 .. t0 + nt - 1 is ONE MMA of nt BN columns (N <= 256) landing in
// accumulators s + t0 .. -- per K step about S + S / (256 / BN) MMAs instead of
// S (S + 1) / 2, each A digit read from shared memory once per MMA instead of once per
// pair.  Every accumulator receives the same digit products as in issue_diagonals, and
// their sums are exact integers, so the results are the same bits.
template <int S>
__device__ __forceinline__ void issue_diagonals_cat(uint32_t acc0, int BN, uint32_t sa,
                                                    uint32_t sb, uint32_t bslot, bool first) {
  const int tmax = 256 / BN;  // B slots per MMA
#pragma unroll
  for (int s = 0; s < S; ++s)
    for (int t0 = 0; t0 < S - s; t0 += tmax) {
      const int nt = S - s - t0 < tmax ? S - s - t0 : tmax;
      const uint32_t idesc = tc::idesc_bf16(128, nt * BN);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
        tc::mma_bf16(acc0 + (uint32_t)((s + t0) * BN),
                     tc::sdesc_k64(a_unit(sa, S, 0, s) + ks * 32),
                     tc::sdesc_k64(b_unit(sb, bslot, S, 0, t0) + ks * 32), idesc,
                     !(first && s == 0 && ks == 0));
    }
}

// The exact-diagonal issue of a policy with one A and one B unit: column-concatenated
// for tiles of up to 64 columns (measured at 290 orbitals with 7 digits: VHS 5.22 ->
// 4.32 ms, stored exchange 4.51 -> 3.48, force bias 2.28 -> 1.92), per pair for wider
// ones (128-column tiles at 4 digits measured 1-2% slower concatenated) or when the
// launch asks for it.
template <int S>
__device__ __forceinline__ void issue_split(const TcCommon& c, uint32_t acc0, uint32_t sa,
                                            uint32_t sb, uint32_t bslot, bool first) {
  if (c.per_pair || c.BN > 64)
    issue_diagonals<S>(acc0, (uint32_t)c.BN, sa, sb, bslot, 0, 0, tc::idesc_bf16(128, c.BN),
                       first);
  else
    issue_diagonals_cat<S>(acc0, c.BN, sa, sb, bslot, first);
}

// Biased exponent field of a double (0 for zero and subnormals).  On B300 the
// FP64 pipe is ~64x slower than the integer pipe, so the row scales, the digits and
// the recombination below are done on the bits with integer instructions.
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// Row exponent e with |x| <= 2^e for a row whose largest exponent field is emax.
__device__ __forceinline__ int row_exponent_field(int emax) { return emax ? emax - 1022 : 0; }


// The same digits returned in q[0..S-1] (q[s] = digit of weight 256^-s; S <= D).
template <int D>
__device__ __forceinline__ void exact_digits(double x, int e, int S, int (&q)[D]) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long v = 0;
  if (E != 0) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = E - 1075 + 7 - e + 8 * (S - 1);
    if (sh >= 0)
      v = sh < 10 ? mant << sh : 0;
    else if (sh > -64)
      v = (mant + (1LL << (-sh - 1))) >> (-sh);
  }
  const bool neg = bits < 0;
#pragma unroll
  for (int s = D - 1; s >= 0; --s) {
    q[s] = 0;
    if (s >= S) continue;
    int d = (int)(v & 255);
    if (d > 128) d -= 256;
    q[s] = neg ? -d : d;
    v = (v - d) >> 8;
  }
}

// The same digits returned as exact floats (q[s] = digit of weight 256^-s, S <= D),
// cut without integer <-> float conversions and with 32-bit arithmetic when D <= 4:
// v = round(|x| 2^(7 - e + 8 (S - 1))) as before; adding 127 to each of the S - 1 low
// bytes of v (w = v + 0x7F...7F) turns the balanced digits in [-127, 128] into the
// plain bytes of w (digit = byte - 127, the top digit = the top byte), and a byte
// permute places byte k of w under the exponent of 2^23, so that one FMA gives
// sign(x) (byte - 127).  The slicing passes that cut every walker's operands each step
// were bound by the integer pipe with the shift-and-mask loop and the conversions.
template <int D>
__device__ __forceinline__ void exact_digits_f(double x, int e, int S, float (&q)[D]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32);
  const int E = (int)((hi >> 20) & 0x7FF);
  const int r = 1068 + e - 8 * (S - 1) - E;  // v = round(mant 2^-r), mant = 1.m 2^52
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const float sg = (int)hi < 0 ? -1.f : 1.f;
  const float ctop = -8388608.f * sg, clow = -8388735.f * sg;  // -(2^23) and -(2^23 + 127)
  if constexpr (D <= 4) {
    unsigned v = 0;  // |x| < 2^e: r >= 22, so v <= 2^31 (2^31 only by rounding up)
    if (E != 0 && r > 0 && r < 54) {
      const unsigned t = (unsigned)(mant >> (r - 1));  // v = (t + 1) / 2 without overflow
      v = (t >> 1) + (t & 1u);
    }
    const unsigned w = v + (0x7F7F7Fu >> (8 * (4 - S)));
#pragma unroll
    for (int s = 0; s < D; ++s) {
      q[s] = 0.f;
      if (s >= S) continue;
      const unsigned b = __byte_perm(w, 0x4B000000u, 0x7440u | (unsigned)(S - 1 - s));
      q[s] = fmaf(__uint_as_float(b), sg, s == 0 ? ctop : clow);
    }
  } else {
    unsigned long long v = 0;
    if (E != 0) {
      if (r <= 0)
        v = r > -10 ? mant << (-r) : 0;
      else if (r < 54)
        v = ((mant >> (r - 1)) + 1ull) >> 1;
    }
    const unsigned long long w = v + (0x7F7F7F7F7F7F7Full >> (8 * (8 - S)));
    const unsigned wl = (unsigned)w, wh = (unsigned)(w >> 32);
#pragma unroll
    for (int s = 0; s < D; ++s) {
      q[s] = 0.f;
      if (s >= S) continue;
      const int k = S - 1 - s;
      const unsigned b = __byte_perm(k < 4 ? wl : wh, 0x4B000000u, 0x7440u | (unsigned)(k & 3));
      q[s] = fmaf(__uint_as_float(b), sg, s == 0 ? ctop : clow);
    }
  }
}

// bfloat16 of an exact digit float (at most 8 significant bits: its low 16 bits are
// zero) and of a pair of them, by moving bits
__device__ __forceinline__ __nv_bfloat16 digit_bf16(float f) {
  return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}
__device__ __forceinline__ __nv_bfloat162 digit_bf16x2(float lo, float hi) {
  const unsigned u = __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632u);
  return *reinterpret_cast<const __nv_bfloat162*>(&u);
}

// Integer digits of x relative to the row scale 2^e (|x| <= 2^e):
// x ~ 2^(e-7) sum_s q_s 256^-s with balanced digits q_s in [-128, 128] (exact in
// bfloat16), written S planes apart.  Rounds x 2^(7-e+8(S-1)) to the nearest
// integer and cuts it into base-256 digits.  D >= S bounds the unrolled digit loops:
// the per-step slicing kernels take D = kFastSlices when S <= 4, so that the digit
// counts beyond 4 cost them neither registers nor instructions.
template <int D = kMaxSlices>
__device__ __forceinline__ void split_exact(double x, int e, int S, __nv_bfloat16* out,
                                            long plane) {
  float q[D];
  exact_digits_f<D>(x, e, S, q);
#pragma unroll
  for (int s = 0; s < D; ++s)
    if (s < S) out[s * plane] = digit_bf16(q[s]);
}

// Scaled digits: the same digits as exact_digits, each written as its value
// q_s 2^(e - 7 - 8 s) (exact in bfloat16: an 8-bit integer times a power of two), S
// planes apart.  Products of scaled digits land at their true weights, so a GEMM over
// them can keep the leading product (0, 0) -- a sum of integer multiples of one power
// of two, exact in FP32 -- in one accumulator and every smaller product in another,
// whose FP32 rounding then only touches digits ~2^-8 below the leading ones.
template <int D = kMaxSlices>
__device__ __forceinline__ void split_scaled(double x, int e, int S, __nv_bfloat16* out,
                                             long plane) {
  int q[D];
  exact_digits<D>(x, e, S, q);
#pragma unroll
  for (int s = 0; s < D; ++s)
    if (s < S) out[s * plane] = __float2bfloat16_rn(ldexpf((float)q[s], e - 7 - 8 * s));
}

// Recombines the S exact diagonal accumulators of one element:
// value = 2^scale_exp sum_d acc_d 256^-d, through one int64 and one conversion for
// S <= 4; for more digits (whose weighted sum would overflow an int64) through two:
// the leading S - 3 diagonals and the last 3, each exact in FP64, added once.
__device__ __forceinline__ double ll_scaled(long long t, int e) {
  if (t == 0) return 0.0;
  return __longlong_as_double(__double_as_longlong(__ll2double_rn(t)) + ((long long)e << 52));
}
template <int S>
__device__ __forceinline__ double combine_exact(const float (&acc)[S], int scale_exp) {
  if constexpr (S <= 4) {
    long long t = 0;
#pragma unroll
    for (int d = 0; d < S; ++d) t += (long long)__float2int_rn(acc[d]) * (1LL << (8 * (S - 1 - d)));
    if (t == 0) return 0.0;
    const double v = __ll2double_rn(t);
    return __longlong_as_double(__double_as_longlong(v) +
                                ((long long)(scale_exp - 8 * (S - 1)) << 52));
  } else {
    constexpr int H = S - 3;
    long long hi = 0, lo = 0;
#pragma unroll
    for (int d = 0; d < H; ++d) hi += (long long)__float2int_rn(acc[d]) * (1LL << (8 * (H - 1 - d)));
#pragma unroll
    for (int d = H; d < S; ++d) lo += (long long)__float2int_rn(acc[d]) * (1LL << (8 * (S - 1 - d)));
    return ll_scaled(hi, scale_exp - 8 * (H - 1)) + ll_scaled(lo, scale_exp - 8 * (S - 1));
  }
}

__device__ __forceinline__ void tmem_row16(uint32_t tmem, int warp, int c0, float (&v)[16]) {
  tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
}

// Split x into S bfloat16 slices written S planes apart.
__device__ __forceinline__ void split_bf16(double x, int S, __nv_bfloat16* out, long plane) {
  double r = x;
  for (int s = 0; s < S; ++s) {
    const __nv_bfloat16 h = __double2bfloat16(r);
    out[s * plane] = h;
    r -= (double)__bfloat162float(h);
  }
}

template <int S, class P>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_split(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const typename P::Args args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  __shared__ int skip;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const typename P::Tile t = P::tile(args);
  const int BN = args.c.BN, nst = args.c.stages;
  const uint32_t bslot = (uint32_t)BN * 64u;
  const uint32_t stage_bytes = S * (P::kUA * kASlot + P::kUB * bslot);
  int* err = args.c.err;
  // another CTA already failed: do nothing (decided once for the whole CTA, before
  // any barrier or TMEM is set up)
  if (threadIdx.x == 0) skip = *(const volatile int*)err;
  __syncthreads();
  if (skip) return;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    fail = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, args.c.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int nkb = t.kb1 - t.kb0;

  if (threadIdx.x == 0) {
    // TMA producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int st = i % nst;
      if (i >= nst && !tc::mbar_wait(&empty[st], ((i / nst) - 1) & 1, err)) {
        fail = 1;
        atomicExch(err, 1);
        break;
      }
      tc::mbar_arrive_expect_tx(&full[st], args.c.tx_bytes);
      uint8_t* sa = smem + st * stage_bytes;
      uint8_t* sb = sa + S * P::kUA * kASlot;
      const int kb = t.kb0 + i;
#pragma unroll
      for (int u = 0; u < P::kUA; ++u)
#pragma unroll
        for (int s = 0; s < S; ++s)
          P::load_a(&tmA, sa + (u * S + s) * kASlot, args, t, u, s, kb, &full[st]);
#pragma unroll
      for (int u = 0; u < P::kUB; ++u)
#pragma unroll
        for (int s = 0; s < S; ++s)
          P::load_b(&tmB, sb + (u * S + s) * bslot, args, t, u, s, kb, &full[st]);
      ++issued;
    }
    // no TMA write may still be in flight when the CTA moves on
    for (int i = issued > nst ? issued - nst : 0; i < issued; ++i)
      tc::mbar_wait(&full[i % nst], (i / nst) & 1, err);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    for (int i = 0; i < nkb; ++i) {
      const int st = i % nst;
      if (!tc::mbar_wait(&full[st], (i / nst) & 1, err)) {
        fail = 1;
        atomicExch(err, 1);
        break;
      }
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
      const uint32_t sb = sa + S * P::kUA * kASlot;
      P::template issue<S>(args, tmem, sa, sb, bslot, i == 0);
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(&done);
  }
  bool ok = tc::mbar_wait(&done, 0, err);
  // the MMAs already issued must finish before TMEM is read or freed: wait again,
  // bounded by time only
  if (!ok) {
    static const int zero = 0;
    ok = tc::mbar_wait(&done, 0, &zero);
  }
  if (!ok) fail = 1;
  tc::fence_after_sync();
  __syncthreads();
  const bool bad = fail != 0;
  __syncwarp();
  if (bad) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    P::template epilogue<S>(args, t, tmem, smem, warp, lane);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, args.c.tmem_cols);
}

// ---------------------------------------------------------------------------- host
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

// BF16 tensor map with the 64-byte swizzle over a dense array; dims[0] is the
// contiguous K axis (its byte size must be a multiple of 16).
inline bool make_tmap(CUtensorMap* tm, const void* base, int rank, const uint64_t* dims,
                      const uint32_t* box) {
  auto fn = encode_fn();
  if (!fn || rank < 1 || rank > 5) return false;
  cuuint64_t gdim[5], gstride[4];
  cuuint32_t bdim[5], estr[5];
  uint64_t stride = 2;
  for (int i = 0; i < rank; ++i) {
    gdim[i] = dims[i];
    bdim[i] = box[i];
    estr[i] = 1;
    if (i > 0) gstride[i - 1] = stride;
    stride *= dims[i];
  }
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), gdim, gstride,
            bdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline uint32_t tmem_cols_for(int cols) {
  uint32_t c = 32;
  while (c < (uint32_t)cols) c <<= 1;
  return c;
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Column tile for `cols` GEMM columns with S TMEM accumulators of BN columns each
// (S BN <= 512, BN a multiple of 16, <= cap): the fewest tiles (wider tiles re-read
// A less often), and among tilings with that count the narrowest (least padding).
inline int pick_bn(int cols, int S, int cap) {
  int hi = 512 / (S > 0 ? S : 1);
  if (hi > cap) hi = cap;
  hi -= hi % 16;
  if (hi < 16) hi = 16;
  const int tiles = (cols + hi - 1) / hi;
  return round_up((cols + tiles - 1) / tiles, 16);
}

// Ring depth and dynamic shared memory for a policy shape; stages = 0 if even one
// stage does not fit.
inline void plan_smem(int S, int kUA, int kUB, int BN, size_t epilogue_bytes, int* stages,
                      size_t* smem) {
  const size_t stage = (size_t)S * (kUA * (size_t)kASlot + kUB * (size_t)BN * 64);
  int n = (int)((kSmemLimit - 2048) / stage);
  if (n > 3) n = 3;
  *stages = n < 1 ? 0 : n;
  const size_t pipe = stage * (size_t)(*stages);
  *smem = (pipe > epilogue_bytes ? pipe : epilogue_bytes) + 1024;
}

template <int S, class P>
cudaError_t launch_tc(dim3 grid, size_t smem, cudaStream_t stream, const CUtensorMap& a,
                      const CUtensorMap& b, const typename P::Args& args) {
  // raised only when it grows, so that no attribute call is issued while a graph is
  // being captured after a first ordinary step
  cudaError_t e = raise_smem_limit((const void*)k_tc_split<S, P>, smem);
  if (e != cudaSuccess) return e;
  k_tc_split<S, P><<<grid, kThreads, smem, stream>>>(a, b, args);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_tc_s(int S, dim3 grid, size_t smem, cudaStream_t stream, const CUtensorMap& a,
                        const CUtensorMap& b, const typename P::Args& args) {
  if (args.c.stages < 1 || args.c.stages > kMaxStages || smem > kSmemLimit)
    return cudaErrorInvalidValue;
  switch (S) {
    case 1: return launch_tc<1, P>(grid, smem, stream, a, b, args);
    case 2: return launch_tc<2, P>(grid, smem, stream, a, b, args);
    case 3: return launch_tc<3, P>(grid, smem, stream, a, b, args);
    case 4: return launch_tc<4, P>(grid, smem, stream, a, b, args);
    case 5: return launch_tc<5, P>(grid, smem, stream, a, b, args);
    case 6: return launch_tc<6, P>(grid, smem, stream, a, b, args);
    case 7: return launch_tc<7, P>(grid, smem, stream, a, b, args);
  }
  return cudaErrorInvalidValue;
}

inline int grid1d(long n) {
  long g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 148 * 32 ? 148 * 32 : g));
}

}  // namespace tce
