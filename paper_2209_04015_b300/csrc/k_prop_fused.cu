// The split-precision propagation Phi_z <- P T_n(A_z) P Phi_z (the walker update of
// Sec. "Review of AFQMC", A_z = i sqrt(dt) V_z) as ONE persistent kernel of
// thread-block clusters: all n + 2 GEMM passes of a walker run back to back inside a
// cluster, and each pass's epilogue cuts the exact digits of the next pass's operand
// itself.
//
// Why clusters.  A digit's scale is a power of two per operand row (walker column j,
// over all orbitals p), and the rows p of one walker span ceil(M / 128) CTAs (the
// 128-row MMA tiles).  The CTAs of one walker form a cluster: each epilogue takes the
// exponent maxima over its own rows, sends them to every peer's shared memory
// (distributed shared memory) and, once all have arrived, cuts its rows of the next
// operand into the digit planes that the next pass loads by TMA.  So no pass leaves
// the chip for a separate slicing launch, the per-step digit planes stay in L2, and
// V_z -- read by the n Taylor passes -- is fetched from HBM once per walker and
// re-read from L2.
//
// Two chains per CTA.  The passes of one column tile are a chain of dependent steps
// (MMAs, then the epilogue and the cluster exchange, then the next MMAs).  Each CTA
// therefore runs two independent chains -- two 32-column tiles of a walker (sharing
// its V_z in L2), or two walkers -- with an accumulator set each in TMEM, interleaved
// pass by pass: the epilogue of one chain (FP64 work, exchange, digit cutting) runs
// while the tensor core works on the other.
//
// Per CTA (one 128-row slab p0..p0+127 of its walkers, brows columns per chain):
//   warp 0    TMA producer: per pass and chain, once the cluster has published the
//             chain's operand (an mbarrier that every CTA of the cluster arrives on),
//             the digit tiles of A (O = P off its diagonal, or V_z) and of the operand
//             into a ring;
//   warp 1    MMA issuer (tcgen05, exact digit diagonals in TMEM, as the per-pass
//             kernel) and TMEM owner;
//   warps 2-9 epilogue: the digits recombined to FP64, the FP64 work of the pass (the
//             first half applies diag(P) to Phi, the Taylor passes add i^k g_k u_k to
//             the FP64 sum, the last half writes Phi), the next operand's exponent
//             exchange and its digits.
// Measured on B300 at 290 orbitals, 52 electrons and 640 walkers it takes about twice
// the per-pass path's time: each chain-pass epilogue (two loads from L2, the FP64
// recombination and Taylor update, the cluster exchange and the digit cutting) is
// latency-bound at ~25 us against ~5 us of arithmetic, and with the Taylor sum in L2
// (neither registers, shared memory nor TMEM can hold it next to the ring and the
// accumulators) two chains do not hide it.  It is kept as the option prop_kernel = 1.
// The arithmetic is the per-pass path's, operation for operation (the same digits,
// exponents, recombination and FP64 updates in the same order), so both give the same
// bits.  Every wait is bounded (time, or the grid-wide error flag); every CTA reaches
// the closing cluster barrier, so no CTA leaves while a peer may still write into its
// shared memory.
#include <cmath>

#include "tc_engine.cuh"

using namespace tce;

namespace {

constexpr int kFWarps = 10;
constexpr int kFEpi = 8;
constexpr int kMaxCluster = 8;  // 128-row slabs per walker: M <= 1024
constexpr int kMaxPasses = 10;  // taylor_order + 2
constexpr int kFBrows = 32;     // walker columns per chain (two accumulator sets fit TMEM)
constexpr int kChains = 2;

struct FusedArgs {
  int M, N, W, Mpad, brows, BN, nkb, npt, njt, nunits, npairs, npass, stages, n;
  int dg[kMaxPasses];     // digits of each pass's operands (pass 0: also Phi's digits)
  double gk[kMaxPasses];  // g_k = dt^(k/2) / k! of Taylor pass k
  uint32_t tmem_cols, set_cols, stage_bytes;
  const int* ea_o;        // row exponents of O per p
  const int* ea_v;        // row exponents of V_z per (z, p)
  const double* pdiag;    // diagonal of P
  double2* phi;           // W x M x N
  double2* accT;          // W x N x M FP64 Taylor sum
  double2* tout;          // W x N x M FP64 next-operand values
  __nv_bfloat16* tsl[2];  // operand digit planes [s][2W][N][Mpad], by round parity
  int* err;
};

// The chain's unit (walker z, first column j0) in pair `pair`; false when empty.
__device__ __forceinline__ bool chain_unit(const FusedArgs& a, int pair, int c, int* z, int* j0) {
  const int u = 2 * pair + c;
  if (u >= a.nunits) return false;
  *z = u / a.njt;
  *j0 = (u - *z * a.njt) * a.brows;
  return true;
}

__device__ __forceinline__ void fused_epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kFEpi * 32) : "memory");
}

// Epilogue of one GEMM pass with S digits (mode 0: first half, 1: Taylor term k,
// 2: last half) for this thread's row p and 8 columns c0..c0+7: the pass's FP64 work,
// the next operand's values into tout and their exponent maxima into ex_loc.  The
// global operands are loaded before the TMEM digits, and all TMEM loads of a part
// (real, imaginary) are in flight together.
template <int S>
__device__ __forceinline__ void epi_pass8(const FusedArgs& a, int mode, int k, int z, int j0, int p,
                                          bool valid, int ea, const int* eb, uint32_t trow, int c0,
                                          int lane, int* ex_loc) {
  const int M = a.M, N = a.N, brows = a.brows;
  double2 g[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = j0 + c0 + jj;
    g[jj] = make_double2(0.0, 0.0);
    if (valid && j < N)
      g[jj] = mode == 0 ? a.phi[((long)z * M + p) * N + j] : a.accT[((long)z * N + j) * M + p];
  }
  uint32_t r[S][8];
  double dre[8];
#pragma unroll
  for (int d = 0; d < S; ++d) tc::tmem_ld8_nowait(trow + (uint32_t)(d * a.BN + c0), r[d]);
  tc::tmem_wait_ld();
#pragma unroll
  for (int d = 0; d < S; ++d) tc::tmem_regs_ready8(r[d]);
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = j0 + c0 + jj;
    float ar[S];
#pragma unroll
    for (int d = 0; d < S; ++d) ar[d] = __uint_as_float(r[d][jj]);
    dre[jj] = (valid && j < N) ? combine_exact<S>(ar, ea + eb[c0 + jj] - 14) : 0.0;
  }
#pragma unroll
  for (int d = 0; d < S; ++d) tc::tmem_ld8_nowait(trow + (uint32_t)(d * a.BN + brows + c0), r[d]);
  tc::tmem_wait_ld();
#pragma unroll
  for (int d = 0; d < S; ++d) tc::tmem_regs_ready8(r[d]);
  int mx[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    mx[jj] = 0;
    const int j = j0 + c0 + jj;
    if (!valid || j >= N) continue;
    float ai[S];
#pragma unroll
    for (int d = 0; d < S; ++d) ai[d] = __uint_as_float(r[d][jj]);
    const double dr = dre[jj], di = combine_exact<S>(ai, ea + eb[c0 + jj] - 14);
    const long ia = ((long)z * N + j) * M + p;  // [z][j][p]
    double2 v;
    if (mode == 0) {
      // u_0 = P Phi = diag(P) Phi + O Phi: also the first term of the Taylor sum
      const double pd = a.pdiag[p];
      v = make_double2(fma(1.0, __dmul_rn(pd, g[jj].x), dr), fma(1.0, __dmul_rn(pd, g[jj].y), di));
      a.accT[ia] = v;
    } else if (mode == 1) {
      // u_k = V u_{k-1}; the sum gains i^k g_k u_k; the next operand is u_k, or the
      // finished sum after the last term
      double2 w = make_double2(dr, di);
      const int kmod = k & 3;
      if (kmod == 1) w = make_double2(-di, dr);
      else if (kmod == 2) w = make_double2(-dr, -di);
      else if (kmod == 3) w = make_double2(di, -dr);
      double2 acc = g[jj];
      acc.x = fma(a.gk[k], w.x, acc.x);
      acc.y = fma(a.gk[k], w.y, acc.y);
      a.accT[ia] = acc;
      v = k == a.n ? acc : make_double2(dr, di);
    } else {
      // Phi = P acc = diag(P) acc + O acc
      const double d = a.pdiag[p];
      a.phi[((long)z * M + p) * N + j] = make_double2(fma(d, g[jj].x, dr), fma(d, g[jj].y, di));
      continue;
    }
    a.tout[ia] = v;
    mx[jj] = max(exp_field(v.x), exp_field(v.y));
  }
  if (mode != 2) {
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int m = __reduce_max_sync(0xffffffffu, mx[jj]);
      if (lane == jj && m > 0) atomicMax(&ex_loc[c0 + jj], m);
    }
  }
}

template <int S>
__device__ __forceinline__ void epi_pass(const FusedArgs& a, int mode, int k, int z, int j0, int p,
                                         bool valid, int ea, const int* eb, uint32_t trow, int c0,
                                         int lane, int* ex_loc) {
  epi_pass8<S>(a, mode, k, z, j0, p, valid, ea, eb, trow, c0, lane, ex_loc);
  epi_pass8<S>(a, mode, k, z, j0, p, valid, ea, eb, trow, c0 + 8, lane, ex_loc);
}

__global__ void __launch_bounds__(32 * kFWarps, 1)
    k_prop_fused(const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmV,
                 const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                 const FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t tfull[kChains];
  __shared__ __align__(8) uint64_t fin;
  __shared__ __align__(8) uint64_t exbar[kChains][2];  // a round's exponent partials arrived
  __shared__ __align__(8) uint64_t bbar[kChains][2];   // the cluster wrote a round's operand
  __shared__ uint32_t tmem_base;
  __shared__ int ep_ok;
  __shared__ int ex_loc[kChains][kFBrows];                     // this CTA's column maxima
  __shared__ int ex_part[kChains][2][kMaxCluster][kFBrows];    // every CTA's, by parity
  __shared__ int eb_s[kChains][2][kFBrows];                    // operand exponents
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = a.stages, BN = a.BN, brows = a.brows, npt = a.npt;
  const uint32_t bslot = (uint32_t)BN * 64u;
  const uint32_t rank = tc::cluster_rank(), cid = tc::cluster_id(), ncl = tc::cluster_count();
  const int p0 = (int)rank * 128;
  int* err = a.err;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&fin, 1);
    for (int c = 0; c < kChains; ++c) {
      tc::mbar_init(&tfull[c], 1);
      for (int b = 0; b < 2; ++b) {
        tc::mbar_init(&exbar[c][b], (uint32_t)npt);
        tc::mbar_init(&bbar[c][b], (uint32_t)npt);
      }
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmO);
    tc::prefetch_tmap(&tmV);
    tc::prefetch_tmap(&tmB0);
    tc::prefetch_tmap(&tmB1);
  }
  for (int i = threadIdx.x; i < kChains * kFBrows; i += blockDim.x) (&ex_loc[0][0])[i] = 0;
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  tc::cluster_sync();  // every peer's barriers exist before the first remote arrival
  const uint32_t tmem = tmem_base;
  const int last = a.npass - 1;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: passes in order, the two chains interleaved
      int it = 0;
      uint32_t R[kChains] = {0, 0};  // rounds consumed per chain
      bool ok = true;
      for (int pair = (int)cid; pair < a.npairs && ok; pair += (int)ncl) {
        for (int pass = 0; pass < a.npass && ok; ++pass) {
          for (int c = 0; c < kChains && ok; ++c) {
            int z, j0;
            if (!chain_unit(a, pair, c, &z, &j0)) continue;
            const uint32_t Rc = R[c]++;
            if (!tc::mbar_wait_cluster(&bbar[c][Rc & 1], (Rc >> 1) & 1, err)) {
              atomicExch(err, 1);
              ok = false;
              break;
            }
            tc::fence_proxy_async_global();
            const int S = a.dg[pass];
            const bool real = pass == 0 || pass == last;
            const int kUA = real ? 1 : 2;
            const CUtensorMap* tb = (Rc & 1) ? &tmB1 : &tmB0;
            const uint32_t tx = (uint32_t)S * (kUA * kASlot + 2u * brows * 64u);
            for (int kb = 0; kb < a.nkb; ++kb, ++it) {
              const int st = it % nst;
              if (it >= nst && !tc::mbar_wait(&empty[st], ((it / nst) - 1) & 1, err)) {
                atomicExch(err, 1);
                ok = false;
                break;
              }
              tc::mbar_arrive_expect_tx(&full[st], tx);
              uint8_t* sa = smem + st * a.stage_bytes;
              uint8_t* sb = sa + S * kUA * kASlot;
              for (int s = 0; s < S; ++s) {
                if (real) {
                  tc::tma_load_3d(sa + s * kASlot, &tmO, kb * kBK, p0, s, &full[st]);
                } else {
                  tc::tma_load_4d(sa + s * kASlot, &tmV, kb * kBK, p0, 2 * z, s, &full[st]);
                  tc::tma_load_4d(sa + (S + s) * kASlot, &tmV, kb * kBK, p0, 2 * z + 1, s,
                                  &full[st]);
                }
                tc::tma_load_4d(sb + s * bslot, tb, kb * kBK, j0, 2 * z, s, &full[st]);
                tc::tma_load_4d(sb + s * bslot + brows * 64, tb, kb * kBK, j0, 2 * z + 1, s,
                                &full[st]);
              }
            }
          }
        }
      }
      // no TMA write may still be in flight when the CTA moves on
      for (int i = it > nst ? it - nst : 0; i < it; ++i)
        tc::mbar_wait(&full[i % nst], (i / nst) & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: the same order; chain c accumulates in TMEM set c
      const uint32_t id_full = tc::idesc_bf16(128, BN);
      const uint32_t id_half = tc::idesc_bf16(128, brows);
      const uint32_t id_half_neg = tc::idesc_bf16(128, brows, true);
      int it = 0;
      bool ok = true;
      for (int pair = (int)cid; pair < a.npairs && ok; pair += (int)ncl) {
        for (int pass = 0; pass < a.npass && ok; ++pass) {
          for (int c = 0; c < kChains && ok; ++c) {
            int z, j0;
            if (!chain_unit(a, pair, c, &z, &j0)) continue;
            const int S = a.dg[pass];
            const bool real = pass == 0 || pass == last;
            const int kUA = real ? 1 : 2;
            const uint32_t acc = tmem + (uint32_t)c * a.set_cols;
            for (int kb = 0; kb < a.nkb; ++kb, ++it) {
              const int st = it % nst;
              if (!tc::mbar_wait(&full[st], (it / nst) & 1, err)) {
                atomicExch(err, 1);
                ok = false;
                break;
              }
              tc::fence_after_sync();
              const uint32_t sa = tc::smem_u32(smem + st * a.stage_bytes);
              const uint32_t sb = sa + (uint32_t)(S * kUA * kASlot);
              const uint32_t sbi = sb + (uint32_t)brows * 64u;
              const bool first = kb == 0;
              switch (S) {
#define AFQ_FUSED_MMA(SS)                                                                    \
  case SS:                                                                                   \
    issue_diagonals<SS>(acc, (uint32_t)BN, sa, sb, bslot, 0, 0, id_full, first);             \
    if (!real) {                                                                             \
      issue_diagonals<SS>(acc, (uint32_t)BN, sa, sbi, bslot, 1, 0, id_half_neg, false);       \
      issue_diagonals<SS>(acc + (uint32_t)brows, (uint32_t)BN, sa, sb, bslot, 1, 0, id_half, \
                          false);                                                            \
    }                                                                                        \
    break;
                AFQ_FUSED_MMA(1)
                AFQ_FUSED_MMA(2)
                AFQ_FUSED_MMA(3)
                AFQ_FUSED_MMA(4)
#undef AFQ_FUSED_MMA
              }
              tc::mma_commit(&empty[st]);
            }
            if (ok) tc::mma_commit(&tfull[c]);
          }
        }
      }
      tc::mma_commit(&fin);
    }
  } else {
    // epilogue warps: TMEM lane quarter lq (rows 32 lq ..), 16 columns c0 .. c0 + 15
    const int q = warp - 2, lq = warp & 3, c0 = 16 * (q >> 2);
    const bool cols = c0 < brows;
    const int row = 32 * lq + lane, p = p0 + row;
    const int M = a.M, N = a.N, Mpad = a.Mpad;
    const long plane = 2L * a.W * N * Mpad;
    uint32_t P[kChains] = {0, 0};  // passes done per chain (tfull phases)
    uint32_t R[kChains] = {0, 0};  // operand rounds published per chain
    bool ok = true;
    for (int pair = (int)cid; pair < a.npairs && ok; pair += (int)ncl) {
      // round -1 of a chain publishes operand 0 (Phi's digits); pass `pass` then
      // publishes operand pass + 1, except the last
      for (int pass = -1; pass < a.npass && ok; ++pass) {
        for (int c = 0; c < kChains && ok; ++c) {
          int z, j0;
          if (!chain_unit(a, pair, c, &z, &j0)) continue;
          int* exl = ex_loc[c];
          if (pass >= 0) {
            if (q == 0 && lane == 0) {
              ep_ok = tc::mbar_wait(&tfull[c], P[c] & 1, err) ? 1 : 0;
              if (!ep_ok) atomicExch(err, 1);
            }
            ++P[c];
            fused_epi_sync();
            if (!ep_ok) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const int mode = pass == 0 ? 0 : (pass == last ? 2 : 1);
            const int ea = p < M ? (mode == 1 ? a.ea_v[(long)z * M + p] : a.ea_o[p]) : 0;
            const int* eb = eb_s[c][(R[c] - 1) & 1];
            const bool valid = p < M;
            const uint32_t trow =
                tmem + (uint32_t)c * a.set_cols + ((uint32_t)(32 * lq) << 16);
            if (cols) {
              switch (a.dg[pass]) {
                case 1: epi_pass<1>(a, mode, pass, z, j0, p, valid, ea, eb, trow, c0, lane, exl); break;
                case 2: epi_pass<2>(a, mode, pass, z, j0, p, valid, ea, eb, trow, c0, lane, exl); break;
                case 3: epi_pass<3>(a, mode, pass, z, j0, p, valid, ea, eb, trow, c0, lane, exl); break;
                case 4: epi_pass<4>(a, mode, pass, z, j0, p, valid, ea, eb, trow, c0, lane, exl); break;
              }
            }
            tc::fence_before_sync();
            if (pass == last) continue;
          } else if (cols) {
            // operand 0: exponent maxima of Phi's columns over this CTA's rows
            for (int h = 0; h < 16; h += 8) {
              double2 v[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + c0 + h + jj;
                v[jj] = (p < M && j < N) ? a.phi[((long)z * M + p) * N + j]
                                         : make_double2(0.0, 0.0);
              }
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int m = __reduce_max_sync(0xffffffffu,
                                                max(exp_field(v[jj].x), exp_field(v[jj].y)));
                if (lane == jj && m > 0) atomicMax(&exl[c0 + h + jj], m);
              }
            }
          }
          // exchange this CTA's column maxima with every CTA of the cluster
          fused_epi_sync();
          const uint32_t Rc = R[c]++;
          const uint32_t par = Rc & 1, ph = (Rc >> 1) & 1;
          if (q == 0) {
            if (lane < brows) {
              const int v = exl[lane];
              exl[lane] = 0;
              const uint32_t loc = tc::smem_u32(&ex_part[c][par][rank][lane]);
              for (int r = 0; r < npt; ++r)
                tc::st_cluster_u32(tc::map_rank(loc, (uint32_t)r), (uint32_t)v);
            }
            tc::fence_cluster();
            __syncwarp();
            if (lane == 0)
              for (int r = 0; r < npt; ++r)
                tc::mbar_arrive_cluster(tc::map_rank(tc::smem_u32(&exbar[c][par]), (uint32_t)r));
          }
          if (q == 0 && lane == 0) {
            ep_ok = tc::mbar_wait_cluster(&exbar[c][par], ph, err) ? 1 : 0;
            if (!ep_ok) atomicExch(err, 1);
          }
          fused_epi_sync();
          if (!ep_ok) {
            ok = false;
            break;
          }
          // the next operand's digits for this CTA's rows (zero rows M <= p < Mpad)
          if (cols && p < Mpad) {
            const int Sn = a.dg[pass + 1 < 0 ? 0 : pass + 1];
            __nv_bfloat16* out = a.tsl[par];
            for (int h = 0; h < 16; h += 8) {
              double2 v[8];
              int e[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int cc = c0 + h + jj, j = j0 + cc;
                int m = 0;
                for (int r = 0; r < npt; ++r) m = max(m, ex_part[c][par][r][cc]);
                e[jj] = row_exponent_field(m);
                v[jj] = make_double2(0.0, 0.0);
                if (p < M && j < N)
                  v[jj] = pass < 0 ? a.phi[((long)z * M + p) * N + j]
                                   : a.tout[((long)z * N + j) * M + p];
              }
              if (row == 0)
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) eb_s[c][par][c0 + h + jj] = e[jj];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + c0 + h + jj;
                if (j >= N) continue;
                int qr[kMaxSlices], qi[kMaxSlices];
                exact_digits(v[jj].x, e[jj], Sn, qr);
                exact_digits(v[jj].y, e[jj], Sn, qi);
                __nv_bfloat16* o = out + ((long)(2 * z) * N + j) * Mpad + p;
#pragma unroll
                for (int s = 0; s < kMaxSlices; ++s)
                  if (s < Sn) {
                    o[s * plane] = __float2bfloat16_rn((float)qr[s]);
                    o[s * plane + (long)N * Mpad] = __float2bfloat16_rn((float)qi[s]);
                  }
              }
            }
          }
          tc::fence_proxy_async_global();
          __threadfence();
          fused_epi_sync();
          if (q == 0 && lane == 0)
            for (int r = 0; r < npt; ++r)
              tc::mbar_arrive_cluster(tc::map_rank(tc::smem_u32(&bbar[c][par]), (uint32_t)r));
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    // the MMAs already issued must finish before TMEM is freed (bounded by time only)
    static const int zero = 0;
    tc::mbar_wait(&fin, 0, &zero);
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, a.tmem_cols);
  }
  tc::cluster_sync();  // no peer writes into this CTA's shared memory any more
}

int sm_count_fused() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace

// Column tile of the cluster kernel's chains: at most 32 walker columns (two
// accumulator sets of 4 digits x 2 x 32 columns fill the 512 TMEM columns).
int fused_prop_rows(int N) { return N >= kFBrows ? kFBrows : (N + 15) / 16 * 16; }

// Phi <- P T_n(A) P Phi for every walker by the cluster kernel.  Returns AFQ_OK, an
// error through afq_fail, or -1 (nothing launched) when this shape cannot take it:
// then the caller runs the per-pass kernels.
int launch_propagate_fused(afq_ctx* ctx) {
  const int M = ctx->M, N = ctx->N, W = ctx->ws.W, n = ctx->p.taylor_order;
  FusedArgs a{};
  a.M = M;
  a.N = N;
  a.W = W;
  a.Mpad = ctx->Mpad;
  a.brows = ctx->prop_rows_fused;
  a.BN = 2 * a.brows;
  a.nkb = ctx->Mpad / kBK;
  a.npt = (M + 127) / 128;
  a.njt = (N + a.brows - 1) / a.brows;
  a.nunits = W * a.njt;
  a.npairs = (a.nunits + 1) / 2;
  a.npass = n + 2;
  a.n = n;
  if (a.npt > kMaxCluster || a.npass > kMaxPasses || a.brows > kFBrows || a.brows < 16 ||
      a.brows % 16)
    return -1;
  int smax = 1;
  for (int k = 0; k < a.npass; ++k) {
    a.dg[k] = ctx->prop_digits[k];
    if (a.dg[k] < 1 || a.dg[k] > kMaxSlices) return -1;
    smax = a.dg[k] > smax ? a.dg[k] : smax;
  }
  double gk = 1.0;
  a.gk[0] = 1.0;
  for (int k = 1; k <= n; ++k) {
    gk *= sqrt(ctx->p.dt) / k;  // the per-pass path's sequence of roundings
    a.gk[k] = gk;
  }
  a.set_cols = (uint32_t)(smax * a.BN);
  if (kChains * a.set_cols > 512) return -1;
  a.tmem_cols = tmem_cols_for(kChains * (int)a.set_cols);
  a.stage_bytes = (uint32_t)(smax * (2 * kASlot + a.BN * 64));
  int nst = (int)((kSmemLimit - 8192 - 1024) / a.stage_bytes);
  if (nst > kMaxStages) nst = kMaxStages;
  if (nst < 2) return -1;
  a.stages = nst;
  const size_t smem = (size_t)a.stage_bytes * nst + 1024;
  a.ea_o = ctx->e_pm;
  a.ea_v = ctx->e_a;
  a.pdiag = ctx->pdiag;
  a.phi = ctx->ws.phi;
  a.accT = ctx->accT;
  a.tout = ctx->tout;
  a.tsl[0] = ctx->T_sl[0];
  a.tsl[1] = ctx->T_sl[1];
  a.err = ctx->flags + 2;

  cudaError_t e = raise_smem_limit((const void*)k_prop_fused, smem);
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("fused propagation: ") + cudaGetErrorString(e));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.npt;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(32 * kFWarps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // persistent: as many clusters as fit at once (asked once per cluster shape)
  static int cached_npt = -1, cached_clusters = 0;
  static size_t cached_smem = 0;
  if (cached_npt != a.npt || cached_smem != smem) {
    cfg.gridDim = dim3((unsigned)(a.npt * (sm_count_fused() / a.npt)));
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_prop_fused, &cfg) != cudaSuccess)
      ncl = 0;
    cudaGetLastError();
    cached_npt = a.npt;
    cached_smem = smem;
    cached_clusters = ncl;
  }
  if (cached_clusters < 1) return -1;
  const int ncl = a.npairs < cached_clusters ? a.npairs : cached_clusters;
  cfg.gridDim = dim3((unsigned)(a.npt * ncl));
  e = cudaLaunchKernelEx(&cfg, k_prop_fused, ctx->tm_pm, ctx->tm_az, ctx->tm_t_fused[0],
                         ctx->tm_t_fused[1], a);
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("fused propagation: ") + cudaGetErrorString(e));
  return AFQ_OK;
}
