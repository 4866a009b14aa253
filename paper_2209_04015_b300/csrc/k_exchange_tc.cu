// Split-precision exchange energy (Sec. "Local energy", precision AFQ_SPLIT_BF16):
// E_K,z = -1/2 sum_s sum_g sum_ij T_ij T_ji with T^{gz} = L~_g,s theta_z,s, as a
// persistent tcgen05 kernel.
//
// The GEMM: A rows (g, i) are G Cholesky indices x n orbitals of L~ (K = Mpad), B rows
// (z, re/im, j) are zb walkers of theta; a 128 x BN accumulator pair holds T^{gz} for
// every (g, z) pair of a tile, and T is never written to HBM.  Both operands are cut
// into S scaled digits (split_scaled: per-row power-of-two scales, each digit stored at
// its true weight): the leading product (0, 0) accumulates exactly (integer multiples
// of one power of two) in a head accumulator and the smaller products in a tail
// accumulator, so the tensor core's biased FP32 accumulation only touches the tail,
// ~2^-8 of T.  Each CTA stays resident and
// walks the tiles in chunks of walker blocks whose theta stays in L2, g-tile major
// inside a chunk (so resident CTAs share each L~ g-tile):
//   warp 0   TMA producer: the S slices of the A and B units of every K block into a
//            ring of stages;
//   warp 1   MMA issuer: the digit products into one of two head / tail TMEM
//            accumulator pairs, then a commit to the epilogue;
//   warps 2-5 epilogue: a few walkers of the tile at a time, their 2n columns are
//            copied from TMEM (head + tail, each warp its 32 lanes) to shared memory, and each warp
//            reduces sum_ij T_ij T_ji of its g-blocks (lanes over (g-block, row i);
//            conflict-free rows and columns; FP32 within the warp, FP64 across warps
//            and tiles).
// With equal spins both spins' tiles run in one launch (the same maps, another
// orbital offset).
// With two accumulator pairs the epilogue of one tile runs under the MMAs of the next.
// Every mbarrier wait is bounded (time, or the grid-wide error flag), as in the
// generic engine.
#include "tc_engine.cuh"

using namespace tce;

namespace {

constexpr int kExWarps = 6;
constexpr int kExThreads = 32 * kExWarps;
constexpr int kEpiWarps = 4;

struct ExArgs {
  // tiles [0, ntiles) cover spin `spin` and, when nspin = 2 (equal spins), spin + 1 with
  // the same maps at column offset `off2`; zc walkers are staged per epilogue round
  int n, off, off2, nspin, G, zb, zc, BN, bstride, X, W, spin, ex_groups, nkb, stages, ngt,
      nzt, zchunk, tiles_per_spin, ntiles, pitch;
  uint32_t tx_bytes, tmem_cols;
  double2* ekp;
  int* err;
};

// Tile order within a spin: walker blocks in chunks of zchunk (whose theta stays in
// L2), and inside a chunk g-tile major, so that resident CTAs share each L~ g-tile.
__device__ __forceinline__ void tile_coords(const ExArgs& a, int tl, int* gt, int* zt) {
  const int per = a.ngt * a.zchunk;
  const int c = tl / per, r = tl - c * per;
  const int zn = min(a.zchunk, a.nzt - c * a.zchunk);
  *gt = r / zn;
  *zt = c * a.zchunk + (r - *gt * zn);
}

__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
}

template <int S>
__global__ void __launch_bounds__(kExThreads, 1)
    k_exchange_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const ExArgs a) {
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
  __shared__ int ep_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = a.stages, n = a.n;
  const uint32_t bslot = (uint32_t)a.BN * 64u;
  const uint32_t stage_bytes = S * (kASlot + bslot);
  float* Ts = reinterpret_cast<float*>(smem + nst * stage_bytes);  // 128 x pitch
  double2* red = reinterpret_cast<double2*>(Ts + 128 * a.pitch);    // zb x 4
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
      tc::mbar_init(&tempty[b], kEpiWarps);
    }
    tc::mbar_init(&fin, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base, a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      int it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
        const int sp = tile / a.tiles_per_spin;
        int gt, zt;
        tile_coords(a, tile % a.tiles_per_spin, &gt, &zt);
        const int g0 = gt * a.G, z0 = zt * a.zb;
        const int off = sp ? a.off2 : a.off;
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const int st = it % nst;
          if (it >= nst && !tc::mbar_wait(&empty[st], ((it / nst) - 1) & 1, err)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[st], a.tx_bytes);
          uint8_t* sa = smem + st * stage_bytes;
          uint8_t* sb = sa + S * kASlot;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            tc::tma_load_4d(sa + s * kASlot, &tmA, kb * kBK, off, g0, s, &full[st]);
            tc::tma_load_4d(sb + s * bslot, &tmB, kb * kBK, off, 2 * z0, s, &full[st]);
          }
        }
      }
      // no TMA write may still be in flight when the CTA moves on
      for (int i = it > nst ? it - nst : 0; i < it; ++i)
        tc::mbar_wait(&full[i % nst], (i / nst) & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t idesc = tc::idesc_bf16(128, a.BN);
      int it = 0, lt = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++lt) {
        const int buf = lt & 1, use = lt >> 1;
        if (use >= 1 && !tc::mbar_wait(&tempty[buf], (use - 1) & 1, err)) {
          atomicExch(err, 1);
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(buf * 2 * a.bstride);
        for (int kb = 0; kb < a.nkb; ++kb, ++it) {
          const int st = it % nst;
          if (!tc::mbar_wait(&full[st], (it / nst) & 1, err)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
          const uint32_t sb = sa + S * kASlot;
          issue_head_tail<S>(acc, acc + (uint32_t)a.bstride, sa, sb, bslot, idesc, kb == 0);
          tc::mma_commit(&empty[st]);
        }
        if (ok) tc::mma_commit(&tfull[buf]);
      }
      tc::mma_commit(&fin);
    }
  } else {
    // epilogue warps: q = warp - 2 picks g-blocks; TMEM lanes 32 (warp % 4) ..
    const int q = warp - 2, lq = warp & 3;
    const int row = 32 * lq + lane;
    const int w2n = 2 * n;
    int lt = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++lt) {
      const int buf = lt & 1;
      // one thread waits for the accumulator; the four warps then agree on the outcome
      if (q == 0 && lane == 0) {
        ep_ok = tc::mbar_wait(&tfull[buf], (lt >> 1) & 1, err) ? 1 : 0;
        if (!ep_ok) atomicExch(err, 1);
      }
      epi_sync();
      if (!ep_ok) break;
      tc::fence_after_sync();
      const int sp = tile / a.tiles_per_spin;
      int gt, zt;
      tile_coords(a, tile % a.tiles_per_spin, &gt, &zt);
      const int g0 = gt * a.G, z0 = zt * a.zb;
      const int gc = min(a.G, a.X - g0);
      const int nblk = gc > q ? (gc - q + kEpiWarps - 1) / kEpiWarps : 0;  // this warp's g-blocks
      const uint32_t acc = tmem + (uint32_t)(buf * 2 * a.bstride) + ((uint32_t)(32 * lq) << 16);
      for (int zr = 0; zr < a.zb; zr += a.zc) {
        // stage walkers zr .. zr + zc - 1: their columns c_lo .. c_hi - 1, row by lane
        const int c_lo = zr * w2n, c_hi = min(a.zb, zr + a.zc) * w2n;
        for (int c0 = c_lo & ~15; c0 < c_hi; c0 += 16) {
          float v[16];
          tc::tmem_ld16(acc + (uint32_t)c0, v);
          if (S > 1) {
            float t[16];
            tc::tmem_ld16(acc + (uint32_t)(a.bstride + c0), t);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] += t[jj];
          }
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int c = c0 + jj;
            if (c >= c_lo && c < c_hi) Ts[row * a.pitch + (c - c_lo)] = v[jj];
          }
        }
        epi_sync();
        for (int zl = zr; zl < min(a.zb, zr + a.zc); ++zl) {
          const int cb = (zl - zr) * w2n;
          float dr = 0.f, di = 0.f;
          // lanes over (g-block of this warp, row i): sum_j T_ij T_ji in FP32, then FP64
          for (int e = lane; e < nblk * n; e += 32) {
            const int b = e / n, i = e - b * n, gl = q + kEpiWarps * b;
            const float* ri = Ts + (gl * n + i) * a.pitch + cb;
            const float* cj = Ts + gl * n * a.pitch + cb + i;
            float sr = 0.f, si = 0.f;
            for (int j = 0; j < n; ++j) {
              const float ar = ri[j], ai = ri[n + j];
              const float br = cj[j * a.pitch], bi = cj[j * a.pitch + n];
              sr = fmaf(ar, br, fmaf(-ai, bi, sr));
              si = fmaf(ar, bi, fmaf(ai, br, si));
            }
            dr += sr;
            di += si;
          }
          // FP32 across the warp (B300's FP64 pipe would cost more than the tile's MMAs
          // leave to the epilogue), FP64 from the warp partials on
          for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_down_sync(0xffffffffu, dr, o);
            di += __shfl_down_sync(0xffffffffu, di, o);
          }
          if (lane == 0) red[zl * kEpiWarps + q] = make_double2((double)dr, (double)di);
        }
        epi_sync();  // Ts is rewritten for the next walkers
      }
      // every TMEM read of this accumulator is done: hand it back to the MMA warp
      tc::fence_before_sync();
      if (lane == 0) tc::mbar_arrive(&tempty[buf]);
      if (q == 0)
        for (int zl = lane; zl < a.zb; zl += 32) {
          const int z = z0 + zl;
          double sr = 0.0, si = 0.0;
#pragma unroll
          for (int k = 0; k < kEpiWarps; ++k) {
            sr += red[zl * kEpiWarps + k].x;
            si += red[zl * kEpiWarps + k].y;
          }
          if (z < a.W)
            a.ekp[((long)z * 2 + a.spin + sp) * a.ex_groups + gt] =
                make_double2(-0.5 * sr, -0.5 * si);
        }
      epi_sync();  // red is rewritten by the next tile
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
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int S>
cudaError_t launch_ex(int grid, size_t smem, cudaStream_t stream, const CUtensorMap& ta,
                      const CUtensorMap& tb, const ExArgs& a) {
  cudaError_t e = raise_smem_limit((const void*)k_exchange_tc<S>, smem);
  if (e != cudaSuccess) return e;
  k_exchange_tc<S><<<grid, kExThreads, smem, stream>>>(ta, tb, a);
  return cudaGetLastError();
}

}  // namespace

int launch_exchange_tc(afq_ctx* ctx, WalkerSet& s) {
  if (ctx->Vsl) return launch_exchange_tcv(ctx, s);  // stored half-rotated tensor
  // equal spins share tile shapes and maps: one launch covers both
  const bool fuse = ctx->na == ctx->nb && ctx->na > 0 && ctx->ex_zb[0] == ctx->ex_zb[1];
  for (int spin = 0; spin < 2; ++spin) {
    const int n = spin ? ctx->nb : ctx->na;
    if (n == 0) continue;
    ExArgs a{};
    a.n = n;
    a.off = spin ? ctx->na : 0;
    a.off2 = ctx->na;
    a.nspin = fuse ? 2 : 1;
    a.G = ctx->ex_G[spin];
    a.zb = ctx->ex_zb[spin];
    a.BN = ctx->ex_BN[spin];
    a.bstride = round_up(a.BN, 32);
    a.X = ctx->X;
    a.W = s.W;
    a.spin = spin;
    a.ex_groups = ctx->ex_groups;
    a.ekp = s.ekp;
    a.err = ctx->flags + 2;
    a.nkb = ctx->Mpad / kBK;
    a.ngt = (ctx->X + a.G - 1) / a.G;
    a.nzt = (s.W + a.zb - 1) / a.zb;
    a.tiles_per_spin = a.ngt * a.nzt;
    {
      // walker blocks per chunk: their theta slices within ~24 MB of L2
      const long bblock = (long)ctx->S * 2 * n * a.zb * ctx->Mpad * 2;
      long zc = (24L << 20) / (bblock > 0 ? bblock : 1);
      a.zchunk = (int)(zc < 1 ? 1 : (zc > a.nzt ? a.nzt : zc));
    }
    a.ntiles = a.tiles_per_spin * a.nspin;
    // walkers staged per epilogue round: 128 rows x (zc 2n + 1) floats within 32 KB
    a.zc = (8192 / 128 - 1) / (2 * n);
    if (a.zc < 1) a.zc = 1;
    if (a.zc > a.zb) a.zc = a.zb;
    a.pitch = a.zc * 2 * n + 1;
    a.tx_bytes = (uint32_t)ctx->S * (kBK * n * a.G * 2 + kBK * n * 2 * a.zb * 2);
    a.tmem_cols = tmem_cols_for(4 * a.bstride);
    if (a.ngt > ctx->ex_groups) return afq_fail(ctx, AFQ_ERR_STATE, "exchange tiles exceed slots");
    if (4 * a.bstride > 512) return afq_fail(ctx, AFQ_ERR_ARG, "exchange tile too wide");
    const size_t stage = (size_t)ctx->S * (kASlot + (size_t)a.BN * 64);
    const size_t fixed = (size_t)128 * a.pitch * 4 + (size_t)a.zb * kEpiWarps * 16 + 1024;
    int nst = (int)((kSmemLimit - 2048 - fixed) / stage);
    if (nst > kMaxStages) nst = kMaxStages;
    if (nst < 1) return afq_fail(ctx, AFQ_ERR_ARG, "exchange tile does not fit in shared memory");
    a.stages = nst;
    const size_t smem = stage * nst + fixed;
    const int grid = a.ntiles < sm_count() ? a.ntiles : sm_count();
    cudaError_t e = cudaErrorInvalidValue;
    switch (ctx->S) {
      case 1: e = launch_ex<1>(grid, smem, ctx->stream, ctx->tm_ex_a[spin], ctx->tm_ex_b[spin], a); break;
      case 2: e = launch_ex<2>(grid, smem, ctx->stream, ctx->tm_ex_a[spin], ctx->tm_ex_b[spin], a); break;
      case 3: e = launch_ex<3>(grid, smem, ctx->stream, ctx->tm_ex_a[spin], ctx->tm_ex_b[spin], a); break;
      case 4: e = launch_ex<4>(grid, smem, ctx->stream, ctx->tm_ex_a[spin], ctx->tm_ex_b[spin], a); break;
    }
    ctx->launches++;
    if (e != cudaSuccess)
      return afq_fail(ctx, AFQ_ERR_CUDA, std::string("exchange tc: ") + cudaGetErrorString(e));
    if (fuse) break;
  }
  return AFQ_OK;
}
