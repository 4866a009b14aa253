// Step kernels of libafqmc: auxiliary fields and force bias, the VHS build, the
// Taylor propagator with the one-body halves, and the phaseless weight update
// (Sec. "Review of AFQMC": hybrid propagation, Eqs. import, ovl, ph and theta).
#include <algorithm>
#include <vector>

#include "afq_internal.cuh"

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers M0, M1, Weyl key
// increments W0, W1, ten rounds; written here from that definition.
constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox_block(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += PH_W0;
      k1 += PH_W1;
    }
    const uint32_t lo0 = PH_M0 * c.x, hi0 = __umulhi(PH_M0, c.x);
    const uint32_t lo1 = PH_M1 * c.z, hi1 = __umulhi(PH_M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// counter (step mod 2^32, walker, pair, step >> 32), key (seed mod 2^32, seed >> 32)
__device__ __forceinline__ uint4 field_words(uint64_t step, uint32_t z, uint32_t m, uint64_t seed) {
  return philox_block(make_uint4((uint32_t)step, z, m, (uint32_t)(step >> 32)), (uint32_t)seed,
                      (uint32_t)(seed >> 32));
}

// 53-bit uniform in (0, 1] from two words: ((a >> 5) 2^26 + (b >> 6) + 1) 2^-53
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)(k + 1) * 0x1p-53;
}

// Box-Muller: the two N(0,1) fields of one (walker, pair)
__device__ __forceinline__ void field_pair(uint64_t step, uint32_t z, uint32_t m, uint64_t seed,
                                           double* g0, double* g1) {
  const uint4 w = field_words(step, z, m, seed);
  const double u1 = uniform53(w.x, w.y), u2 = uniform53(w.z, w.w);
  const double r = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  double sn, cs;
  sincos(ang, &sn, &cs);
  *g0 = r * cs;
  *g1 = r * sn;
}

__device__ __forceinline__ double2 warp_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__device__ double2 block_sum2(double2 v, double2* red) {
  v = warp_sum2(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double2 s = cmk(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = cadd(s, red[i]);
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// K3: fields xi (given or Philox), force bias xbar = -i sqrt(dt) (c - vbar) with
// optional cap, shifted fields y = xi - xbar, cfb = sum (xi xbar - xbar^2/2) and
// cmf = -i sqrt(dt) sum y vbar.  One CTA per walker.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fields(int X, double sdt, double cap,
                                                const double* __restrict__ xi_in, uint64_t seed,
                                                const unsigned long long* __restrict__ step_dev,
                                                const double2* __restrict__ c,
                                                const double* __restrict__ vbar,
                                                double2* __restrict__ xbar, double2* __restrict__ y,
                                                double2* __restrict__ cfb,
                                                double2* __restrict__ cmf) {
  __shared__ double2 red[8];
  const int z = blockIdx.x;
  const int npair = (X + 1) / 2;
  // the step counter lives on the device so that a captured graph draws new fields
  // on every replay
  const uint64_t step = *step_dev;
  double2 sfb = cmk(0.0, 0.0), smf = cmk(0.0, 0.0);
  for (int m = threadIdx.x; m < npair; m += 256) {
    double xi2[2];
    if (xi_in) {
      xi2[0] = xi_in[(long)z * X + 2 * m];
      xi2[1] = 2 * m + 1 < X ? xi_in[(long)z * X + 2 * m + 1] : 0.0;
    } else {
      field_pair(step, (uint32_t)z, (uint32_t)m, seed, &xi2[0], &xi2[1]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * m + h;
      if (g < X) {
        const double2 cz = c[(long)z * X + g];
        const double vb = vbar[g];
        double2 xb = cmk(sdt * cz.y, -sdt * (cz.x - vb));
        if (cap > 0.0) {
          const double mag = hypot(xb.x, xb.y);
          if (mag > cap) xb = cscale(xb, cap / mag);
        }
        const double x = xi2[h];
        const double2 yy = cmk(x - xb.x, -xb.y);
        const double2 xb2 = cmul(xb, xb);
        sfb = cadd(sfb, cmk(x * xb.x - 0.5 * xb2.x, x * xb.y - 0.5 * xb2.y));
        smf = cadd(smf, cscale(yy, vb));
        xbar[(long)z * X + g] = xb;
        y[(long)z * X + g] = yy;
      }
    }
  }
  sfb = block_sum2(sfb, red);
  smf = block_sum2(smf, red);
  if (threadIdx.x == 0) {
    cfb[z] = sfb;
    cmf[z] = cmk(sdt * smf.y, -sdt * smf.x);
  }
}

__global__ void k_philox_fields(int W, int X, uint64_t seed, uint64_t step, double* out,
                                uint32_t* words) {
  const int npair = (X + 1) / 2;
  const long total = (long)W * npair;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int z = (int)(e / npair), m = (int)(e % npair);
    if (words) {
      const uint4 w = field_words(step, z, m, seed);
      words[4 * e + 0] = w.x;
      words[4 * e + 1] = w.y;
      words[4 * e + 2] = w.z;
      words[4 * e + 3] = w.w;
    }
    if (out) {
      double g0, g1;
      field_pair(step, z, m, seed, &g0, &g1);
      out[(long)z * X + 2 * m] = g0;
      if (2 * m + 1 < X) out[(long)z * X + 2 * m + 1] = g1;
    }
  }
}

// ---------------------------------------------------------------------------
// K4 (FP64): A_z = i sqrt(dt) sum_g y_zg L_g over the packed upper triangle,
// written to both triangles of the dense symmetric W x M x M output.
// ---------------------------------------------------------------------------
constexpr int VZ = 8, VT = 64, VK = 32;
// One tile: packed rows t0 = bx VT .. + VT of walkers z0 = by VZ .. + VZ (256 threads).
__device__ __forceinline__ void vhs_tile(int W, int X, int M, int Mp, double sdt,
                                         const double2* __restrict__ y,
                                         const double* __restrict__ Lpk,
                                         const int2* __restrict__ tpq, double2* __restrict__ A,
                                         double* __restrict__ Asum, int bx, int by) {
  __shared__ double2 Ys[VZ][VK];
  __shared__ double Ls[VK][VT];
  const int t0 = bx * VT, z0 = by * VZ;
  const int tz = threadIdx.x / 32, tt = threadIdx.x % 32;
  double2 a0 = cmk(0.0, 0.0), a1 = cmk(0.0, 0.0);
  for (int k0 = 0; k0 < X; k0 += VK) {
    {
      const int r = threadIdx.x / VK, kk = threadIdx.x % VK;
      Ys[r][kk] = (z0 + r < W && k0 + kk < X) ? y[(long)(z0 + r) * X + k0 + kk] : cmk(0.0, 0.0);
    }
    for (int e = threadIdx.x; e < VK * VT; e += 256) {
      const int kk = e / VT, cc = e % VT;
      Ls[kk][cc] = (k0 + kk < X && t0 + cc < Mp) ? Lpk[(long)(k0 + kk) * Mp + t0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < VK; ++kk) {
      const double2 yv = Ys[tz][kk];
      const double l0 = Ls[kk][tt], l1 = Ls[kk][tt + 32];
      a0.x = fma(yv.x, l0, a0.x);
      a0.y = fma(yv.y, l0, a0.y);
      a1.x = fma(yv.x, l1, a1.x);
      a1.y = fma(yv.y, l1, a1.y);
    }
    __syncthreads();
  }
  const int z = z0 + tz;
  if (z >= W) return;
  double2* Az = A + (long)z * M * M;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = t0 + tt + 32 * h;
    if (t < Mp) {
      const double2 a = h ? a1 : a0;
      const double2 v = cmk(-sdt * a.y, sdt * a.x);  // i sqrt(dt) a
      const int2 pq = tpq[t];
      Az[(long)pq.x * M + pq.y] = v;
      if (pq.x != pq.y) Az[(long)pq.y * M + pq.x] = v;
      if (Asum) {  // Re A + Im A, the third operand of the 3-product complex multiply
        double* Sz = Asum + (long)z * M * M;
        Sz[(long)pq.x * M + pq.y] = v.x + v.y;
        if (pq.x != pq.y) Sz[(long)pq.y * M + pq.x] = v.x + v.y;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_vhs_fp64(int W, int X, int M, int Mp, double sdt,
                                                  const double2* __restrict__ y,
                                                  const double* __restrict__ Lpk,
                                                  const int2* __restrict__ tpq,
                                                  double2* __restrict__ A,
                                                  double* __restrict__ Asum) {
  vhs_tile(W, X, M, Mp, sdt, y, Lpk, tpq, A, Asum, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// K5 (FP64): Phi_z[:, cols] <- P T_n(A_z) P Phi_z[:, cols] for a chunk of NC
// columns.  One thread per orbital row p; P and A_z are symmetric, so row q of
// each is read with the lanes running over p (coalesced), and the column chunk
// of the current Taylor term is broadcast from shared memory.
// ---------------------------------------------------------------------------
template <int NC, int NCg>
__device__ __forceinline__ void sym_apply_real(int M, int p, const double* __restrict__ S,
                                               const double2* __restrict__ in, int cb,
                                               double2 out[NCg]) {
#pragma unroll
  for (int c = 0; c < NCg; ++c) out[c] = cmk(0.0, 0.0);
  int q = 0;
  for (; q + 4 <= M; q += 4) {
    double s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = S[(long)(q + u) * M + p];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NCg; ++c) {
        const double2 b = in[(q + u) * NC + cb + c];
        out[c].x = fma(s[u], b.x, out[c].x);
        out[c].y = fma(s[u], b.y, out[c].y);
      }
  }
  for (; q < M; ++q) {
    const double sv = S[(long)q * M + p];
#pragma unroll
    for (int c = 0; c < NCg; ++c) {
      const double2 b = in[q * NC + cb + c];
      out[c].x = fma(sv, b.x, out[c].x);
      out[c].y = fma(sv, b.y, out[c].y);
    }
  }
}

// out[c] = sum_q S_qp in[q][cb + c] for a complex symmetric S (row p read as column p).
template <int NC, int NCg>
__device__ __forceinline__ void sym_apply_cplx(int M, int p, const double2* __restrict__ S,
                                               const double2* __restrict__ in, int cb,
                                               double2 out[NCg]) {
#pragma unroll
  for (int c = 0; c < NCg; ++c) out[c] = cmk(0.0, 0.0);
  int q = 0;
  for (; q + 4 <= M; q += 4) {
    double2 s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = S[(long)(q + u) * M + p];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NCg; ++c) {
        const double2 b = in[(q + u) * NC + cb + c];
        out[c].x = fma(s[u].x, b.x, fma(-s[u].y, b.y, out[c].x));
        out[c].y = fma(s[u].x, b.y, fma(s[u].y, b.x, out[c].y));
      }
  }
  for (; q < M; ++q) {
    const double2 sv = S[(long)q * M + p];
#pragma unroll
    for (int c = 0; c < NCg; ++c) {
      const double2 b = in[q * NC + cb + c];
      out[c].x = fma(sv.x, b.x, fma(-sv.y, b.y, out[c].x));
      out[c].y = fma(sv.x, b.y, fma(sv.y, b.x, out[c].y));
    }
  }
}

// out[c] = sum_q S_qp in[q][cb + c] for a complex symmetric S by Gauss's three real
// products: with Ssum = Re S + Im S and insum = Re in + Im in,
//   Re = sum Re S Re in - sum Im S Im in,  Im = sum Ssum insum - (the two sums above),
// 3 multiply-adds per complex term instead of 4 (the sums cost M and M NC additions).
template <int NC, int NCg>
__device__ __forceinline__ void sym_apply_cplx3(int M, int p, const double2* __restrict__ S,
                                                const double* __restrict__ Ssum,
                                                const double2* __restrict__ in,
                                                const double* __restrict__ insum, int cb,
                                                double2 out[NCg]) {
  double p1[NCg], p2[NCg], p3[NCg];
#pragma unroll
  for (int c = 0; c < NCg; ++c) p1[c] = p2[c] = p3[c] = 0.0;
  int q = 0;
  for (; q + 4 <= M; q += 4) {
    double2 s[4];
    double ss[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s[u] = S[(long)(q + u) * M + p];
      ss[u] = Ssum[(long)(q + u) * M + p];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NCg; ++c) {
        const double2 b = in[(q + u) * NC + cb + c];
        p1[c] = fma(s[u].x, b.x, p1[c]);
        p2[c] = fma(s[u].y, b.y, p2[c]);
        p3[c] = fma(ss[u], insum[(q + u) * NC + cb + c], p3[c]);
      }
  }
  for (; q < M; ++q) {
    const double2 sv = S[(long)q * M + p];
    const double sv2 = Ssum[(long)q * M + p];
#pragma unroll
    for (int c = 0; c < NCg; ++c) {
      const double2 b = in[q * NC + cb + c];
      p1[c] = fma(sv.x, b.x, p1[c]);
      p2[c] = fma(sv.y, b.y, p2[c]);
      p3[c] = fma(sv2, insum[q * NC + cb + c], p3[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NCg; ++c) out[c] = cmk(p1[c] - p2[c], p3[c] - p1[c] - p2[c]);
}

// K5 (FP64): Phi <- P T_n(A) P Phi for NC walker columns c0 .. c0 + NC - 1 of walker
// z, the current Taylor term in shared memory (sm: propagate_fp64_smem bytes).  G
// threads share each row p (each owns NC/G of the columns), so that G M threads fill
// whole warps for M not a multiple of 32.  The unit runs on nthr threads (thread t of
// them); a unit that is not live only takes part in the CTA's barriers.
template <int NC, int G>
__device__ __forceinline__ void prop_unit(int M, int N, int order, const double* __restrict__ P,
                                          const double2* __restrict__ A,
                                          const double* __restrict__ Asum,
                                          double2* __restrict__ phi, int z, int c0, int t,
                                          int nthr, unsigned char* sm, bool live) {
  constexpr int NCg = NC / G;
  double2* cur = reinterpret_cast<double2*>(sm);  // M x NC
  double2* nxt = cur + M * NC;
  double2* acc = nxt + M * NC;
  double* curs = reinterpret_cast<double*>(acc + M * NC);  // Re + Im of cur (M x NC)
  double* nxts = curs + M * NC;
  const bool act = live && t < G * M;
  const int p = act ? t % M : 0, cb = act ? (t / M) * NCg : 0;
  const double2* Az = A + (long)z * M * M;
  const double* Sz = Asum + (long)z * M * M;
  double2* phz = phi + (long)z * M * N;
  if (live)
    for (int e = t; e < M * NC; e += nthr) {
      const int q = e / NC, c = e % NC;
      cur[e] = c0 + c < N ? phz[(long)q * N + c0 + c] : cmk(0.0, 0.0);
    }
  __syncthreads();
  double2 r[NCg];
  if (act) {
    sym_apply_real<NC, NCg>(M, p, P, cur, cb, r);
#pragma unroll
    for (int c = 0; c < NCg; ++c) {
      acc[p * NC + cb + c] = r[c];
      nxt[p * NC + cb + c] = r[c];
      nxts[p * NC + cb + c] = r[c].x + r[c].y;
    }
  }
  __syncthreads();
  {
    double2* tt = cur;
    cur = nxt;
    nxt = tt;
    double* ts = curs;
    curs = nxts;
    nxts = ts;
  }
  for (int k = 1; k <= order; ++k) {
    const double inv = 1.0 / k;
    if (act) {
      sym_apply_cplx3<NC, NCg>(M, p, Az, Sz, cur, curs, cb, r);
#pragma unroll
      for (int c = 0; c < NCg; ++c) {
        const double2 v = cscale(r[c], inv);
        nxt[p * NC + cb + c] = v;
        nxts[p * NC + cb + c] = v.x + v.y;
        acc[p * NC + cb + c] = cadd(acc[p * NC + cb + c], v);
      }
    }
    __syncthreads();
    double2* tt = cur;
    cur = nxt;
    nxt = tt;
    double* ts = curs;
    curs = nxts;
    nxts = ts;
  }
  if (act) {
    sym_apply_real<NC, NCg>(M, p, P, acc, cb, r);
#pragma unroll
    for (int c = 0; c < NCg; ++c)
      if (c0 + cb + c < N) phz[(long)p * N + c0 + cb + c] = r[c];
  }
}

// One CTA per (column chunk, walker).
template <int NC, int G>
__global__ void k_propagate_fp64(int M, int N, int order, const double* __restrict__ P,
                                 const double2* __restrict__ A, const double* __restrict__ Asum,
                                 double2* __restrict__ phi) {
  extern __shared__ __align__(16) unsigned char smraw[];
  prop_unit<NC, G>(M, N, order, P, A, Asum, phi, blockIdx.y, blockIdx.x * NC, threadIdx.x,
                   blockDim.x, smraw, true);
}

// ---------------------------------------------------------------------------
// Grouped launches for batches of uneven systems: one persistent launch per stage
// (the VHS build, the Taylor propagation) whose CTAs take tiles of every system from
// a descriptor table, the next tile from a device counter.  A tile runs the same
// device code as the system's own launch, so results are bit-identical to it.
// ---------------------------------------------------------------------------
struct VhsDesc {
  int W, X, M, Mp;
  double sdt;
  const double2* y;
  const double* Lpk;
  const int2* tpq;
  double2* A;
  double* Asum;
  int tx;     // packed-row tiles of VT rows
  int tile0;  // first tile of this system in the launch
};

struct PropDesc {
  int M, N, order, G;
  int T;       // threads of one unit (one walker's column chunk): 32 ceil(G M / 32)
  int U;       // units per CTA (U T <= the CTA's threads)
  int chunks;  // column chunks per walker
  int units;   // chunks x W
  int tile0;   // first CTA tile of this system in the launch
  int unit_smem;  // shared-memory bytes of one unit (a multiple of 16)
  const double* P;
  const double2* A;
  const double* Asum;
  double2* phi;
};

// The next tile of a persistent grouped launch (every thread gets the same value).
__device__ __forceinline__ int next_tile(int* counter) {
  __shared__ int tile;
  __syncthreads();  // every thread has read the previous value
  if (threadIdx.x == 0) tile = atomicAdd(counter, 1);
  __syncthreads();
  return tile;
}

__global__ void __launch_bounds__(256) k_vhs_fp64_grouped(const VhsDesc* __restrict__ d, int ns,
                                                          int total, int* __restrict__ counter) {
  for (;;) {
    const int tile = next_tile(counter);
    if (tile >= total) return;
    int s = 0;
    while (s + 1 < ns && tile >= d[s + 1].tile0) ++s;
    const VhsDesc g = d[s];
    const int local = tile - g.tile0;
    vhs_tile(g.W, g.X, g.M, g.Mp, g.sdt, g.y, g.Lpk, g.tpq, g.A, g.Asum, local % g.tx,
             local / g.tx);
  }
}

// Each CTA tile holds U units of one system side by side (threads u T .. u T + T - 1
// and shared memory u unit_smem .. of unit u); G is the system's threads per row.
template <int NC>
__global__ void __launch_bounds__(1024, 1)
    k_propagate_fp64_grouped(const PropDesc* __restrict__ d, int ns, int total,
                             int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smraw[];
  for (;;) {
    const int tile = next_tile(counter);
    if (tile >= total) return;
    int s = 0;
    while (s + 1 < ns && tile >= d[s + 1].tile0) ++s;
    const PropDesc g = d[s];
    const int sub = (int)threadIdx.x / g.T;
    const int unit = (tile - g.tile0) * g.U + sub;
    const bool live = sub < g.U && unit < g.units;
    const int z = live ? unit / g.chunks : 0, c0 = live ? (unit % g.chunks) * NC : 0;
    const int t = (int)threadIdx.x - (sub < g.U ? sub : 0) * g.T;
    unsigned char* sm = smraw + (size_t)(sub < g.U ? sub : 0) * g.unit_smem;
    if (NC >= 4 && g.G == 4)
      prop_unit<NC, (NC >= 4 ? 4 : 1)>(g.M, g.N, g.order, g.P, g.A, g.Asum, g.phi, z, c0, t, g.T,
                                       sm, live);
    else if (NC >= 2 && g.G == 2)
      prop_unit<NC, (NC >= 2 ? 2 : 1)>(g.M, g.N, g.order, g.P, g.A, g.Asum, g.phi, z, c0, t, g.T,
                                       sm, live);
    else
      prop_unit<NC, 1>(g.M, g.N, g.order, g.P, g.A, g.Asum, g.phi, z, c0, t, g.T, sm, live);
  }
}

// ---------------------------------------------------------------------------
// K8: overlap ratio R = (O'/O) e^{cmf}, importance I = R e^{cfb} e^{log_const},
// phaseless weight w <- w |I| max(0, cos arg R) (or w <- w I in free projection).
// ---------------------------------------------------------------------------
// With e_shift_dev set, log_const = -dt (base - E_shift) takes E_shift from the device
// (the block driver's energy-shift feedback); base = e0 - 1/2 sum vbar^2, the same
// operations in the same order as the host's value.
__global__ void k_weights(int W, double log_const, const double* __restrict__ e_shift_dev,
                          double dt, double base, int free_proj, const double2* __restrict__ det,
                          const double2* __restrict__ cfb, const double2* __restrict__ cmf,
                          double2* __restrict__ ovlp, double2* __restrict__ w, int* flags,
                          unsigned long long* __restrict__ step_dev) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z == 0) *step_dev += 1;  // the step's fields were drawn by k_fields earlier in order
  if (z >= W) return;
  if (e_shift_dev) log_const = -dt * (base - *e_shift_dev);
  const double2 onew = cmul(det[2 * z], det[2 * z + 1]);
  const double2 ratio = cmul(cdiv(onew, ovlp[z]), cexp(cmf[z]));
  const double2 imp = cmul(cmul(ratio, cexp(cfb[z])), cmk(exp(log_const), 0.0));
  double2 wn;
  if (free_proj) {
    wn = cmul(w[z], imp);
  } else {
    const double cth = cos(atan2(ratio.y, ratio.x));
    wn = cmk(w[z].x * cabs(imp) * (cth > 0.0 ? cth : 0.0), 0.0);
  }
  if (!isfinite(wn.x) || !isfinite(wn.y) || !isfinite(onew.x) || !isfinite(onew.y))
    atomicAdd(&flags[1], 1);
  w[z] = wn;
  ovlp[z] = onew;
}

// sum_z w_z Re E_L,z / sum_z w_z (complex ratio, real part, in free projection)
__global__ void __launch_bounds__(256) k_emix(int W, int free_proj, const double2* __restrict__ w,
                                              const double2* __restrict__ energy,
                                              double* __restrict__ out) {
  __shared__ double2 red[8];
  double2 num = cmk(0.0, 0.0), den = cmk(0.0, 0.0);
  for (int z = threadIdx.x; z < W; z += 256) {
    const double2 el = energy[4 * z + 3];
    if (free_proj) {
      num = cadd(num, cmul(w[z], el));
      den = cadd(den, w[z]);
    } else {
      num.x += w[z].x * el.x;
      den.x += w[z].x;
    }
  }
  num = block_sum2(num, red);
  den = block_sum2(den, red);
  if (threadIdx.x == 0) out[0] = free_proj ? cdiv(num, den).x : num.x / den.x;
}

}  // namespace

int launch_fields(afq_ctx* ctx, const double* xi_dev) {
  k_fields<<<ctx->ws.W, 256, 0, ctx->stream>>>(ctx->X, sqrt(ctx->p.dt), ctx->p.fb_cap, xi_dev,
                                               ctx->p.seed, ctx->d_step, ctx->ws.c, ctx->vbar,
                                               ctx->xbar, ctx->y, ctx->cfb, ctx->cmf);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_philox_fields(afq_ctx* ctx, uint64_t step, double* out, uint32_t* words) {
  const long total = (long)ctx->ws.W * ((ctx->X + 1) / 2);
  int grid = (int)((total + 255) / 256);
  if (grid > 148 * 16) grid = 148 * 16;
  k_philox_fields<<<grid, 256, 0, ctx->stream>>>(ctx->ws.W, ctx->X, ctx->p.seed, step, out,
                                                 words);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_vhs_fp64(afq_ctx* ctx) {
  dim3 grid((ctx->Mp + VT - 1) / VT, (ctx->ws.W + VZ - 1) / VZ);
  k_vhs_fp64<<<grid, 256, 0, ctx->stream>>>(ctx->ws.W, ctx->X, ctx->M, ctx->Mp, sqrt(ctx->p.dt),
                                            ctx->y, ctx->Lpk, ctx->tpq, ctx->A, ctx->Asum);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// Shared memory of one CTA of the FP64 propagator: three complex planes (the walker
// columns, the current and the next Taylor term) and two real ones of M x NC.
size_t propagate_fp64_smem(int M, int NC) {
  return (size_t)3 * M * NC * sizeof(double2) + (size_t)2 * M * NC * 8;
}

template <int NC, int G>
int launch_propagate_g(afq_ctx* ctx) {
  const int threads = 32 * ((G * ctx->M + 31) / 32);
  const size_t smem = propagate_fp64_smem(ctx->M, NC);
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_propagate_fp64<NC, G>, smem));
  dim3 grid((ctx->N + NC - 1) / NC, ctx->ws.W);
  if (!ctx->Asum) return afq_fail(ctx, AFQ_ERR_STATE, "FP64 propagation needs Re A + Im A");
  k_propagate_fp64<NC, G><<<grid, threads, smem, ctx->stream>>>(
      ctx->M, ctx->N, ctx->p.taylor_order, ctx->P, ctx->A, ctx->Asum, ctx->ws.phi);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// Threads per row: the G (dividing NC, G M <= 1024) that leaves the fewest idle
// lanes in the last warp.
int propagate_rows_per_thread(int M, int NC) {
  int best = 1;
  double eff = 0.0;
  for (int G = 1; G <= NC; G *= 2) {
    if (G * M > 1024) break;
    const double e = (double)(G * M) / (32.0 * ((G * M + 31) / 32));
    if (e > eff + 1e-9) {
      eff = e;
      best = G;
    }
  }
  return best;
}

template <int NC>
int launch_propagate_nc(afq_ctx* ctx) {
  switch (propagate_rows_per_thread(ctx->M, NC)) {
    case 2: if (NC >= 2) return launch_propagate_g<NC, (NC >= 2 ? 2 : 1)>(ctx); break;
    case 4: if (NC >= 4) return launch_propagate_g<NC, (NC >= 4 ? 4 : 1)>(ctx); break;
    case 8: if (NC >= 8) return launch_propagate_g<NC, (NC >= 8 ? 8 : 1)>(ctx); break;
    default: break;
  }
  return launch_propagate_g<NC, 1>(ctx);
}

// Column chunk NC (2, 4 or 8 walker columns per CTA) as chosen by the autotuner,
// narrowed while its planes do not fit one CTA's shared memory (227 KB: NC = 4
// up to M = 908, NC = 2 up to M = 1816).
int launch_propagate_fp64(afq_ctx* ctx) {
  int nc = ctx->prop_nc == 2 || ctx->prop_nc == 8 ? ctx->prop_nc : 4;
  while (nc > 2 && propagate_fp64_smem(ctx->M, nc) > 227 * 1024) nc /= 2;
  switch (nc) {
    case 2: return launch_propagate_nc<2>(ctx);
    case 8: return launch_propagate_nc<8>(ctx);
    default: return launch_propagate_nc<4>(ctx);
  }
}

int launch_weights(afq_ctx* ctx, double log_const, const double* e_shift_dev) {
  k_weights<<<(ctx->ws.W + 127) / 128, 128, 0, ctx->stream>>>(
      ctx->ws.W, log_const, e_shift_dev, ctx->p.dt, ctx->e0 - 0.5 * ctx->sum_vbar2,
      ctx->p.free_projection, ctx->ws.det, ctx->cfb, ctx->cmf, ctx->ws.ovlp, ctx->ws.w,
      ctx->flags, ctx->d_step);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_emix(afq_ctx* ctx, WalkerSet& s, double* out) {
  k_emix<<<1, 256, 0, ctx->stream>>>(s.W, ctx->p.free_projection, s.w, s.energy, out);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// ---------------------------------------------------------------------------
// Grouped launches: descriptor tables (host side)
// ---------------------------------------------------------------------------
struct GroupedStep {
  int ns = 0, nc = 4, prop_threads = 0, vhs_total = 0, prop_total = 0;
  int vhs_grid = 0, prop_grid = 0;
  size_t prop_smem = 0;
  VhsDesc* vd = nullptr;  // device tables
  PropDesc* pd = nullptr;
  int* counters = nullptr;  // [0] VHS, [1] propagation; zeroed before each VHS launch
};

namespace {

template <int NC>
const void* grouped_prop_kernel() {
  return (const void*)k_propagate_fp64_grouped<NC>;
}

const void* grouped_prop_fn(int nc) {
  return nc == 2 ? grouped_prop_kernel<2>() : grouped_prop_kernel<4>();
}

}  // namespace

void grouped_step_free(GroupedStep* g) {
  if (!g) return;
  if (g->vd) cudaFree(g->vd);
  if (g->pd) cudaFree(g->pd);
  if (g->counters) cudaFree(g->counters);
  delete g;
}

// Tiles of the systems in order of decreasing cost per tile (the dynamic tile counter
// then hands the long tiles out first); one column chunk NC for all systems: 2 when
// every system's autotuned chunk is 2, else 4 (8 columns would spill at the 64
// registers a thread of a 1024-thread CTA has).  Each column's arithmetic does not
// depend on NC, so the results are those of the systems' own launches.
int grouped_step_create(GroupedStep** out, afq_ctx* const* ctxs, int n, std::string* err) {
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || ctxs[i]->mixed || !ctxs[i]->Asum || !ctxs[i]->have_walkers) {
      *err = "grouped launches take FP64 contexts with walkers";
      return AFQ_ERR_ARG;
    }
  int nc = 2;
  for (int i = 0; i < n; ++i)
    if (ctxs[i]->prop_nc != 2) nc = 4;
  constexpr int kThreads = 1024;
  constexpr size_t kSmem = 227 * 1024;
  for (int i = 0; i < n; ++i)
    while (nc > 2 && propagate_fp64_smem(ctxs[i]->M, nc) > kSmem) nc /= 2;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::vector<VhsDesc> vd(n);
  std::vector<PropDesc> pd(n);
  // VHS: a tile costs VZ walkers x VT packed rows x X
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return ctxs[a]->X > ctxs[b]->X; });
  int tile = 0;
  for (int k = 0; k < n; ++k) {
    const afq_ctx* c = ctxs[order[k]];
    VhsDesc& d = vd[k];
    d.W = c->ws.W;
    d.X = c->X;
    d.M = c->M;
    d.Mp = c->Mp;
    d.sdt = sqrt(c->p.dt);
    d.y = c->y;
    d.Lpk = c->Lpk;
    d.tpq = c->tpq;
    d.A = c->A;
    d.Asum = c->Asum;
    d.tx = (c->Mp + VT - 1) / VT;
    d.tile0 = tile;
    tile += d.tx * ((c->ws.W + VZ - 1) / VZ);
  }
  const int vhs_total = tile;
  // propagation: a CTA tile costs U units x order x M^2 NC
  size_t smem = 0;
  std::vector<double> cost(n);
  std::vector<PropDesc> tmp(n);
  for (int i = 0; i < n; ++i) {
    const afq_ctx* c = ctxs[i];
    PropDesc& d = tmp[i];
    d.M = c->M;
    d.N = c->N;
    d.order = c->p.taylor_order;
    d.G = propagate_rows_per_thread(c->M, nc);
    d.T = 32 * ((d.G * c->M + 31) / 32);
    if (d.T > kThreads) {
      *err = "grouped propagation: too many orbitals";
      return AFQ_ERR_ARG;
    }
    d.unit_smem = (int)((propagate_fp64_smem(c->M, nc) + 15) / 16 * 16);
    d.U = kThreads / d.T;
    while (d.U > 1 && (size_t)d.U * d.unit_smem > kSmem) --d.U;
    d.chunks = (c->N + nc - 1) / nc;
    d.units = d.chunks * c->ws.W;
    d.P = c->P;
    d.A = c->A;
    d.Asum = c->Asum;
    d.phi = c->ws.phi;
    smem = std::max(smem, (size_t)d.U * d.unit_smem);
    cost[i] = (double)d.U * d.order * c->M * c->M;
  }
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  tile = 0;
  for (int k = 0; k < n; ++k) {
    pd[k] = tmp[order[k]];
    pd[k].tile0 = tile;
    tile += (pd[k].units + pd[k].U - 1) / pd[k].U;
  }
  const int prop_total = tile;

  GroupedStep* g = new (std::nothrow) GroupedStep();
  if (!g) return AFQ_ERR_NOMEM;
  g->ns = n;
  g->nc = nc;
  g->prop_threads = kThreads;
  g->prop_smem = smem;
  g->vhs_total = vhs_total;
  g->prop_total = prop_total;
  int per_sm = 0;
  bool ok = cudaMalloc((void**)&g->vd, n * sizeof(VhsDesc)) == cudaSuccess &&
            cudaMalloc((void**)&g->pd, n * sizeof(PropDesc)) == cudaSuccess &&
            cudaMalloc((void**)&g->counters, 2 * sizeof(int)) == cudaSuccess &&
            cudaMemcpy(g->vd, vd.data(), n * sizeof(VhsDesc), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(g->pd, pd.data(), n * sizeof(PropDesc), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            raise_smem_limit(grouped_prop_fn(nc), smem) == cudaSuccess;
  int dev = 0, sms = 148;
  ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vhs_fp64_grouped, 256, 0) ==
                 cudaSuccess;
  g->vhs_grid = std::min(vhs_total, sms * std::max(per_sm, 1));
  ok = ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_prop_fn(nc), kThreads,
                                                           smem) == cudaSuccess;
  g->prop_grid = std::min(prop_total, sms * std::max(per_sm, 1));
  if (!ok) {
    cudaGetLastError();
    grouped_step_free(g);
    *err = "grouped launches: device tables";
    return AFQ_ERR_CUDA;
  }
  *out = g;
  return AFQ_OK;
}

// The grouped VHS build of every system (zeroes both tile counters first).
cudaError_t grouped_step_vhs(GroupedStep* g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g->counters, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_vhs_fp64_grouped<<<g->vhs_grid, 256, 0, st>>>(g->vd, g->ns, g->vhs_total, g->counters);
  return cudaGetLastError();
}

// The grouped Taylor propagation of every system (after grouped_step_vhs).
cudaError_t grouped_step_propagate(GroupedStep* g, cudaStream_t st) {
  if (g->nc == 2)
    k_propagate_fp64_grouped<2><<<g->prop_grid, g->prop_threads, g->prop_smem, st>>>(
        g->pd, g->ns, g->prop_total, g->counters + 1);
  else
    k_propagate_fp64_grouped<4><<<g->prop_grid, g->prop_threads, g->prop_smem, st>>>(
        g->pd, g->ns, g->prop_total, g->counters + 1);
  return cudaGetLastError();
}
