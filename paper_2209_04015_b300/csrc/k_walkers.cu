// Per-walker kernels of libafqmc: overlap, theta and determinant (Sec. "Overlap",
// Eq. halfgf), the force-bias / Coulomb contraction (Eq. rfb), the fused exchange
// energy (Sec. "Local energy"), energy assembly and the QR re-orthogonalisation.
//
// FP64 on B300 runs on the FP64 pipe at about 1 TFLOP/s, so these kernels are
// bound by the number of DFMA instructions: they stage operands in shared memory
// so every DFMA is fed without global-memory waits, and size grids in the
// thousands of CTAs so all 148 SMs keep their FP64 pipes busy.
#include "afq_internal.cuh"
#include "df_arith.cuh"

namespace {

constexpr int OT = 256;                                     // threads, overlap kernel
constexpr int PC = 32;                                      // Phi rows per chunk
constexpr int MAXO1 = (AFQ_NMAX * AFQ_NMAX + OT - 1) / OT;  // S entries per thread

__device__ __forceinline__ double2 warp_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Deterministic block sum of a complex value; result valid in thread 0.
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
// K1: S_s = Psi_s^T Phi_s, Gauss-Jordan inverse with partial pivoting giving
// det S_s and S_s^-1, theta_s^T = S_s^-T Phi_s^T, and E1_s = sum h~ . theta.
// One CTA per (walker, spin).
// ---------------------------------------------------------------------------

// det S and S^-1 of the split-precision walker ensemble when theta is formed on the
// tensor cores: one block of kGjWarps warps per (walker, spin) matrix, in-place
// Gauss-Jordan elimination with partial row pivoting (ties -> lowest row) on
// double-floats (n^3 complex updates instead of the augmented form's ~1.5 n^3).  Per
// pivot warp 0 finds the pivot, swaps the rows, forms the reciprocal (an FP32
// reciprocal refined by a Newton step in double-floats) and scales the pivot row; then
// every warp updates its share of the rows, lanes over columns, four rows at a time for
// independent chains.  The row swaps are undone on the columns at the end.  det S is
// accumulated in FP64 from the pivots; S^-1 is written in FP64 ([k][j], nmax apart);
// E1 follows from S^-1 and H = h~ Phi (both exact to FP64 quality), not from theta.
// A pivot with |p|^2 below 1e-36 (the double-float range) is flagged as singular.
// Nine blocks per SM (<= 56 registers): the 2 x 640 matrices of 640 walkers then run in
// one wave on 148 SMs, where eight left a second wave of 96 (0.80 -> 0.76 ms for the
// overlap class at 290 orbitals; two warps or one warp per matrix measured 0.78).
constexpr int kGjWarps = 4;
__global__ void __launch_bounds__(32 * kGjWarps, 9) k_gj_df(int units, int na, int nb, int nmax,
                                                         const double2* __restrict__ Spre,
                                                         const double2* __restrict__ H,
                                                         double2* __restrict__ sinv,
                                                         double2* __restrict__ det,
                                                         double2* __restrict__ e1, int* flags) {
  extern __shared__ __align__(16) unsigned char gjraw[];
  __shared__ DF2 s_inv;
  __shared__ int perm[AFQ_NMAX];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const long unit = blockIdx.x;
  if (unit >= units) return;
  const int n = (unit & 1) ? nb : na;
  if (n == 0) {
    if (tid == 0) {
      det[unit] = cmk(1.0, 0.0);
      e1[unit] = cmk(0.0, 0.0);
    }
    return;
  }
  DF2* a = reinterpret_cast<DF2*>(gjraw);  // n x n
  DF2* fk = a + nmax * nmax;               // column k
  const double2* Sz = Spre + unit * nmax * nmax;
  for (int e = tid; e < n * n; e += 32 * kGjWarps) a[e] = df_from(Sz[(long)(e / n) * nmax + e % n]);
  __syncthreads();
  double2 dt = cmk(1.0, 0.0);  // thread 0
  const DF2 zero = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int k = 0; k < n; ++k) {
    if (wid == 0) {
      float best = -1.f;
      int bi = k;
      for (int i = k + lane; i < n; i += 32) {
        const float2 h = a[i * n + k].hi;
        const float v = h.x * h.x + h.y * h.y;
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (bi != k)
        for (int j = lane; j < n; j += 32) {
          const DF2 t = a[k * n + j];
          a[k * n + j] = a[bi * n + j];
          a[bi * n + j] = t;
        }
      __syncwarp();
      DF2 pv = a[k * n + k];
      const float m2 = pv.hi.x * pv.hi.x + pv.hi.y * pv.hi.y;
      if (!(m2 >= 1e-36f)) {
        if (lane == 0) atomicAdd(&flags[0], 1);
        pv = DF2{make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
      }
      if (lane == 0) {
        perm[k] = bi;
        const double2 d = cmul(dt, df_to_double(pv));
        dt = bi != k ? cmk(-d.x, -d.y) : d;
      }
      const DF2 inv = df_crecip(pv);
      for (int j = lane; j < n; j += 32) a[k * n + j] = j == k ? inv : df_cmul(a[k * n + j], inv);
      for (int i = lane; i < n; i += 32) fk[i] = a[i * n + k];
      if (lane == 0) s_inv = inv;
    }
    __syncthreads();
    const DF2 inv = s_inv;
    for (int j = lane; j < n; j += 32) {
      const DF2 akj = j == k ? inv : a[k * n + j];
      // this warp's rows wid, wid + kGjWarps, ...: four at a time (independent chains)
      for (int i0 = wid; i0 < n; i0 += 4 * kGjWarps) {
        DF2 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * kGjWarps;
          if (i < n && i != k) r[u] = df_cfms(fk[i], akj, j == k ? zero : a[i * n + j]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * kGjWarps;
          if (i < n && i != k) a[i * n + j] = r[u];
        }
      }
    }
    __syncthreads();
  }
  // undo the row swaps on the columns: each thread owns a row
  for (int i = tid; i < n; i += 32 * kGjWarps)
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k) {
        const DF2 t = a[i * n + k];
        a[i * n + k] = a[i * n + p];
        a[i * n + p] = t;
      }
    }
  __syncthreads();
  double2* so = sinv + unit * nmax * nmax;
  for (int e = tid; e < n * n; e += 32 * kGjWarps)
    so[(long)(e / n) * nmax + e % n] = df_to_double(a[e]);
  if (wid == 0) {
    // E1 = sum_jp h~_jp theta_pj = tr(H S^-1) with H = h~ Phi (trial i x walker j, from
    // the overlap GEMM): lanes over the walker index j, sum over i of H_ij (S^-1)_ji
    const double2* Hz = H + unit * nmax * nmax;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int j = lane; j < n; j += 32)
      for (int i = 0; i < n; ++i) {
        const DF2 h = df_from(Hz[(long)i * nmax + j]);
        const DF2 b = a[j * n + i];
        df_mac_rn(rh, rl, h.hi.x, h.lo.x, b.hi.x, b.lo.x);
        df_mac_rn(rh, rl, -h.hi.y, -h.lo.y, b.hi.y, b.lo.y);
        df_mac_rn(ih, il, h.hi.x, h.lo.x, b.hi.y, b.lo.y);
        df_mac_rn(ih, il, h.hi.y, h.lo.y, b.hi.x, b.lo.x);
      }
    df_renorm(rh, rl);
    df_renorm(ih, il);
    df_warp_sum(rh, rl);
    df_warp_sum(ih, il);
    if (lane == 0) {
      det[unit] = dt;
      e1[unit] = cmk(f2d_bits(rh) + f2d_bits(rl), f2d_bits(ih) + f2d_bits(il));
    }
  }
}

// MO: S entries per thread (n^2 <= OT MO); the launch picks the smallest that fits,
// so that the accumulators do not hold registers sized for 64 electrons.
template <bool DF, int MO>
__global__ void __launch_bounds__(OT) k_overlap_theta(int M, int N, int na, int nb,
                                                      const double* __restrict__ psiT,
                                                      const double* __restrict__ ht,
                                                      const double2* __restrict__ phi,
                                                      double2* __restrict__ thetaT,
                                                      double2* __restrict__ det,
                                                      double2* __restrict__ e1, int* flags,
                                                      const double2* __restrict__ Spre,
                                                      int nmax, int pcr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double2 red[OT / 32];
  __shared__ int s_piv;
  __shared__ double2 s_det;
  const int z = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) {
    if (tid == 0) {
      det[2 * z + s] = cmk(1.0, 0.0);
      e1[2 * z + s] = cmk(0.0, 0.0);
    }
    return;
  }
  const int n2 = 2 * n, ldn = n | 1;
  double2* aug = reinterpret_cast<double2*>(smraw);  // n x 2n  [S | I] -> [I | S^-1]
  double2* cphi = aug + n * n2;                      // PC x ldn
  double* cpsi = reinterpret_cast<double*>(cphi + PC * ldn);  // PC x ldn
  double2* fac = reinterpret_cast<double2*>(cpsi + PC * ldn + (PC * ldn & 1));  // n
  const double2* phiz = phi + (long)z * M * N;

  // 1. S_ij = sum_p Psi_pi Phi_pj (or, with Spre, the product formed on the tensor cores:
  // W x 2 x nmax x nmax, to FP64 quality)
  double2 acc[MO];
#pragma unroll
  for (int k = 0; k < MO; ++k) acc[k] = cmk(0.0, 0.0);
  if (Spre) {
    const double2* Sz = Spre + ((long)z * 2 + s) * nmax * nmax;
#pragma unroll
    for (int k = 0; k < MO; ++k) {
      const int o = tid + k * OT;
      if (o < n * n) acc[k] = Sz[(o / n) * nmax + o % n];
    }
  }
  for (int p0 = 0; p0 < M && !Spre; p0 += PC) {
    const int pc = min(PC, M - p0);
    for (int e = tid; e < PC * n; e += OT) {
      const int pp = e / n, j = e % n;
      cphi[pp * ldn + j] = pp < pc ? phiz[(long)(p0 + pp) * N + off + j] : cmk(0.0, 0.0);
      cpsi[pp * ldn + j] = pp < pc ? psiT[(long)(off + j) * M + p0 + pp] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MO; ++k) {
      const int o = tid + k * OT;
      if (o < n * n) {
        const int i = o / n, j = o % n;
        double2 a = acc[k];
        for (int pp = 0; pp < pc; ++pp) {
          const double ps = cpsi[pp * ldn + i];
          const double2 ph = cphi[pp * ldn + j];
          a.x = fma(ps, ph.x, a.x);
          a.y = fma(ps, ph.y, a.y);
        }
        acc[k] = a;
      }
    }
    __syncthreads();
  }
  const int wid = tid >> 5, lane = tid & 31;
  if constexpr (!DF) {
#pragma unroll
    for (int k = 0; k < MO; ++k) {
      const int o = tid + k * OT;
      if (o < n * n) {
        const int i = o / n, j = o % n;
        aug[i * n2 + j] = acc[k];
        aug[i * n2 + n + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
      }
    }
    if (tid == 0) s_det = cmk(1.0, 0.0);
    __syncthreads();

    // 2. Gauss-Jordan elimination with partial pivoting (ties -> lowest row).  Per pivot
    // three barriers: warp 0 picks the pivot row and its reciprocal; all threads swap
    // the pivot row into place scaled by the reciprocal and keep the column-kc factors
    // of the other rows; then every other row is updated on the columns not yet reduced
    // (left columns > kc and the whole right half), warps over rows, lanes over columns.
    __shared__ double2 s_inv, s_old;
    for (int kc = 0; kc < n; ++kc) {
      if (tid < 32) {
        double best = -1.0;
        int bi = kc;
        for (int r = kc + tid; r < n; r += 32) {
          const double v = cabs2(aug[r * n2 + kc]);
          if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          double2 pv = aug[bi * n2 + kc];
          const bool bad = !(cabs2(pv) >= 1e-300);
          if (bad) atomicAdd(&flags[0], 1);
          const double2 d = cmul(s_det, pv);
          s_det = bi != kc ? cmk(-d.x, -d.y) : d;
          if (bad) pv = cmk(1.0, 0.0);
          s_inv = cdiv(cmk(1.0, 0.0), pv);
          s_old = aug[kc * n2 + kc];  // column kc of the row that moves to row bi
          s_piv = bi;
        }
      }
      __syncthreads();
      const int piv = s_piv;
      const double2 inv = s_inv;
      // factors of column kc for the rows after the swap (row piv receives old row kc;
      // the swap below writes only rows kc and piv, so the other reads are unaffected)
      for (int r = tid; r < n; r += OT)
        if (r != kc) fac[r] = r == piv ? s_old : aug[r * n2 + kc];
      for (int c = kc + tid; c < n2; c += OT) {
        const double2 top = aug[piv * n2 + c];
        if (piv != kc) aug[piv * n2 + c] = aug[kc * n2 + c];
        aug[kc * n2 + c] = cmul(top, inv);
      }
      __syncthreads();
      for (int r = wid; r < n; r += OT / 32) {
        if (r == kc) continue;
        const double2 f = fac[r];
        for (int c = kc + 1 + lane; c < n2; c += 32)
          aug[r * n2 + c] = cfms(f, aug[kc * n2 + c], aug[r * n2 + c]);
      }
      __syncthreads();
    }
  } else {
    // 2'. The same elimination on double-floats (split-precision walker ensembles):
    // the FP64 pipe runs 2 lanes per clock on B300 and bound the FP64 form, while a
    // double-float complex update costs ~50 FP32 operations on a 64x faster pipe.  The
    // pivot search compares the FP32 heads; the pivot's reciprocal and the determinant
    // are formed in FP64 by one thread.  Each update rounds at ~2^-47 of |f a|
    // (FP64: 2^-53), so S^-1 and det S keep ~2^-44 relative for the overlap matrices of
    // normalised walkers -- theta is formed in double-floats anyway.
    DF2* adf = reinterpret_cast<DF2*>(aug);  // n x 2n  [S | I] -> [I | S^-1]
    DF2* fdf = reinterpret_cast<DF2*>(fac);
    __shared__ DF2 s_invd, s_oldd;
    const DF2 dzero = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int k = 0; k < MO; ++k) {
      const int o = tid + k * OT;
      if (o < n * n) {
        const int i = o / n, j = o % n;
        adf[i * n2 + j] = df_from(acc[k]);
        DF2 e = dzero;
        if (i == j) e.hi.x = 1.f;
        adf[i * n2 + n + j] = e;
      }
    }
    if (tid == 0) s_det = cmk(1.0, 0.0);
    __syncthreads();
    for (int kc = 0; kc < n; ++kc) {
      if (tid < 32) {
        float best = -1.f;
        int bi = kc;
        for (int r = kc + tid; r < n; r += 32) {
          const float2 h = adf[r * n2 + kc].hi;
          const float v = h.x * h.x + h.y * h.y;
          if (v > best) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          double2 pv = df_to_double(adf[bi * n2 + kc]);
          const bool bad = !(cabs2(pv) >= 1e-300);
          if (bad) atomicAdd(&flags[0], 1);
          const double2 d = cmul(s_det, pv);
          s_det = bi != kc ? cmk(-d.x, -d.y) : d;
          if (bad) pv = cmk(1.0, 0.0);
          s_invd = df_from(cdiv(cmk(1.0, 0.0), pv));
          s_oldd = adf[kc * n2 + kc];
          s_piv = bi;
        }
      }
      __syncthreads();
      const int piv = s_piv;
      const DF2 inv = s_invd;
      for (int r = tid; r < n; r += OT)
        if (r != kc) fdf[r] = r == piv ? s_oldd : adf[r * n2 + kc];
      for (int c = kc + tid; c < n2; c += OT) {
        const DF2 top = adf[piv * n2 + c];
        if (piv != kc) adf[piv * n2 + c] = adf[kc * n2 + c];
        adf[kc * n2 + c] = df_cmul(top, inv);
      }
      __syncthreads();
      for (int r = wid; r < n; r += OT / 32) {
        if (r == kc) continue;
        const DF2 f = fdf[r];
        for (int c = kc + 1 + lane; c < n2; c += 32)
          adf[r * n2 + c] = df_cfms(f, adf[kc * n2 + c], adf[r * n2 + c]);
      }
      __syncthreads();
    }
  }

  // 3. theta^T_jp = sum_k (S^-1)_kj Phi_pk and E1 = sum_jp h~_jp theta^T_jp
  double2 e1acc = cmk(0.0, 0.0);
  if (DF) {
    // S^-1 as double-floats: the right half of the eliminated augmented matrix
    const DF2* sdf = reinterpret_cast<const DF2*>(aug) + n;  // [k][j] at slot k * n2 + j
    DF2* pdf = reinterpret_cast<DF2*>(cphi);  // Phi chunk as double-floats
    for (int p0 = 0; p0 < M; p0 += pcr) {
      const int pc = min(pcr, M - p0);
      __syncthreads();
      for (int e = tid; e < pc * n; e += OT) {
        const int pp = e / n, j = e % n;
        pdf[pp * ldn + j] = df_from(phiz[(long)(p0 + pp) * N + off + j]);
      }
      __syncthreads();
      for (int e = tid; e < n * pc; e += OT) {
        const int j = e / pc, pp = e % pc;
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int k = 0; k < n; ++k) {
          const DF2 a = sdf[k * n2 + j];
          const DF2 b = pdf[pp * ldn + k];
          df_mac(rh, rl, a.hi.x, a.lo.x, b.hi.x, b.lo.x);
          df_mac(rh, rl, -a.hi.y, -a.lo.y, b.hi.y, b.lo.y);
          df_mac(ih, il, a.hi.x, a.lo.x, b.hi.y, b.lo.y);
          df_mac(ih, il, a.hi.y, a.lo.y, b.hi.x, b.lo.x);
        }
        const double2 t = cmk(f2d_bits(rh) + f2d_bits(rl), f2d_bits(ih) + f2d_bits(il));
        thetaT[((long)z * N + off + j) * M + p0 + pp] = t;
        const double hv = ht[(long)(off + j) * M + p0 + pp];
        e1acc.x = fma(hv, t.x, e1acc.x);
        e1acc.y = fma(hv, t.y, e1acc.y);
      }
    }
  }
  for (int p0 = 0; p0 < M && !DF; p0 += pcr) {
    const int pc = min(pcr, M - p0);
    for (int e = tid; e < pc * n; e += OT) {
      const int pp = e / n, j = e % n;
      cphi[pp * ldn + j] = phiz[(long)(p0 + pp) * N + off + j];
    }
    __syncthreads();
    for (int e = tid; e < n * pc; e += OT) {
      const int j = e / pc, pp = e % pc;
      {
        double2 t = cmk(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
          const double2 sv = aug[k * n2 + n + j];
          const double2 ph = cphi[pp * ldn + k];
          t.x = fma(sv.x, ph.x, fma(-sv.y, ph.y, t.x));
          t.y = fma(sv.x, ph.y, fma(sv.y, ph.x, t.y));
        }
        const long idx = ((long)z * N + off + j) * M + p0 + pp;
        thetaT[idx] = t;
        const double hv = ht[(long)(off + j) * M + p0 + pp];
        e1acc.x = fma(hv, t.x, e1acc.x);
        e1acc.y = fma(hv, t.y, e1acc.y);
      }
    }
    __syncthreads();
  }
  const double2 tot = block_sum2(e1acc, red);
  if (tid == 0) {
    e1[2 * z + s] = tot;
    det[2 * z + s] = s_det;
  }
}

// ---------------------------------------------------------------------------
// K2 (FP64): c_zg = sum_k L~_g,k theta^T_z,k over k = (sigma, j, p), K = N M.
// 32 g x 8 walkers per CTA, one complex output per thread.
// ---------------------------------------------------------------------------
constexpr int FG = 32, FZ = 16, FK = 64;
__global__ void __launch_bounds__(256) k_force_bias_fp64(int X, int W, int K, int kchunk,
                                                         const double* __restrict__ Lt,
                                                         const double2* __restrict__ thetaT,
                                                         double2* __restrict__ out) {
  __shared__ double As[FG][FK + 1];
  __shared__ double2 Bs[FZ][FK];
  const int g0 = blockIdx.x * FG, z0 = blockIdx.y * FZ;
  const int tg = threadIdx.x % 32, tz = threadIdx.x / 32;  // walkers tz and tz + 8
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  double2 acc0 = cmk(0.0, 0.0), acc1 = cmk(0.0, 0.0);
  for (int k0 = kb; k0 < ke; k0 += FK) {
    for (int e = threadIdx.x; e < FG * FK; e += 256) {
      const int r = e / FK, kk = e % FK;
      As[r][kk] = (g0 + r < X && k0 + kk < ke) ? Lt[(long)(g0 + r) * K + k0 + kk] : 0.0;
    }
    for (int e = threadIdx.x; e < FZ * FK; e += 256) {
      const int r = e / FK, kk = e % FK;
      Bs[r][kk] = (z0 + r < W && k0 + kk < ke) ? thetaT[(long)(z0 + r) * K + k0 + kk]
                                               : cmk(0.0, 0.0);
    }
    __syncthreads();
    const int kc = min(FK, ke - k0);
    for (int kk = 0; kk < kc; ++kk) {
      const double a = As[tg][kk];
      const double2 b0 = Bs[tz][kk], b1 = Bs[tz + 8][kk];
      acc0.x = fma(a, b0.x, acc0.x);
      acc0.y = fma(a, b0.y, acc0.y);
      acc1.x = fma(a, b1.x, acc1.x);
      acc1.y = fma(a, b1.y, acc1.y);
    }
    __syncthreads();
  }
  // out: c (W x X) without a K split, else the partial sums [split][W][X]
  double2* o = out + (long)blockIdx.z * W * X;
  if (g0 + tg < X) {
    if (z0 + tz < W) o[(long)(z0 + tz) * X + g0 + tg] = acc0;
    if (z0 + tz + 8 < W) o[(long)(z0 + tz + 8) * X + g0 + tg] = acc1;
  }
}

__global__ void k_fb64_reduce(long n, int ks, const double2* __restrict__ part,
                              double2* __restrict__ c) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    double2 v = part[e];
    for (int k = 1; k < ks; ++k) v = cadd(v, part[(long)k * n + e]);
    c[e] = v;
  }
}

// ---------------------------------------------------------------------------
// K6 (FP64): exchange.  For walker z, spin s and a group of G Cholesky indices,
// T^g = L~_g,s theta_s (n x n, K = M) is formed in registers, staged in shared
// memory, and consumed at once as sum_ij T_ij T_ji; T never reaches HBM.
// ---------------------------------------------------------------------------
constexpr int ET = 256, EKC = 32;
constexpr int MAXO6 = (64 * AFQ_NMAX + ET - 1) / ET;
__global__ void __launch_bounds__(ET) k_exchange_fp64(int M, int N, int na, int nb, int X,
                                                      int G, int slots,
                                                      const double* __restrict__ Lt,
                                                      const double2* __restrict__ thetaT,
                                                      double2* __restrict__ ekp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double2 red[ET / 32];
  const int grp = blockIdx.x, z = blockIdx.y, s = blockIdx.z, tid = threadIdx.x;
  const int n = s ? nb : na, off = s ? na : 0;
  const long oidx = ((long)z * 2 + s) * slots + grp;
  if (n == 0) {
    if (tid == 0) ekp[oidx] = cmk(0.0, 0.0);
    return;
  }
  const int g0 = grp * G, gc = min(G, X - g0), R = gc * n, total = R * n;
  const int lda = EKC + 1;
  double* As = reinterpret_cast<double*>(smraw);                       // R x lda
  double2* Bs = reinterpret_cast<double2*>(As + G * n * lda + ((G * n * lda) & 1));  // n x lda
  double2* Ts = Bs + n * lda;                                          // R x n
  double2 acc[MAXO6];
#pragma unroll
  for (int k = 0; k < MAXO6; ++k) acc[k] = cmk(0.0, 0.0);
  const double2* thz = thetaT + ((long)z * N + off) * M;
  for (int p0 = 0; p0 < M; p0 += EKC) {
    for (int e = tid; e < R * EKC; e += ET) {
      const int r = e / EKC, kk = e % EKC;
      const int g = g0 + r / n, i = r % n;
      As[r * lda + kk] = p0 + kk < M ? Lt[((long)g * N + off + i) * M + p0 + kk] : 0.0;
    }
    for (int e = tid; e < n * EKC; e += ET) {
      const int j = e / EKC, kk = e % EKC;
      Bs[j * lda + kk] = p0 + kk < M ? thz[(long)j * M + p0 + kk] : cmk(0.0, 0.0);
    }
    __syncthreads();
    // the last chunk of a ragged M runs only over its valid orbitals (no FMAs on the
    // zero padding: at M = 100 that was 28 of every 128)
    const int kc = min(EKC, M - p0);
#pragma unroll
    for (int k = 0; k < MAXO6; ++k) {
      const int o = tid + k * ET;
      if (o < total) {
        const int r = o / n, j = o % n;
        double2 a = acc[k];
        if (kc == EKC) {
#pragma unroll 8
          for (int kk = 0; kk < EKC; ++kk) {
            const double l = As[r * lda + kk];
            const double2 t = Bs[j * lda + kk];
            a.x = fma(l, t.x, a.x);
            a.y = fma(l, t.y, a.y);
          }
        } else {
#pragma unroll 4
          for (int kk = 0; kk < kc; ++kk) {
            const double l = As[r * lda + kk];
            const double2 t = Bs[j * lda + kk];
            a.x = fma(l, t.x, a.x);
            a.y = fma(l, t.y, a.y);
          }
        }
        acc[k] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < MAXO6; ++k) {
    const int o = tid + k * ET;
    if (o < total) Ts[o] = acc[k];
  }
  __syncthreads();
  double2 part = cmk(0.0, 0.0);
  const int nn = n * n;
  for (int e = tid; e < gc * nn; e += ET) {
    const int g = e / nn, ij = e % nn, i = ij / n, j = ij % n;
    part = cadd(part, cmul(Ts[(g * n + i) * n + j], Ts[(g * n + j) * n + i]));
  }
  const double2 tot = block_sum2(part, red);
  if (tid == 0) ekp[oidx] = cscale(tot, -0.5);
}

// E1, EJ = 1/2 sum_g c_g^2, EK and E_L = e0 + E1 + EJ + EK per walker.
__global__ void __launch_bounds__(256) k_energy_assemble(int X, int ngroups, double e0,
                                                         const double2* __restrict__ e1,
                                                         const double2* __restrict__ c,
                                                         const double2* __restrict__ ekp,
                                                         double2* __restrict__ energy) {
  __shared__ double2 red[8];
  const int z = blockIdx.x;
  double2 ej = cmk(0.0, 0.0);
  for (int g = threadIdx.x; g < X; g += 256) {
    const double2 v = c[(long)z * X + g];
    ej = cadd(ej, cmul(v, v));
  }
  ej = block_sum2(ej, red);
  double2 ek = cmk(0.0, 0.0);
  for (int e = threadIdx.x; e < 2 * ngroups; e += 256) ek = cadd(ek, ekp[(long)z * 2 * ngroups + e]);
  ek = block_sum2(ek, red);
  if (threadIdx.x == 0) {
    const double2 one = cadd(e1[2 * z], e1[2 * z + 1]);
    const double2 coul = cscale(ej, 0.5);
    energy[4 * z + 0] = one;
    energy[4 * z + 1] = coul;
    energy[4 * z + 2] = ek;
    energy[4 * z + 3] = cadd(cmk(e0, 0.0), cadd(one, cadd(coul, ek)));
  }
}

// ---------------------------------------------------------------------------
// K7: QR of each spin block by classical Gram-Schmidt with reorthogonalisation
// (Daniel, Gragg, Kaufman and Stewart, Math. Comp. 30, 1976): a column is projected
// once, and a second time only when the first projection removed more than half of
// its squared norm (|v'|^2 < |v|^2 / 2); otherwise the one pass already leaves it
// orthogonal to working precision.  Walkers re-orthogonalised every few steps are
// close to orthonormal, so the second pass (half of classical Gram-Schmidt twice) is
// rarely taken.  diag(R) comes out real and positive.  Works on a column-major copy Qw.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_qr(int M, int N, int na, int nb,
                                            double2* __restrict__ phi, double2* __restrict__ Qw,
                                            double* __restrict__ detR, int* flags) {
  __shared__ double2 rs[AFQ_NMAX + 1];
  __shared__ double2 red[32];
  __shared__ double s_norm;
  __shared__ int s_again;
  __shared__ double rdiag[AFQ_NMAX];  // diag R, logged once at the end
  const int z = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nt = blockDim.x, nw = nt >> 5;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) {
    if (tid == 0) detR[2 * z + s] = 1.0;
    return;
  }
  double2* phz = phi + (long)z * M * N;
  double2* Q = Qw + ((long)z * N + off) * M;  // column j at Q + j * M
  for (int e = tid; e < M * n; e += nt) {
    const int p = e / n, j = e % n;
    Q[(long)j * M + p] = phz[(long)p * N + off + j];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double2* v = Q + (long)j * M;
    for (int pass = 0; pass < 2; ++pass) {
      if (j > 0) {
        // r_i = q_i^H v for i < j; the first pass also takes |v|^2 as index j
        const int last = pass == 0 ? j : j - 1;
        for (int i = wid; i <= last; i += nw) {
          const double2* qi = i < j ? Q + (long)i * M : v;
          double2 d = cmk(0.0, 0.0);
          for (int p = lane; p < M; p += 32) d = cfma_conj(qi[p], v[p], d);
          d = warp_sum2(d);
          if (lane == 0) rs[i] = d;
        }
        __syncthreads();
        for (int p = tid; p < M; p += nt) {
          double2 t = v[p];
          for (int i = 0; i < j; ++i) t = cfms(Q[(long)i * M + p], rs[i], t);
          v[p] = t;
        }
        __syncthreads();
      }
      double2 nr = cmk(0.0, 0.0);
      for (int p = tid; p < M; p += nt) nr.x += cabs2(v[p]);
      nr = block_sum2(nr, red);
      if (tid == 0) {
        const int again = pass == 0 && j > 0 && nr.x < 0.5 * rs[j].x;
        s_again = again;
        if (!again) {
          const double rjj = sqrt(nr.x);
          if (!(rjj > 0.0)) atomicAdd(&flags[0], 1);
          s_norm = rjj > 0.0 ? 1.0 / rjj : 1.0;
          rdiag[j] = rjj > 0.0 ? rjj : 1.0;
        }
      }
      __syncthreads();
      if (!s_again) break;
    }
    const double inv = s_norm;
    for (int p = tid; p < M; p += nt) v[p] = cscale(v[p], inv);
    __syncthreads();
  }
  // log det R = sum_j log R_jj, the logs in parallel off the column loop
  double lg = 0.0;
  for (int j = tid; j < n; j += nt) lg += log(rdiag[j]);
  const double logdet = block_sum2(cmk(lg, 0.0), red).x;
  for (int e = tid; e < M * n; e += nt) {
    const int p = e / n, j = e % n;
    phz[(long)p * N + off + j] = Q[(long)j * M + p];
  }
  if (tid == 0) detR[2 * z + s] = exp(logdet);
}

// The same Gram-Schmidt QR with reorthogonalisation on double-floats (the walker
// ensembles of split-precision contexts).  B300 runs FP64 at 2 lanes per clock per SM,
// which bound the FP64 form of this kernel (M n^2 complex multiply-adds per matrix);
// double-float products and sums run on the 64x faster FP32 pipe at ~2^-44 relative,
// far below the ~2^-31 that the split-precision propagation leaves in the walkers.
// R's diagonal, its logarithms and the reorthogonalisation test are FP64.  Qw holds
// the double-float columns (the same 16 bytes per complex entry as the FP64 form).
__global__ void __launch_bounds__(256) k_qr_df(int M, int N, int na, int nb,
                                               double2* __restrict__ phi, DF2* __restrict__ Qw,
                                               double* __restrict__ detR, int* flags) {
  __shared__ DF2 rs[AFQ_NMAX + 1];
  __shared__ float2 red[32];
  __shared__ double2 redd[32];
  __shared__ float s_inv_h, s_inv_l;
  __shared__ int s_again;
  __shared__ double rdiag[AFQ_NMAX];
  const int z = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nt = blockDim.x, nw = nt >> 5;
  const int n = s ? nb : na, off = s ? na : 0;
  if (n == 0) {
    if (tid == 0) detR[2 * z + s] = 1.0;
    return;
  }
  double2* phz = phi + (long)z * M * N;
  DF2* Q = Qw + ((long)z * N + off) * M;  // column j at Q + j * M
  for (int e = tid; e < M * n; e += nt) {
    const int p = e / n, j = e % n;
    Q[(long)j * M + p] = df_from(phz[(long)p * N + off + j]);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    DF2* v = Q + (long)j * M;
    for (int pass = 0; pass < 2; ++pass) {
      if (j > 0) {
        // r_i = q_i^H v for i < j; the first pass also takes |v|^2 as index j
        const int last = pass == 0 ? j : j - 1;
        for (int i = wid; i <= last; i += nw) {
          const DF2* qi = i < j ? Q + (long)i * M : v;
          float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
          for (int p = lane; p < M; p += 32) {
            const DF2 a = qi[p], b = v[p];
            df_mac_rn(rh, rl, a.hi.x, a.lo.x, b.hi.x, b.lo.x);
            df_mac_rn(rh, rl, a.hi.y, a.lo.y, b.hi.y, b.lo.y);
            df_mac_rn(ih, il, a.hi.x, a.lo.x, b.hi.y, b.lo.y);
            df_mac_rn(ih, il, -a.hi.y, -a.lo.y, b.hi.x, b.lo.x);
          }
          df_renorm(rh, rl);
          df_renorm(ih, il);
          df_warp_sum(rh, rl);
          df_warp_sum(ih, il);
          if (lane == 0) rs[i] = DF2{make_float2(rh, ih), make_float2(rl, il)};
        }
        __syncthreads();
        for (int p = tid; p < M; p += nt) {
          DF2 t = v[p];
          for (int i = 0; i < j; ++i) t = df_cfms(Q[(long)i * M + p], rs[i], t);
          v[p] = t;
        }
        __syncthreads();
      }
      float nh = 0.f, nl = 0.f;
      for (int p = tid; p < M; p += nt) {
        const DF2 b = v[p];
        df_mac_rn(nh, nl, b.hi.x, b.lo.x, b.hi.x, b.lo.x);
        df_mac_rn(nh, nl, b.hi.y, b.lo.y, b.hi.y, b.lo.y);
      }
      df_renorm(nh, nl);
      df_warp_sum(nh, nl);
      if (lane == 0) red[wid] = make_float2(nh, nl);
      __syncthreads();
      if (tid == 0) {
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < nw; ++w) df_add(th, tl, red[w].x, red[w].y);
        const double nr = f2d_bits(th) + f2d_bits(tl);
        const double before = f2d_bits(rs[j].hi.x) + f2d_bits(rs[j].lo.x);
        const int again = pass == 0 && j > 0 && nr < 0.5 * before;
        s_again = again;
        if (!again) {
          const double rjj = sqrt(nr);
          if (!(rjj > 0.0)) atomicAdd(&flags[0], 1);
          float ih2, il2;
          df_split(rjj > 0.0 ? 1.0 / rjj : 1.0, ih2, il2);
          s_inv_h = ih2;
          s_inv_l = il2;
          rdiag[j] = rjj > 0.0 ? rjj : 1.0;
        }
      }
      __syncthreads();
      if (!s_again) break;
    }
    const float ih = s_inv_h, il = s_inv_l;
    for (int p = tid; p < M; p += nt) {
      const DF2 b = v[p];
      float rh = 0.f, rl = 0.f, qh = 0.f, ql = 0.f;
      df_mac_rn(rh, rl, b.hi.x, b.lo.x, ih, il);
      df_mac_rn(qh, ql, b.hi.y, b.lo.y, ih, il);
      df_renorm(rh, rl);
      df_renorm(qh, ql);
      v[p] = DF2{make_float2(rh, qh), make_float2(rl, ql)};
    }
    __syncthreads();
  }
  // log det R = sum_j log R_jj, the logs in parallel off the column loop
  double lg = 0.0;
  for (int j = tid; j < n; j += nt) lg += log(rdiag[j]);
  const double logdet = block_sum2(cmk(lg, 0.0), redd).x;
  for (int e = tid; e < M * n; e += nt) {
    const int p = e / n, j = e % n;
    phz[(long)p * N + off + j] = df_to_double(Q[(long)j * M + p]);
  }
  if (tid == 0) detR[2 * z + s] = exp(logdet);
}

__global__ void k_qr_finish(int W, const double* __restrict__ detR, double2* __restrict__ ovlp) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < W) ovlp[z] = cscale(ovlp[z], 1.0 / (detR[2 * z] * detR[2 * z + 1]));
}

__global__ void k_init_overlap(int W, const double2* __restrict__ det, double2* __restrict__ ovlp) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < W) ovlp[z] = cmul(det[2 * z], det[2 * z + 1]);
}

size_t overlap_smem(int n) {
  const int ldn = n | 1;
  return (size_t)n * 2 * n * 16 + (size_t)PC * ldn * 16 + (size_t)PC * ldn * 8 + 8 + (size_t)n * 16;
}

size_t exchange_smem(int G, int n) {
  const int lda = EKC + 1;
  return (size_t)G * n * lda * 8 + 8 + (size_t)n * lda * 16 + (size_t)G * n * n * 16;
}

}  // namespace

int exchange_group_size(int nmax) { return nmax > 0 ? (64 / nmax > 1 ? 64 / nmax : 1) : 1; }

// Rows of Phi per theta chunk (<= PC): each chunk's n x rows outputs are spread over
// the OT threads, so the count minimising the number of thread passes over all chunks,
// ceil(M / rows) ceil(n rows / OT), keeps every thread busy (290 orbitals and 26
// electrons: 29 rows, 30 passes instead of 37 with 32 rows).  Larger rows win ties.
int theta_chunk_rows(int M, int n) {
  int best = PC;
  long best_passes = -1;
  for (int r = PC; r >= 1; --r) {
    const long passes = (long)((M + r - 1) / r) * ((long)(n * r + OT - 1) / OT);
    if (best_passes < 0 || passes < best_passes) {
      best_passes = passes;
      best = r;
    }
  }
  return best;
}

// df: the elimination and theta in double-float arithmetic (split-precision walker
// ensembles); S is FP64 (or the tensor cores' product to FP64 quality), det S and the
// one-body energy accumulate in FP64 either way.
template <bool DF, int MO>
int launch_overlap_mo(afq_ctx* ctx, WalkerSet& s) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  const size_t smem = overlap_smem(nmax);
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_overlap_theta<DF, MO>, smem));
  // split-precision walker ensembles take S from the tensor cores (k_overlap_tc.cu)
  const double2* Spre = nullptr;
  if (DF && ctx->ov_S && &s == &ctx->ws) {
    AFQ_TRY(launch_overlap_s_tc(ctx, s));
    Spre = ctx->ov_S;
  }
  k_overlap_theta<DF, MO><<<dim3(s.W, 2), OT, smem, ctx->stream>>>(
      ctx->M, ctx->N, ctx->na, ctx->nb, ctx->psiT, ctx->ht, s.phi, s.thetaT, s.det, s.e1,
      ctx->flags, Spre, nmax, theta_chunk_rows(ctx->M, nmax));
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

template <bool DF>
int launch_overlap_df(afq_ctx* ctx, WalkerSet& s) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  const int need = (nmax * nmax + OT - 1) / OT;
  if (need <= 1) return launch_overlap_mo<DF, 1>(ctx, s);
  if (need <= 2) return launch_overlap_mo<DF, 2>(ctx, s);
  if (need <= 4) return launch_overlap_mo<DF, 4>(ctx, s);
  if (need <= 8) return launch_overlap_mo<DF, 8>(ctx, s);
  return launch_overlap_mo<DF, MAXO1>(ctx, s);
}

// The split-precision walker ensemble with the tensor-core theta: S and H = h~ Phi on
// the tensor cores (7 digits), det S, S^-1 and E1 by one block per matrix, theta on the
// tensor cores (the force bias's and the exchange's digit count).
int launch_overlap_gj_tc(afq_ctx* ctx, WalkerSet& s) {
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  AFQ_TRY(launch_overlap_s_tc(ctx, s));
  const size_t smem = (size_t)(nmax * nmax + nmax) * sizeof(DF2);
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_gj_df, smem));
  const long units = 2L * s.W;
  k_gj_df<<<(unsigned)units, 32 * kGjWarps, smem, ctx->stream>>>(
      (int)units, ctx->na, ctx->nb, nmax, ctx->ov_S, ctx->ov_H, ctx->th_sinv, s.det, s.e1,
      ctx->flags);
  AFQ_LAUNCHED(ctx);
  return launch_theta_tc(ctx, s);
}

// theta of the walker ensemble to double-float precision (~2^-44) whichever form the
// step used: the mixed estimators read theta itself, not only its digits
int launch_theta_precise(afq_ctx* ctx) { return launch_overlap_df<true>(ctx, ctx->ws); }

int launch_overlap_theta(afq_ctx* ctx, WalkerSet& s, bool df) {
  if (df && ctx->ov_S && ctx->th_sinv && &s == &ctx->ws) return launch_overlap_gj_tc(ctx, s);
  return df ? launch_overlap_df<true>(ctx, s) : launch_overlap_df<false>(ctx, s);
}

// c = L~ theta over K = N M.  Small grids are split over K (partial sums reduced in a
// fixed order, so the result does not depend on scheduling) when the walker set fits
// the context's partial-sum buffer.
int launch_force_bias_fp64(afq_ctx* ctx, WalkerSet& s) {
  const int K = ctx->N * ctx->M;
  dim3 grid((ctx->X + FG - 1) / FG, (s.W + FZ - 1) / FZ, 1);
  const long tiles = (long)grid.x * grid.y;
  int ks = (int)((4 * 148 + tiles - 1) / tiles);
  const int kblocks = (K + FK - 1) / FK;
  if (ks > kblocks) ks = kblocks;
  if (ks > kFbSplitMax) ks = kFbSplitMax;
  if (ks < 1 || !ctx->fb64_part || (long)s.W * ctx->X > ctx->fb64_part_wx) ks = 1;
  const int kchunk = ((kblocks + ks - 1) / ks) * FK;
  ks = (K + kchunk - 1) / kchunk;
  grid.z = ks;
  k_force_bias_fp64<<<grid, 256, 0, ctx->stream>>>(ctx->X, s.W, K, kchunk, ctx->Lt, s.thetaT,
                                                   ks > 1 ? ctx->fb64_part : s.c);
  AFQ_LAUNCHED(ctx);
  if (ks > 1) {
    const long n = (long)s.W * ctx->X;
    k_fb64_reduce<<<(int)((n + 255) / 256 < 148 * 16 ? (n + 255) / 256 : 148 * 16), 256, 0,
                    ctx->stream>>>(n, ks, ctx->fb64_part, s.c);
    AFQ_LAUNCHED(ctx);
  }
  return AFQ_OK;
}

// Largest g-group for n_max electrons per spin: G n^2 outputs fit the per-thread
// register tile and the shared memory of one CTA.
int exchange_group_max(int nmax) {
  if (nmax <= 0) return 1;
  int g = (64 * AFQ_NMAX) / (nmax * nmax);
  while (g > 1 && exchange_smem(g, nmax) > 200 * 1024) --g;
  return g < 1 ? 1 : g;
}

int launch_exchange_fp64(afq_ctx* ctx, WalkerSet& s) {
  if (ctx->ex_stored) return launch_exchange_v(ctx, s);
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  const int G = ctx->ex_G_fp64 > 0 ? ctx->ex_G_fp64 : exchange_group_size(nmax);
  const int ngroups = (ctx->X + G - 1) / G;
  if (ngroups > ctx->ex_groups) return afq_fail(ctx, AFQ_ERR_STATE, "exchange groups exceed slots");
  const size_t smem = exchange_smem(G, nmax);
  AFQ_CUDA(ctx, raise_smem_limit((const void*)k_exchange_fp64, smem));
  k_exchange_fp64<<<dim3(ngroups, s.W, 2), ET, smem, ctx->stream>>>(
      ctx->M, ctx->N, ctx->na, ctx->nb, ctx->X, G, ctx->ex_groups, ctx->Lt, s.thetaT, s.ekp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

// The exchange kernel with explicit device pointers and stream (no context): the
// partial sums go to ekp, W x 2 x ceil(X / G) complex slots.
cudaError_t launch_exchange_fp64_raw(int M, int X, int na, int nb, int W, const double* Lt,
                                     const double2* thetaT, double2* ekp, cudaStream_t stream) {
  const int nmax = na > nb ? na : nb;
  const int G = exchange_group_size(nmax);
  const int ngroups = (X + G - 1) / G;
  const size_t smem = exchange_smem(G, nmax);
  // shared with the context path: never lowers the limit its launches rely on
  cudaError_t e = raise_smem_limit((const void*)k_exchange_fp64, smem);
  if (e != cudaSuccess) return e;
  k_exchange_fp64<<<dim3(ngroups, W, 2), ET, smem, stream>>>(M, na + nb, na, nb, X, G, ngroups,
                                                             Lt, thetaT, ekp);
  return cudaGetLastError();
}

int launch_energy_assemble(afq_ctx* ctx, WalkerSet& s) {
  k_energy_assemble<<<s.W, 256, 0, ctx->stream>>>(ctx->X, ctx->ex_groups, ctx->e0, s.e1, s.c,
                                                  s.ekp, s.energy);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_qr(afq_ctx* ctx, WalkerSet& s, double2* Qw) {
  // one thread per orbital row up to 256 (whole warps); larger M loops over the rows
  // (the FP64 pipe is already busy with several 256-thread CTAs per SM: measured no
  // gain from 320 threads at M = 290)
  int nt = (ctx->M + 31) / 32 * 32;
  if (nt < 64) nt = 64;
  if (nt > 256) nt = 256;
  if (ctx->mixed && &s == &ctx->ws)  // split-precision walkers: double-float QR
    k_qr_df<<<dim3(s.W, 2), nt, 0, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb, s.phi,
                                                   reinterpret_cast<DF2*>(Qw), ctx->detR,
                                                   ctx->flags);
  else
    k_qr<<<dim3(s.W, 2), nt, 0, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb, s.phi, Qw,
                                                ctx->detR, ctx->flags);
  AFQ_LAUNCHED(ctx);
  k_qr_finish<<<(s.W + 127) / 128, 128, 0, ctx->stream>>>(s.W, ctx->detR, s.ovlp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_init_overlap(afq_ctx* ctx, WalkerSet& s) {
  k_init_overlap<<<(s.W + 127) / 128, 128, 0, ctx->stream>>>(s.W, s.det, s.ovlp);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
