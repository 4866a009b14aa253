// Mixed <S^2> estimator (Sec. "Customized mixed estimators"): S^2 commutes with H, so
// its mixed estimate is unbiased, and for a single-determinant trial
//   S2_z = N_beta + M_S (M_S + 1) - tr(G_alpha G_beta),   M_S = (N_alpha - N_beta) / 2
// (the trace follows from Wick's theorem on S^2 = S_- S_+ + S_z (S_z + 1)).  With
// G_s = Psi_s theta_s^T the trace is sum_{i < nb, j < na} A_ij B_ji for
// A = theta_beta^T Psi_alpha and B = theta_alpha^T Psi_beta, 2 M na nb multiply-adds
// per walker instead of forming the M x M Green's functions.  FP64, from the theta
// the last step (or set-up) left in the walker set.
#include "afq_internal.cuh"

namespace {

constexpr int ST = 256;  // threads per walker
constexpr int SC = 32;   // orbital rows per shared-memory chunk

size_t s2_smem(int N) { return (size_t)N * (SC + 1) * (sizeof(double2) + sizeof(double)); }

// One CTA per walker; thread t owns the (beta i, alpha j) pairs t, t + ST, ...
// (PT of them at most).
template <int PT>
__global__ void __launch_bounds__(ST)
    k_spin_squared(int M, int N, int na, int nb, const double* __restrict__ psiT,
                   const double2* __restrict__ thetaT, double2* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int ld = SC + 1;
  double2* th = reinterpret_cast<double2*>(smraw);      // N x ld: theta^T rows, a chunk of p
  double* ps = reinterpret_cast<double*>(th + N * ld);  // N x ld: Psi^T rows
  __shared__ double2 red[ST / 32];
  const int z = blockIdx.x, tid = threadIdx.x;
  const int P = na * nb;
  double2 a[PT], b[PT];
#pragma unroll
  for (int k = 0; k < PT; ++k) a[k] = b[k] = cmk(0.0, 0.0);
  const double2* tz = thetaT + (long)z * N * M;
  for (int p0 = 0; p0 < M; p0 += SC) {
    const int pc = min(SC, M - p0);
    for (int e = tid; e < N * SC; e += ST) {
      const int n = e / SC, pp = e % SC;
      th[n * ld + pp] = pp < pc ? tz[(long)n * M + p0 + pp] : cmk(0.0, 0.0);
      ps[n * ld + pp] = pp < pc ? psiT[(long)n * M + p0 + pp] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      const int o = tid + k * ST;
      if (o < P) {
        const int i = o / na, j = o % na;  // beta i, alpha j
        const double2* thb = th + (na + i) * ld;
        const double2* tha = th + j * ld;
        const double* psa = ps + j * ld;
        const double* psb = ps + (na + i) * ld;
        double2 ak = a[k], bk = b[k];
        for (int pp = 0; pp < pc; ++pp) {
          ak.x = fma(thb[pp].x, psa[pp], ak.x);  // A_ij = sum_p theta_beta,pi Psi_alpha,pj
          ak.y = fma(thb[pp].y, psa[pp], ak.y);
          bk.x = fma(tha[pp].x, psb[pp], bk.x);  // B_ji = sum_p theta_alpha,pj Psi_beta,pi
          bk.y = fma(tha[pp].y, psb[pp], bk.y);
        }
        a[k] = ak;
        b[k] = bk;
      }
    }
    __syncthreads();
  }
  double2 t = cmk(0.0, 0.0);
#pragma unroll
  for (int k = 0; k < PT; ++k)
    if (tid + k * ST < P) t = cadd(t, cmul(a[k], b[k]));
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_down_sync(0xffffffffu, t.x, o);
    t.y += __shfl_down_sync(0xffffffffu, t.y, o);
  }
  if ((tid & 31) == 0) red[tid >> 5] = t;
  __syncthreads();
  if (tid == 0) {
    double2 tr = cmk(0.0, 0.0);
    for (int w = 0; w < ST / 32; ++w) tr = cadd(tr, red[w]);
    const double ms = 0.5 * (na - nb);
    out[z] = cmk(nb + ms * (ms + 1.0) - tr.x, -tr.y);
  }
}

// Re(sum_z w_z v_z / sum_z w_z) (phaseless weights: sum w Re v / sum w); one CTA.
__global__ void __launch_bounds__(256)
    k_weighted_mean(int W, int free_proj, const double2* __restrict__ w,
                    const double2* __restrict__ v, double* __restrict__ out) {
  __shared__ double2 rn[8], rd[8];
  double2 num = cmk(0.0, 0.0), den = cmk(0.0, 0.0);
  for (int z = threadIdx.x; z < W; z += 256) {
    if (free_proj) {
      num = cadd(num, cmul(w[z], v[z]));
      den = cadd(den, w[z]);
    } else {
      num.x += w[z].x * v[z].x;
      den.x += w[z].x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    num.x += __shfl_down_sync(0xffffffffu, num.x, o);
    num.y += __shfl_down_sync(0xffffffffu, num.y, o);
    den.x += __shfl_down_sync(0xffffffffu, den.x, o);
    den.y += __shfl_down_sync(0xffffffffu, den.y, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rn[threadIdx.x >> 5] = num;
    rd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 n = cmk(0.0, 0.0), d = cmk(0.0, 0.0);
    for (int i = 0; i < 8; ++i) {
      n = cadd(n, rn[i]);
      d = cadd(d, rd[i]);
    }
    out[0] = free_proj ? cdiv(n, d).x : n.x / d.x;
  }
}

template <int PT>
cudaError_t launch_s2(const afq_ctx* ctx, const WalkerSet& s, double2* out) {
  const size_t smem = s2_smem(ctx->N);
  if (smem > 48 * 1024) {
    const cudaError_t e = raise_smem_limit((const void*)k_spin_squared<PT>, smem);
    if (e != cudaSuccess) return e;
  }
  k_spin_squared<PT><<<s.W, ST, smem, ctx->stream>>>(ctx->M, ctx->N, ctx->na, ctx->nb,
                                                      ctx->psiT, s.thetaT, out);
  return cudaGetLastError();
}

// sum_z w_z theta^T_z (N x M complex) and sum_z w_z: one thread per element, the
// walkers added in index order.
__global__ void __launch_bounds__(256)
    k_theta_wsum(int W, long NM, const double2* __restrict__ w,
                 const double2* __restrict__ thetaT, double2* __restrict__ out,
                 double2* __restrict__ wsum) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < NM;
       e += (long)gridDim.x * blockDim.x) {
    double2 a = cmk(0.0, 0.0);
    for (int z = 0; z < W; ++z) a = cadd(a, cmul(w[z], thetaT[(long)z * NM + e]));
    out[e] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double2 t = cmk(0.0, 0.0);
    for (int z = 0; z < W; ++z) t = cadd(t, w[z]);
    *wsum = t;
  }
}

// <G^s>_pq = sum_j Psi_s,pj Thetabar_s,qj / sum_z w_z (G_pq = sum_j Psi_pj theta_qj),
// both spins: out is 2 x M x M complex.
__global__ void __launch_bounds__(256)
    k_one_rdm(int M, int na, int nb, const double* __restrict__ psiT,
              const double2* __restrict__ tbar, const double2* __restrict__ wsum,
              double2* __restrict__ out) {
  const long MM = (long)M * M;
  const double2 ws = *wsum;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * MM;
       e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e / MM);
    const long r = e - s * MM;
    const int p = (int)(r / M), q = (int)(r - (long)p * M);
    const int n = s ? nb : na, off = s ? na : 0;
    double2 a = cmk(0.0, 0.0);
    for (int j = 0; j < n; ++j) {
      const double ps = psiT[(long)(off + j) * M + p];
      const double2 t = tbar[(long)(off + j) * M + q];
      a.x = fma(ps, t.x, a.x);
      a.y = fma(ps, t.y, a.y);
    }
    out[e] = cdiv(a, ws);
  }
}

// grid-stride launches: enough CTAs to fill the machine, at most one per 256 elements
int stride_grid(long n) {
  const long g = (n + 255) / 256;
  return (int)(g < 148L * 16 ? (g > 0 ? g : 1) : 148L * 16);
}

}  // namespace

// Weighted mixed one-body density matrix of both spins into out_dev (2 x M x M
// complex); work: N x M complex + 1 (device scratch).
int launch_one_rdm(afq_ctx* ctx, WalkerSet& s, double2* work_dev, double2* out_dev) {
  const long NM = (long)ctx->N * ctx->M;
  k_theta_wsum<<<stride_grid(NM), 256, 0, ctx->stream>>>(s.W, NM, s.w, s.thetaT, work_dev,
                                                    work_dev + NM);
  AFQ_LAUNCHED(ctx);
  k_one_rdm<<<stride_grid(2L * ctx->M * ctx->M), 256, 0, ctx->stream>>>(
      ctx->M, ctx->na, ctx->nb, ctx->psiT, work_dev, work_dev + NM, out_dev);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_spin_squared(afq_ctx* ctx, WalkerSet& s, double2* out_dev, double* mix_dev) {
  const int pairs = ctx->na * ctx->nb;
  const int pt = (pairs + ST - 1) / ST;
  cudaError_t e;
  if (pt <= 1)
    e = launch_s2<1>(ctx, s, out_dev);
  else if (pt <= 2)
    e = launch_s2<2>(ctx, s, out_dev);
  else if (pt <= 4)
    e = launch_s2<4>(ctx, s, out_dev);
  else if (pt <= 8)
    e = launch_s2<8>(ctx, s, out_dev);
  else
    e = launch_s2<16>(ctx, s, out_dev);  // na nb <= 64 * 64 = 16 ST
  ctx->launches++;
  if (e != cudaSuccess)
    return afq_fail(ctx, AFQ_ERR_CUDA, std::string("spin squared: ") + cudaGetErrorString(e));
  if (mix_dev) {
    k_weighted_mean<<<1, 256, 0, ctx->stream>>>(s.W, ctx->p.free_projection, s.w, out_dev,
                                                mix_dev);
    AFQ_LAUNCHED(ctx);
  }
  return AFQ_OK;
}
