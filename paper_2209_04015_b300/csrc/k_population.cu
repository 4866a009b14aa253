// Population control by the comb, and the per-block energy sums of the block
// workflow (blocks of propagation steps, each followed by one energy evaluation, as
// in the paper's example workflow, Sec. "Interface with PySCF"; the paper names
// population control among the light parts of AFQMC, Sec. "Introduction", without
// fixing an algorithm).
//
// Comb (systematic resampling): running sums C_z = w_0 + ... + w_z of the phaseless
// weights (capped at w_cap when w_cap > 0), T = C_{W-1}; W teeth t_k = (k + u)(T / W)
// for one offset u in [0, 1); new walker k copies the walker z with
// C_{z-1} <= t_k < C_z (walker matrix and stored overlap) and gets weight T / W.
// A tooth at or above C_{W-1} (rounding) goes to the last walker with positive
// weight.  The running sums are formed by one thread in index order and every
// operation is a correctly rounded FP64 add, multiply or divide, so the selection
// is a fixed function of the weights and u.
#include "afq_internal.cuh"

namespace {

constexpr int kCombThreads = 256;

__global__ void __launch_bounds__(kCombThreads)
    k_comb_select(int W, double u, double w_cap, const double2* __restrict__ w,
                  double* __restrict__ C, int* __restrict__ parents,
                  double* __restrict__ spacing, int* __restrict__ flags) {
  __shared__ double s_spacing;
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    double s = 0.0;
    int last = -1;
    for (int z = 0; z < W; ++z) {
      double wz = w[z].x;
      if (w_cap > 0.0 && wz > w_cap) wz = w_cap;
      s = __dadd_rn(s, wz);
      C[z] = s;
      if (wz > 0.0) last = z;
    }
    const bool ok = s > 0.0 && isfinite(s) && last >= 0;
    if (!ok) atomicAdd(&flags[3], 1);
    s_spacing = ok ? __ddiv_rn(s, (double)W) : -1.0;
    s_last = last;
    *spacing = s_spacing;
  }
  __syncthreads();
  const double sp = s_spacing;
  for (int k = threadIdx.x; k < W; k += kCombThreads) {
    if (!(sp > 0.0)) {  // no valid population: keep every walker where it is
      parents[k] = k;
      continue;
    }
    const double t = __dmul_rn(__dadd_rn((double)k, u), sp);
    int lo = 0, hi = W;  // first z with C_z > t (C is non-decreasing)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (C[mid] <= t)
        lo = mid + 1;
      else
        hi = mid;
    }
    parents[k] = lo < s_last ? lo : s_last;
  }
}

// New walker k <- walker parents[k]: matrix into phi_out, stored overlap into
// ovlp_out, weight T / W in place (the old weights are no longer read).  Grid
// (chunks of the matrix, walkers strided by gridDim.y).
__global__ void __launch_bounds__(256)
    k_comb_gather(int W, long MN, const int* __restrict__ parents,
                  const double* __restrict__ spacing, const double2* __restrict__ phi,
                  double2* __restrict__ phi_out, const double2* __restrict__ ovlp,
                  double2* __restrict__ ovlp_out, double2* __restrict__ w) {
  const double sp = *spacing;
  for (int k = blockIdx.y; k < W; k += gridDim.y) {
    const int z = parents[k];
    const double2* src = phi + (long)z * MN;
    double2* dst = phi_out + (long)k * MN;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
         e += (long)gridDim.x * blockDim.x)
      dst[e] = src[e];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ovlp_out[k] = ovlp[z];
      if (sp > 0.0) w[k] = make_double2(sp, 0.0);
    }
  }
}

// (sum_z w_z, sum_z w_z E_L,z) as [Re, Im, Re, Im]; one CTA, fixed reduction order.
__global__ void __launch_bounds__(256)
    k_block_sums(int W, const double2* __restrict__ w, const double2* __restrict__ energy,
                 double* __restrict__ out) {
  __shared__ double2 red_w[8], red_e[8];
  double2 sw = cmk(0.0, 0.0), se = cmk(0.0, 0.0);
  for (int z = threadIdx.x; z < W; z += 256) {
    sw = cadd(sw, w[z]);
    se = cadd(se, cmul(w[z], energy[4 * z + 3]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw.x += __shfl_down_sync(0xffffffffu, sw.x, o);
    sw.y += __shfl_down_sync(0xffffffffu, sw.y, o);
    se.x += __shfl_down_sync(0xffffffffu, se.x, o);
    se.y += __shfl_down_sync(0xffffffffu, se.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red_w[wid] = sw;
    red_e[wid] = se;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 tw = cmk(0.0, 0.0), te = cmk(0.0, 0.0);
    for (int i = 0; i < 8; ++i) {
      tw = cadd(tw, red_w[i]);
      te = cadd(te, red_e[i]);
    }
    out[0] = tw.x;
    out[1] = tw.y;
    out[2] = te.x;
    out[3] = te.y;
  }
}

// Population feedback on the energy shift (the usual diffusion Monte Carlo control):
// E_shift <- E_b - ln(T_b / W) / (dt n), with E_b = Re(sum w E_L / sum w) the block's
// mixed estimate, T_b = |sum w| its total weight and n the steps of a block, so that
// the next block brings the total weight back towards W.  With phaseless weights
// (imaginary parts zero) E_b is a real division of the real parts.
__global__ void k_shift_from_block(int free_proj, int W, double dt_n,
                                   const double* __restrict__ sums, double* __restrict__ e_shift) {
  if (threadIdx.x != 0) return;
  const double2 den = cmk(sums[0], sums[1]), num = cmk(sums[2], sums[3]);
  const double eb = free_proj ? cdiv(num, den).x : num.x / den.x;
  const double tb = free_proj ? cabs(den) : den.x;
  const double e = eb - log(tb / W) / dt_n;
  if (isfinite(e)) *e_shift = e;
}

__global__ void k_set_scalar(double* __restrict__ dst, double v) {
  if (threadIdx.x == 0) *dst = v;
}

}  // namespace

int launch_shift_from_block(afq_ctx* ctx, const double* sums_dev, int steps,
                            double* e_shift_dev) {
  k_shift_from_block<<<1, 32, 0, ctx->stream>>>(ctx->p.free_projection, ctx->ws.W,
                                                ctx->p.dt * steps, sums_dev, e_shift_dev);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int launch_set_scalar(afq_ctx* ctx, double* dst_dev, double value) {
  k_set_scalar<<<1, 32, 0, ctx->stream>>>(dst_dev, value);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}

int comb_walkers(afq_ctx* ctx, double u, double w_cap) {
  WalkerSet& s = ctx->ws;
  const int W = s.W;
  const long MN = (long)ctx->M * ctx->N;
  if (!ctx->comb_phi) {
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->comb_phi, (size_t)W * MN * sizeof(double2)));
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->comb_ovlp, (size_t)W * sizeof(double2)));
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->comb_cum, (size_t)(W + 1) * sizeof(double)));
    AFQ_CUDA(ctx, cudaMalloc((void**)&ctx->comb_parents, (size_t)W * sizeof(int)));
  }
  k_comb_select<<<1, kCombThreads, 0, ctx->stream>>>(W, u, w_cap, s.w, ctx->comb_cum,
                                                      ctx->comb_parents, ctx->comb_cum + W,
                                                      ctx->flags);
  AFQ_LAUNCHED(ctx);
  const int chunks = (int)std::min<long>((MN + 255) / 256, 8);
  k_comb_gather<<<dim3(chunks, std::min(W, 65535)), 256, 0, ctx->stream>>>(
      W, MN, ctx->comb_parents, ctx->comb_cum + W, s.phi, ctx->comb_phi, s.ovlp, ctx->comb_ovlp,
      s.w);
  AFQ_LAUNCHED(ctx);
  AFQ_CUDA(ctx, cudaMemcpyAsync(s.phi, ctx->comb_phi, (size_t)W * MN * sizeof(double2),
                                cudaMemcpyDeviceToDevice, ctx->stream));
  AFQ_CUDA(ctx, cudaMemcpyAsync(s.ovlp, ctx->comb_ovlp, (size_t)W * sizeof(double2),
                                cudaMemcpyDeviceToDevice, ctx->stream));
  return AFQ_OK;
}

void comb_free(afq_ctx* ctx) {
  for (void* p : {(void*)ctx->comb_phi, (void*)ctx->comb_ovlp, (void*)ctx->comb_cum,
                  (void*)ctx->comb_parents})
    if (p) cudaFree(p);
  ctx->comb_phi = nullptr;
  ctx->comb_ovlp = nullptr;
  ctx->comb_cum = nullptr;
  ctx->comb_parents = nullptr;
}

int launch_block_sums(afq_ctx* ctx, double* out_dev) {
  k_block_sums<<<1, 256, 0, ctx->stream>>>(ctx->ws.W, ctx->ws.w, ctx->ws.energy, out_dev);
  AFQ_LAUNCHED(ctx);
  return AFQ_OK;
}
