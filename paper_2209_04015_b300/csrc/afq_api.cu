// C ABI of libafqmc (declared in include/afqmc.h): context, input validation,
// set-up sequence and the per-step launch sequence on the context's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "afq_internal.cuh"

int afq_fail(afq_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

cudaError_t raise_smem_limit(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;  // largest size set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = limit[{dev, fn}];
  if (smem <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

namespace {

void drop_graph(afq_ctx* ctx);

template <class T>
int dalloc(afq_ctx* ctx, T** p, size_t n) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return afq_fail(ctx, AFQ_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return AFQ_OK;
}

template <class T>
void dfree(T** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

int free_walker_set(WalkerSet& s) {
  dfree(&s.phi);
  dfree(&s.thetaT);
  dfree(&s.det);
  dfree(&s.e1);
  dfree(&s.c);
  dfree(&s.ekp);
  dfree(&s.energy);
  dfree(&s.w);
  dfree(&s.ovlp);
  s.W = 0;
  return AFQ_OK;
}

int alloc_walker_set(afq_ctx* ctx, WalkerSet& s, int W) {
  free_walker_set(s);
  const size_t M = ctx->M, N = ctx->N, X = ctx->X;
  AFQ_TRY(dalloc(ctx, &s.phi, W * M * N));
  AFQ_TRY(dalloc(ctx, &s.thetaT, W * N * M));
  AFQ_TRY(dalloc(ctx, &s.det, 2 * (size_t)W));
  AFQ_TRY(dalloc(ctx, &s.e1, 2 * (size_t)W));
  AFQ_TRY(dalloc(ctx, &s.c, W * X));
  AFQ_TRY(dalloc(ctx, &s.ekp, (size_t)W * 2 * ctx->ex_groups));
  AFQ_TRY(dalloc(ctx, &s.energy, 4 * (size_t)W));
  AFQ_TRY(dalloc(ctx, &s.w, W));
  AFQ_TRY(dalloc(ctx, &s.ovlp, W));
  // exchange slots that a tiling leaves unwritten must read as zero
  AFQ_CUDA(ctx, cudaMemsetAsync(s.ekp, 0, (size_t)W * 2 * ctx->ex_groups * sizeof(double2),
                                ctx->stream));
  s.W = W;
  return AFQ_OK;
}

int sync(afq_ctx* ctx) {
  AFQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return AFQ_OK;
}

// Reads and clears the device flags; maps them to a status.
int check_flags(afq_ctx* ctx) {
  int h[4] = {0, 0, 0, 0};
  AFQ_CUDA(ctx, cudaMemcpyAsync(h, ctx->flags, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(h), ctx->stream));
  AFQ_TRY(sync(ctx));
  const std::string all = " (singular pivots " + std::to_string(h[0]) + ", non-finite values " +
                          std::to_string(h[1]) + ", tensor-core time-outs " + std::to_string(h[2]) + ")";
  if (h[2]) return afq_fail(ctx, AFQ_ERR_CUDA, "tensor-core pipeline wait timed out" + all);
  if (h[0]) return afq_fail(ctx, AFQ_ERR_SINGULAR, "singular pivot(s)" + all);
  if (h[1]) return afq_fail(ctx, AFQ_ERR_NAN, "non-finite weight(s)" + all);
  if (h[3])
    return afq_fail(ctx, AFQ_ERR_NAN,
                    "population control: total weight not positive and finite (walkers kept)");
  return AFQ_OK;
}

cudaEvent_t take_event(afq_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs one launch wrapper, bracketed by an event pair when profiling is on.
template <class F>
int timed(afq_ctx* ctx, int kid, F&& launch) {
  if (!ctx->profiling || ctx->capturing) return launch();
  afq_ctx::ProfRec r{kid, take_event(ctx), take_event(ctx)};
  AFQ_CUDA(ctx, cudaEventRecord(r.a, ctx->stream));
  int rc = launch();
  AFQ_CUDA(ctx, cudaEventRecord(r.b, ctx->stream));
  ctx->prof.push_back(r);
  return rc;
}

// Folds finished event pairs into the per-class totals.
int drain_profile(afq_ctx* ctx) {
  if (ctx->prof.empty()) return AFQ_OK;
  AFQ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->prof) {
    float ms = 0.f;
    AFQ_CUDA(ctx, cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->prof_ms[r.kid] += ms;
    ctx->prof_n[r.kid] += 1;
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->prof.clear();
  return AFQ_OK;
}

// Green's-function intermediates of a walker set: theta, det, E1 and c.  The
// walker ensemble of a split-precision context takes the tensor-core force bias;
// other sets (the trial at set-up) always use FP64.
int green_and_bias(afq_ctx* ctx, WalkerSet& s) {
  const bool tc = ctx->mixed && &s == &ctx->ws;
  AFQ_TRY(timed(ctx, AFQ_K_OVERLAP, [&] { return launch_overlap_theta(ctx, s, tc); }));
  if (tc) {
    AFQ_TRY(timed(ctx, AFQ_K_FORCE_BIAS, [&] {
      int rc = launch_slice_theta(ctx, s);
      return rc != AFQ_OK ? rc : launch_force_bias_tc(ctx, s);
    }));
  } else {
    AFQ_TRY(timed(ctx, AFQ_K_FORCE_BIAS, [&] { return launch_force_bias_fp64(ctx, s); }));
  }
  return AFQ_OK;
}

int energy_kernels(afq_ctx* ctx, WalkerSet& s) {
  const bool tc = ctx->mixed && &s == &ctx->ws;
  if (tc) {
    AFQ_TRY(timed(ctx, AFQ_K_EXCHANGE, [&] { return launch_exchange_tc(ctx, s); }));
  } else {
    AFQ_TRY(timed(ctx, AFQ_K_EXCHANGE, [&] { return launch_exchange_fp64(ctx, s); }));
  }
  AFQ_TRY(timed(ctx, AFQ_K_ENERGY, [&] { return launch_energy_assemble(ctx, s); }));
  return AFQ_OK;
}

int free_walkers(afq_ctx* ctx) {
  chain_free(ctx);
  comb_free(ctx);
  free_walker_set(ctx->ws);
  dfree(&ctx->xi);
  dfree(&ctx->xbar);
  dfree(&ctx->y);
  dfree(&ctx->cfb);
  dfree(&ctx->cmf);
  dfree(&ctx->A);
  dfree(&ctx->Asum);
  dfree(&ctx->detR);
  dfree(&ctx->fb64_part);
  ctx->fb64_part_wx = 0;
  ctx->have_walkers = false;
  return AFQ_OK;
}

int free_trial(afq_ctx* ctx) {
  mixed_free(ctx);
  dfree(&ctx->psiT);
  dfree(&ctx->Lt);
  dfree(&ctx->ht);
  dfree(&ctx->vbar);
  dfree(&ctx->hpp);
  dfree(&ctx->P);
  dfree(&ctx->Vx);
  ctx->ex_stored = false;
  ctx->have_trial = false;
  return free_walkers(ctx);
}

bool symmetric(const double* a, int M, double* dev_out) {
  double mx = 0.0, dv = 0.0;
  for (int p = 0; p < M; ++p)
    for (int q = 0; q < M; ++q) {
      mx = std::fmax(mx, std::fabs(a[(size_t)p * M + q]));
      if (q > p) dv = std::fmax(dv, std::fabs(a[(size_t)p * M + q] - a[(size_t)q * M + p]));
    }
  *dev_out = dv;
  return dv <= 1e-12 * (mx > 0.0 ? mx : 1.0) && std::isfinite(mx);
}

// One hybrid-propagation step (Sec. "Review of AFQMC") on the context's stream.
// A step in three parts: the fields, the VHS build and propagation (which a batch in
// grouped mode launches for all its systems at once), and the rest.
int step_fields(afq_ctx* ctx, const double* xi_dev) {
  return timed(ctx, AFQ_K_FIELDS, [&] { return launch_fields(ctx, xi_dev); });
}

int step_finish(afq_ctx* ctx, const double* e_shift_dev) {
  const double log_const = -ctx->p.dt * (ctx->e0 - 0.5 * ctx->sum_vbar2 - ctx->e_shift);
  AFQ_TRY(green_and_bias(ctx, ctx->ws));
  AFQ_TRY(timed(ctx, AFQ_K_WEIGHTS, [&] { return launch_weights(ctx, log_const, e_shift_dev); }));
  ctx->step++;
  if (ctx->p.qr_period > 0 && ctx->step % (uint64_t)ctx->p.qr_period == 0)
    AFQ_TRY(timed(ctx, AFQ_K_QR, [&] { return launch_qr(ctx, ctx->ws, ctx->A); }));
  return AFQ_OK;
}

int one_step(afq_ctx* ctx, const double* xi_dev, const double* e_shift_dev = nullptr) {
  AFQ_TRY(step_fields(ctx, xi_dev));
  if (ctx->mixed) {
    AFQ_TRY(timed(ctx, AFQ_K_VHS, [&] { return launch_vhs_tc(ctx); }));
    AFQ_TRY(timed(ctx, AFQ_K_PROPAGATE, [&] { return launch_propagate_tc(ctx); }));
  } else {
    AFQ_TRY(timed(ctx, AFQ_K_VHS, [&] { return launch_vhs_fp64(ctx); }));
    AFQ_TRY(timed(ctx, AFQ_K_PROPAGATE, [&] { return launch_propagate_fp64(ctx); }));
  }
  return step_finish(ctx, e_shift_dev);
}

}  // namespace

extern "C" {

void afq_default_params(afq_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dt = 0.005;
  p->taylor_order = 6;
  p->qr_period = 5;
  p->seed = 1;
  p->precision = AFQ_FP64;
  p->has_e_shift = 0;
  p->e_shift = 0.0;
  p->fb_cap = 0.0;
  p->free_projection = 0;
  p->split_slices = 4;
  p->prop_slices = 4;
  p->exchange = AFQ_EXCHANGE_AUTO;
  p->prop_kernel = 0;
}

int afq_create(afq_ctx** out, const afq_params* params, void* cuda_stream) {
  if (!out) return AFQ_ERR_ARG;
  *out = nullptr;
  afq_ctx* ctx = new (std::nothrow) afq_ctx();
  if (!ctx) return AFQ_ERR_NOMEM;
  if (params) {
    ctx->p = *params;
  } else {
    afq_default_params(&ctx->p);
  }
  if (ctx->p.split_slices == 0) ctx->p.split_slices = 4;
  if (ctx->p.prop_slices == 0) ctx->p.prop_slices = 4;
  if (!(ctx->p.dt > 0.0) || ctx->p.taylor_order < 1 || ctx->p.taylor_order > 32 ||
      ctx->p.qr_period < 0 ||
      (ctx->p.precision != AFQ_FP64 && ctx->p.precision != AFQ_SPLIT_BF16) ||
      ctx->p.split_slices < 1 || ctx->p.split_slices > 7 || ctx->p.prop_slices < 1 ||
      ctx->p.prop_slices > 7 || ctx->p.exchange < AFQ_EXCHANGE_AUTO ||
      ctx->p.exchange > AFQ_EXCHANGE_STORED || ctx->p.prop_kernel < 0 ||
      ctx->p.prop_kernel > 2) {
    delete ctx;
    return AFQ_ERR_ARG;
  }
  ctx->mixed = ctx->p.precision == AFQ_SPLIT_BF16;
  ctx->S = ctx->p.split_slices;
  ctx->Sp = ctx->p.prop_slices;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    delete ctx;
    return AFQ_ERR_CUDA;
  }
  if (cudaMalloc((void**)&ctx->flags, 4 * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->flags, 0, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_step, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->d_step, 0, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->emix, sizeof(double)) != cudaSuccess) {
    cudaFree(ctx->flags);
    delete ctx;
    return AFQ_ERR_CUDA;
  }
  *out = ctx;
  return AFQ_OK;
}

int afq_destroy(afq_ctx* ctx) {
  if (!ctx) return AFQ_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  free_trial(ctx);
  dfree(&ctx->h1);
  dfree(&ctx->L);
  dfree(&ctx->Lpk);
  dfree(&ctx->tpq);
  drop_graph(ctx);
  dfree(&ctx->flags);
  dfree(&ctx->d_step);
  dfree(&ctx->emix);
  dfree(&ctx->scratch);
  for (auto& r : ctx->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
  return AFQ_OK;
}

const char* afq_last_error(const afq_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int afq_init_hamiltonian(afq_ctx* ctx, int M, int X, const double* h1, const double* L, double e0) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!h1 || !L) return afq_fail(ctx, AFQ_ERR_ARG, "h1 and L must not be NULL");
  if (M < 1 || M > AFQ_MMAX) return afq_fail(ctx, AFQ_ERR_ARG, "M out of range [1, 1024]");
  if (X < 1) return afq_fail(ctx, AFQ_ERR_ARG, "X must be >= 1");
  if (!std::isfinite(e0)) return afq_fail(ctx, AFQ_ERR_ARG, "e0 not finite");
  double dv;
  if (!symmetric(h1, M, &dv))
    return afq_fail(ctx, AFQ_ERR_ARG, "h1 not symmetric (max |h - h^T| = " + std::to_string(dv) + ")");
  for (int g = 0; g < X; ++g)
    if (!symmetric(L + (size_t)g * M * M, M, &dv))
      return afq_fail(ctx, AFQ_ERR_ARG, "L_" + std::to_string(g) + " not symmetric");
  free_trial(ctx);
  ctx->M = M;
  ctx->X = X;
  ctx->Mp = M * (M + 1) / 2;
  ctx->e0 = e0;
  const size_t MM = (size_t)M * M;
  AFQ_TRY(dalloc(ctx, &ctx->h1, MM));
  AFQ_TRY(dalloc(ctx, &ctx->L, (size_t)X * MM));
  AFQ_TRY(dalloc(ctx, &ctx->Lpk, (size_t)X * ctx->Mp));
  AFQ_TRY(dalloc(ctx, &ctx->tpq, (size_t)ctx->Mp));
  std::vector<int2> tpq(ctx->Mp);
  for (int p = 0, t = 0; p < M; ++p)
    for (int q = p; q < M; ++q) tpq[t++] = make_int2(p, q);
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->h1, h1, MM * 8, cudaMemcpyHostToDevice, ctx->stream));
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->L, L, (size_t)X * MM * 8, cudaMemcpyHostToDevice, ctx->stream));
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->tpq, tpq.data(), tpq.size() * sizeof(int2),
                                cudaMemcpyHostToDevice, ctx->stream));
  AFQ_TRY(launch_pack_L(ctx));
  AFQ_TRY(sync(ctx));
  ctx->have_ham = true;
  return AFQ_OK;
}

int afq_init_trial(afq_ctx* ctx, int na, int nb, const double* psi_a, const double* psi_b) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_ham) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_hamiltonian first");
  if (na < 0 || nb < 0 || na > AFQ_NMAX || nb > AFQ_NMAX || na + nb < 1)
    return afq_fail(ctx, AFQ_ERR_ARG, "need 0 <= na, nb <= 64 and na + nb >= 1");
  if (na > ctx->M || nb > ctx->M) return afq_fail(ctx, AFQ_ERR_ARG, "more electrons than orbitals");
  if ((na && !psi_a) || (nb && !psi_b)) return afq_fail(ctx, AFQ_ERR_ARG, "trial pointer NULL");
  free_trial(ctx);
  const int M = ctx->M, X = ctx->X, N = na + nb;
  ctx->na = na;
  ctx->nb = nb;
  ctx->N = N;
  ctx->ex_groups = X;  // one slot per g: room for any g-group size
  ctx->ex_G_fp64 = 0;
  ctx->prop_nc = 4;
  const size_t MM = (size_t)M * M;
  std::vector<double> psiT((size_t)N * M);
  for (int p = 0; p < M; ++p) {
    for (int i = 0; i < na; ++i) psiT[(size_t)i * M + p] = psi_a[(size_t)p * na + i];
    for (int i = 0; i < nb; ++i) psiT[(size_t)(na + i) * M + p] = psi_b[(size_t)p * nb + i];
  }
  for (double v : psiT)
    if (!std::isfinite(v)) return afq_fail(ctx, AFQ_ERR_ARG, "trial not finite");
  AFQ_TRY(dalloc(ctx, &ctx->psiT, (size_t)N * M));
  AFQ_TRY(dalloc(ctx, &ctx->Lt, (size_t)X * N * M));
  AFQ_TRY(dalloc(ctx, &ctx->ht, (size_t)N * M));
  AFQ_TRY(dalloc(ctx, &ctx->vbar, (size_t)X));
  AFQ_TRY(dalloc(ctx, &ctx->hpp, MM));
  AFQ_TRY(dalloc(ctx, &ctx->P, MM));
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->psiT, psiT.data(), psiT.size() * 8, cudaMemcpyHostToDevice,
                                ctx->stream));
  // L~_g = Psi^T L_g (N x M per g) and h~ = Psi^T h1
  AFQ_TRY(launch_dgemm(ctx, N, M, M, 1.0, ctx->psiT, M, 1, 0, ctx->L, M, 1, (long)MM, 0.0, ctx->Lt,
                       M, 1, (long)N * M, X, 1));
  AFQ_TRY(launch_dgemm(ctx, N, M, M, 1.0, ctx->psiT, M, 1, 0, ctx->h1, M, 1, 0, 0.0, ctx->ht, M,
                       1, 0, 1, 1));
  AFQ_TRY(launch_vbar(ctx));
  // sum_g L_g L_g as one GEMM over k = (g, r): A(p, k) = L[k M + p] (L_g symmetric)
  const int tiles = ((M + 31) / 32) * ((M + 31) / 32);
  int ksplit = (600 + tiles - 1) / tiles;
  if (ksplit > X * M / 64) ksplit = X * M / 64 > 0 ? X * M / 64 : 1;
  if (ksplit > 256) ksplit = 256;
  double* s2part = nullptr;
  AFQ_TRY(dalloc(ctx, &s2part, (size_t)ksplit * MM));
  int rc = launch_dgemm(ctx, M, M, X * M, 1.0, ctx->L, 1, M, 0, ctx->L, M, 1, 0, 0.0, s2part, M, 1,
                        (long)MM, 1, ksplit);
  if (rc == AFQ_OK) rc = launch_hpp(ctx, s2part, ksplit);
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&s2part);
  AFQ_TRY(rc);
  // P = exp(-dt h''/2) by scaling and squaring of a degree-18 Taylor polynomial
  std::vector<double> hpp(MM), vbar(X);
  AFQ_CUDA(ctx, cudaMemcpy(hpp.data(), ctx->hpp, MM * 8, cudaMemcpyDeviceToHost));
  AFQ_CUDA(ctx, cudaMemcpy(vbar.data(), ctx->vbar, (size_t)X * 8, cudaMemcpyDeviceToHost));
  ctx->sum_vbar2 = 0.0;
  for (double v : vbar) ctx->sum_vbar2 += v * v;
  double norm1 = 0.0;
  for (int q = 0; q < M; ++q) {
    double s = 0.0;
    for (int p = 0; p < M; ++p) s += std::fabs(hpp[(size_t)p * M + q]);
    norm1 = std::fmax(norm1, s);
  }
  norm1 *= 0.5 * ctx->p.dt;
  if (!std::isfinite(norm1)) return afq_fail(ctx, AFQ_ERR_NAN, "h'' not finite");
  int sq = 0;
  while (norm1 / std::ldexp(1.0, sq) > 0.5) ++sq;
  double *Bm = nullptr, *E = nullptr, *T = nullptr;
  rc = dalloc(ctx, &Bm, MM);
  if (rc == AFQ_OK) rc = dalloc(ctx, &E, MM);
  if (rc == AFQ_OK) rc = dalloc(ctx, &T, MM);
  if (rc == AFQ_OK) rc = launch_axpby(ctx, (int)MM, -0.5 * ctx->p.dt / std::ldexp(1.0, sq), ctx->hpp, 0.0, Bm);
  if (rc == AFQ_OK) rc = launch_set_identity(ctx, M, E);
  for (int k = 18; k >= 1 && rc == AFQ_OK; --k) {
    rc = launch_set_identity(ctx, M, T);
    if (rc == AFQ_OK)
      rc = launch_dgemm(ctx, M, M, M, 1.0 / k, Bm, M, 1, 0, E, M, 1, 0, 1.0, T, M, 1, 0, 1, 1);
    std::swap(E, T);
  }
  for (int k = 0; k < sq && rc == AFQ_OK; ++k) {
    rc = launch_dgemm(ctx, M, M, M, 1.0, E, M, 1, 0, E, M, 1, 0, 0.0, T, M, 1, 0, 1, 1);
    std::swap(E, T);
  }
  if (rc == AFQ_OK)
    rc = cudaMemcpyAsync(ctx->P, E, MM * 8, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess
             ? AFQ_OK
             : afq_fail(ctx, AFQ_ERR_CUDA, "copy P");
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&Bm);
  dfree(&E);
  dfree(&T);
  AFQ_TRY(rc);
  // Exchange: the stored half-rotated tensor when asked for, or (AUTO) when it fits a
  // quarter of the free memory (at most 16 GiB) and needs fewer multiply-adds than
  // forming T per (walker, g): (n M)^2 against 2 X n^2 M.  Split-precision contexts
  // add the bf16 planes of V' for the tensor-core form.
  {
    double vbytes = 8.0 * ((double)na * M * na * M + (double)nb * M * nb * M);
    if (ctx->mixed) vbytes += exchange_tcv_bytes(ctx, (M + 31) / 32 * 32);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
    const double budget = std::fmin(0.25 * (double)fr, 16.0 * 1073741824.0);
    ctx->ex_stored = ctx->p.exchange == AFQ_EXCHANGE_STORED ||
                     (ctx->p.exchange == AFQ_EXCHANGE_AUTO && vbytes <= budget && M < 1.5 * X);
    // the direct tensor-core exchange keeps a float tail accumulator (at most 4 digits);
    // more digits (the FP64-quality setting) take the stored form when it fits at all
    if (ctx->mixed && ctx->S > 4 && !ctx->ex_stored) {
      if (ctx->p.exchange == AFQ_EXCHANGE_AUTO && vbytes <= 0.9 * (double)fr)
        ctx->ex_stored = true;
      else
        return afq_fail(ctx, AFQ_ERR_ARG,
                        "split_slices > 4 needs the stored exchange (the direct tensor-core "
                        "exchange takes at most 4 digits)");
    }
    if (ctx->ex_stored) {
      AFQ_TRY(build_exchange_v(ctx));
      const int slots = exchange_v_slots(ctx);
      if (slots > ctx->ex_groups) ctx->ex_groups = slots;
    }
  }
  ctx->have_trial = true;
  // trial energy: the energy kernels on a one-walker set equal to the trial
  WalkerSet t;
  rc = alloc_walker_set(ctx, t, 1);
  std::vector<double2> phi((size_t)M * N);
  for (int p = 0; p < M; ++p)
    for (int j = 0; j < N; ++j) phi[(size_t)p * N + j] = make_double2(psiT[(size_t)j * M + p], 0.0);
  if (rc == AFQ_OK)
    rc = cudaMemcpyAsync(t.phi, phi.data(), phi.size() * 16, cudaMemcpyHostToDevice, ctx->stream) ==
                 cudaSuccess
             ? AFQ_OK
             : afq_fail(ctx, AFQ_ERR_CUDA, "copy trial");
  if (rc == AFQ_OK) rc = green_and_bias(ctx, t);   // FP64: t is not the walker ensemble
  if (rc == AFQ_OK) rc = energy_kernels(ctx, t);
  double2 e[4];
  if (rc == AFQ_OK)
    rc = cudaMemcpyAsync(e, t.energy, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess
             ? AFQ_OK
             : afq_fail(ctx, AFQ_ERR_CUDA, "copy energy");
  if (rc == AFQ_OK) rc = sync(ctx);
  free_walker_set(t);
  AFQ_TRY(rc);
  AFQ_TRY(check_flags(ctx));
  ctx->e_trial = e[3].x;
  ctx->e_shift = ctx->p.has_e_shift ? ctx->p.e_shift : ctx->e_trial;
  if (ctx->mixed) {
    AFQ_TRY(mixed_init_trial(ctx));
    if (ctx->ex_stored) AFQ_TRY(mixed_exchange_v_init(ctx));
    AFQ_TRY(mixed_prop_init_trial(ctx));
    AFQ_TRY(sync(ctx));
  }
  return AFQ_OK;
}

int afq_trial_energy(afq_ctx* ctx, double* e_out) {
  if (!ctx || !e_out) return AFQ_ERR_ARG;
  if (!ctx->have_trial) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_trial first");
  *e_out = ctx->e_trial;
  return AFQ_OK;
}

int afq_exchange_algorithm(afq_ctx* ctx, int* algo_out) {
  if (!ctx || !algo_out) return AFQ_ERR_ARG;
  if (!ctx->have_trial) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_trial first");
  *algo_out = ctx->ex_stored ? AFQ_EXCHANGE_STORED : AFQ_EXCHANGE_DIRECT;
  return AFQ_OK;
}

int afq_prop_digits(afq_ctx* ctx, int* digits, int count, double* x_out) {
  if (!ctx || !digits || count < 0) return AFQ_ERR_ARG;
  if (!ctx->have_trial || !ctx->mixed)
    return afq_fail(ctx, AFQ_ERR_STATE, "split-precision context with a trial needed");
  const int n = ctx->p.taylor_order + 2;
  for (int i = 0; i < n && i < count; ++i) digits[i] = ctx->prop_digits[i];
  if (x_out) *x_out = ctx->prop_x;
  return AFQ_OK;
}

int afq_init_walkers(afq_ctx* ctx, int W, const double* phi, const double* w) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_trial) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_trial first");
  if (W < 1 || W > (1 << 24)) return afq_fail(ctx, AFQ_ERR_ARG, "W out of range");
  free_walkers(ctx);
  const size_t M = ctx->M, N = ctx->N, X = ctx->X;
  AFQ_TRY(alloc_walker_set(ctx, ctx->ws, W));
  AFQ_TRY(dalloc(ctx, &ctx->xi, W * X));
  AFQ_TRY(dalloc(ctx, &ctx->xbar, W * X));
  AFQ_TRY(dalloc(ctx, &ctx->y, W * X));
  AFQ_TRY(dalloc(ctx, &ctx->cfb, (size_t)W));
  AFQ_TRY(dalloc(ctx, &ctx->cmf, (size_t)W));
  // A holds i sqrt(dt) V per walker during a step and is the QR workspace after it
  AFQ_TRY(dalloc(ctx, &ctx->A, (size_t)W * M * (M > N ? M : N)));
  if (!ctx->mixed) AFQ_TRY(dalloc(ctx, &ctx->Asum, (size_t)W * M * M));
  AFQ_TRY(dalloc(ctx, &ctx->detR, 2 * (size_t)W));
  AFQ_TRY(dalloc(ctx, &ctx->fb64_part, (size_t)kFbSplitMax * W * ctx->X));
  ctx->fb64_part_wx = (long)W * ctx->X;
  AFQ_CUDA(ctx, cudaMemsetAsync(ctx->xbar, 0, W * X * 16, ctx->stream));
  std::vector<double2> h;
  if (phi) {
    AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.phi, phi, W * M * N * 16, cudaMemcpyHostToDevice,
                                  ctx->stream));
  } else {
    std::vector<double> psiT(N * M);
    AFQ_CUDA(ctx, cudaMemcpy(psiT.data(), ctx->psiT, N * M * 8, cudaMemcpyDeviceToHost));
    h.resize(W * M * N);
    for (int z = 0; z < W; ++z)
      for (size_t p = 0; p < M; ++p)
        for (size_t j = 0; j < N; ++j) h[(z * M + p) * N + j] = make_double2(psiT[j * M + p], 0.0);
    AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.phi, h.data(), h.size() * 16, cudaMemcpyHostToDevice,
                                  ctx->stream));
  }
  std::vector<double2> wv(W);
  for (int z = 0; z < W; ++z) wv[z] = make_double2(w ? w[z] : 1.0, 0.0);
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.w, wv.data(), W * 16, cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->mixed) {
    AFQ_TRY(mixed_init_walkers(ctx));
    AFQ_TRY(mixed_prop_init_walkers(ctx));
  }
  AFQ_TRY(green_and_bias(ctx, ctx->ws));
  AFQ_TRY(launch_init_overlap(ctx, ctx->ws));
  AFQ_CUDA(ctx, cudaMemsetAsync(ctx->d_step, 0, sizeof(unsigned long long), ctx->stream));
  AFQ_TRY(sync(ctx));
  ctx->step = 0;
  ctx->have_walkers = true;
  return check_flags(ctx);
}

static int propagate_impl(afq_ctx* ctx, const double* fields, int nsteps, bool dev) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (nsteps < 0) return afq_fail(ctx, AFQ_ERR_ARG, "nsteps < 0");
  const size_t WX = (size_t)ctx->ws.W * ctx->X;
  for (int k = 0; k < nsteps; ++k) {
    const double* xi = nullptr;
    if (fields && dev) {
      xi = fields + k * WX;
    } else if (fields) {
      AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->xi, fields + k * WX, WX * 8, cudaMemcpyHostToDevice,
                                    ctx->stream));
      xi = ctx->xi;
    }
    AFQ_TRY(one_step(ctx, xi));
  }
  if (dev) return AFQ_OK;
  return check_flags(ctx);
}

int afq_propagate(afq_ctx* ctx, const double* fields, int nsteps) {
  return propagate_impl(ctx, fields, nsteps, false);
}

int afq_propagate_dev(afq_ctx* ctx, const double* fields_dev, int nsteps) {
  return propagate_impl(ctx, fields_dev, nsteps, true);
}

static int energy_impl(afq_ctx* ctx) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  AFQ_TRY(energy_kernels(ctx, ctx->ws));
  AFQ_TRY(timed(ctx, AFQ_K_ENERGY, [&] { return launch_emix(ctx, ctx->ws, ctx->emix); }));
  return AFQ_OK;
}

int afq_local_energy(afq_ctx* ctx, double* e_out, double* e_mix) {
  AFQ_TRY(energy_impl(ctx));
  if (e_out)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_out, ctx->ws.energy, (size_t)ctx->ws.W * 4 * 16,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  if (e_mix)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_mix, ctx->emix, 8, cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_TRY(sync(ctx));
  return check_flags(ctx);
}

int afq_local_energy_dev(afq_ctx* ctx, double* e_out_dev, double* e_mix_dev) {
  AFQ_TRY(energy_impl(ctx));
  if (e_out_dev)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_out_dev, ctx->ws.energy, (size_t)ctx->ws.W * 4 * 16,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  if (e_mix_dev)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_mix_dev, ctx->emix, 8, cudaMemcpyDeviceToDevice, ctx->stream));
  return AFQ_OK;
}

int afq_orthogonalise(afq_ctx* ctx) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  chain_free(ctx);  // a chain tape refers to the walkers before this QR
  AFQ_TRY(timed(ctx, AFQ_K_QR, [&] { return launch_qr(ctx, ctx->ws, ctx->A); }));
  AFQ_TRY(sync(ctx));
  return check_flags(ctx);
}

static int comb_checks(afq_ctx* ctx, double w_cap) {
  if (ctx->p.free_projection)
    return afq_fail(ctx, AFQ_ERR_STATE, "the comb needs the phaseless (real) weights");
  if (!(w_cap >= 0.0) || !std::isfinite(w_cap))
    return afq_fail(ctx, AFQ_ERR_ARG, "w_cap must be finite and >= 0");
  return AFQ_OK;
}

int afq_comb(afq_ctx* ctx, double u, double w_cap, int* parents) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  AFQ_TRY(comb_checks(ctx, w_cap));
  if (!(u >= 0.0 && u < 1.0)) return afq_fail(ctx, AFQ_ERR_ARG, "comb offset u outside [0, 1)");
  chain_free(ctx);  // a chain tape refers to the walkers before the comb
  AFQ_TRY(comb_walkers(ctx, u, w_cap));
  AFQ_TRY(green_and_bias(ctx, ctx->ws));
  if (parents)
    AFQ_CUDA(ctx, cudaMemcpyAsync(parents, ctx->comb_parents, (size_t)ctx->ws.W * sizeof(int),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_TRY(sync(ctx));
  return check_flags(ctx);
}

int afq_run_blocks(afq_ctx* ctx, int nblocks, int steps_per_block, const double* u,
                   double w_cap, int shift_feedback, double* sums) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (nblocks < 0 || steps_per_block < 1)
    return afq_fail(ctx, AFQ_ERR_ARG, "nblocks < 0 or steps_per_block < 1");
  if (nblocks > 0 && !sums) return afq_fail(ctx, AFQ_ERR_ARG, "sums is NULL");
  if (u) {
    AFQ_TRY(comb_checks(ctx, w_cap));
    for (int b = 0; b < nblocks; ++b)
      if (!(u[b] >= 0.0 && u[b] < 1.0))
        return afq_fail(ctx, AFQ_ERR_ARG, "comb offset u outside [0, 1)");
  }
  if (nblocks == 0) return AFQ_OK;
  chain_free(ctx);
  double* d = nullptr;  // nblocks x 4 block sums, then the device energy shift
  AFQ_TRY(dalloc(ctx, &d, (size_t)nblocks * 4 + 1));
  double* es = shift_feedback ? d + (size_t)nblocks * 4 : nullptr;
  int rc = es ? launch_set_scalar(ctx, es, ctx->e_shift) : AFQ_OK;
  for (int b = 0; b < nblocks && rc == AFQ_OK; ++b) {
    for (int k = 0; k < steps_per_block && rc == AFQ_OK; ++k) rc = one_step(ctx, nullptr, es);
    if (rc == AFQ_OK) rc = energy_kernels(ctx, ctx->ws);
    if (rc == AFQ_OK) rc = launch_block_sums(ctx, d + 4 * (size_t)b);
    if (rc == AFQ_OK && es)
      rc = launch_shift_from_block(ctx, d + 4 * (size_t)b, steps_per_block, es);
    if (rc == AFQ_OK && u) {
      rc = comb_walkers(ctx, u[b], w_cap);
      if (rc == AFQ_OK) rc = green_and_bias(ctx, ctx->ws);
    }
  }
  if (rc == AFQ_OK &&
      cudaMemcpyAsync(sums, d, (size_t)nblocks * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy block sums");
  double shift = ctx->e_shift;
  if (rc == AFQ_OK && es &&
      cudaMemcpyAsync(&shift, es, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy energy shift");
  if (rc == AFQ_OK) rc = sync(ctx);
  if (rc == AFQ_OK) ctx->e_shift = shift;  // later steps continue with the fed-back shift
  dfree(&d);
  return rc == AFQ_OK ? check_flags(ctx) : rc;
}

int afq_get_e_shift(afq_ctx* ctx, double* e_shift) {
  if (!ctx || !e_shift) return AFQ_ERR_ARG;
  *e_shift = ctx->e_shift;
  return AFQ_OK;
}

int afq_spin_squared(afq_ctx* ctx, double* s2_out, double* s2_mix) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  const size_t W = ctx->ws.W;
  // split precision forms the step's theta at the force bias's digit count: the
  // estimator takes it in double-floats
  if (ctx->mixed && ctx->th_sinv) AFQ_TRY(launch_theta_precise(ctx));
  double* d = nullptr;  // W complex values, then the weighted estimate
  AFQ_TRY(dalloc(ctx, &d, 2 * W + 1));
  int rc = launch_spin_squared(ctx, ctx->ws, reinterpret_cast<double2*>(d), d + 2 * W);
  if (rc == AFQ_OK && s2_out &&
      cudaMemcpyAsync(s2_out, d, 2 * W * sizeof(double), cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy S^2");
  if (rc == AFQ_OK && s2_mix &&
      cudaMemcpyAsync(s2_mix, d + 2 * W, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy weighted S^2");
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&d);
  return rc == AFQ_OK ? check_flags(ctx) : rc;
}

int afq_one_rdm(afq_ctx* ctx, double* g_out) {
  if (!ctx || !g_out) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  const size_t NM = (size_t)ctx->N * ctx->M, MM2 = 2 * (size_t)ctx->M * ctx->M;
  if (ctx->mixed && ctx->th_sinv) AFQ_TRY(launch_theta_precise(ctx));  // as for S^2
  double* d = nullptr;  // Thetabar (N x M complex), sum w, then the two matrices
  AFQ_TRY(dalloc(ctx, &d, 2 * (NM + 1 + MM2)));
  double2* work = reinterpret_cast<double2*>(d);
  double2* out = work + NM + 1;
  int rc = launch_one_rdm(ctx, ctx->ws, work, out);
  if (rc == AFQ_OK &&
      cudaMemcpyAsync(g_out, out, MM2 * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy one-body density matrix");
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&d);
  return rc == AFQ_OK ? check_flags(ctx) : rc;
}

static int get_impl(afq_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (!ctx || !dst) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  AFQ_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return sync(ctx);
}

int afq_get_walkers(afq_ctx* ctx, double* phi) {
  if (!ctx) return AFQ_ERR_ARG;
  return get_impl(ctx, phi, ctx->ws.phi, (size_t)ctx->ws.W * ctx->M * ctx->N * 16);
}
int afq_get_weights(afq_ctx* ctx, double* w) {
  if (!ctx) return AFQ_ERR_ARG;
  return get_impl(ctx, w, ctx->ws.w, (size_t)ctx->ws.W * 16);
}
int afq_get_overlaps(afq_ctx* ctx, double* o) {
  if (!ctx) return AFQ_ERR_ARG;
  return get_impl(ctx, o, ctx->ws.ovlp, (size_t)ctx->ws.W * 16);
}
int afq_get_force_bias(afq_ctx* ctx, double* xbar) {
  if (!ctx) return AFQ_ERR_ARG;
  return get_impl(ctx, xbar, ctx->xbar, (size_t)ctx->ws.W * ctx->X * 16);
}
int afq_get_step(afq_ctx* ctx, uint64_t* step) {
  if (!ctx || !step) return AFQ_ERR_ARG;
  *step = ctx->step;
  return AFQ_OK;
}

int afq_set_state(afq_ctx* ctx, const double* phi, const double* w, const double* ovlp,
                  uint64_t step) {
  if (!ctx || !phi || !w) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  chain_free(ctx);
  const size_t W = ctx->ws.W;
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.phi, phi, W * ctx->M * ctx->N * 16, cudaMemcpyHostToDevice,
                                ctx->stream));
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.w, w, W * 16, cudaMemcpyHostToDevice, ctx->stream));
  AFQ_TRY(green_and_bias(ctx, ctx->ws));
  if (ovlp) {
    AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->ws.ovlp, ovlp, W * 16, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    AFQ_TRY(launch_init_overlap(ctx, ctx->ws));
  }
  ctx->step = step;
  const unsigned long long st = step;
  AFQ_CUDA(ctx, cudaMemcpyAsync(ctx->d_step, &st, sizeof(st), cudaMemcpyHostToDevice, ctx->stream));
  AFQ_TRY(sync(ctx));
  return check_flags(ctx);
}

int afq_philox_fields(afq_ctx* ctx, uint64_t step, double* out) {
  if (!ctx || !out) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  double* d = nullptr;
  AFQ_TRY(dalloc(ctx, &d, (size_t)ctx->ws.W * ctx->X));
  int rc = launch_philox_fields(ctx, step, d, nullptr);
  if (rc == AFQ_OK)
    rc = cudaMemcpyAsync(out, d, (size_t)ctx->ws.W * ctx->X * 8, cudaMemcpyDeviceToHost,
                         ctx->stream) == cudaSuccess
             ? AFQ_OK
             : afq_fail(ctx, AFQ_ERR_CUDA, "copy fields");
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&d);
  return rc;
}

int afq_philox_words(afq_ctx* ctx, uint64_t step, uint32_t* out) {
  if (!ctx || !out) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  const size_t n = (size_t)ctx->ws.W * ((ctx->X + 1) / 2) * 4;
  uint32_t* d = nullptr;
  AFQ_TRY(dalloc(ctx, &d, n));
  int rc = launch_philox_fields(ctx, step, nullptr, d);
  if (rc == AFQ_OK)
    rc = cudaMemcpyAsync(out, d, n * 4, cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess
             ? AFQ_OK
             : afq_fail(ctx, AFQ_ERR_CUDA, "copy words");
  if (rc == AFQ_OK) rc = sync(ctx);
  dfree(&d);
  return rc;
}

int afq_profile_enable(afq_ctx* ctx, int on) {
  if (!ctx) return AFQ_ERR_ARG;
  AFQ_TRY(drain_profile(ctx));
  if (on)
    for (int k = 0; k < AFQ_K_COUNT; ++k) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_n[k] = 0;
    }
  ctx->profiling = on != 0;
  return AFQ_OK;
}

int afq_profile_read(afq_ctx* ctx, int kernel, double* total_ms, uint64_t* launches) {
  if (!ctx || kernel < 0 || kernel >= AFQ_K_COUNT) return AFQ_ERR_ARG;
  AFQ_TRY(drain_profile(ctx));
  if (total_ms) *total_ms = ctx->prof_ms[kernel];
  if (launches) *launches = ctx->prof_n[kernel];
  return AFQ_OK;
}

const char* afq_kernel_name(int kernel) {
  static const char* names[AFQ_K_COUNT] = {"fields", "vhs", "propagate", "overlap_theta",
                                           "force_bias", "weights", "qr", "exchange", "energy"};
  return kernel >= 0 && kernel < AFQ_K_COUNT ? names[kernel] : nullptr;
}


// ===========================================================================
// CUDA graphs, batches of systems and the autotuner
// ===========================================================================
}  // extern "C"

struct afq_batch {
  std::vector<afq_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nsteps = 0;
  int grouped = 0;              // 1: VHS and propagation as grouped launches (FP64)
  GroupedStep* gs = nullptr;    // their descriptor tables (built at capture)
  std::string err;
};

namespace {

// Records nsteps steps (device Philox fields) and the local energy after each one
// on ctx->stream, which is being captured; the host step mirror is restored.
int record_steps(afq_ctx* ctx, int nsteps) {
  const uint64_t step0 = ctx->step;
  ctx->capturing = true;
  int rc = AFQ_OK;
  for (int k = 0; k < nsteps && rc == AFQ_OK; ++k) {
    rc = one_step(ctx, nullptr);
    if (rc == AFQ_OK) rc = energy_impl(ctx);
  }
  ctx->capturing = false;
  ctx->step = step0;
  return rc;
}

// Stage-major recording of a batch in grouped mode, on the batch's streams (being
// captured from b->origin): per step, every system's fields on its own branch, the
// grouped VHS build and propagation of all systems on the origin stream, then the
// rest of every system's step and its local energy on the branches again.
int record_grouped(afq_batch* b, int nsteps) {
  const size_t n = b->ctx.size();
  std::vector<cudaStream_t> own(n);
  std::vector<uint64_t> step0(n);
  for (size_t i = 0; i < n; ++i) {
    own[i] = b->ctx[i]->stream;
    step0[i] = b->ctx[i]->step;
    b->ctx[i]->stream = b->streams[i];
    b->ctx[i]->capturing = true;
  }
  auto fork = [&]() {
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) return AFQ_ERR_CUDA;
    for (size_t i = 0; i < n; ++i)
      if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return AFQ_ERR_CUDA;
    return AFQ_OK;
  };
  auto join = [&]() {
    for (size_t i = 0; i < n; ++i)
      if (cudaEventRecord(b->events[i], b->streams[i]) != cudaSuccess ||
          cudaStreamWaitEvent(b->origin, b->events[i], 0) != cudaSuccess)
        return AFQ_ERR_CUDA;
    return AFQ_OK;
  };
  int rc = AFQ_OK;
  for (int k = 0; k < nsteps && rc == AFQ_OK; ++k) {
    rc = fork();
    for (size_t i = 0; i < n && rc == AFQ_OK; ++i) rc = step_fields(b->ctx[i], nullptr);
    if (rc == AFQ_OK) rc = join();
    if (rc == AFQ_OK && (grouped_step_vhs(b->gs, b->origin) != cudaSuccess ||
                         grouped_step_propagate(b->gs, b->origin) != cudaSuccess))
      rc = AFQ_ERR_CUDA;
    if (rc == AFQ_OK) rc = fork();
    for (size_t i = 0; i < n && rc == AFQ_OK; ++i) {
      rc = step_finish(b->ctx[i], nullptr);
      if (rc == AFQ_OK) rc = energy_impl(b->ctx[i]);
      if (rc != AFQ_OK) b->err = b->ctx[i]->err;
    }
    if (rc == AFQ_OK) rc = join();
  }
  for (size_t i = 0; i < n; ++i) {
    b->ctx[i]->stream = own[i];
    b->ctx[i]->capturing = false;
    b->ctx[i]->step = step0[i];
  }
  if (rc != AFQ_OK && b->err.empty()) b->err = "grouped capture failed";
  return rc;
}

int check_capturable(afq_ctx* ctx, int nsteps) {
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (nsteps < 1) return afq_fail(ctx, AFQ_ERR_ARG, "nsteps < 1");
  const int q = ctx->p.qr_period;
  if (q > 0 && (nsteps % q != 0 || ctx->step % (uint64_t)q != 0))
    return afq_fail(ctx, AFQ_ERR_ARG,
                    "a captured block must hold whole QR periods and start on one");
  return AFQ_OK;
}

void drop_graph(afq_ctx* ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph_exec = nullptr;
  ctx->graph = nullptr;
  ctx->graph_steps = 0;
}

// Times one launch sequence (after one warm-up run) with events on the stream.
template <class F>
float time_launch(afq_ctx* ctx, F&& f, int reps = 3) {
  if (f() != AFQ_OK) return 1e30f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, ctx->stream);
  int rc = AFQ_OK;
  for (int r = 0; r < reps && rc == AFQ_OK; ++r) rc = f();
  cudaEventRecord(b, ctx->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc == AFQ_OK ? ms / reps : 1e30f;
}

}  // namespace

extern "C" {

int afq_graph_capture(afq_ctx* ctx, int nsteps) {
  if (!ctx) return AFQ_ERR_ARG;
  AFQ_TRY(check_capturable(ctx, nsteps));
  drop_graph(ctx);
  AFQ_TRY(sync(ctx));
  // the legacy default stream cannot be captured: record on a private stream
  cudaStream_t s = ctx->stream, rec = nullptr;
  if (!s) {
    AFQ_CUDA(ctx, cudaStreamCreateWithFlags(&rec, cudaStreamNonBlocking));
    ctx->stream = rec;
  }
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? record_steps(ctx, nsteps) : afq_fail(ctx, AFQ_ERR_CUDA, "begin capture");
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->stream = s;
  if (rec) cudaStreamDestroy(rec);
  if (rc != AFQ_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return afq_fail(ctx, AFQ_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
  ctx->graph = g;
  AFQ_CUDA(ctx, cudaGraphInstantiate(&ctx->graph_exec, g, 0));
  ctx->graph_steps = nsteps;
  return AFQ_OK;
}

int afq_graph_launch(afq_ctx* ctx, int nreplays) {
  if (!ctx || nreplays < 0) return AFQ_ERR_ARG;
  if (!ctx->graph_exec) return afq_fail(ctx, AFQ_ERR_STATE, "afq_graph_capture first");
  for (int r = 0; r < nreplays; ++r) {
    AFQ_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->launches++;
  }
  ctx->step += (uint64_t)ctx->graph_steps * nreplays;
  return AFQ_OK;
}

int afq_get_energy(afq_ctx* ctx, double* e_out, double* e_mix) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (e_out)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_out, ctx->ws.energy, (size_t)ctx->ws.W * 4 * 16,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  if (e_mix)
    AFQ_CUDA(ctx, cudaMemcpyAsync(e_mix, ctx->emix, 8, cudaMemcpyDeviceToHost, ctx->stream));
  AFQ_TRY(sync(ctx));
  return check_flags(ctx);
}

int afq_batch_create(afq_batch** out, int n, afq_ctx* const* ctxs) {
  if (!out || n < 1 || !ctxs) return AFQ_ERR_ARG;
  *out = nullptr;
  afq_batch* b = new (std::nothrow) afq_batch();
  if (!b) return AFQ_ERR_NOMEM;
  bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) {
    if (!ctxs[i] || !ctxs[i]->have_walkers) ok = false;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    b->ctx.push_back(ctxs[i]);
    b->streams.push_back(st);
    b->events.push_back(ev);
  }
  if (!ok) {
    afq_batch_destroy(b);
    return AFQ_ERR_ARG;
  }
  *out = b;
  return AFQ_OK;
}

int afq_batch_destroy(afq_batch* b) {
  if (!b) return AFQ_ERR_ARG;
  if (b->origin) cudaStreamSynchronize(b->origin);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  grouped_step_free(b->gs);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->events)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
  return AFQ_OK;
}

const char* afq_batch_last_error(const afq_batch* b) { return b ? b->err.c_str() : "null batch"; }

int afq_batch_set_grouped(afq_batch* b, int grouped) {
  if (!b || (grouped != 0 && grouped != 1)) return AFQ_ERR_ARG;
  if (grouped)
    for (auto* c : b->ctx)
      if (c->mixed) {
        b->err = "grouped launches take FP64 contexts";
        return AFQ_ERR_ARG;
      }
  b->grouped = grouped;
  return AFQ_OK;
}

int afq_batch_capture(afq_batch* b, int nsteps) {
  if (!b) return AFQ_ERR_ARG;
  for (auto* c : b->ctx) {
    int rc = check_capturable(c, nsteps);
    if (rc == AFQ_OK) rc = sync(c);
    if (rc != AFQ_OK) {
      b->err = c->err;
      return rc;
    }
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  grouped_step_free(b->gs);
  b->gs = nullptr;
  if (b->grouped) {  // descriptor tables of the current walker buffers
    const int rc = grouped_step_create(&b->gs, b->ctx.data(), (int)b->ctx.size(), &b->err);
    if (rc != AFQ_OK) return rc;
  }
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    b->err = "begin capture";
    return AFQ_ERR_CUDA;
  }
  int rc = cudaEventRecord(b->fork, b->origin) == cudaSuccess ? AFQ_OK : AFQ_ERR_CUDA;
  if (rc == AFQ_OK && b->grouped) rc = record_grouped(b, nsteps);
  // one branch per system: its steps run concurrently with the other systems'
  for (size_t i = 0; i < b->ctx.size() && rc == AFQ_OK && !b->grouped; ++i) {
    afq_ctx* c = b->ctx[i];
    cudaStream_t own = c->stream;
    c->stream = b->streams[i];
    rc = cudaStreamWaitEvent(c->stream, b->fork, 0) == cudaSuccess ? AFQ_OK : AFQ_ERR_CUDA;
    if (rc == AFQ_OK) rc = record_steps(c, nsteps);
    if (rc == AFQ_OK && (cudaEventRecord(b->events[i], c->stream) != cudaSuccess ||
                         cudaStreamWaitEvent(b->origin, b->events[i], 0) != cudaSuccess))
      rc = AFQ_ERR_CUDA;
    if (rc != AFQ_OK) b->err = c->err.empty() ? "capture failed" : c->err;
    c->stream = own;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->origin, &g);
  if (rc != AFQ_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (b->err.empty()) b->err = std::string("end capture: ") + cudaGetErrorString(e);
    return rc != AFQ_OK ? rc : AFQ_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    b->err = "graph instantiate";
    return AFQ_ERR_CUDA;
  }
  b->nsteps = nsteps;
  return AFQ_OK;
}

int afq_batch_launch(afq_batch* b, int nreplays) {
  if (!b || nreplays < 0) return AFQ_ERR_ARG;
  if (!b->exec) {
    b->err = "afq_batch_capture first";
    return AFQ_ERR_STATE;
  }
  // work already queued on the systems' own streams comes first ...
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (cudaEventRecord(b->events[i], b->ctx[i]->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->origin, b->events[i], 0) != cudaSuccess)
      return AFQ_ERR_CUDA;
  for (int r = 0; r < nreplays; ++r)
    if (cudaGraphLaunch(b->exec, b->origin) != cudaSuccess) {
      b->err = "graph launch";
      return AFQ_ERR_CUDA;
    }
  // ... and later work on them waits for the replays
  if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) return AFQ_ERR_CUDA;
  for (auto* c : b->ctx) {
    if (cudaStreamWaitEvent(c->stream, b->fork, 0) != cudaSuccess) return AFQ_ERR_CUDA;
    c->step += (uint64_t)b->nsteps * nreplays;
    c->launches += (uint64_t)nreplays;
  }
  return AFQ_OK;
}

int afq_batch_synchronize(afq_batch* b) {
  if (!b) return AFQ_ERR_ARG;
  if (cudaStreamSynchronize(b->origin) != cudaSuccess) return AFQ_ERR_CUDA;
  for (auto* c : b->ctx) {
    const int rc = check_flags(c);
    if (rc != AFQ_OK) {
      b->err = c->err;
      return rc;
    }
  }
  return AFQ_OK;
}

int afq_autotune(afq_ctx* ctx) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (ctx->capturing) return afq_fail(ctx, AFQ_ERR_STATE, "cannot tune while capturing");
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  WalkerSet& s = ctx->ws;
  const int nmax = ctx->na > ctx->nb ? ctx->na : ctx->nb;
  int rc = AFQ_OK;
  if (!ctx->mixed) {
    // FP64 exchange (direct form): g-group size (pure: it only rewrites its partial sums)
    float best = 1e30f;
    int bestG = exchange_group_size(nmax);
    for (int G = 1; !ctx->ex_stored && G <= exchange_group_max(nmax);
         G = G < 4 ? G + 1 : G * 3 / 2) {
      ctx->ex_G_fp64 = G;
      const float ms = time_launch(ctx, [&] { return launch_exchange_fp64(ctx, s); });
      if (ms < best) {
        best = ms;
        bestG = G;
      }
    }
    ctx->ex_G_fp64 = bestG;
    // FP64 propagator column chunk: timed on a copy, the walkers are restored
    double2* backup = nullptr;
    const size_t bytes = (size_t)s.W * ctx->M * ctx->N * sizeof(double2);
    if (cudaMalloc((void**)&backup, bytes) != cudaSuccess) rc = AFQ_ERR_NOMEM;
    if (rc == AFQ_OK && cudaMemcpyAsync(backup, s.phi, bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) rc = AFQ_ERR_CUDA;
    if (rc == AFQ_OK) rc = launch_fields(ctx, nullptr);
    if (rc == AFQ_OK) rc = launch_vhs_fp64(ctx);
    best = 1e30f;
    int bestNC = 4;
    for (int nc : {2, 4, 8}) {
      if (rc != AFQ_OK) break;
      ctx->prop_nc = nc;
      const float ms = time_launch(ctx, [&] {
        if (cudaMemcpyAsync(s.phi, backup, bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
          return (int)AFQ_ERR_CUDA;
        return launch_propagate_fp64(ctx);
      });
      if (ms < best) {
        best = ms;
        bestNC = nc;
      }
    }
    ctx->prop_nc = bestNC;
    if (backup) {
      cudaMemcpyAsync(s.phi, backup, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      cudaFree(backup);
    }
  } else {
    rc = mixed_autotune(ctx);
  }
  // slots written under another tiling must not leak into the energy
  if (rc == AFQ_OK)
    rc = cudaMemsetAsync(s.ekp, 0, (size_t)s.W * 2 * ctx->ex_groups * sizeof(double2),
                         ctx->stream) == cudaSuccess ? AFQ_OK : AFQ_ERR_CUDA;
  if (rc == AFQ_OK) rc = green_and_bias(ctx, s);  // theta and c are recomputed unchanged
  if (rc == AFQ_OK) rc = sync(ctx);
  ctx->profiling = prof;
  return rc == AFQ_OK ? check_flags(ctx) : rc;
}

int afq_local_energy_backward_dev(afq_ctx* ctx, const double* gE_dev, double* dh1_dev,
                                  double* dL_dev, double* dphi_dev) {
  if (!ctx || !gE_dev) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (ctx->capturing) return afq_fail(ctx, AFQ_ERR_STATE, "not during capture");
  AFQ_TRY(adjoint_local_energy(ctx, reinterpret_cast<const double2*>(gE_dev), dh1_dev, dL_dev,
                               reinterpret_cast<double2*>(dphi_dev)));
  return check_flags(ctx);  // the backward synchronises the stream before returning
}

int afq_local_energy_backward(afq_ctx* ctx, const double* gE, double* dh1, double* dL,
                              double* dphi) {
  if (!ctx || !gE) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  const size_t W = ctx->ws.W, M = ctx->M, N = ctx->N, X = ctx->X;
  double *g = nullptr, *a = nullptr, *b = nullptr, *c = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&g, W * 16) != cudaSuccess ||
      (dh1 && cudaMalloc((void**)&a, M * M * 8) != cudaSuccess) ||
      (dL && cudaMalloc((void**)&b, X * M * M * 8) != cudaSuccess) ||
      (dphi && cudaMalloc((void**)&c, W * M * N * 16) != cudaSuccess))
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "backward outputs");
  if (rc == AFQ_OK && cudaMemcpyAsync(g, gE, W * 16, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy gE");
  if (rc == AFQ_OK) rc = adjoint_local_energy(ctx, reinterpret_cast<double2*>(g), a, b,
                                              reinterpret_cast<double2*>(c));
  if (rc == AFQ_OK && dh1) rc = cudaMemcpy(dh1, a, M * M * 8, cudaMemcpyDeviceToHost) == cudaSuccess ? rc : AFQ_ERR_CUDA;
  if (rc == AFQ_OK && dL) rc = cudaMemcpy(dL, b, X * M * M * 8, cudaMemcpyDeviceToHost) == cudaSuccess ? rc : AFQ_ERR_CUDA;
  if (rc == AFQ_OK && dphi) rc = cudaMemcpy(dphi, c, W * M * N * 16, cudaMemcpyDeviceToHost) == cudaSuccess ? rc : AFQ_ERR_CUDA;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(g);
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  if (c) cudaFree(c);
  return rc != AFQ_OK ? rc : check_flags(ctx);
}

static int chain_forward_impl(afq_ctx* ctx, int K, const double* fields, bool dev,
                              double* e_out, bool e_dev) {
  if (!ctx) return AFQ_ERR_ARG;
  if (!ctx->have_walkers) return afq_fail(ctx, AFQ_ERR_STATE, "afq_init_walkers first");
  if (ctx->capturing) return afq_fail(ctx, AFQ_ERR_STATE, "not during capture");
  if (ctx->mixed) return afq_fail(ctx, AFQ_ERR_ARG, "the chain adjoint needs an FP64 context");
  if (ctx->p.fb_cap > 0.0)
    return afq_fail(ctx, AFQ_ERR_ARG, "the chain adjoint needs fb_cap = 0 (a cap is not smooth)");
  if (K < 0) return afq_fail(ctx, AFQ_ERR_ARG, "K must be >= 0");
  chain_free(ctx);
  ChainTape& t = ctx->chain;
  const size_t W = ctx->ws.W, WX = W * ctx->X, WMN = W * ctx->M * ctx->N;
  const int qr = ctx->p.qr_period;
  t.K = K;
  t.W = (int)W;
  t.s0 = ctx->step;
  t.seg_cap = qr > 0 ? qr : (int)std::ceil(std::sqrt((double)(K > 1 ? K : 1)));
  // segments end after every QR and after seg_cap steps; checkpoints hold the walkers
  // at the chain start, after every QR and at every inner segment boundary
  std::vector<int> ck_step{0};
  int last = 0;
  for (int k = 1; k <= K; ++k) {
    const bool q = qr > 0 && (t.s0 + k) % (uint64_t)qr == 0;
    if (q || k - last >= t.seg_cap || k == K) {
      ChainSeg sg;
      sg.start = last;
      sg.len = k - last;
      sg.ck_in = (int)ck_step.size() - 1;
      sg.qr_end = q;
      if (q || k < K) {
        ck_step.push_back(k);
        sg.ck_out = (int)ck_step.size() - 1;
      }
      t.segs.push_back(sg);
      last = k;
    }
  }
  t.nck = (int)ck_step.size();
  if (cudaMalloc((void**)&t.fields, (K > 0 ? (size_t)K : 1) * WX * 8) != cudaSuccess ||
      cudaMalloc((void**)&t.ckpt, (size_t)t.nck * WMN * 16) != cudaSuccess) {
    chain_free(ctx);
    return afq_fail(ctx, AFQ_ERR_NOMEM, "chain tape");
  }
  int rc = AFQ_OK;
  if (K > 0 && fields) {
    if (cudaMemcpyAsync(t.fields, fields, (size_t)K * WX * 8,
                        dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess)
      rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy chain fields");
  } else {
    for (int k = 0; k < K && rc == AFQ_OK; ++k)
      rc = launch_philox_fields(ctx, t.s0 + k, t.fields + (size_t)k * WX, nullptr);
  }
  if (rc == AFQ_OK &&
      cudaMemcpyAsync(t.ckpt, ctx->ws.phi, WMN * 16, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "chain checkpoint");
  size_t ci = 1;
  for (int k = 1; k <= K && rc == AFQ_OK; ++k) {
    rc = one_step(ctx, t.fields + (size_t)(k - 1) * WX);
    if (rc == AFQ_OK && ci < ck_step.size() && ck_step[ci] == k) {
      if (cudaMemcpyAsync(t.ckpt + ci * WMN, ctx->ws.phi, WMN * 16, cudaMemcpyDeviceToDevice,
                          ctx->stream) != cudaSuccess)
        rc = afq_fail(ctx, AFQ_ERR_CUDA, "chain checkpoint");
      ++ci;
    }
  }
  if (rc == AFQ_OK) rc = energy_impl(ctx);
  if (rc == AFQ_OK && e_out &&
      cudaMemcpyAsync(e_out, ctx->ws.energy, W * 4 * 16,
                      e_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy chain energies");
  if (rc == AFQ_OK) rc = sync(ctx);
  if (rc == AFQ_OK) rc = check_flags(ctx);
  if (rc != AFQ_OK) {
    chain_free(ctx);
    return rc;
  }
  t.valid = true;
  return AFQ_OK;
}

int afq_chain_forward(afq_ctx* ctx, int K, const double* fields, double* e_out) {
  return chain_forward_impl(ctx, K, fields, false, e_out, false);
}

int afq_chain_forward_dev(afq_ctx* ctx, int K, const double* fields_dev, double* e_out_dev) {
  return chain_forward_impl(ctx, K, fields_dev, true, e_out_dev, true);
}

int afq_chain_backward_dev(afq_ctx* ctx, const double* gE_dev, double* dh1_dev, double* dL_dev,
                           double* dphi0_dev) {
  if (!ctx || !gE_dev) return AFQ_ERR_ARG;
  if (ctx->capturing) return afq_fail(ctx, AFQ_ERR_STATE, "not during capture");
  AFQ_TRY(chain_backward(ctx, reinterpret_cast<const double2*>(gE_dev), dh1_dev, dL_dev,
                         reinterpret_cast<double2*>(dphi0_dev)));
  return check_flags(ctx);  // the backward synchronises the stream before returning
}

int afq_chain_backward(afq_ctx* ctx, const double* gE, double* dh1, double* dL, double* dphi0) {
  if (!ctx || !gE) return AFQ_ERR_ARG;
  if (!ctx->chain.valid) return afq_fail(ctx, AFQ_ERR_STATE, "afq_chain_forward first");
  const size_t W = ctx->chain.W, M = ctx->M, N = ctx->N, X = ctx->X;
  double *g = nullptr, *a = nullptr, *b = nullptr, *c = nullptr;
  int rc = AFQ_OK;
  if (cudaMalloc((void**)&g, W * 16) != cudaSuccess ||
      (dh1 && cudaMalloc((void**)&a, M * M * 8) != cudaSuccess) ||
      (dL && cudaMalloc((void**)&b, X * M * M * 8) != cudaSuccess) ||
      (dphi0 && cudaMalloc((void**)&c, W * M * N * 16) != cudaSuccess))
    rc = afq_fail(ctx, AFQ_ERR_NOMEM, "chain backward outputs");
  if (rc == AFQ_OK && cudaMemcpyAsync(g, gE, W * 16, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    rc = afq_fail(ctx, AFQ_ERR_CUDA, "copy gE");
  if (rc == AFQ_OK)
    rc = chain_backward(ctx, reinterpret_cast<double2*>(g), a, b, reinterpret_cast<double2*>(c));
  if (rc == AFQ_OK && dh1 && cudaMemcpy(dh1, a, M * M * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = AFQ_ERR_CUDA;
  if (rc == AFQ_OK && dL && cudaMemcpy(dL, b, X * M * M * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = AFQ_ERR_CUDA;
  if (rc == AFQ_OK && dphi0 && cudaMemcpy(dphi0, c, W * M * N * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = AFQ_ERR_CUDA;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(g);
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  if (c) cudaFree(c);
  return rc != AFQ_OK ? rc : check_flags(ctx);
}

int afq_get_tiles(afq_ctx* ctx, int* tiles, int n) {
  if (!ctx || !tiles || n < 1) return AFQ_ERR_ARG;
  const int v[5] = {ctx->ex_G_fp64, ctx->prop_nc, ctx->ex_zb[0], ctx->ex_zb[1], ctx->fb_ksplit};
  for (int i = 0; i < n && i < 5; ++i) tiles[i] = v[i];
  return AFQ_OK;
}

int afq_launch_count(afq_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return AFQ_ERR_ARG;
  *count = ctx->launches;
  return AFQ_OK;
}

}  // extern "C"
