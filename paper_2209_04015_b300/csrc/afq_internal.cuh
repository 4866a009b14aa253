// Internal declarations of libafqmc: the context, device buffers, complex helpers
// and the host-side launch wrappers of every kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "afqmc.h"

#define AFQ_NMAX 64    // electrons per spin
#define AFQ_MMAX 1024  // orbitals

// ----------------------------------------------------------------------------
// complex helpers (double2 = re, im)
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return cmk(a.x * s, a.y * s); }
// acc + a b, acc - a b and acc + conj(a) b as four fused multiply-adds (the unfused
// forms cost six FP64 operations, on a pipe that runs 2 lanes per clock per SM)
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  return cmk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 acc) {
  return cmk(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  return cmk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // a / b with scaling by the larger component of b
  double s = fabs(b.x) > fabs(b.y) ? fabs(b.x) : fabs(b.y);
  double2 bs = cmk(b.x / s, b.y / s);
  double d = bs.x * bs.x + bs.y * bs.y;
  double2 n = cmul(a, cconj(bs));
  return cmk(n.x / (d * s), n.y / (d * s));
}
__device__ __forceinline__ double2 cexp(double2 a) {
  double e = exp(a.x), s, c;
  sincos(a.y, &s, &c);
  return cmk(e * c, e * s);
}

constexpr int kFbSplitMax = 8;  // K splits of the FP64 force bias

// ----------------------------------------------------------------------------
// walker-set buffers: everything the overlap / force-bias / energy kernels need
// ----------------------------------------------------------------------------
struct WalkerSet {
  int W = 0;
  double2* phi = nullptr;     // W x M x N   walker matrices, alpha columns first
  double2* thetaT = nullptr;  // W x N x M   theta^T = (Phi S^-1)^T per spin block
  double2* det = nullptr;     // W x 2       det(Psi_s^T Phi_s)
  double2* e1 = nullptr;      // W x 2       one-body energy per spin
  double2* c = nullptr;       // W x X       Coulomb vector / mixed <v_g>
  double2* ekp = nullptr;     // W x 2 x G   exchange partial sums per g-group
  double2* energy = nullptr;  // W x 4       E1, EJ, EK, E_L
  double2* w = nullptr;       // W           weights
  double2* ovlp = nullptr;    // W           stored overlaps
};

// Tape of a K-step chain for its adjoint (k_chain.cu): the fields of every step and
// the walkers at segment boundaries (chain start, after every QR, and every seg_cap
// steps); the backward recomputes each segment from its checkpoint.
struct ChainSeg {
  int start = 0, len = 0;  // chain steps start .. start + len - 1 (0-based)
  int ck_in = 0;           // checkpoint holding the walkers before step start
  int ck_out = -1;         // checkpoint after the segment (the QR output), or -1
  bool qr_end = false;     // the segment's last step ends with a QR
};
struct ChainTape {
  bool valid = false;
  int K = 0, W = 0, nck = 0, seg_cap = 0;
  uint64_t s0 = 0;           // step counter at the chain start
  double* fields = nullptr;  // K x W x X
  double2* ckpt = nullptr;   // nck x W x M x N
  std::vector<ChainSeg> segs;
};

struct afq_ctx {
  afq_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  uint64_t launches = 0;

  int M = 0, X = 0, na = 0, nb = 0, N = 0, Mp = 0;
  double e0 = 0.0, e_trial = 0.0, e_shift = 0.0, sum_vbar2 = 0.0;
  bool have_ham = false, have_trial = false, have_walkers = false;
  uint64_t step = 0;                   // host mirror of the step counter
  unsigned long long* d_step = nullptr; // device step counter (Philox fields, graphs)
  int ex_groups = 0;  // exchange partial-sum slots per (walker, spin)
  int ex_G_fp64 = 0;  // g-group of the FP64 exchange (0: default), autotuned
  int prop_nc = 4;    // walker columns per CTA of the FP64 propagator, autotuned
  bool capturing = false;  // a CUDA graph is being captured: no host syncs, no events
  cudaGraph_t graph = nullptr;          // afq_graph_capture: a block of steps
  cudaGraphExec_t graph_exec = nullptr;
  int graph_steps = 0;

  // Hamiltonian
  double* h1 = nullptr;   // M x M
  double* L = nullptr;    // X x M x M (kept for the trial set-up and gradients)
  double* Lpk = nullptr;  // X x Mp packed upper triangles, Mp = M (M + 1) / 2
  int2* tpq = nullptr;    // Mp packed index -> (p, q), p <= q
  // trial
  double* psiT = nullptr;  // N x M   rows: alpha orbitals then beta orbitals
  double* Lt = nullptr;    // X x N x M half-rotated Cholesky vectors
  double* ht = nullptr;    // N x M   Psi^T h1
  double* vbar = nullptr;  // X
  double* hpp = nullptr;   // M x M   h''
  double* P = nullptr;     // M x M   exp(-dt h''/2)
  // walkers
  WalkerSet ws;
  double* xi = nullptr;      // W x X fields of the current step
  double2* xbar = nullptr;   // W x X
  double2* y = nullptr;      // W x X shifted fields
  double2* cfb = nullptr;    // W
  double2* cmf = nullptr;    // W
  double2* A = nullptr;      // W x M x M  i sqrt(dt) V, symmetric
  double* Asum = nullptr;    // W x M x M  Re A + Im A (FP64 propagation, 3-product form)
  double* detR = nullptr;    // W x 2
  double2* fb64_part = nullptr;  // kFbSplitMax x W x X: K-split partials of the FP64 force bias
  long fb64_part_wx = 0;         // W X the buffer was sized for
  double* emix = nullptr;    // 1
  int* flags = nullptr;      // [0] singular pivots, [1] non-finite values,
                             // [2] tensor-core pipeline time-outs,
                             // [3] population control without positive total weight
  // population control (comb) workspace, allocated on first use
  double2* comb_phi = nullptr;   // W x M x N gathered walkers
  double2* comb_ovlp = nullptr;  // W gathered stored overlaps
  double* comb_cum = nullptr;    // W running weight sums, then T / W
  int* comb_parents = nullptr;   // W parent index of each new walker
  double* scratch = nullptr; // set-up workspace
  size_t scratch_bytes = 0;

  // split-precision (AFQ_SPLIT_BF16) state
  bool mixed = false;
  int S = 4;                          // exact digits per operand (force bias, exchange)
  int Sp = 4;                         // exact digits per operand (propagation)
  int Mpad = 0;                       // M rounded up to the 32-wide K block
  __nv_bfloat16* Lt_sl = nullptr;     // S x X x N x Mpad scaled digits of L~ (direct exchange)
  __nv_bfloat16* th_sl = nullptr;     // S x W x 2 x N x Mpad scaled digits of theta (direct exchange)
  __nv_bfloat16* Lt_ex = nullptr;     // S x X x N x Mpad integer digits of L~ (force bias)
  int* e_fb = nullptr;                // X row exponents of Lt_ex
  double* fb_part = nullptr;          // ksplit x 2W x X force-bias partial sums (exact, FP64)
  int fb_BN = 0, fb_kbper = 0, fb_ksplit = 0, fb_ksplit_cap = 0;
  int ex_G[2] = {0, 0}, ex_zb[2] = {0, 0}, ex_BN[2] = {0, 0};
  CUtensorMap tm_fb_a, tm_fb_b, tm_ex_a[2], tm_ex_b[2];
  // split-precision propagation operands (k_mixed_prop.cu)
  int Xpad = 0, vhs_BN = 0, prop_rows = 0;  // prop_rows: walker columns per propagation tile
  // exact digits per propagation GEMM pass: [0] the first P, [1..n] the Taylor powers,
  // [n+1] the last P (at most Sp; fewer for the small high powers), and the estimate
  // x = sqrt(dt) |V|_2 they were chosen for
  int prop_digits[40] = {};
  double prop_x = 0.0;
  __nv_bfloat16* LT_sl = nullptr;     // S x M^2 x Xpad: L^T, the VHS operand
  __nv_bfloat16* Pm_sl = nullptr;     // S x M x Mpad: the off-diagonal part of P
  double* pdiag = nullptr;            // M: the diagonal of P, applied in FP64
  __nv_bfloat16* y_sl = nullptr;      // S x 2W x Xpad: shifted fields (re, im rows)
  __nv_bfloat16* A_sl = nullptr;      // S x 2W x M x Mpad: i sqrt(dt) V (re, im planes)
  __nv_bfloat16* T_sl[2] = {nullptr, nullptr};  // S x 2W x N x Mpad: Taylor operands [Re; Im]
  double2* accT = nullptr;            // W x N x M FP64 accumulator of the propagated walker
  double2* tout = nullptr;            // W x N x M FP64 operand between propagation launches
  int *e_lt = nullptr, *e_pm = nullptr, *e_y = nullptr, *e_a = nullptr;  // row exponents
  int* e_t[2] = {nullptr, nullptr};
  CUtensorMap tm_vhs_a, tm_vhs_b, tm_pm, tm_az, tm_t[2];
  __nv_bfloat16* T_neg[2] = {nullptr, nullptr};  // S x W x N x Mpad: -Im of the operands (<= 4 digits)
  CUtensorMap tm_t_real[2];  // the same operands in prop_rows_real-row boxes (P passes and
                             // the column-concatenated complex passes)
  CUtensorMap tm_tneg[2];    // T_neg in prop_rows_real-row boxes
  int prop_rows_real = 0;    // walker columns per tile of the real P passes
  CUtensorMap tm_t_fused[2]; // the same operands in prop_rows_fused-row boxes (cluster kernel)
  int prop_rows_fused = 0;   // walker columns per chain of the cluster kernel
  // theta's integer digit planes (S x 2W x N x Mpad, one exponent per (z, re/im)):
  // the B operand of the force bias and of the stored exchange.  Stored exchange
  // (k_exchange_tcv.cu): S integer-digit planes of V' per spin (n Mpad)^2 with row
  // exponents, y^T (2W x max n Mpad FP64) and the maps of both GEMM operands
  __nv_bfloat16* Vsl = nullptr;
  int* exv_ea = nullptr;
  __nv_bfloat16* exv_th = nullptr;
  int* exv_eb = nullptr;
  double* exv_y = nullptr;
  int exv_BN = 0;
  CUtensorMap tm_exv_a[2], tm_exv_b;

  // overlap product S = Psi^T Phi of the split-precision walker ensemble on the tensor
  // cores (k_overlap_tc.cu): 7 exact digits of Psi^T and h~ (2N x Mpad per digit) with row
  // exponents, of Phi^T (2W N x Mpad per digit) with exponents per (z, j), and S itself
  // (W x 2 x nmax x nmax complex)
  __nv_bfloat16* ov_psi_sl = nullptr;
  int* ov_ea = nullptr;
  __nv_bfloat16* ov_phi_sl = nullptr;
  int* ov_eb = nullptr;
  double2* ov_S = nullptr;
  double2* ov_H = nullptr;  // h~ Phi per (z, spin), same layout: E1 = tr(S^-1 H)
  CUtensorMap tm_ov_a, tm_ov_b;
  // theta = Phi S^-1 of the split-precision walker ensemble on the tensor cores
  // (k_mixed_prop.cu), per unit u = (z, spin): th_S exact digits of Phi's rows p over
  // the spin's columns k (A: th_S x 2W x re/im x M x th_K) and of S^-1's columns j over
  // k (B: th_S x 2W x re/im x nmax x th_K, and -Im: th_S x 2W x nmax x th_K), their
  // exponents per (u, p) and (u, j), and S^-1 itself in FP64 (2W x nmax x nmax, written
  // by the Gauss-Jordan kernel); E1 is summed by the pass that takes theta's exponents
  int th_S = 0, th_K = 0, th_brows = 0;
  __nv_bfloat16 *th_a_sl = nullptr, *th_b_sl = nullptr, *th_bn_sl = nullptr;
  int *th_ea = nullptr, *th_eb = nullptr;
  double2* th_sinv = nullptr;
  CUtensorMap tm_tha, tm_thb, tm_thbn;

  ChainTape chain;  // afq_chain_forward
  // half-rotated exchange tensor V_s[(j,p),(i,q)] = sum_g L~_g,s[j][q] L~_g,s[i][p] per
  // spin (alpha block, then beta block): built by afq_init_trial when the stored
  // exchange is chosen, else on the first local-energy adjoint; kept with the trial
  double* Vx = nullptr;
  bool ex_stored = false;  // FP64 exchange from Vx (else T per (walker, g))

  // built-in profiler: event pairs around launches of each kernel class
  bool profiling = false;
  struct ProfRec {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[AFQ_K_COUNT] = {};
  uint64_t prof_n[AFQ_K_COUNT] = {};
};

// status helpers -------------------------------------------------------------
int afq_fail(afq_ctx* ctx, int code, const std::string& msg);

// Make the dynamic shared-memory limit of kernel fn on the current device at least
// smem bytes.  The limit is a process-wide attribute of the kernel that every caller
// (every context, stream and host thread) shares, so it is only ever raised: a
// smaller request after a larger one keeps the larger limit, and launches sized for
// the larger request stay valid.  The largest size set per (device, kernel) is kept
// under a mutex, so the attribute call is issued only when the limit grows (none in
// steady state, and none while a graph captured after a first ordinary step runs).
cudaError_t raise_smem_limit(const void* fn, size_t smem);
#define AFQ_CUDA(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return afq_fail(ctx, AFQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define AFQ_TRY(x)                 \
  do {                             \
    int rc_ = (x);                 \
    if (rc_ != AFQ_OK) return rc_; \
  } while (0)
#define AFQ_LAUNCHED(ctx)                                                                \
  do {                                                                                   \
    (ctx)->launches++;                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return afq_fail(ctx, AFQ_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// ----------------------------------------------------------------------------
// launch wrappers (each returns AFQ_OK or an error code via afq_fail)
// ----------------------------------------------------------------------------
// set-up (k_setup.cu)
// stored-tensor exchange (k_exchange_v.cu; split precision: k_exchange_tcv.cu)
int build_exchange_v(afq_ctx* ctx);
double exchange_tcv_bytes(const afq_ctx* ctx, int Mpad);
int mixed_exchange_v_init(afq_ctx* ctx);
int mixed_exchange_v_walkers(afq_ctx* ctx);
int launch_exchange_tcv(afq_ctx* ctx, WalkerSet& s);
int exchange_v_slots(const afq_ctx* ctx);
int launch_exchange_v(afq_ctx* ctx, WalkerSet& s);
int launch_dgemm(afq_ctx* ctx, int m, int n, int k, double alpha, const double* A, long sam,
                 long sak, long sab, const double* B, long sbk, long sbn, long sbb, double beta,
                 double* C, long scm, long scn, long scb, int batch, int ksplit);
int launch_pack_L(afq_ctx* ctx);
int launch_vbar(afq_ctx* ctx);
int launch_hpp(afq_ctx* ctx, const double* s2part, int ksplit);
int launch_axpby(afq_ctx* ctx, int n, double a, const double* x, double b, double* y);
int launch_set_identity(afq_ctx* ctx, int M, double* out);

// walker kernels (k_walkers.cu)
int launch_overlap_theta(afq_ctx* ctx, WalkerSet& s, bool df = false);
int launch_theta_precise(afq_ctx* ctx);  // the walker ensemble's theta in double-floats
int launch_force_bias_fp64(afq_ctx* ctx, WalkerSet& s);
int launch_exchange_fp64(afq_ctx* ctx, WalkerSet& s);
int launch_energy_assemble(afq_ctx* ctx, WalkerSet& s);
int launch_qr(afq_ctx* ctx, WalkerSet& s, double2* Qw);  // Qw: W x N x M workspace
int exchange_group_size(int nmax);
int exchange_group_max(int nmax);
int launch_init_overlap(afq_ctx* ctx, WalkerSet& s);

// step kernels (k_step.cu)
int launch_fields(afq_ctx* ctx, const double* xi_dev);
int launch_philox_fields(afq_ctx* ctx, uint64_t step, double* out, uint32_t* words);
int launch_vhs_fp64(afq_ctx* ctx);
int launch_propagate_fp64(afq_ctx* ctx);
// grouped VHS and propagation of several FP64 systems (batches; k_step.cu)
struct GroupedStep;
int grouped_step_create(GroupedStep** out, afq_ctx* const* ctxs, int n, std::string* err);
void grouped_step_free(GroupedStep* g);
cudaError_t grouped_step_vhs(GroupedStep* g, cudaStream_t st);
cudaError_t grouped_step_propagate(GroupedStep* g, cudaStream_t st);
int launch_weights(afq_ctx* ctx, double log_const, const double* e_shift_dev = nullptr);
int launch_emix(afq_ctx* ctx, WalkerSet& s, double* out);
int comb_walkers(afq_ctx* ctx, double u, double w_cap);  // k_population.cu
void comb_free(afq_ctx* ctx);
int launch_block_sums(afq_ctx* ctx, double* out_dev);
int launch_shift_from_block(afq_ctx* ctx, const double* sums_dev, int steps, double* e_shift_dev);
int launch_set_scalar(afq_ctx* ctx, double* dst_dev, double value);
int launch_spin_squared(afq_ctx* ctx, WalkerSet& s, double2* out_dev, double* mix_dev);  // k_estimators.cu
int launch_one_rdm(afq_ctx* ctx, WalkerSet& s, double2* work_dev, double2* out_dev);

// adjoint of the local energy (k_adjoint.cu)
int adjoint_local_energy(afq_ctx* ctx, const double2* gE, double* dh1, double* dL, double2* dphi);
// t holds theta and c of its walkers.  F (X x N x M, accumulated) may be NULL; out
// receives the walker cotangent: mode 0 g conj(dE/dPhi), mode 1 conj(g) dE/dPhi.
int adjoint_energy_core(afq_ctx* ctx, WalkerSet& t, const double2* gE, double* dh1, double* F,
                        double2* out, int mode);
// lam += (I - Psi theta^T) lamT^T S^-T per walker (the adjoint of theta = Phi S^-1)
int launch_bwd_theta(afq_ctx* ctx, WalkerSet& t, const double2* lamT, double2* lam);

// K-step chain adjoint (k_chain.cu)
void chain_free(afq_ctx* ctx);
int chain_backward(afq_ctx* ctx, const double2* gE, double* dh1, double* dL, double2* dphi0);
// out = exp(scale * src) (n x n, FP64) by scaling and squaring of a degree-18 Taylor
// polynomial; norm1 bounds ||scale * src||_1.
int expm_taylor(afq_ctx* ctx, const double* src, double scale, int n, double norm1, double* out);

// split-precision tensor-core path (k_mixed.cu)
int mixed_init_trial(afq_ctx* ctx);
int mixed_init_walkers(afq_ctx* ctx);
void mixed_free(afq_ctx* ctx);
int launch_slice_theta(afq_ctx* ctx, WalkerSet& s);
int launch_force_bias_tc(afq_ctx* ctx, WalkerSet& s);
int launch_exchange_tc(afq_ctx* ctx, WalkerSet& s);
int mixed_autotune(afq_ctx* ctx);
void mixed_prop_free(afq_ctx* ctx);
int mixed_prop_init_trial(afq_ctx* ctx);
int mixed_prop_init_walkers(afq_ctx* ctx);
int launch_vhs_tc(afq_ctx* ctx);
int launch_propagate_tc(afq_ctx* ctx);
// theta^T of the walker ensemble on the tensor cores from S^-1 in ctx->th_sinv
int theta_tc_init_walkers(afq_ctx* ctx);
void theta_tc_free(afq_ctx* ctx);
int launch_theta_tc(afq_ctx* ctx, WalkerSet& s);
// S = Psi^T Phi on the tensor cores (k_overlap_tc.cu)
int overlap_tc_init_trial(afq_ctx* ctx);
int overlap_tc_init_walkers(afq_ctx* ctx);
void overlap_tc_free(afq_ctx* ctx);
int launch_overlap_s_tc(afq_ctx* ctx, WalkerSet& s);
// the cluster kernel of every propagation pass (k_prop_fused.cu): AFQ_OK, an error,
// or -1 when the shape cannot take it (nothing launched)
int launch_propagate_fused(afq_ctx* ctx);
int fused_prop_rows(int N);  // walker columns per chain of that kernel
