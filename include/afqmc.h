/*
 * afqmc.h - C ABI of the B300 phaseless-AFQMC walker-step library (libafqmc.so).
 *
 * The library runs one imaginary-time step of phaseless auxiliary-field QMC for a
 * batch of single-determinant walkers under a Cholesky-factorised Hamiltonian
 * (Malone, Mahajan, Spencer, Lee, arXiv:2209.04015, Sec. "Review of AFQMC" and
 * Sec. "Implementational details"), entirely in CUDA kernels for sm_103a.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Arrays are row-major C arrays.  Complex numbers are interleaved (re, im)
 *    pairs of doubles, so a "W x X complex" array holds 2*W*X doubles.
 *  - Pointers are HOST pointers unless the function name ends in _dev, in which
 *    case they are DEVICE pointers that the kernels read or write on the
 *    context's stream (for example torch tensors' data_ptr()).
 *  - The library copies every host input into device memory that it owns; the
 *    caller keeps ownership of all its buffers, host or device.  Host outputs are
 *    complete when the call returns; _dev outputs are complete in stream order.
 *  - Every function returns an afq_status.  On failure nothing is written to the
 *    caller's outputs, and afq_last_error() returns a message.
 *  - Spin blocks: walker matrices hold the alpha columns first, then the beta
 *    columns (na + nb columns in all).
 *  - Sizes: 1 <= na, nb <= 64 (na or nb may be 0), M <= 1024, X >= 1, W >= 1.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afq_ctx afq_ctx;

typedef enum afq_status {
  AFQ_OK = 0,
  AFQ_ERR_ARG = 1,      /* bad pointer, size or call order                  */
  AFQ_ERR_CUDA = 2,     /* a CUDA runtime call failed                        */
  AFQ_ERR_SINGULAR = 3, /* an overlap matrix Psi^T Phi had a zero pivot      */
  AFQ_ERR_NAN = 4,      /* a weight, overlap or energy became NaN/Inf        */
  AFQ_ERR_STATE = 5,    /* hamiltonian / trial / walkers not initialised     */
  AFQ_ERR_NOMEM = 6     /* device allocation failed                          */
} afq_status;

typedef enum afq_precision {
  AFQ_FP64 = 0,       /* every contraction in float64                         */
  AFQ_SPLIT_BF16 = 1, /* force bias, exchange, VHS and propagator contractions as
                         bf16 tensor-core GEMMs (tcgen05) on exact 8-bit integer
                         digits of their operands; the overlap matrix S and
                         h~ Phi on 7 digits (FP64 quality); det S, S^-1 and the QR
                         in double-float arithmetic (~2^-44 relative); theta on
                         the force bias's digits up to 4 (double-float beyond, and
                         for afq_spin_squared / afq_one_rdm); weights float64 */
  AFQ_SPLIT_TF32 = 2  /* reserved: afq_create rejects it (AFQ_ERR_ARG)          */
} afq_precision;

typedef enum afq_exchange {
  AFQ_EXCHANGE_AUTO = 0,   /* STORED when its tensor fits the memory budget (1/4 of the
                              free device memory at afq_init_trial, at most 16 GiB) and
                              takes fewer multiply-adds (M < 1.5 X); else DIRECT      */
  AFQ_EXCHANGE_DIRECT = 1, /* T_zg = L~_g theta_z formed and consumed per (walker, g)
                              (Sec. "Local energy"): 2 X n^2 M multiply-adds per walker
                              and spin, no extra memory                             */
  AFQ_EXCHANGE_STORED = 2  /* the half-rotated two-electron tensor
                              V[(j,p),(i,q)] = sum_g L~_g,jq L~_g,ip kept per spin
                              (na^2 M^2 + nb^2 M^2 doubles, built by afq_init_trial):
                              E_K = -1/2 sum_s theta_s^T V_s theta_s, about (n M)^2
                              multiply-adds per walker and spin (V is symmetric:
                              only its upper blocks are read).  AFQ_SPLIT_BF16
                              contexts also keep split_slices exact-digit planes of
                              V in the padded layout, blocks above the diagonal
                              doubled (2 S (n Mpad)^2 bytes per spin), and run
                              V theta for both spins as one tensor-core GEMM      */
} afq_exchange;

typedef struct afq_params {
  double dt;           /* imaginary time step (the paper's Delta tau)            */
  int taylor_order;    /* order n of the Taylor series of exp(A); default 6      */
  int qr_period;       /* QR re-orthogonalisation after every qr_period-th step;
                          0 disables it                                           */
  uint64_t seed;       /* Philox key for device-drawn fields                     */
  int precision;       /* an afq_precision                                       */
  int has_e_shift;     /* 0: E_shift = trial energy, 1: use e_shift              */
  double e_shift;      /* energy shift in exp(-dt (H - E_shift))                 */
  double fb_cap;       /* |xbar_g| cap; 0 = off                                  */
  int free_projection; /* 1: complex weights w <- w I (no phaseless cut)         */
  int split_slices;    /* AFQ_SPLIT_BF16: digits S per FP64 operand of the force bias
                          and the exchange, 1..7; 0 = 4.  Force bias and stored
                          exchange: exact 8-bit digits, the products of digit
                          orders s + t <= S - 1 each in its own exact TMEM
                          accumulator; direct exchange (S <= 4 only; more digits
                          take the stored exchange, AFQ_ERR_ARG at afq_init_trial
                          when it is asked for or does not fit): the same digits
                          stored at their weights, the leading product in an exact
                          TMEM accumulator and the smaller ones in a second (FP32).
                          7 digits (55 bits) with prop_slices = 7 give FP64
                          quality (the FP64 path's 1e-10 parity with the oracle);
                          6 with 6 pass the same parity tests               */
  int prop_slices;     /* AFQ_SPLIT_BF16: exact 8-bit digits per FP64 operand of the
                          VHS and propagator GEMMs, 1..7 (per-row power-of-two scale,
                          one exact TMEM accumulator per digit order; the Taylor
                          powers take fewer where their terms are small); 0 = 4  */
  int exchange;        /* an afq_exchange: algorithm of the exchange energy        */
  int prop_kernel;     /* AFQ_SPLIT_BF16 propagation: 0 = one launch per GEMM pass with
                          digit slicing launches between them (default); the real
                          passes and the complex passes of 3 or more digits issue one
                          MMA per A digit over the concatenated B digits (32-column
                          tiles; two TMEM accumulator sets up to 4 digits, two ring
                          stages per K block from 5);
                          1 = one persistent kernel of thread-block clusters for all
                          GEMM passes of a step (each walker's 128-row slabs form a
                          cluster that exchanges the digit exponents on chip; about
                          2x slower on this part, kept as an option), falling back
                          to 0 where a shape cannot take it; 2 = the per-pass
                          kernels with one MMA per digit pair (64-column complex
                          tiles), and so every other split GEMM (force bias, VHS,
                          stored exchange, overlap product), which otherwise issue
                          one MMA per A digit over the concatenated B digits.  All
                          give the same bits.                                      */
} afq_params;

/* Fill *p with the defaults: dt 0.005, Taylor order 6, QR every 5 steps, seed 1,
   FP64, E_shift = trial energy, no cap, phaseless; in split mode 4 exact digits for
   the force bias, the exchange and the propagation; exchange AUTO. */
void afq_default_params(afq_params* p);

/* Create a context bound to cuda_stream (a cudaStream_t, or NULL for the legacy
   default stream) on the current CUDA device.  *ctx receives the handle; the
   caller releases it with afq_destroy. */
int afq_create(afq_ctx** ctx, const afq_params* params, void* cuda_stream);
int afq_destroy(afq_ctx* ctx);
/* Message of the last failed call on ctx (never NULL; "" when none). */
const char* afq_last_error(const afq_ctx* ctx);

/* Hamiltonian of Eq. Habinitio with the Cholesky factorisation (pr|qs) =
   sum_g L_g,pr L_g,qs (Sec. "Review of AFQMC").
   h1: M x M, symmetric.  L: X x M x M, each L_g symmetric.  e0: constant energy.
   Symmetry is checked to 1e-12 relative (AFQ_ERR_ARG otherwise). */
int afq_init_hamiltonian(afq_ctx* ctx, int M, int X, const double* h1, const double* L,
                         double e0);

/* Single-determinant trial Psi_T (Sec. "Overlap"): psi_a M x na, psi_b M x nb, real,
   with orthonormal columns.  Builds the half-rotated vectors L~_g = Psi^T L_g
   (Sec. "One-body Green's function and force bias"), the rotated h~ = Psi^T h1, the
   mean field vbar_g, h'' = h1 - 1/2 sum_g L_g L_g + sum_g vbar_g L_g, the
   half-step propagator exp(-dt h''/2) and, with the stored exchange (see
   afq_exchange), the half-rotated tensor V.  Needs afq_init_hamiltonian first. */
int afq_init_trial(afq_ctx* ctx, int na, int nb, const double* psi_a,
                   const double* psi_b);
/* Local energy of the trial determinant itself (its Hartree-Fock energy). */
int afq_trial_energy(afq_ctx* ctx, double* e_out);
/* The exchange algorithm afq_init_trial resolved params.exchange to:
   AFQ_EXCHANGE_DIRECT or AFQ_EXCHANGE_STORED. */
int afq_exchange_algorithm(afq_ctx* ctx, int* algo_out);
/* AFQ_SPLIT_BF16: exact digits of each propagation GEMM pass chosen by
   afq_init_trial -- digits[0] the first P, digits[1..n] the Taylor powers,
   digits[n+1] the last P (n = taylor_order; a power with x^k / k! small gets fewer,
   at most prop_slices) -- and x_out the estimate of sqrt(dt) |V|_2 behind them.
   Writes min(n + 2, count) entries; AFQ_ERR_STATE in FP64 contexts. */
int afq_prop_digits(afq_ctx* ctx, int* digits, int count, double* x_out);

/* Walker ensemble of Eq. stat_wfs.  phi: W x M x (na+nb) complex, or NULL for W
   copies of the trial.  w: W real weights, or NULL for all ones.  Computes the
   stored overlaps <Psi_T|phi_z> and the Green's-function intermediates, and resets
   the step counter to 0. */
int afq_init_walkers(afq_ctx* ctx, int W, const double* phi, const double* w);

/* nsteps hybrid-propagation steps (Sec. "Review of AFQMC": force bias, shifted
   fields, B(x - xbar), overlap ratio Eq. ovl, importance function Eq. import,
   phaseless weight Eqs. ph and theta, walker update), with QR after every
   qr_period-th step.  fields: nsteps x W x X N(0,1) auxiliary fields, or NULL to
   draw them on the device from Philox4x32-10 at the current step counter.
   AFQ_ERR_SINGULAR / AFQ_ERR_NAN are reported after the last step. */
int afq_propagate(afq_ctx* ctx, const double* fields, int nsteps);
/* Same with device-resident fields (nsteps x W x X doubles) or NULL. */
int afq_propagate_dev(afq_ctx* ctx, const double* fields_dev, int nsteps);

/* Mixed local energy (Sec. "Local energy"): per walker E1, EJ, EK and
   E_L = e0 + E1 + EJ + EK as complex numbers (e_out: W x 4 complex, may be NULL),
   and the weighted estimate sum_z w_z Re E_L,z / sum_z w_z (e_mix, may be NULL). */
int afq_local_energy(afq_ctx* ctx, double* e_out, double* e_mix);
/* Same with device outputs; no host synchronisation. */
int afq_local_energy_dev(afq_ctx* ctx, double* e_out_dev, double* e_mix_dev);

/* QR re-orthogonalisation of every walker's spin blocks, Phi_s = Q R with diag(R)
   real and positive; Phi_s <- Q and the stored overlap is divided by
   prod_s det R_s. */
int afq_orthogonalise(afq_ctx* ctx);

/* Population control by the comb.  The paper counts population control among the
   light parts of AFQMC (Sec. "Introduction") without fixing an algorithm; the comb
   (systematic resampling) is the reading taken.  With the phaseless weights w_z,
   first capped at w_cap when w_cap > 0 (0 = no cap), their running sums
   C_z = w_0 + ... + w_z in index order and T = C_{W-1}, the teeth
   t_k = (k + u) (T / W), k = 0..W-1, select parents: new walker k copies the walker
   z with C_{z-1} <= t_k < C_z (its matrix and stored overlap; a tooth at or above
   C_{W-1} goes to the last walker with positive weight) and every new walker gets
   weight T / W.  theta, the determinants and the Coulomb vector are then rebuilt,
   and a chain tape is discarded.
   u: the comb's offset in [0, 1), drawn by the caller (AFQ_ERR_ARG outside).
   parents: host array of W ints receiving the parent of each new walker, or NULL.
   AFQ_ERR_STATE in free projection (complex weights); AFQ_ERR_NAN when T is not
   positive and finite (the walkers are then left as they were). */
int afq_comb(afq_ctx* ctx, double u, double w_cap, int* parents);

/* The block workflow of the paper's example (Sec. "Interface with PySCF": blocks of
   propagation steps, typically 25, each followed by one energy evaluation): for each
   block b, steps_per_block steps with the device fields (QR at its cadence), then the
   local energies and the block sums written to sums[4 b .. 4 b + 3] =
   (Re, Im of sum_z w_z; Re, Im of sum_z w_z E_L,z), then, when u is not NULL, the comb
   with offset u[b] and cap w_cap (as afq_comb).  sums: host, nblocks x 4 doubles.
   shift_feedback != 0: after each block the energy shift E_shift of the weight factor
   exp(-dt (e0 - 1/2 sum vbar^2 - E_shift)) becomes E_b - ln(T_b / W) / (dt
   steps_per_block), on the device, with E_b = Re(sum w E_L / sum w) the block's
   estimate and T_b = |sum w| its total weight (population feedback: the total weight
   returns towards W; the shift multiplies every weight of a step by the same factor,
   so ratio estimators do not change); the context keeps the last shift afterwards
   (afq_get_e_shift).  0: E_shift stays as set at afq_init_trial.
   One host synchronisation at the end; errors of any block are reported then.
   AFQ_ERR_ARG for nblocks < 0, steps_per_block < 1 or an offset outside [0, 1). */
int afq_run_blocks(afq_ctx* ctx, int nblocks, int steps_per_block, const double* u,
                   double w_cap, int shift_feedback, double* sums);
/* The energy shift the weight update uses now (AFQ_ERR_ARG for a NULL pointer). */
int afq_get_e_shift(afq_ctx* ctx, double* e_shift);

/* Mixed estimator of S^2 (Sec. "Customized mixed estimators"; S^2 commutes with H,
   so the mixed estimate is unbiased): per walker
     <Psi_T|S^2|Phi_z> / <Psi_T|Phi_z> = N_beta + M_S (M_S + 1) - tr(G_alpha G_beta),
   M_S = (na - nb) / 2, G_s the walker's Green's function of spin s (the trace of
   the product, from Wick's theorem; the paper's printed sum drops the transpose,
   which only agrees for symmetric G).  FP64 from the walkers' current theta (an
   AFQ_SPLIT_BF16 context first recomputes theta in double-float arithmetic: its step
   forms theta at the force bias's digit count).
   s2_out: W complex (host) or NULL; s2_mix: Re(sum w S2 / sum w) (host) or NULL.
   AFQ_ERR_STATE before afq_init_walkers. */
int afq_spin_squared(afq_ctx* ctx, double* s2_out, double* s2_mix);

/* Weighted mixed one-body density matrix of each spin (a Green's-function mixed
   estimator, Sec. "Customized mixed estimators"):
     <G^s>_pq = sum_z w_z G^s_z,pq / sum_z w_z,   G_pq = <a+_p a_q> = sum_j Psi_pj theta_qj,
   formed as Psi_s (sum_z w_z theta_z,s)^T / sum_z w_z from the walkers' current theta
   (FP64; complex weights in free projection; double-float theta recomputed first in
   AFQ_SPLIT_BF16 contexts, as for afq_spin_squared).  g_out: host, 2 x M x M complex, the
   alpha matrix first (AFQ_ERR_ARG if NULL); AFQ_ERR_STATE before afq_init_walkers. */
int afq_one_rdm(afq_ctx* ctx, double* g_out);

/* Getters (host outputs): walkers W x M x (na+nb) complex; weights W complex
   (imaginary parts are zero in phaseless mode); stored overlaps W complex; the
   force bias xbar of the last step, W x X complex. */
int afq_get_walkers(afq_ctx* ctx, double* phi);
int afq_get_weights(afq_ctx* ctx, double* w);
int afq_get_overlaps(afq_ctx* ctx, double* ovlp);
int afq_get_force_bias(afq_ctx* ctx, double* xbar);
int afq_get_step(afq_ctx* ctx, uint64_t* step);
/* Restore a saved state (checkpoint/resume): walkers, weights (W complex),
   overlaps (W complex, or NULL to recompute) and the step counter. */
int afq_set_state(afq_ctx* ctx, const double* phi, const double* w, const double* ovlp,
                  uint64_t step);

/* The device Philox4x32-10 field stream of one step: out is W x X doubles.  Counter
   (step mod 2^32, walker, g/2, step >> 32), key (seed mod 2^32, seed >> 32);
   Box-Muller of two 53-bit uniforms gives the fields for g = 2m and 2m+1. */
int afq_philox_fields(afq_ctx* ctx, uint64_t step, double* out);
/* The raw Philox words of the same stream: out is W x ceil(X/2) x 4 uint32. */
int afq_philox_words(afq_ctx* ctx, uint64_t step, uint32_t* out);

/* Number of kernel launches this context has issued since creation. */
int afq_launch_count(afq_ctx* ctx, uint64_t* count);

/* Kernel classes timed by the built-in profiler (CUDA events recorded on the
   context's stream around each launch of that class). */
typedef enum afq_kernel {
  AFQ_K_FIELDS = 0,   /* fields, force bias, shifted fields, cfb, cmf          */
  AFQ_K_VHS = 1,      /* VHS build A = i sqrt(dt) sum_g y_g L_g                */
  AFQ_K_PROPAGATE = 2,/* P T_n(A) P applied to every walker                    */
  AFQ_K_OVERLAP = 3,  /* overlap, determinant, theta, one-body energy          */
  AFQ_K_FORCE_BIAS = 4,/* c = L~ theta (force bias and Coulomb vector)         */
  AFQ_K_WEIGHTS = 5,  /* overlap ratio and phaseless weight                    */
  AFQ_K_QR = 6,       /* QR re-orthogonalisation                               */
  AFQ_K_EXCHANGE = 7, /* fused exchange energy                                 */
  AFQ_K_ENERGY = 8,   /* energy assembly and weighted estimate                 */
  AFQ_K_COUNT = 9
} afq_kernel;

/* on != 0 starts recording event pairs around every launch (and clears earlier
   records); on == 0 stops.  Recording adds two event records per launch. */
int afq_profile_enable(afq_ctx* ctx, int on);
/* Total device time in ms and launch count of one kernel class over the records
   taken since afq_profile_enable(ctx, 1); synchronises the stream. */
int afq_profile_read(afq_ctx* ctx, int kernel, double* total_ms, uint64_t* launches);
/* Name of a kernel class, or NULL when kernel is out of range. */
const char* afq_kernel_name(int kernel);

/* ---- Adjoint of the mixed local energy (the paper lists automatic differentiation
   as future work, Sec. "Customized mixed estimators"; closed forms of the local
   energy of Sec. "Local energy") ----
   For a cotangent gE (W complex; PyTorch's convention gE = dLoss/dRe E + i dLoss/dIm E)
   of Loss(E_L), at the current walkers:
     dh1  (M x M)          = Re sum_z conj(g_z) G_z   (G = the mixed one-body density
                            matrix sum_s Psi_s theta_s^T; dE/dh1 = G)
     dL   (X x M x M)      = Re sum_z conj(g_z) (c_zg G_z - sum_s G^s_z L_g^T G^s_z)
     dphi (W x M x N cplx) = g_z conj(dE_z/dPhi_z) = dLoss/dRe Phi + i dLoss/dIm Phi
   h1 and L_g entries are treated as independent (no symmetrisation).  Any output
   may be NULL.  FP64 in both precision modes.  The first call with dphi keeps a
   trial-fixed tensor of na^2 M^2 + nb^2 M^2 doubles on the device (released with the
   trial); a dL request takes a temporary workspace of max(na, nb)^2 M^2 doubles.
   AFQ_ERR_NOMEM when either cannot be allocated. */
int afq_local_energy_backward(afq_ctx* ctx, const double* gE, double* dh1, double* dL,
                              double* dphi);
int afq_local_energy_backward_dev(afq_ctx* ctx, const double* gE_dev, double* dh1_dev,
                                  double* dL_dev, double* dphi_dev);

/* ---- Adjoint of a K-step chain (FP64 contexts, fb_cap = 0) ----
   Objective: Loss = sum_z Re(conj(g_z) E_L(Phi_z^K)) after K steps of the hybrid
   propagation (Sec. "Review of AFQMC") from the walkers Phi^0 held at the call, with
   the fields xi of every step held fixed.  The force bias is differentiated through
   (it depends on Phi and L); the weights are not part of the objective (the phaseless
   max(0, cos) is not differentiable); vbar, L~ and P = exp(-dt h''/2) depend on h1
   and L.  QR re-orthogonalisation is a gauge (E_L and theta are invariant under
   Phi -> Phi C), so the cotangent maps through it as lam_pre = lam_post R^-T.

   afq_chain_forward runs K ordinary steps (weights, overlaps and QR as afq_propagate;
   fields: K x W x X N(0,1) values, or NULL for the device Philox stream at the
   current step counter), keeps a tape (the fields and the walkers at the chain start,
   after every QR and every ceil(sqrt(K)) steps when qr_period = 0) and returns the
   energies at Phi^K in e_out (W x 4 complex, as afq_local_energy; may be NULL).
   afq_chain_backward then gives, for a cotangent gE (W complex):
     dh1   (M x M)          symmetrised dLoss/dh1
     dL    (X x M x M)      symmetrised dLoss/dL_g
     dphi0 (W x M x N cplx) dLoss/dRe Phi^0 + i dLoss/dIm Phi^0
   recomputing each segment from its checkpoint and keeping, for every step of the
   longest segment, the walkers, i sqrt(dt) V and the taylor_order + 1 Taylor terms
   (about (taylor_order + 2) W M N + W M^2 complex values per step) until it returns.
   Any output may be NULL.  It fails
   with AFQ_ERR_STATE if the walkers changed after the forward (a step, QR, set_state
   or init_walkers).  The context's walkers, weights and force bias are left as the
   forward left them. */
int afq_chain_forward(afq_ctx* ctx, int K, const double* fields, double* e_out);
int afq_chain_forward_dev(afq_ctx* ctx, int K, const double* fields_dev, double* e_out_dev);
int afq_chain_backward(afq_ctx* ctx, const double* gE, double* dh1, double* dL, double* dphi0);
int afq_chain_backward_dev(afq_ctx* ctx, const double* gE_dev, double* dh1_dev, double* dL_dev,
                           double* dphi0_dev);

/* ---- CUDA graphs, batches of systems, autotuning (no counterpart in the paper:
   these serve the data-parallel step at scale) ---- */

/* Capture nsteps steps (fields drawn by the device Philox stream, whose step
   counter lives in device memory) each followed by the local energy, as one CUDA
   graph on the context's stream.  With qr_period > 0, nsteps must be a multiple of
   qr_period and the context's step counter must sit on a QR boundary, so that every
   replay performs the same QR cadence.  No host work runs during a replay. */
int afq_graph_capture(afq_ctx* ctx, int nsteps);
/* Launch the captured graph nreplays times (asynchronous, on the context's stream);
   the step counter advances by nreplays * nsteps. */
int afq_graph_launch(afq_ctx* ctx, int nreplays);
/* Energies of the last local-energy evaluation (from a graph or afq_local_energy_dev):
   e_out W x 4 complex and/or e_mix, host outputs; synchronises the stream. */
int afq_get_energy(afq_ctx* ctx, double* e_out, double* e_mix);

/* A batch of independent systems (contexts with walkers, possibly of uneven M, N,
   X and W) stepped by one CUDA graph in which every system is its own concurrent
   branch.  The batch owns its streams; the contexts stay owned by the caller and
   must outlive the batch. */
typedef struct afq_batch afq_batch;
int afq_batch_create(afq_batch** batch, int n, afq_ctx* const* ctxs);
int afq_batch_destroy(afq_batch* batch);
const char* afq_batch_last_error(const afq_batch* batch);
/* Launch layout of the next afq_batch_capture (Eq. Bx and the Taylor walker update
   of Sec. "Review of AFQMC", per system).  grouped = 0 (default): every system's
   step is its own graph branch.  grouped = 1 (FP64 contexts only, else
   AFQ_ERR_ARG): per step the fields of every system run on its branch, then ONE
   persistent launch builds the VHS of all systems and ONE propagates all their
   walkers -- CTAs take tiles of every system from a per-system descriptor table
   (M, N, X, W, device pointers) in order of decreasing cost, the next tile from a
   device counter -- and the rest of the step and the local energy run on the
   branches.  Results are bit-identical to the per-system launches.  The tables
   hold the contexts' current device buffers: re-capture after afq_init_walkers or
   afq_set_state changes a walker count. */
int afq_batch_set_grouped(afq_batch* batch, int grouped);
/* Capture nsteps steps + local energies of every system (same rules as
   afq_graph_capture, for each context). */
int afq_batch_capture(afq_batch* batch, int nsteps);
/* Replay nreplays times after the work already queued on the contexts' streams;
   later work on those streams waits for the replays. */
int afq_batch_launch(afq_batch* batch, int nreplays);
/* Wait for the replays and report the contexts' device flags. */
int afq_batch_synchronize(afq_batch* batch);

/* Autotuner: times candidate tiles of the kernels on the context's current walkers
   with CUDA events and keeps the fastest.  FP64: the g-group of the exchange kernel
   and the walker-column chunk of the propagator (timed on a copy, walkers
   restored).  AFQ_SPLIT_BF16: walkers per exchange tile for each spin and the
   split-K depth of the force bias.  Results do not change values beyond rounding
   order; they are read back with afq_get_tiles. */
int afq_autotune(afq_ctx* ctx);
/* tiles[0..n): FP64 exchange g-group (0 = default), FP64 propagator columns,
   split exchange walkers per tile (alpha, beta), force-bias split-K depth. */
int afq_get_tiles(afq_ctx* ctx, int* tiles, int n);

/* Exchange energy without any device allocation.  The paper has no counterpart:
   this exists for callers that cannot call cudaMalloc, such as a host framework
   that owns all device memory through its own pool or fixed arena, or a
   latency-critical loop that must avoid the device synchronisation of
   cudaMalloc / cudaFree.
   Inputs (device pointers, read on cuda_stream): Lt_dev, the half-rotated Cholesky
   vectors L~_g = Psi^T L_g as X x (na+nb) x M doubles (alpha rows first);
   thetaT_dev, theta^T of each walker as W x (na+nb) x M complex (theta_s =
   Phi_s (Psi_s^T Phi_s)^-1 per spin block).  Output: ek_dev, W complex values
   E_K,z = -1/2 sum_s sum_g sum_ij T_ij T_ji, the same as column EK of
   afq_local_energy.  The caller owns every buffer.
   The kernel's partial sums live in a file-scope device array of
   AFQ_STATIC_EXCHANGE_SLOTS complex doubles (4 MiB, held by each GPU that loads
   the library until exit).  A call needs W * 2 * ceil(X / G) slots, with
   G = max(1, 64 / max(na, nb)); larger calls return AFQ_ERR_ARG with a message on
   stderr.  The first call on a device looks up the array's device address (make
   that first call before any stream capture).  All calls share the array, so
   calls that overlap on the GPU race; each call writes every slot it reads.
   The exchange kernel's shared-memory limit is a process-wide attribute that the
   context path shares: a call only ever raises it (never lowers it), so it does
   not affect launches of contexts on other streams or host threads.
   Returns AFQ_OK, AFQ_ERR_ARG or AFQ_ERR_CUDA. */
#define AFQ_STATIC_EXCHANGE_SLOTS 262144
int afq_exchange_energy_static(int M, int X, int na, int nb, int W, const double* Lt_dev,
                               const double* thetaT_dev, double* ek_dev, void* cuda_stream);

/* Measured FP64 fused multiply-add throughput of the current device in TFLOP/s (2
   flops per FMA): 8 CTAs of 256 threads per SM, 16 independent FMA chains per thread,
   CUDA-event timed on cuda_stream, best of five launches after three untimed ones
   (about 0.3 s).  A measurement helper with no counterpart in the paper, reported
   beside the FP64 kernels' roofline.  Returns AFQ_OK, AFQ_ERR_ARG (NULL output) or
   AFQ_ERR_CUDA. */
int afq_fp64_fma_rate(double* tflops, void* cuda_stream);

/* Split-precision real GEMM on the tensor cores: C = A B^T with A m x k, B n x k and
   C m x n, all row-major FP64 DEVICE arrays, read and written on cuda_stream.  Each
   operand is cut into `slices` bfloat16 slices (1..4) and the slice products with
   s + t <= slices - 1 are accumulated in FP32 by tcgen05.mma; this is the
   contraction engine of the AFQ_SPLIT_BF16 force bias (Eq. rfb) and exchange
   (Sec. "Local energy").  Allocates its slice workspace, synchronises the stream
   before returning.  Returns AFQ_OK, AFQ_ERR_ARG, AFQ_ERR_NOMEM or AFQ_ERR_CUDA. */
int afq_gemm_split_bf16(int m, int n, int k, int slices, const double* A_dev, const double* B_dev,
                        double* C_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
