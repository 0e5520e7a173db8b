/*
 * ltmp2.h -- C ABI of the GB300 (sm_103a) Laplace-transformed MP2 hot path.
 *
 * Method: Schaefer, Ramberger, Kresse, "Quartic scaling MP2 for solids: a highly
 * parallelized algorithm in the plane wave basis" (arXiv:1611.06797).  Gamma
 * point; closed shell, spin restricted (Sec. II B: sum over spins -> 2), with a
 * spin-unrestricted pairing of two contexts (ltmp2_energy_uhf).  Beside the
 * Green's-function route below, the paper's own stored-overlap-density route
 * (ltmp2_set_route) and its internal auxiliary-cutoff extrapolation
 * (ltmp2_set_extrapolation) are available.
 *
 * For each Laplace point tau (Eq. SCHLT) the library builds the tau-scaled
 * virtual Green's function P_v(tau) = sum_a |a> e^{-(e_a - mu) tau} <a| in the
 * plane-wave basis, the transformed occupied states
 *     w_j^{(G' tau)} = e^{(e_j - mu) tau} P_v(tau) e^{-iG'r} |j>       (Eqs. SCHnewstate, SCHtransmatrix)
 * forms the pair co-densities <i| e^{-iGr} |w_j^{(G' tau)}> with batched 3D FFTs,
 * weights them with the Coulomb kernel v(G) = 4 pi / G^2 (Eq. SCH2EI) and
 * contracts the exchange (Fock-like, Eq. SCHfocklike) and direct (Hartree-like,
 * Eq. dLTMP2Compact at q = 0) terms.  No sum over virtual orbitals is done
 * after P_v is built.  The energies are
 *     E_x = sum_k w_k/Omega^2 sum_{G,G' in A} v(G) v(G') sum_ij M_ij(G;G') M_ji(-G;-G')
 *     E_d = -2 sum_k w_k/Omega^2 sum_{G,G' in A} v(G) v(G') sum_ij M_ii(G;G') M_jj(-G;-G')
 * with M_ij(G;G') = <i|e^{-iGr}|w_j^{(G' tau_k)}> and A the auxiliary set
 * {G != 0 : |G|^2/2 <= E_cut^aux} (Sec. II A).  This equals closed-shell MP2
 * (Eq. CanMP2 with Eqs. MP2direct, MP2exchange) with 1/Delta replaced by
 * -sum_k w_k exp(Delta tau_k).
 *
 * Conventions
 *   - Hartree atomic units; energies are per simulation cell.
 *   - Overlap densities are grid-discrete: phi_n(r_t) = Omega^{-1/2} sum_p c_n(p)
 *     e^{i G_p r_t} on the FFT grid and rho_mn(G) = (Omega/N_FFT) sum_t
 *     phi_m^*(r_t) phi_n(r_t) e^{-i G r_t} (aliasing included).
 *   - The G = 0 Coulomb term is dropped (rho_ia(0) = 0 for occupied/virtual pairs).
 *   - Every function returns LTMP2_OK (0) or a negative status; ltmp2_strerror()
 *     names it.  Nothing is printed.  On error no output is written.
 *   - A context is thread-compatible, not thread-safe: calls on one context must
 *     not overlap.  Different contexts are independent.
 *   - All pointers in these signatures are HOST pointers unless stated.
 */
#ifndef LTMP2_H
#define LTMP2_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define LTMP2_OK 0
#define LTMP2_ERR_INVALID_ARG (-1)     /* NULL pointer, size <= 0, NaN, unsorted eigenvalues ... */
#define LTMP2_ERR_GAP (-2)             /* e_LUMO - e_HOMO < 1e-6 Ha: the Laplace transform needs a gap */
#define LTMP2_ERR_NOT_ORTHONORMAL (-3) /* sampled <m|n> deviates from delta_mn by more than 1e-8 */
#define LTMP2_ERR_GRID (-4)            /* grid not cubic/5-smooth/supported, or a sphere does not fit it */
#define LTMP2_ERR_OOM (-5)             /* device allocation failed */
#define LTMP2_ERR_CUDA (-6)            /* a CUDA call failed (no device, launch error ...) */
#define LTMP2_ERR_TIMEOUT (-7)         /* a bounded device wait ran out (persistent batch kernel) */
#define LTMP2_ERR_UNSUPPORTED (-8)     /* option not available for these sizes */
#define LTMP2_ERR_NO_CONVERGENCE (-9)  /* Laplace-grid fit did not converge */
#define LTMP2_ERR_NOT_REAL (-10)       /* LTMP2_FLAG_REAL_ORBITALS set but c(-G) != conj c(G) */

/* ---------------------------------------------------------------- precision */
/* LTMP2_FP64: complex128 FFTs, FP64 GEMMs, FP64 accumulation (the plain path).   */
/* LTMP2_FP32: complex64 FFTs; transformed-state GEMM on tcgen05 tensor cores in  */
/*             3xTF32 split precision (hi*hi + hi*lo + lo*hi), each 16-wide k    */
/*             block's tensor-memory partial added to FP32 register sums; with   */
/*             real orbitals the Green's function P_r = R_v^T D R_v and the      */
/*             direct-term products sum_G v M_ii conj(M_jj) per G' too (general  */
/*             orbitals: CUDA cores, compensated FP32 sums); per-pair, per-tau   */
/*             and final sums in FP64.                                           */
#define LTMP2_FP64 0
#define LTMP2_FP32 1

/* ---------------------------------------------------------------- flags */
/* Orbitals are real in real space, c_n(-G) = conj(c_n(G)) (time-reversal symmetry,
 * Sec. II D, at k = 0).  Then w_j^{(-G')} = conj(w_j^{(G')}) in real space and only
 * half of the G' set is transformed; the library checks the property in setup.  */
#define LTMP2_FLAG_REAL_ORBITALS 1
/* Run the dense products on the CUDA cores instead of the tcgen05 tensor cores: in
 * LTMP2_FP32 the transformed-state GEMM in FP32 with two-level summation instead of the
 * 3xTF32 kernel; in LTMP2_FP64 the Green's function and transformed-state GEMMs in FP64
 * instead of the exact-slice products (see ltmp2_dgemm_nt).  For comparisons.       */
#define LTMP2_FLAG_SIMT_GEMM 2

typedef struct ltmp2_ctx ltmp2_ctx; /* opaque; owns all device memory of one system */

/* Mean-field input of one system (Sec. II A; the paper takes HF orbitals, Fig. SerialGamma).
 *   lattice   [9]  rows a1, a2, a3 of the cell (bohr), row-major; Omega = |det|.
 *   grid      [3]  FFT grid n1, n2, n3.  Must be cubic (n1 = n2 = n3) with
 *                  n in {8,10,12,16,18,20,24,25,27,30,32,36,40}.
 *   n_pw           number of plane waves of the orbital basis (|G|^2/2 <= E_cut).
 *   miller    [n_pw][3] int: G_p = m1 b1 + m2 b2 + m3 b3.  Each |m_k| < n_k/2, and
 *                  for every (m1, m2) its m3 values must form one contiguous range (true
 *                  for a sphere); with LTMP2_FLAG_REAL_ORBITALS the set must also be
 *                  inversion symmetric.
 *   n_orb, n_occ   orbitals (ascending energy); the first n_occ are doubly occupied,
 *                  all others virtual.  1 <= n_occ < n_orb <= n_pw.
 *   coeff     [n_orb][n_pw] complex128 as interleaved (re, im) doubles, row-major,
 *                  orthonormal rows (the library samples <m|n>).
 *   eps       [n_orb] orbital energies in Hartree, non-decreasing.
 *   ecut_aux       E_cut^aux in Hartree; <= 0 selects 2/3 of the largest |G_p|^2/2
 *                  ("commonly chosen as 2/3 E_cut", Sec. II A).
 *   precision      LTMP2_FP64 or LTMP2_FP32.
 *   flags          0 or LTMP2_FLAG_REAL_ORBITALS, optionally | LTMP2_FLAG_SIMT_GEMM.
 */
typedef struct {
  double lattice[9];
  int grid[3];
  int n_pw;
  const int *miller;
  int n_orb;
  int n_occ;
  const double *coeff;
  const double *eps;
  double ecut_aux;
  int precision;
  int flags;
} ltmp2_system;

/* Validate the input, copy it to the current CUDA device and precompute the
 * tau-independent parts (occupied orbitals on the grid, the aux set A and v(G),
 * index tables).  The caller keeps ownership of every array in *sys; nothing is
 * retained.  On success *out owns the device memory until ltmp2_destroy().
 * Errors: INVALID_ARG, GAP, NOT_ORTHONORMAL, GRID, NOT_REAL, OOM, CUDA.           */
int ltmp2_setup(const ltmp2_system *sys, ltmp2_ctx **out);

/* Run all later work of ctx on this CUDA stream (a cudaStream_t passed as void*;
 * NULL = the legacy default stream).  The stream must belong to the device that
 * was current at setup and must outlive the calls that use it.                  */
int ltmp2_set_stream(ltmp2_ctx *ctx, void *stream);

/* Laplace quadrature for the energy denominator (Eq. SCHLT; the paper uses a
 * minimax grid, Sec. II C and Sec. III A, without printing it):
 *     1/x ~= sum_{k<n_tau} w_k exp(-x tau_k)   on  x in [2 gap, 2 width],
 * fitted to minimise max_x |1 - x sum_k w_k exp(-x tau_k)| (relative error).
 *   gap   = e_LUMO - e_HOMO > 0,  width = e_max - e_min >= gap  (Hartree).
 *   n_tau in [1, 24].  tau, w: caller arrays of n_tau doubles, ascending tau.
 *   max_err (may be NULL): the achieved maximum relative error, measured on
 *   20000 log-spaced points.  Host only; no device is touched.
 * Errors: INVALID_ARG, NO_CONVERGENCE.                                          */
int ltmp2_laplace_grid(double gap, double width, int n_tau, double *tau, double *w,
                       double *max_err);

/* E_direct and E_exchange (and per-pair energies) for the quadrature (tau, w).
 *   n_tau >= 1; tau[k] > 0, w[k] finite (host arrays, copied).
 *   e_direct, e_exchange: one double each (host).
 *   e_pair: NULL or [n_occ][n_occ] doubles (host, row-major) receiving
 *           e_ij = e^d_ij + e^x_ij, symmetric, summing to E_d + E_x.
 * The call is synchronous: it returns after the results are on the host.
 * Errors: INVALID_ARG, OOM, CUDA.                                               */
int ltmp2_energy(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w,
                 double *e_direct, double *e_exchange, double *e_pair);

/* The contribution of the outer-loop plane waves G' in the half-open range
 * [gp_begin, gp_end) of the ordered primary set (Sec. III B: the G' loop splits
 * into independent, communication-free pieces).  Primary G' are the aux vectors
 * whose first non-zero Miller index is positive; each carries its partner -G'.
 * Summing the outputs over a partition of [0, ltmp2_num_primary_gprime()) gives
 * exactly the ltmp2_energy() result up to summation order.
 *   e_pair_direct, e_pair_exchange: NULL or [n_occ][n_occ] doubles (host).
 * Errors: INVALID_ARG, OOM, CUDA.                                               */
int ltmp2_energy_partial(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w,
                         int gp_begin, int gp_end, double *e_direct, double *e_exchange,
                         double *e_pair_direct, double *e_pair_exchange);

/* Primary G' vectors processed per slab (one pass of the transformed-state GEMM,
 * the FFT kernels and the contraction).  Setup picks the largest slab that fits a
 * share of the free device memory; n in [1, that capacity] lowers it (smaller
 * launches, same result up to summation order), n <= 0 restores it.  Returns the
 * slab size in effect, or a negative status.                                     */
int ltmp2_set_slab_size(ltmp2_ctx *ctx, int n);

/* ---------------------------------------------------------------- batching form
 * Several systems of uneven grids and orbital counts in one launch.  The outer loops
 * of Sec. III A (tau points, then slabs of the G' loop, Sec. III B) of every system are
 * captured into one CUDA graph, so a run is a single graph launch.  When every system
 * allows it (Gamma point, one precision, no cutoff levels, the Green's-function route,
 * at most 16 systems) and the systems need similar numbers of (tau, slab) rounds (the
 * most at most twice the fewest), the graph runs in rounds: round r takes the r-th (tau, slab) of every
 * system that still has one; each system's gather, transformed-state GEMM and z transform
 * run on its own branch, then ONE persistent plane-FFT launch and ONE persistent column
 * launch serve the co-density items of all those systems (resident thread blocks take
 * (system, column, plane) and (system, pair) items from a device counter), then each
 * system's direct term and accumulation.  Otherwise every system is one graph branch.
 * FP64 energies equal ltmp2_energy's to rounding of the summation order.              */

/* Autotuner: times one slab of the path for each candidate (slab sizes down from the
 * setup capacity; in LTMP2_FP32 also the two tensor-core GEMM layouts) and keeps the
 * fastest per primary G', then the plane FFT kernel and its block shape.  The choice is cached per (grid, n_pw, n_occ, |A|, precision,
 * real-orbital flag) for the process and applied to ctx.  slab, gemm_variant: NULL or
 * receive the choice (gemm_variant = -1 in LTMP2_FP64).  Errors: INVALID_ARG, CUDA,
 * TIMEOUT.                                                                          */
int ltmp2_autotune(ltmp2_ctx *ctx, int *slab, int *gemm_variant);

/* Settings in effect for ctx: values[0] slab size, [1] tensor-core GEMM layout (-1 in
 * FP64 or with LTMP2_FLAG_SIMT_GEMM), [2] plane FFT kernel (0 full-plane passes,
 * 1 compacted passes, 2 product in registers with a compact intermediate, 3 the same with
 * every warp on its own occupied planes and no block barriers; set-up chooses 3 in
 * LTMP2_FP32 and 2 in LTMP2_FP64), [3] occupied planes per plane-kernel block, for
 * kernel 3 per warp step (0 = default), [4] the precision form's
 * Green's function on the tensor cores (1; 3xTF32, set up at first use) or on the CUDA
 * cores with compensated sums (0, the default: the tensor-core build's plain FP32 sums
 * over K = n_v left 4x the error in E_d on the 36^3 workload), [5] its direct-term
 * contraction on the tensor cores (1, the default) or the CUDA cores (0); [4] and [5] are
 * -1 where there is no choice (FP64, general orbitals, LTMP2_FLAG_SIMT_GEMM).
 * The autotuner also chooses [2] and [3], timing the plane kernel alone.  values holds
 * LTMP2_TUNING_VALUES entries.                                                          */
#define LTMP2_TUNING_VALUES 6
int ltmp2_get_tuning(const ltmp2_ctx *ctx, int *values);

/* Apply settings by hand, same layout as ltmp2_get_tuning; a negative entry keeps the
 * current value.  Every choice gives the same energies up to rounding.  INVALID_ARG for
 * a slab outside 1..capacity, a GEMM layout without the tensor-core path (or other than
 * 5 for real orbitals), a plane-kernel shape over 1024 threads or 200 KB of shared
 * memory, or a value of [4] / [5] other than -1 where there is no choice.             */
int ltmp2_set_tuning(ltmp2_ctx *ctx, const int *values);

typedef struct ltmp2_batch ltmp2_batch; /* opaque; a captured, instantiated graph */

/* Capture the full energy evaluation of n distinct contexts (each with its own
 * quadrature: n_tau[i], tau[i][*], w[i][*], host arrays copied into the graph) into one
 * CUDA graph.  The contexts must stay alive, on one device and with unchanged slab /
 * tuning settings, until ltmp2_batch_destroy.  Nothing runs yet.
 * Errors: INVALID_ARG (NULL, duplicate ctx, bad tau), OOM, CUDA.                     */
int ltmp2_batch_create(ltmp2_ctx *const *ctxs, int n, const int *n_tau, const double *const *tau,
                       const double *const *w, ltmp2_batch **out);

/* One graph launch on the stream of ctxs[0]; waits for it and writes E_direct[i] and
 * E_exchange[i] (host arrays of n).  Per-pair energies stay readable through each
 * context's accumulators only via ltmp2_energy.  Errors: INVALID_ARG, CUDA, TIMEOUT. */
int ltmp2_batch_run(ltmp2_batch *b, double *e_direct, double *e_exchange);

/* Number of kernel nodes in the batch graph (all systems).                          */
int ltmp2_batch_kernel_nodes(const ltmp2_batch *b, long long *count);

/* *persistent = 1 when b runs in rounds with the shared persistent FFT stages, else 0. */
int ltmp2_batch_mode(const ltmp2_batch *b, int *persistent);

void ltmp2_batch_destroy(ltmp2_batch *b);

/* Autotune every context, then create, run once and destroy a batch.                */
int ltmp2_energy_batch(ltmp2_ctx *const *ctxs, int n, const int *n_tau, const double *const *tau,
                       const double *const *w, double *e_direct, double *e_exchange);

/* ---------------------------------------------------------------- learned form
 * Weak occupied pairs are screened: their exchange co-densities (the N_o^2 part of
 * step (iv.b), Sec. III C) are not formed and their exchange energy is estimated by a
 * small pair-energy model instead; the direct term (step (iv.a)) stays exact for all
 * pairs.  The paper has no counterpart.  ltmp2_energy_screened runs the whole form:
 * descriptors, the model's estimates, the screening rule and the combined energy.     */

/* keep: NULL (every pair contracted) or [n_occ][n_occ] bytes, symmetric, keep[i][i] != 0;
 * keep[i][j] == 0 leaves pair (i, j) out of the exchange contraction in later
 * ltmp2_energy* calls (their e^x_ij, and so E_exchange, omit it).  Errors: INVALID_ARG,
 * OOM, CUDA.                                                                           */
int ltmp2_set_pair_mask(ltmp2_ctx *ctx, const unsigned char *keep);

/* Cheap descriptors of every unordered occupied pair i <= j (row order i, then j),
 * LTMP2_NUM_DESC doubles each: e_i - mu, e_j - mu (Ha), log10 S_ij / sqrt(S_ii S_jj)
 * with S_ij = (1/N) sum_r |u_i|^2 |u_j|^2, centroid distance (bohr, periodic centroids, minimum
 * image), spreads of i and j (bohr), i == j, distance / (spread_i + spread_j).
 * desc: host array of n_occ (n_occ + 1) / 2 * LTMP2_NUM_DESC doubles.             */
#define LTMP2_NUM_DESC 8
int ltmp2_pair_descriptors(ltmp2_ctx *ctx, double *desc);

/* Pair-energy surrogate: a perceptron n_in -> width -> width -> 1 (tanh, FP32;
 * n_in <= 16, width <= 64), trained with Adam on standardised inputs and targets by
 * hand-written kernels on the current device.                                         */
typedef struct ltmp2_mlp ltmp2_mlp;
int ltmp2_mlp_create(int n_in, int width, unsigned long long seed, ltmp2_mlp **out);
/* X [n][n_in], y [n] host arrays; full-batch Adam for `epochs` steps at rate lr;
 * final_loss (may be NULL): mean squared error of the standardised targets.         */
int ltmp2_mlp_train(ltmp2_mlp *net, const float *X, const float *y, int n, int epochs, float lr,
                    float *final_loss);
/* y[n] = model(X[n][n_in]) in the units of the training targets.                    */
int ltmp2_mlp_predict(const ltmp2_mlp *net, const float *X, int n, float *y);
/* Root-mean-square residual of the last training run, in the units of the targets (0
 * before any training).                                                              */
int ltmp2_mlp_residual(const ltmp2_mlp *net, float *sigma);
void ltmp2_mlp_destroy(ltmp2_mlp *net);

/* Training set of the pair model from one exact all-pairs evaluation of ctx (Gamma point):
 *   X [n_occ (n_occ + 1) / 2][LTMP2_NUM_DESC] the descriptors of ltmp2_pair_descriptors,
 *   y [n_occ (n_occ + 1) / 2] the target ln|e^x_ij| of each unordered pair i <= j, where
 *     e^x_ij is the exchange energy of the ordered pairs (i, j) and (j, i) together (of
 *     (i, i) for i = j), from the contraction of every pair (any pair mask is cleared).
 * Host arrays.  Errors: INVALID_ARG, UNSUPPORTED (k-point contexts), OOM, CUDA.       */
int ltmp2_learned_training_data(ltmp2_ctx *ctx, int n_tau, const double *tau, const double *w, float *X,
                                float *y);

/* The screening rule.  est [n_occ (n_occ + 1) / 2]: non-negative estimates of |e^x_ij|
 * per unordered pair (row order i, then j >= i).  Off-diagonal pairs are screened in
 * ascending order of est (ties in row order) while the sum of the screened estimates
 * stays <= budget (Ha); diagonal pairs are never screened.  keep [n_occ][n_occ] receives
 * the pair mask (symmetric, 0 = screened); n_screened and est_screened (may be NULL) the
 * number of screened unordered pairs and the sum of their estimates.  Host only.
 * Errors: INVALID_ARG (sizes, a negative or non-finite estimate or budget), OOM.       */
int ltmp2_screen_select(int n_occ, const double *est, double budget, unsigned char *keep, int *n_screened,
                        double *est_screened);

/* Learned-form energy.  The model net (LTMP2_NUM_DESC inputs, trained on the targets of
 * ltmp2_learned_training_data) predicts y_ij ~ ln|e^x_ij| for every unordered pair from
 * the descriptors.  Selecting the smallest predictions favours the pairs the model
 * underestimates, so the screening decision runs on an upper bound: ltmp2_screen_select
 * takes margin x exp(y_ij) against the budget (Ha, e.g. 0.1 meV/atom x atoms), where
 * margin >= 1 is the caller's validated bound on |e^x| / exp(y) for the lowest predictions
 * (from systems held out of training).  A screened pair contributes exp(y_ij).  The
 * screened pairs' exchange co-densities are not formed:
 *   e_direct   = E_d of every pair (exact),
 *   e_exchange = E_x of the contracted pairs + the screened pairs' estimates.
 * info (may be NULL) [4]: screened unordered pairs, their estimated exchange (Ha), the
 * contracted exchange (Ha), unordered pairs.  The pair mask of ctx is cleared afterwards.
 * Errors: INVALID_ARG (also margin < 1), UNSUPPORTED (k-point contexts), OOM, CUDA, TIMEOUT. */
int ltmp2_energy_screened(ltmp2_ctx *ctx, const ltmp2_mlp *net, int n_tau, const double *tau, const double *w,
                          double budget, double margin, double *e_direct, double *e_exchange, double *info);

/* ---------------------------------------------------------------- failure-path self-test
 * (no counterpart in the paper)  Every device-side wait of this library (the tcgen05
 * GEMM's mbarrier waits) is bounded: when its budget runs out the kernel raises a device
 * error word, finishes and returns, and the entry point reports LTMP2_ERR_TIMEOUT; the
 * context stays usable.  This call exercises that path on demand: one thread waits, with
 * the same bounded wait, on an mbarrier that nothing ever completes, for budget_us
 * microseconds (1 .. 10^6).  Returns LTMP2_ERR_TIMEOUT (the expected outcome: the wait
 * ran out and was reported), LTMP2_OK only if the wait completed (a broken timer), or
 * INVALID_ARG / OOM / CUDA.                                                           */
int ltmp2_selftest_wait(ltmp2_ctx *ctx, int budget_us);

/* ---------------------------------------------------------------- spin-unrestricted form
 * Eqs. MP2direct and MP2exchange with the spin sums kept (Sec. II B): alpha and beta
 * electrons occupy different orbital sets.  With <ij|ab> between orbitals of the stated
 * spins and D the Laplace denominator of Eq. SCHLT,
 *   E_direct   = 1/2 sum_{s s'} sum_{i j a b} |<i s, j s'|a s, b s'>|^2 D,
 *   E_exchange = -1/2 sum_s sum_{i j a b} <i s, j s|a s, b s> <a s, b s|j s, i s> D.
 * Each channel runs the closed-shell path on its own orbitals (its exchange and same-spin
 * direct sums, reweighted: 1/2 per (s, s') and per s instead of 2 and 1), and the
 * opposite-spin direct term contracts the two channels' diagonal co-densities
 * M^alpha_ii(G;G') and M^beta_jj(-G;-G') at the same tau and G' (the paper notes that
 * the spin-unrestricted case costs twice the restricted one, Sec. III C).
 *   alpha, beta: contexts set up from the two channels' orbitals and energies, each with
 *     its own n_occ (singly occupied orbitals, >= 1) and mid-gap shift; they must share
 *     the lattice, grid, plane-wave set, auxiliary set, precision and real-orbital flag
 *     (else INVALID_ARG).  Both run on alpha's stream; extrapolation levels and pair
 *     masks are not supported here (UNSUPPORTED).  The first call allocates alpha's
 *     opposite-spin scratch.
 *   tau, w: a quadrature valid for both channels' denominators.
 *   e_direct, e_exchange: Ha per cell.  e_spin: NULL or [3] = same-spin alpha, same-spin
 *     beta and opposite-spin parts of E_direct + E_exchange.                            */
int ltmp2_energy_uhf(ltmp2_ctx *alpha, ltmp2_ctx *beta, int n_tau, const double *tau, const double *w,
                     double *e_direct, double *e_exchange, double *e_spin);

/* ---------------------------------------------------------------- transformed-state route
 * How step (iii) of Sec. III A builds w_j^{(G' tau)} (Eqs. SCHnewstate, SCHtransmatrix):
 *   LTMP2_ROUTE_GREEN (default): the virtual Green's function P_v(tau) is built per tau by a
 *     GEMM over the virtuals and applied to the gathered e^{-iG'r}|j>; nothing is stored.
 *   LTMP2_ROUTE_OVERLAP: the paper's own route: step (i) computes and stores the overlap
 *     densities rho_aj(G') = <a|e^{-iG'r}|j> (Eq. SCHovrlp) once for every virtual a,
 *     occupied j and primary G' (n_prim x n_occ x n_v complex values: 1.35 GB in FP64 for
 *     3071 plane waves, 32 occupied), and per tau and G' the transformation matrix
 *     e^{(e_j-mu)tau} rho_aj(G') e^{-(e_a-mu)tau} multiplies the virtual coefficients.
 * Both give the same energies up to rounding.                                          */
#define LTMP2_ROUTE_GREEN 0
#define LTMP2_ROUTE_OVERLAP 1
/* Select the route for later ltmp2_energy* calls.  LTMP2_ROUTE_OVERLAP computes and stores
 * the overlap densities during this call (first use allocates them) and needs
 * LTMP2_FLAG_REAL_ORBITALS (UNSUPPORTED otherwise); its transformed-state product runs on
 * the CUDA cores in both precisions.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.       */
int ltmp2_set_route(ltmp2_ctx *ctx, int route);

/* ---------------------------------------------------------------- FP64 products on the tensor cores
 * The FP64 path's products in the real basis (the Green's function P_r, the transformed
 * states W^T = (U S)^T P_r of step (iii), Sec. III A, and at large tau the two products
 * through the kept virtuals) run on the tcgen05 tensor cores with FP64 accuracy, unless
 * LTMP2_FLAG_SIMT_GEMM is set: every row of both operands is scaled by a power of two and
 * cut into 8 slices of 7 bits (exact in TF32); the 36 slice products with s + t < 8 are
 * accumulated per order s + t in FP32 tensor memory, where sums of at most 400 k stay
 * below 2^24 and are therefore exact, and combined in FP64 registers.  A dropped term is
 * at most 7 x 2^-56 of the product of the two rows' largest magnitudes; the result
 * differs from an FP64 GEMM by about its own rounding.
 * ltmp2_dgemm_nt: C = A B^T with that scheme.  A [m][lda], B [n][ldb], C [m][ldc]: DEVICE
 * pointers to row-major doubles (first k columns of A and B used), lda, ldb >= k,
 * ldc >= n.  Allocates and frees its own slice buffers (about 32 (m + n) k bytes) and
 * synchronises the device.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (a bounded wait
 * inside the kernel ran out; C is then not written).                                     */
int ltmp2_dgemm_nt(int m, int n, int k, const double *a, int lda, const double *b, int ldb, double *c, int ldc);

/* ---------------------------------------------------------------- virtuals per Laplace point
 * The Laplace factor of Eq. SCHLT weights virtual a at point tau by e^{-(e_a-mu)tau}.
 * Relative to the LUMO's weight, the virtuals with e^{-(e_a - e_LUMO) tau} < 2^-L add
 * terms below the rounding of an FP64 product over the others (L = 64 by default; the
 * product's own rounding is about 2^-53 of the sum of its terms' magnitudes), so they are
 * left out of the Green's function and of step (iii)'s transformation at that tau.
 * Energies ascend, so the kept virtuals are the first n_v(tau).  When the transformed
 * states are then cheaper through the virtual space, W = R_v'^T D' (R_v' U S), than
 * through the Green's function (4 n_pw n_v(tau) against 2 n_pw^2 multiply-adds per
 * column; real orbitals, CUDA-core GEMMs: the FP64 path and LTMP2_FLAG_SIMT_GEMM), the
 * library takes that route for that tau and builds no Green's function.
 *   LTMP2_VIRTUALS_ALL:   every virtual at every tau, W through the Green's function.
 *   LTMP2_VIRTUALS_AUTO:  the default described above.
 *   LTMP2_VIRTUALS_SPACE: as AUTO, but W through the virtual space at every tau where
 *                         the route exists (a test setting: slower at small tau).
 * k-point contexts keep every virtual (UNSUPPORTED).                                   */
#define LTMP2_VIRTUALS_ALL 0
#define LTMP2_VIRTUALS_AUTO 1
#define LTMP2_VIRTUALS_SPACE 2
/* mode as above; 53 <= log2_cut <= 1100 is L.  Applies to later ltmp2_energy* calls.
 * Errors: INVALID_ARG, UNSUPPORTED.                                                      */
int ltmp2_set_virtual_cut(ltmp2_ctx *ctx, int mode, double log2_cut);
/* For each of n_tau points tau[k] > 0: n_virt[k] = the virtuals kept at tau[k] and, when
 * w_virtual is not NULL, w_virtual[k] = 1 if the transformed states go through the virtual
 * space there (host arithmetic only; no device work).  Errors: INVALID_ARG.              */
int ltmp2_tau_virtuals(ltmp2_ctx *ctx, int n_tau, const double *tau, int *n_virt, int *w_virtual);

/* ---------------------------------------------------------------- internal cutoff extrapolation
 * Sec. III D, Eq. CutDecay: the MP2 energy converges with the auxiliary cutoff as
 * E(E_aux) - E(inf) ~ E_aux^(-3/2).  With n_c levels, every later ltmp2_energy* call
 * also evaluates the energy on the nested spheres A_n = {G : |G|^2/2 <= E_aux[n]},
 * E_aux[n] = E_aux / alpha^(n-1), n = 1..n_c (A_1 = A; both the inner G-sum and the
 * outer G'-sum are truncated), in the same pass: only the column and direct-term
 * contractions group their G-sums by level, plus one accumulation launch per slab.   */

/* n_c <= 1 switches the levels off; 2 <= n_c <= LTMP2_MAX_LEVELS, alpha > 1 (the paper
 * uses n_c = 8, alpha = 1.05).  The first call allocates the level accumulators
 * (2 x 16 x slab capacity x n_occ^2 x 16 bytes).  Errors: INVALID_ARG; UNSUPPORTED when
 * the column kernel's shared memory (2 |A| complex values) exceeds 200 KB (FP64 with
 * |A| > 6400); OOM; CUDA.                                                            */
#define LTMP2_MAX_LEVELS 16
int ltmp2_set_extrapolation(ltmp2_ctx *ctx, int n_c, double alpha);

/* Per level n (arrays of n_c entries on the host, any may be NULL): the cutoff E_aux[n]
 * (Ha), |A_n| (G = 0 excluded), and E_direct[n], E_exchange[n] (Ha per cell) of the
 * last ltmp2_energy* call made with these levels (level 1 equals that call's result).
 * INVALID_ARG when the levels are off, or energies are asked for before such a call. */
int ltmp2_level_energies(const ltmp2_ctx *ctx, double *ecut_aux, int *n_aux, double *e_direct,
                         double *e_exchange);

/* Least-squares line y = a + b x through the n >= 2 points y = energy[k],
 * x = ecut_aux[k]^(-3/2) (Eq. CutDecay): *e_inf = a (the extrapolated energy),
 * *slope = b, *sigma = standard error of a from the residuals (0 for n = 2); slope
 * and sigma may be NULL.  Host arithmetic only.  INVALID_ARG on non-positive or equal
 * cutoffs.                                                                           */
int ltmp2_extrapolate(int n, const double *ecut_aux, const double *energy, double *e_inf, double *slope,
                      double *sigma);

/* Number of primary G' vectors (half of |A|); returns < 0 on a NULL ctx.        */
int ltmp2_num_primary_gprime(const ltmp2_ctx *ctx);

/* Sizes of a set-up system: n_aux = |A| (G = 0 excluded), n_pw, n_occ, grid n. */
int ltmp2_sizes(const ltmp2_ctx *ctx, int *n_aux, int *n_pw, int *n_occ, int *grid_n);

/* Imaginary residues of the last ltmp2_energy* call: the exact sums are real, so
 * these measure rounding (and, for LTMP2_FLAG_REAL_ORBITALS, the symmetry).       */
int ltmp2_last_imag(const ltmp2_ctx *ctx, double *im_direct, double *im_exchange);

/* Per-stage device timing.  When enabled (on != 0), every later ltmp2_energy*
 * call records CUDA events around each kernel launch on the context's stream and
 * accumulates, per stage, the number of launches and their summed duration (ms).
 * Stages: 0 Green's-function GEMM, 1 transformed-state GEMM, 2 gather and
 * w z-transform, 3 plane FFT kernel, 4 column FFT + exchange contraction,
 * 5 direct-term contraction, 6 accumulation.  ltmp2_stage_times() copies
 * min(n, 7) entries and resets nothing; ltmp2_reset_stage_times() zeroes them.   */
#define LTMP2_NUM_STAGES 7
int ltmp2_set_profiling(ltmp2_ctx *ctx, int on);
int ltmp2_stage_times(const ltmp2_ctx *ctx, int n, double *ms, long long *launches);
int ltmp2_reset_stage_times(ltmp2_ctx *ctx);

/* Cumulative number of this library's kernel launches made for ctx (all calls). */
int ltmp2_kernel_launches(const ltmp2_ctx *ctx, long long *count);

/* 64-bit hash of every input that determines the energies of ctx: lattice, grid,
 * plane-wave set, coefficients, eigenvalues, n_occ, the resolved E_aux, precision and
 * flags (the paper has no counterpart; checkpoint files are keyed by it).  Two set-ups
 * of the same inputs give the same value.  Errors: INVALID_ARG.                      */
int ltmp2_fingerprint(const ltmp2_ctx *ctx, unsigned long long *out);

/* Fixed-order FP64 sum of the results of n ltmp2_energy_partial calls over disjoint G'
 * ranges (Sec. III B: the pieces are additive), chunk 0 first, so that a checkpointed
 * and resumed evaluation sums exactly as an uninterrupted one.
 *   e [n][2] (E_d, E_x per chunk); pd, px: NULL or [n][n_occ][n_occ] pair energies.
 *   e_out [2]; pd_out, px_out: NULL or [n_occ][n_occ].  Host arithmetic only.
 * Errors: INVALID_ARG (sizes, NULL where outputs are asked for, non-finite totals). */
int ltmp2_sum_partials(int n, int n_occ, const double *e, const double *pd, const double *px, double *e_out,
                       double *pd_out, double *px_out);

/* ltmp2_setup + ltmp2_energy in one call that makes no device allocation (the paper
 * has no counterpart; this serves callers that cannot call cudaMalloc: a process whose
 * device-memory budget is already held by its own pool, code that must not trigger
 * the device-wide synchronisation cudaMalloc/cudaFree can cause, or a plug-in whose
 * host application owns all device memory).
 *   sys, n_tau, tau, w, e_direct, e_exchange, e_pair: as for ltmp2_setup and
 *           ltmp2_energy (host pointers; e_pair may be NULL).
 *   stream: a cudaStream_t as void* (NULL = legacy default stream) on the current device.
 * Every device buffer of the path lives in one 32 MiB array that is part of the
 * library image (each GPU that loads the library holds it until the process exits).
 * Systems whose buffers do not fit return LTMP2_ERR_UNSUPPORTED; as a guide, the
 * 12^3 grid with 515 plane waves and 4 occupied orbitals fits in both precisions.
 * In LTMP2_FP32 the transformed-state GEMM runs on the CUDA cores, as it does in
 * ltmp2_energy with LTMP2_FLAG_SIMT_GEMM (so that flag is not accepted here).
 * The first call on a device looks up the array's device address and uploads the FFT
 * tables; make that first call before any stream capture.  The address is cached per
 * device, so calls after a cudaDeviceReset of that device are not supported.  Every
 * call reuses the same array (the previous call's contents stay until overwritten; the
 * accumulators are cleared by each call), so calls whose GPU work overlaps, from any
 * thread or stream, race and must be serialised by the caller.  The call returns after
 * the results are on the host.  Input validation is ltmp2_setup's (the same checks,
 * the orthonormality sample included).  Errors: as ltmp2_setup and ltmp2_energy, plus
 * UNSUPPORTED.                                                                       */
int ltmp2_energy_noalloc(const ltmp2_system *sys, int n_tau, const double *tau, const double *w,
                         double *e_direct, double *e_exchange, double *e_pair, void *stream);

/* Measured FMA rate of the current GPU's CUDA cores (the paper has no counterpart):
 * independent FMA chains in every thread of a full grid, timed with CUDA events, best of
 * five launches after one warm-up.  precision: LTMP2_FP64 or LTMP2_FP32; *tflops receives
 * 2 x FMAs / s / 1e12.  The roofline denominators of the CUDA-core kernels.  Allocates and
 * frees a small device buffer.  Errors: INVALID_ARG, OOM, CUDA.                      */
int ltmp2_alu_peak(int precision, double *tflops);

/* ---------------------------------------------------------------- k-point sampling
 * Sec. II C-D: the MP2 energy per unit cell with the Brillouin zone sampled on a
 * Gamma-centred n1 x n2 x n3 mesh, k = sum_i (kappa_i / n_i) b_i, kappa_i = 0 .. n_i - 1
 * (k-point index (kappa_1 n_2 + kappa_2) n_3 + kappa_3).  Bloch orbitals
 * phi_{nk}(r) = e^{ikr} sum_m c_{nk}(m) e^{iG_m r} / sqrt(N_k Omega_0) over one plane-wave
 * set shared by every k; the two-electron integrals (Eq. 2eIPLWV) conserve crystal
 * momentum, k1 + k2 = k3 + k4 + G, and carry the shifted Coulomb kernel
 * 4 pi / |G + k3 - k1|^2.  With the outer loop over the momentum transfers
 * Q' = G' + q' of the Born-von Karman supercell, every transformed state
 * w_{j k}^{(Q' tau)} = e^{(e_{jk}-mu) tau} P_v^{k - q'}(tau) e^{-iQ'r} |j k> (Eqs. StateDec,
 * DecompCoeff) uses the Green's function of its own k - q', and the exchange and direct
 * contractions (Eqs. xLTMP2, dLTMP2Compact) run over every occupied pair (i k1, j k2): the
 * N_k^3 loop over (k1, k2, q).  The energies equal the Gamma-point energies of the
 * supercell divided by N_k.  General complex orbitals (no time-reversal shortcut).
 *
 *   lattice, grid       unit cell and its FFT grid, as in ltmp2_system
 *   mesh [3]            n1, n2, n3 >= 1, N_k = n1 n2 n3 <= 64
 *   n_pw, miller        the plane-wave set of every k ([n_pw][3]; each |m_i| < n_i/2, every
 *                       (m1, m2) column one contiguous m3 range; no inversion symmetry needed)
 *   n_orb, n_occ        orbitals and doubly occupied orbitals per k (1 <= n_occ < n_orb <= n_pw)
 *   coeff               [N_k][n_orb][n_pw] complex128 (re, im), orthonormal rows per k
 *   eps                 [N_k][n_orb] Hartree, non-decreasing per k; the indirect gap
 *                       min_k e_{n_occ, k} - max_k e_{n_occ - 1, k} must be >= 1e-6 Ha
 *   ecut_aux            E_aux (Ha) of the momentum transfers |Q|^2 / 2; <= 0: 2/3 of the
 *                       largest |G_m|^2 / 2
 *   precision           LTMP2_FP64 or LTMP2_FP32 (CUDA-core products in both); flags 0.
 * The context works with ltmp2_energy, ltmp2_energy_partial (ranges of the primary Q'),
 * ltmp2_num_primary_gprime, ltmp2_set_slab_size, ltmp2_set_stream, profiling and
 * ltmp2_destroy; energies are per unit cell, and pair energies and ltmp2_sizes' n_occ
 * index the N_k n_occ composite occupied orbitals k n_occ + i.  The route, extrapolation,
 * pair-mask, batching, autotuning, descriptor and spin-unrestricted calls return
 * UNSUPPORTED.  Errors: as ltmp2_setup.                                            */
typedef struct {
  double lattice[9];
  int grid[3];
  int mesh[3];
  int n_pw;
  const int *miller;
  int n_orb;
  int n_occ;
  const double *coeff;
  const double *eps;
  double ecut_aux;
  int precision;
  int flags;
} ltmp2_kpoint_system;
int ltmp2_setup_kpoints(const ltmp2_kpoint_system *sys, ltmp2_ctx **out);

/* Free all device memory of ctx.  NULL is ignored.                              */
void ltmp2_destroy(ltmp2_ctx *ctx);

/* Static description of a status code (never NULL).                             */
const char *ltmp2_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LTMP2_H */
