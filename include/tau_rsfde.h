/*
 * tau_rsfde.h — C ABI of the GB300 (sm_103a) τ-preconditioned GMRES solver for the
 * quasi-compact Crank–Nicolson discretisation of the d-dimensional
 * variable-coefficient Riesz space-fractional diffusion equation
 * (She, Zhang, Gu, Serra-Capizzano, arXiv:2404.10221).
 *
 * Problem (§1, Eq. (RSFDE)):  e(x,t) u_t = sum_i kappa_i d^{alpha_i}_{x_i} u + f  on
 * Omega = prod (L_i, R_i), u = 0 on the boundary, u(x,0) = psi(x).
 * Each Crank–Nicolson step (§2, Eq. (tls)) solves
 *     A^{(m)} u^{(m+1)} = b^{(m)},   A^{(m)} = B_alpha E^{(m+1/2)} + S_alpha,
 *     b^{(m)} = (B_alpha E^{(m+1/2)} - S_alpha) u^{(m)} + dt F^{(m+1/2)},
 * with B_alpha = B_{alpha_d} ⊗ ... ⊗ B_{alpha_1} (Eq. (Ha)), S_alpha the Kronecker sum of
 * Eq. (Salpha) built from the fractional-weight Toeplitz matrices of Eq. (eq0), by GMRES
 * left-preconditioned with the τ preconditioner of Eq. (Pa) (one-sided form, Eq. (one-sided)).
 * The library runs the algebraically identical form  M^{-1} A u = M^{-1} b  with
 * M = B_alpha P_alpha = ebar B_alpha + tau(S_alpha); the τ matrices commute (§3), so
 * P^{-1} Ã = M^{-1} A and P^{-1} b̃ = M^{-1} b and the Krylov iterates are the same.
 * M^{-1} is applied as a d-dimensional DST-I, a pointwise divide by the eigenvalues
 * mu_k = ebar prod beta + sum_i eta_i q^{(i)} prod_{l!=i} beta (Eqs. (diag), (q), Lemma Heig,
 * Lemma le:eig), and a second DST-I.
 *
 * Conventions shared by every call:
 *   - Grid vectors hold the interior nodes x_J, J in prod {1..n_i}, in lexicographic order
 *     with x_1 fastest (§2); length n_tot = prod n_i; FP64.
 *   - Calls return tau_status: 0 = TAU_OK, negative = error.  tau_last_error() returns a
 *     thread-local message for the last failing call of the calling thread.
 *   - No call aborts, traps or spins without bound.  Device-side waits are bounded and end
 *     with TAU_ETIMEOUT.
 *   - The library owns every tau_problem and every device buffer it allocates.  Callers own
 *     the host arrays and device pointers they pass; the library never frees them and never
 *     keeps them past the call, except where a call says otherwise.
 *   - All device work of a problem is issued on the CUDA stream given to tau_create
 *     (NULL = legacy default stream).  Device pointers passed to a call must be usable on
 *     that stream; calls that take device pointers are asynchronous with respect to the host
 *     unless stated otherwise.
 */
#ifndef TAU_RSFDE_H
#define TAU_RSFDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tau_status;
#define TAU_OK 0
#define TAU_EINVAL (-1)       /* invalid argument (size, order alpha, NULL pointer, ...) */
#define TAU_ECUDA (-2)        /* a CUDA runtime call failed; the message names it */
#define TAU_ENOMEM (-3)       /* device allocation failed */
#define TAU_ETIMEOUT (-4)     /* a bounded device wait ran out */
#define TAU_ESTATE (-5)       /* call out of order (e.g. tau_solve before tau_setup) */
#define TAU_EUNSUPPORTED (-6) /* valid request the build does not support (message says why) */
#define TAU_ENOTCONV (-7)     /* GMRES hit max_iter without meeting tol (result still written) */

#define TAU_X0_ZERO 0         /* GMRES initial guess 0 for every step */
#define TAU_X0_PREV 1         /* GMRES initial guess u^{(m)} */

#define TAU_FP64 0            /* plain FP64 arithmetic everywhere */
#define TAU_MIXED 1           /* FP64 iterative refinement (residual b - A x, correction, stopping)
                                 around an inner flexible GMRES whose matvec, tau solve and Arnoldi
                                 vectors are FP32 */
#define TAU_DF64 2            /* the plain method with every solver vector, transform and Arnoldi
                                 product in double-float arithmetic (pairs of FP32 numbers, ~48
                                 significant bits) on the FP32 pipes; scalars (Givens, least squares)
                                 in FP64; u, e and f cross the API in FP64 */

#define TAU_OPGM 0            /* one-sided: GMRES on P^{-1} Ã u = P^{-1} b̃ (§3), run in the equivalent
                                 A-form M^{-1} A u = M^{-1} b with M = ebar B + tau(S) */
#define TAU_TPGM 1            /* two-sided: GMRES on P^{-1/2} Ã P^{-1/2} ũ = P^{-1/2} b̃ (Eq. (Pls)),
                                 u = P^{-1/2} ũ; both P^{-1/2} and P^{-1/2} B^{-1} are DST-diag-DST
                                 products, so an iteration costs one more τ solve than OPGM.
                                 TAU_FP64 only */
#define TAU_SPGM 2            /* the paper's comparison method (Table 1, Eq. (Pcir)): GMRES on
                                 P_c^{-1} Ã u = P_c^{-1} b̃ with the Strang circulant preconditioner
                                 P_c = ebar I + c(B)^{-1} c(S); P_c^{-1} by the separable orthonormal
                                 Hartley transform (dense, O(n_i) per element), B^{-1} by the DST.
                                 TAU_FP64 only; meant for comparisons at small n */

#define TAU_TC_AUTO 0
#define TAU_TC_OFF 1
#define TAU_TC_ON 2

#define TAU_ROUTE_AUTO 0      /* per-dimension choice: FFT when n_i+1 is a power of two (<= 4096),
                                 else chirp for 128 <= n_i < 4096 (when one line fits in shared
                                 memory), else dense; d = 1: FFT for n+1 = 2^p <= 512, dense for
                                 n < 128, long otherwise (one line in one CTA would leave the
                                 other SMs idle) */
#define TAU_ROUTE_FFT 1       /* shared-memory FFT route (requires n_i+1 = 2^p, 2 <= n_i+1 <= 4096) */
#define TAU_ROUTE_DENSE 2     /* explicit n_i x n_i mode products (any n_i <= 8192) */
#define TAU_ROUTE_CHIRP 3     /* any n_i < 4096: Toeplitz products through a power-of-two circulant
                                 embedding of length 2K (K the power of two >= n_i+1), DST-I of two
                                 lines at once as one Bluestein DFT of length n_i+1 through a
                                 convolution of power-of-two length >= 2 n_i (O(log n_i) per
                                 element).
                                 Every route needs one line (the n_i values plus the route's work
                                 row) in at most 200 KB of shared memory: TAU_DF64 (16-byte
                                 elements) fits the chirp route up to n_i = 2047 and the dense
                                 route up to n_i = 4266; otherwise tau_create returns
                                 TAU_EUNSUPPORTED for a forced route */
#define TAU_ROUTE_LONG 4      /* d = 1 only, any n (automatic from n = 128): the chirp route's
                                 convolutions (length F = 2 K_T, K_T the power of two >= n+1) as
                                 four-step FFTs over global memory, a few launches per operator
                                 instead of one CTA per line; not with TAU_SPGM */

#define TAU_TUNE_AUTO 0       /* measure new choices (and reuse recorded ones) for problems of >= 65536
                                 unknowns; TAU_AUTOTUNE=1/0 in the environment forces it on/off */
#define TAU_TUNE_ON 1         /* measure new choices, reuse recorded ones */
#define TAU_TUNE_OFF 2        /* the rules and heuristics only */
#define TAU_TUNE_RECORDED 3   /* recorded choices where present (this process, or the autotune file),
                                 the rules otherwise; nothing is measured (setup stays short) */

typedef struct tau_problem tau_problem;

/* Problem and solver parameters (§1 Eq. (RSFDE); §4 for the GMRES settings). */
typedef struct {
  int d;                /* spatial dimension, 1..3 */
  int64_t n[3];         /* interior points per dimension, n_i >= 1; h_i = (R_i - L_i)/(n_i + 1) */
  double L[3], R[3];    /* interval ends, L_i < R_i */
  double alpha[3];      /* fractional orders, 1 < alpha_i < 2 */
  double kappa[3];      /* kappa_i >= 0, sum kappa_i > 0 */
  double T;             /* final time > 0 */
  int64_t M;            /* number of Crank–Nicolson steps, dt = T / M */
  double tol;           /* GMRES stop: ||r_k|| <= tol ||r_0|| on the preconditioned residual */
  int max_iter;         /* GMRES iteration cap per step, 1..1000 (no restart) */
  int x0_mode;          /* TAU_X0_ZERO or TAU_X0_PREV */
  int precision;        /* TAU_FP64, TAU_MIXED or TAU_DF64 */
  int route[3];         /* TAU_ROUTE_* per dimension */
  double e_min, e_max;  /* bounds of e over the grid and all t_{m+1/2} for ebar (Eqs. (bard),
                           (dhat)); pass NaN for both to let tau_setup scan them */
  /* TAU_MIXED only (0 selects the default): */
  double refine_tol;    /* stop refining at ||b - A x||_2 <= refine_tol ||b - A x_0||_2 (FP64); 1e-10 */
  int inner_max_iter;   /* inner FGMRES iterations per refinement sweep, 1..1000; 30 */
  int max_sweeps;       /* refinement sweeps per step; 10 */
  double inner_tol;     /* inner FGMRES relative residual target of the first sweep; 1e-5.  A later
                           sweep targets the reduction still needed, 0.3 refine_tol rho_0 / rho,
                           kept within [min(1e-6, inner_tol), inner_tol] */
  int method;           /* TAU_OPGM (0, default), TAU_TPGM or TAU_SPGM */
  int tc;               /* TAU_MIXED only: the DST-I passes of the FP32 τ solve on dimensions with
                           n_i <= 256 as tensor-core (tcgen05, TF32) mode products (relative error
                           ~1e-3: the flexible inner GMRES takes the result as its preconditioner).
                           When every n_i <= 256 the FP32 matvec can also run its Toeplitz
                           products on the tensor cores from split TF32 operands (FP32-level
                           accuracy).  TAU_TC_AUTO (0, default): tau_setup times both operators
                           both ways and keeps the faster of each (cached per grid shape);
                           TAU_TC_OFF (1): line passes; TAU_TC_ON (2): tensor cores wherever
                           n_i <= 256 */
  int autotune;         /* TAU_TUNE_AUTO (0, default), TAU_TUNE_ON, TAU_TUNE_OFF or TAU_TUNE_RECORDED:
                           whether tau_setup times the route of each dimension (d >= 2), the lines
                           per CTA of the line passes and (TAU_TC_AUTO) the tensor-core choice */
} tau_problem_desc;

/* A field g(x,t) = sum_{r<rank} c_r(t) prod_i phi_{r,i}(x_i) given as tables (host memory,
 * copied by tau_set_fields; the caller keeps ownership):
 *   time_coef[k*rank + r] = c_r(t_k)   for the n_times time levels the field needs
 *                                       (e and f: t_{m+1/2}, m = 0..M-1, so n_times = M;
 *                                        psi: n_times = 1),
 *   space[i][r*(n_i+2) + j] = phi_{r,i}(x_{i,j}),  j = 0..n_i+1 (boundary nodes included). */
typedef struct {
  int rank;
  int64_t n_times;
  const double* time_coef;
  const double* space[3];
} tau_field;

/* Fields as device arrays, for e and f of any form (not only separable expansions): the
 * problem statement (§1, Eq. (RSFDE)) allows any positive e(x,t) and any source f(x,t), and each
 * Crank–Nicolson step (Eq. (tls)) needs them only at t_{m+1/2} on the grid.
 *   e:   e(x_J, t_{m+1/2}) at the interior nodes (x_1 fastest), step m at e + m * e_step;
 *        e_step = n_tot (M slabs of n_tot doubles) or 0 (e does not depend on t: one slab).
 *   f:   f(x, t_{m+1/2}) on the padded grid prod_i (n_i + 2) (boundary nodes included, x_1
 *        fastest), step m at f + m * f_step; f_step = prod(n_i + 2) or 0.  NULL: f = 0.
 *        The library forms F = interior restriction of (⊗_l 𝓗_{alpha_l}) f (Eq. (2.2), Appendix A).
 *   psi: u^{(0)} = psi(x_J) at the interior nodes (n_tot doubles); NULL: psi = 0.
 * All three are device pointers of the problem's device, owned by the caller, who keeps them
 * alive and their contents as given until tau_destroy: the library keeps the pointers (no copy)
 * and reads e and f of step m, on the problem's stream, when that step runs (so a caller may
 * write a step's slab on that stream any time before the step is enqueued); tau_setup reads all
 * of e (the ebar scan, unless desc bounds are given) and psi. */
typedef struct {
  const double* e;
  int64_t e_step;
  const double* f;
  int64_t f_step;
  const double* psi;
} tau_field_device;

/* Per-problem statistics (host copy). */
typedef struct {
  int64_t steps_done;       /* m: number of completed steps */
  int64_t total_iters;      /* sum of GMRES iterations over completed steps */
  int last_iters;           /* iterations of the last step */
  int max_iters_step;       /* largest per-step count so far */
  double last_relres;       /* |g_k| / ||r_0|| of the last step (preconditioned, Givens estimate) */
  double ebar, e_hat, e_check; /* Eqs. (bard), (dhat) */
  int route[3];             /* route chosen per dimension (TAU_ROUTE_FFT, _DENSE, _CHIRP or _LONG) */
  int graph;                /* 1 if steps run as CUDA-graph launches with device-side loop control */
  int64_t device_bytes;     /* device memory held by the problem */
  int64_t kernels_prologue; /* kernels of one step: prologue + iters * per_iter + epilogue */
  int64_t kernels_per_iter;
  int64_t kernels_epilogue;
  int64_t kernels_total;    /* kernels launched by the completed steps */
  int64_t total_sweeps;     /* TAU_MIXED: refinement sweeps over the completed steps (iters count the
                               inner FGMRES iterations) */
  int lines_per_cta[3];     /* grid lines per CTA of the line-pass kernel per dimension (FP64), chosen
                               by the setup's autotuner (problems with >= 65536 unknowns, or
                               TAU_AUTOTUNE=1; TAU_AUTOTUNE=0 keeps the shared-memory heuristic) */
  int lines_per_cta_f32[3]; /* the same for the FP32 passes of a TAU_MIXED problem */
  int tc_dims;              /* bit i set: the FP32 τ solve runs its DST-I along dimension i on the
                               tensor cores (TAU_TC_ON, or TAU_TC_AUTO where it timed faster); bit 8
                               set: the FP32 matvec runs as split-TF32 tensor-core passes */
  int route_source[3];      /* how route[i] was chosen: 0 by the rule of TAU_ROUTE_AUTO (or forced),
                               1 measured by this tau_setup (d >= 2, TAU_ROUTE_AUTO, tuning on: the
                               FFT or chirp route against the dense route, FP64 passes timed), 2 from
                               an earlier measurement on this device and shape (in memory, or the
                               autotune file: $TAU_TUNE_CACHE, default
                               $XDG_CACHE_HOME/tau_rsfde/autotune.txt or ~/.cache/tau_rsfde/...;
                               "off" disables the file) */
  double route_ms[3];       /* measured device time of the chosen route's representative passes (one
                               matvec pass and one DST pass along dimension i, ms); 0 if not measured */
  double route_alt_ms[3];   /* the same for the fastest rejected candidate; 0 if none */
  int resid_precision;      /* TAU_MIXED: precision of the outer residual b - A x (TAU_FP64, or
                               TAU_DF64 where its rounding floor 2^-48 * 8 * max_i eta_i 2 s_0(alpha_i)
                               / ebar is at most refine_tol / 2); otherwise desc.precision */
} tau_stats;

/* Create a problem: validates desc, allocates device state (Krylov basis of
 * (max_iter+1) * n_tot doubles plus O(n_tot) work vectors).  `stream` is a cudaStream_t or NULL.
 * Errors: TAU_EINVAL (bad desc), TAU_EUNSUPPORTED (route/size not supported), TAU_ENOMEM, TAU_ECUDA. */
tau_status tau_create(const tau_problem_desc* desc, void* stream, tau_problem** out);

/* Copy the field tables of e (Eq. (tls): E^{(m+1/2)} = diag e(G, t_{m+1/2})), f (source, evaluated
 * at t_{m+1/2} on the padded grid) and psi (u^{(0)} = psi(G)) to the device.
 * Requires e->n_times == f->n_times == M and psi->n_times == 1.  Synchronous. */
tau_status tau_set_fields(tau_problem* p, const tau_field* e, const tau_field* f, const tau_field* psi);

/* The device-array form of tau_set_fields (tau_field_device above); either call sets the fields
 * once.  Errors: TAU_EINVAL (NULL e, a step that is neither 0 nor the slab size), TAU_ESTATE
 * (fields already set).  Enqueues nothing. */
tau_status tau_set_fields_device(tau_problem* p, const tau_field_device* fields);

/* One-time setup (Remark after Theorem GMRES: the preconditioner does not depend on the step):
 * FCD weights (§2), Toeplitz spectra, tau eigenvalues q (Eq. (q)), beta (Lemma Heig), 1/mu,
 * ebar (scan of e over G x {t_{m+1/2}} unless desc bounds are given), u^{(0)} = psi(G), m = 0.
 * Synchronous. */
tau_status tau_setup(tau_problem* p);

/* Advance `count` Crank–Nicolson steps (count <= M - m).  Asynchronous: the host only enqueues
 * work; per-step statistics are read by tau_get_stats (which synchronises).  Returns TAU_ENOTCONV
 * from tau_get_stats/tau_sync if any step hit max_iter. */
tau_status tau_step(tau_problem* p, int64_t count);

/* All remaining steps, then synchronise; returns TAU_ENOTCONV if some step hit max_iter. */
tau_status tau_solve(tau_problem* p);

/* Wait for enqueued work; return TAU_ENOTCONV if some completed step hit max_iter. */
tau_status tau_sync(tau_problem* p);

/* Copy u^{(m)} (n_tot doubles) to `out` (host memory if is_device == 0, else a device pointer);
 * *m_out (optional) receives m.  Host copies are synchronous; device copies are enqueued. */
tau_status tau_get_solution(tau_problem* p, double* out, int is_device, int64_t* m_out);

/* Replace u^{(m)} and m (resume from a checkpoint; 0 <= m <= M).  Same memory rules. */
tau_status tau_set_solution(tau_problem* p, const double* u, int is_device, int64_t m);

/* Statistics (synchronises the stream). */
tau_status tau_get_stats(tau_problem* p, tau_stats* out);

/* GMRES iterations of steps 0..min(cap, m)-1 into iters[] (host; synchronises). */
tau_status tau_get_iters(tau_problem* p, int* iters, int64_t cap);

/* Free everything the problem owns (synchronises its stream first).  NULL is accepted. */
tau_status tau_destroy(tau_problem* p);

/* Thread-local message of the last failed call ("" if none). */
const char* tau_last_error(void);

/* ---- operator-level entry points (device pointers, n_tot doubles each, enqueued on the
 *      problem's stream; require tau_setup).  They expose each step of the solver on its own. */

/* y = A^{(m)} x = B_alpha (e(.,t_{m+1/2}) ∘ x) + S_alpha x, Eq. (tls), 0 <= m < M. */
tau_status tau_apply_A(tau_problem* p, int64_t m, const double* x, double* y);

/* z = M^{-1} r with M = ebar B_alpha + tau(S_alpha) (Eqs. (Pa), (tauSalpha), (diag)). */
tau_status tau_apply_Minv(tau_problem* p, const double* r, double* z);

/* z = M^{-1} A^{(m)} x: one preconditioned matvec of the GMRES loop (fused kernels). */
tau_status tau_apply_MinvA(tau_problem* p, int64_t m, const double* x, double* z);

/* b = (B_alpha E^{(m+1/2)} - S_alpha) u + dt F^{(m+1/2)}, Eq. (tls) with F from Eq. (2.2)/Appendix A. */
tau_status tau_rhs(tau_problem* p, int64_t m, const double* u, double* b);

/* y = S_d x: orthonormal d-dimensional DST-I, S = sqrt(2/(n+1)) [sin(pi j k/(n+1))] (§3). */
tau_status tau_dst(tau_problem* p, const double* x, double* y);

/* y = (I ⊗ .. ⊗ S_{alpha_dim} ⊗ .. ⊗ I) x: the fractional-weight Toeplitz matrix of Eq. (eq0)
 * along dimension dim (0-based; unscaled, no eta). */
tau_status tau_toeplitz_mode(tau_problem* p, int dim, const double* x, double* y);

/* FP32 operators of the inner solve of a TAU_MIXED problem (device float vectors of n_tot):
 * y = A^{(m)} x and z = M^{-1} r with every step in FP32 (tables rounded from their FP64 values). */
tau_status tau_apply_A_f32(tau_problem* p, int64_t m, const float* x, float* y);
tau_status tau_apply_Minv_f32(tau_problem* p, const float* r, float* z);

/* ebar, e_hat, e_check (Eqs. (bard), (dhat)); requires tau_setup. */
tau_status tau_get_ebar(tau_problem* p, double* ebar, double* e_hat, double* e_check);

/* Measured FP64 FMA throughput of the current device in FLOP/s (diagnostic used for the
 * roofline of the FP64-bound kernels; runs a bounded kernel for a few milliseconds). */
tau_status tau_measure_fp64_peak(void* stream, double* flops_per_s);

/* Host only (no CUDA call; usable without a GPU): the faster precision form that still resolves
 * this problem's operator.  TAU_MIXED when an FP32 matvec resolves it,
 *     2^-23 max_i eta_i 2 s_0(alpha_i) / e_min <= 0.05,
 * eta_i = kappa_i dt / (2 h_i^alpha_i) (Eq. (tls)), s_0(alpha) = Gamma(alpha+1)/Gamma(alpha/2+1)^2 the
 * diagonal fractional weight and 2 s_0 a bound of the weights' 1-norm (Eq. (As1)); otherwise
 * TAU_DF64: the FP32 rounding error of eta_i T x (about eps_32 eta_i ||s||_1 |x|) would swamp the
 * O(e |x|) value that the cancelling Toeplitz sum leaves, and the inner solve could not converge.
 * Reads d, n, L, R, alpha, kappa, T, M and e_min (a positive number, not NaN; a lower bound of e
 * over the grid and all t_{m+1/2}).  Errors: TAU_EINVAL. */
tau_status tau_choose_precision(const tau_problem_desc* desc, int* precision);

/* Self-test of the bounded waits of the tensor-core kernels: one CTA waits on an mbarrier that
 * nothing arrives at, with a limit of 1e5 polls, and *gave_up (host int) is set to 1 when the wait
 * ran out and the kernel returned as it must (0 would mean a wait that could not time out).  Runs
 * on `stream` (NULL = default) and synchronizes it.  Errors: TAU_EINVAL (NULL gave_up), TAU_ECUDA. */
tau_status tau_selftest_bounded_wait(void* stream, int* gave_up);

/* Test hook of the error path of the bounded device waits: sets, on the problem's stream, the
 * device flag that a tensor-core kernel sets when one of its mbarrier waits runs out.  The next
 * tau_sync / tau_solve / tau_batch_sync of the problem returns TAU_ETIMEOUT and clears the flag
 * (an expired wait is reported once); the syncs after that return to normal.  No device wait is
 * made to run out.  Errors: TAU_EINVAL (NULL), TAU_ECUDA. */
tau_status tau_inject_wait_timeout(tau_problem* p);

/* ---- batching: many independent problems advanced by one graph launch per step.
 *
 * tau_batch_create groups `count` problems that have completed tau_setup, share the CUDA device,
 * and stand at the same step m with the same M, into one CUDA graph: one branch per problem, each
 * holding that problem's whole step (right-hand side, its own device-controlled GMRES or
 * refinement loop, update).  Branches have no dependencies on one another, so the GPU overlaps
 * the problems' kernels; a problem's arithmetic is the same as when it is stepped alone.
 * The batch does not own the problems (destroy the batch first).  Problems may mix precisions,
 * sizes and dimensions.  While a batch exists, do not step its problems individually.
 * Errors: TAU_EINVAL (NULL, count < 1, problems at different m or M), TAU_ESTATE (not set up),
 * TAU_EUNSUPPORTED (graph construction failed), TAU_ENOMEM. */
typedef struct tau_batch tau_batch;
tau_status tau_batch_create(tau_problem* const* problems, int count, void* stream, tau_batch** out);
/* Grouped execution.  Mixed-precision problems on the line-pass routes (TAU_MIXED with the tensor
 * cores off, no long-line dimension) that share d, the residual precision chosen by tau_setup and
 * x0_mode form a group: the group's branch of the graph is the mixed step with every kernel one
 * launch over all of its problems (each CTA works for one problem, from a table of their argument
 * blocks), its loops running while any problem still iterates and problems that finished skipping
 * their work.  The number of kernels per step then no longer grows with the number of problems.  A
 * problem's arithmetic is unchanged (same kernels, tiles and reduction order as alone).  Other
 * problems get a branch each.  TAU_BATCH_GROUPS=0 in the environment turns grouping off. */
typedef struct {
  int groups;                         /* groups formed */
  int grouped_problems;               /* problems in them */
  int branches;                       /* independent branches of the graph (groups + single problems) */
  int64_t launches_prologue_epilogue; /* grouped launches per step outside the loops (sum over groups) */
  int64_t launches_per_sweep;         /* grouped launches per refinement sweep around the inner loop */
  int64_t launches_per_inner_iter;    /* grouped launches per inner FGMRES iteration */
} tau_batch_info;
tau_status tau_batch_get_info(tau_batch* b, tau_batch_info* info);
/* Advance every problem of the batch by `count` steps (asynchronous; one graph launch per step). */
tau_status tau_batch_step(tau_batch* b, int64_t count);
/* Wait for the batch's work; TAU_ENOTCONV if some problem's step hit its iteration cap. */
tau_status tau_batch_sync(tau_batch* b);
tau_status tau_batch_destroy(tau_batch* b);

/* ---- serving: a continuous-batching request loop for whole time-marching solves.
 *
 * tau_server_create starts a worker thread on the current CUDA device.  tau_server_submit copies a
 * request (problem description and field tables, as for tau_create / tau_set_fields) into a FIFO
 * queue.  The worker admits queued requests while the estimated device memory of the admitted
 * ones stays within `device_bytes_budget` and fewer than `max_active` are admitted; each admitted
 * request gets its own stream and a tau_problem whose Krylov basis and solution stay on the
 * device until its last step.  Admitted TAU_MIXED requests run their inner solve on the line
 * passes (the server sets tc = TAU_TC_OFF) and, unless the request asks for TAU_TUNE_ON or _OFF,
 * take the recorded autotuning choices only (TAU_TUNE_RECORDED: admission measures nothing).
 * Requests of at most 2^20 unknowns of the same kind (d, the residual precision tau_setup chose,
 * x0_mode; no long-line dimension) batch their iterations together: one step graph
 * whose kernels are each one launch over all of them (the grouped execution of tau_batch), rebuilt
 * whenever the set changes, every launch advancing each member by one step.  Larger requests fill
 * the GPU by themselves and step on their own streams, as do the others.  TAU_BATCH_GROUPS=0 in the
 * environment at tau_server_create turns the shared launches off.  The worker issues `steps_per_launch` steps at a time (a group: at most the
 * steps its nearest-to-finish member has left), so requests that arrive while others run are
 * admitted as memory frees up and join the next group or overlap on the GPU.  A request's result is
 * the same alone and in the mix (its arithmetic does not depend on the group).  A finished request's solution u^(M) is
 * copied to host memory and its device memory returns to the budget.  A request whose estimate
 * exceeds the whole budget fails at once with TAU_ENOMEM.  All host waits are bounded.
 * Times are seconds since tau_server_create. */
#define TAU_REQ_QUEUED 0
#define TAU_REQ_RUNNING 1
#define TAU_REQ_DONE 2
#define TAU_REQ_FAILED 3
typedef struct tau_server tau_server;
typedef struct {
  int64_t id;
  int state;                  /* TAU_REQ_* */
  tau_status status;          /* TAU_OK, TAU_ENOTCONV (done, some step hit its cap) or the failure */
  double t_submit, t_admit, t_finish;
  int64_t unknowns, steps, gmres_iters;
  int64_t device_bytes;       /* device memory the request held while admitted */
} tau_request_info;
typedef struct {
  int64_t completed, failed, queued, active;
  int64_t device_bytes_in_use;    /* estimated bytes of the admitted requests */
  double latency_p50_s, latency_p99_s, latency_mean_s;   /* submit -> u^(M) on the host, completed */
  double unknowns_steps;          /* sum of n_tot * M over completed requests */
  double span_s;                  /* first submit -> last completion */
  double throughput;              /* unknowns_steps / span_s */
  int64_t group_launches;         /* step-graph launches shared by a group of requests */
  int64_t group_rebuilds;         /* group graphs built (the set of requests changed) */
  int64_t group_request_steps;    /* request steps taken inside shared launches */
} tau_server_stats;
tau_status tau_server_create(int64_t device_bytes_budget, int max_active, int steps_per_launch, tau_server** out);
tau_status tau_server_submit(tau_server* s, const tau_problem_desc* desc, const tau_field* e, const tau_field* f,
                             const tau_field* psi, int64_t* id_out);
tau_status tau_server_poll(tau_server* s, int64_t id, tau_request_info* info);
/* Wait until the request is done or failed, at most timeout_s seconds (TAU_ETIMEOUT otherwise). */
tau_status tau_server_wait(tau_server* s, int64_t id, double timeout_s, tau_request_info* info);
/* Copy a finished request's solution (n doubles, host memory). */
tau_status tau_server_result(tau_server* s, int64_t id, double* u_host, int64_t n);
/* Forget a finished or failed request (frees its host copy of the solution). */
tau_status tau_server_release(tau_server* s, int64_t id);
tau_status tau_server_summary(tau_server* s, tau_server_stats* out);
/* Cancel queued requests, let admitted ones finish, stop the worker, free everything. */
tau_status tau_server_destroy(tau_server* s);

/* ---- allocation-free entry point (the paper has no counterpart).
 *
 * y = A x = B_alpha (e ∘ x) + S_alpha x for the grid and coefficients of `desc` (d, n, L, R, alpha,
 * kappa, T, M give h_i, dt and eta_i; route[i] must be TAU_ROUTE_AUTO; the other fields are
 * ignored), without a tau_problem and without allocating device memory.  The entry point picks
 * its own route per dimension: the FFT route when n_i + 1 is a power of two, dense O(n_i) sums
 * otherwise (a forced route returns TAU_EINVAL).  For callers that cannot call cudaMalloc: code living inside
 * a host application whose memory pool owns the device, plugins that must not change the
 * device's memory footprint, and latency-critical loops where an allocation (which may
 * synchronise the device) is not acceptable.
 *   e, x: device pointers to n_tot doubles (e = e(x_J, t) at the interior nodes); y: device
 *   output of n_tot doubles (must not alias x or e).  Enqueued on `stream` (cudaStream_t or NULL).
 * Scratch (FCD weights, circulant spectra, twiddles, the two Kronecker channels) lives in one
 * static device array of about 5.2 MB that every GPU loading the library holds until process
 * exit; it is rebuilt on each call.  Limits: n_i <= 4095 per dimension and n_tot <= 262,144;
 * larger problems return TAU_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  Every call shares the array: calls that overlap on the GPU race. */
tau_status tau_apply_A_noalloc(const tau_problem_desc* desc, const double* e, const double* x, double* y,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TAU_RSFDE_H */
