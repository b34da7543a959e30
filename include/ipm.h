/*
 * ipm.h -- C ABI of the GB300 reduced-space interior-point hot path.
 *
 * The library solves the two-stage block nonlinear program of §2 (eqs. (2)-(3))
 * for stochastic AC optimal power flow (§4.1.1): N scenarios share the
 * controls u (generator voltages and non-slack active powers) and own their
 * states x_i (angles, load-bus voltages).  At every interior-point iteration
 * it evaluates each scenario's Jacobians and Lagrangian Hessian, condenses the
 * inequalities into a barrier diagonal (Prop. 2.1/2.2), eliminates the states
 * through a batched sparse LU of G_x and the multi-RHS solves
 * Z = -G_x^{-1} G_u (Prop. 2.3), accumulates the dense reduced Hessian
 * Z^T K Z over scenarios (the Schur complement of Prop. 2.4) and factors it
 * by dense Cholesky.
 *
 * Precision (ipm_options.precision): IPM_PREC_FP64 runs every step in FP64.
 * IPM_PREC_MIXED runs the multi-RHS solves in FP32 and the Z^T Y products as
 * three-term BF16 split products on the tensor cores (FP32 accumulation per
 * 64-wide block, FP64 across blocks); the LU of G_x, the Cholesky and the
 * recovery stay FP64, and the reduced step is refined to FP64 accuracy by
 * conjugate gradients on the exact FP64 reduced operator, preconditioned by
 * the mixed-precision factor.  When that factor is not positive definite or
 * the refinement meets non-positive curvature (K_hat ill-conditioned near
 * the solution), the iteration is condensed again in FP64 and the inertia
 * decision is taken on the exact K_hat.  IPM_PREC_FP64_TC is the FP64 path
 * with the Z^T Y contraction emulated on the BF16 tensor cores: per 512
 * contraction rows and column, FP64 operands (rows balanced by powers of
 * two) are scaled by a power of two and split into eight 7-bit integer
 * slices; the 36 slice products that matter are accumulated exactly (integer
 * sums of at most 2^24 in FP32), combined into one exact 64-bit integer per
 * group and accumulated in FP64; each row's product is off by about 2^-52 of
 * the product of the group's largest entries of the two columns; a
 * non-finite result falls back to the FP64 units.
 *
 * Conventions (all entry points):
 *  - Every call returns an ipm_status; nothing aborts or traps.  On error,
 *    ipm_last_error() describes the failure.
 *  - "stream" is a cudaStream_t passed as void* (0 = legacy default stream).
 *    Work is enqueued on it; calls that must read a device scalar (a
 *    positive-definiteness flag, a KKT error, a line-search merit value)
 *    synchronise that stream before returning.
 *  - Host arrays passed to ipm_create are copied; the caller keeps ownership.
 *  - Device pointers passed in are caller-owned, must hold the stated number
 *    of doubles, and are accessed through "stream".
 *  - A context is not thread-safe; use one stream per context at a time.
 */
#ifndef IPM_H
#define IPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipm_ctx ipm_ctx;

typedef enum {
  IPM_OK = 0,
  IPM_ERR_ARG = 1,          /* invalid argument (sizes, NaN/negative loads, bad indices) */
  IPM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  IPM_ERR_OOM = 3,          /* device allocation failed */
  IPM_ERR_SINGULAR_GX = 4,  /* a static LU pivot of G_x is (numerically) zero */
  IPM_ERR_NOT_PD = 5,       /* inertia correction exceeded its largest delta_w */
  IPM_ERR_LINESEARCH = 6,   /* backtracking fell below the minimum step */
  IPM_ERR_MAXITER = 7,      /* iteration limit reached */
  IPM_ERR_TIMEOUT = 8,      /* a bounded device wait gave up */
  IPM_ERR_STATE = 9         /* call out of order (e.g. solve before factor) */
} ipm_status;

/* One network (per-unit).  Lines use the pi model without taps or shunts
 * (Y_ff = Y_tt = y + j b/2, Y_ft = Y_tf = -y, y = 1/(r + j x)).
 * gen_bus[0] must be 0: generator 0 is the slack (its Pg is the dependent
 * function P_0 + Pd_0).  Pg bounds are [0, pmax]; Qg bounds [-qmax, qmax];
 * V bounds [vmin, vmax] at every bus.  rate: NULL (no line-flow limits,
 * m = n_gen + 1) or [n_line] positive finite apparent-power ratings: the
 * operational constraints of §4.1.1 then include |S_f|^2 <= rate^2 and
 * |S_t|^2 <= rate^2 at both ends of every line, 2 n_line more rows of h
 * (m = n_gen + 1 + 2 n_line, the count of the paper's instance table): row
 * n_gen + 1 + l is the from end of line l, row n_gen + 1 + n_line + l its to
 * end, each h = P^2 + Q^2 of the power entering the line there. */
typedef struct {
  int n_bus, n_line, n_gen;
  const int *from, *to;        /* [n_line] */
  const int *gen_bus;          /* [n_gen] distinct buses, gen_bus[0] == 0 */
  const double *r, *x, *b;     /* [n_line] */
  const double *pmax, *qmax;   /* [n_gen] */
  const double *c2, *c1;       /* [n_gen] cost c2 Pg^2 + c1 Pg */
  const double *vmin, *vmax;   /* [n_bus] */
  const double *rate;          /* [n_line] or NULL */
} ipm_network;

enum { IPM_PREC_FP64 = 0, IPM_PREC_MIXED = 1, IPM_PREC_FP64_TC = 2 };

enum { IPM_BARRIER_MONOTONE = 0, IPM_BARRIER_ADAPTIVE = 1 };

enum { IPM_REDUCTION_DENSE = 0, IPM_REDUCTION_ADJOINT = 1, IPM_REDUCTION_AUTO = 2 };

typedef struct {
  double tol;            /* KKT residual E_0 target (1e-8) */
  int max_iter;          /* 200 */
  int precision;         /* IPM_PREC_FP64, IPM_PREC_MIXED or IPM_PREC_FP64_TC */
  int max_refine;        /* mixed path: conjugate-gradient iterations on the exact reduced
                            operator, preconditioned by the BF16x3 factor (default 60); an
                            iteration whose CG does not reach 1e-10 is condensed again in FP64 */
  int solve_threads;     /* threads per CTA of the multi-RHS solves: 128 or 256 (0 = 256,
                            or the autotuner's choice) */
  int barrier_rule;      /* IPM_BARRIER_ADAPTIVE (default): mu = max(tol/10, sigma * mean
                            complementarity) at every iteration; IPM_BARRIER_MONOTONE:
                            mu <- max(tol/10, min(0.2 mu, mu^1.5)) when E_mu <= 10 mu */
  int graphs;            /* 1: replay the condensation as CUDA graphs captured on its first
                            call (needs a non-NULL stream; ignored while profiling) */
  int autotune;          /* 1: at the first condensation, time the candidate launch shapes
                            (solve threads, scenario groups of the reduced-Hessian
                            contraction) and keep the fastest; results are cached per
                            (n_x, n_u, N, precision) for the process */
  int poison;            /* 1: fill every device buffer with NaN when it is allocated (a check
                            that nothing is read before it is written; results must not change) */
  int lu_pair;           /* 1 (default): factor G_x on a cluster of two CTAs per scenario when its
                            dense trailing block fits their shared memory; 0: one CTA */
  int aug_refine;        /* steps of FP64 iterative refinement on the residual of the augmented
                            system eq. (6) after the reduced solve (default 10, every path): the
                            residual of the step is formed from J, K and the right-hand sides,
                            the correction is solved through the same condensation and
                            reduction, and refinement stops at a relative residual (max norm,
                            against the right-hand side) <= 1e-12 or when a step no longer
                            halves it; 0 = no residual check */
  int reduction;         /* how K_hat = sum_i Z_i^T Y_i is formed on the FP64 paths:
                            IPM_REDUCTION_DENSE (default) the contraction of Z and Y;
                            IPM_REDUCTION_ADJOINT the paper's local reduction by adjoint solves
                            (§3.2: K_hat V = L_u - G_u^T G_x^{-T} L_x with V = I, one more
                            multi-RHS solve with G_x^T instead of the contraction);
                            IPM_REDUCTION_AUTO: the autotuner (autotune = 1) times both at the
                            first condensation and keeps the faster (dense without it) */
  int big_block;         /* 0 (default): the dense trailing block of the LU of G_x is factored
                            and solved in shared memory when it has at most 400 states and by
                            the batched global-memory kernels above that (the block then also
                            takes the sparse pivots just before it that reach a sixth of it);
                            1: the global-memory kernels whatever its size */
  double sigma;          /* centring factor of the adaptive rule (0.1) */
  int tc_solve;          /* mixed path with a dense trailing block too large for shared memory
                            (big_block): 1 (default) the block updates of the multi-RHS solve as
                            BF16x3 products on the tensor cores (FP32 accumulation), 0 FP32 on
                            the SIMT units */
} ipm_options;

/* Sizes of a context.  state_len = 4 N n_x + 4 N m + 3 n_u + 3; the state
 * vector layout is, in doubles:
 *   x[N][n_x], u[n_u], s[N][m], y[N][n_x], z[N][m],
 *   zl_x[N][n_x], zu_x[N][n_x], zl_u[n_u], zu_u[n_u], zl_s[N][m], zu_s[N][m],
 *   mu, rho, delta_last.
 * step_len = 2 N n_x + 2 N m + n_u (p_x, p_u, p_s, p_y, p_z in that order). */
typedef struct {
  int n_bus, n_line, n_gen, n_scen;
  int n_x, n_u, m;
  long long state_len, step_len;
  long long nnz_lu;      /* stored entries of the static-pivot LU of G_x */
  int lu_levels;         /* level-schedule depth of the LU / triangular solves */
  int nnz_kx, nnz_ku;    /* entries of the rows of [K_xx K_xu] and [K_ux] per scenario (the
                            products Y = K_x [Z; I], Y_u = K_u [Z; I]) */
  int nd;                /* states in the dense trailing block of the LU of G_x */
  int big_block;         /* 1 if that block is handled by the global-memory kernels */
  long long lu_sparse_ops; /* multiply-adds of the sparse pivots per scenario (level lists and
                              products into the trailing block) */
} ipm_dims;

ipm_status ipm_default_options(ipm_options *opt);

/* Create a context for one network and N scenarios.
 * pd, qd: host [n_scen][n_bus] loads (scenario-major).  Builds the symbolic
 * structures (orderings, LU pattern, level schedules) on the host, uploads
 * everything, allocates all device workspaces and sets the cold-start state.
 * Errors: IPM_ERR_ARG on bad sizes/indices/non-finite or negative loads,
 * IPM_ERR_OOM, IPM_ERR_CUDA. */
ipm_status ipm_create(const ipm_network *net, int n_scen, const double *pd,
                      const double *qd, const ipm_options *opt, ipm_ctx **out);
ipm_status ipm_destroy(ipm_ctx *ctx);
ipm_status ipm_get_dims(const ipm_ctx *ctx, ipm_dims *out);
const char *ipm_last_error(const ipm_ctx *ctx);

/* Cold start (§2.2 reading): theta = 0, V = 1, Pg = Pmax/2, pushed inside the
 * boxes; s = -h pushed; y = z = 0; bound duals 1; mu = 0.1; rho = 1. */
ipm_status ipm_init_state(ipm_ctx *ctx, void *stream);

/* Copy a full state in/out (layout above).  on_device != 0: the pointer is a
 * device pointer, else a host pointer (pinned or pageable).
 * The state is the primal-dual point of the interior-point method of §2.2:
 * the primal variables (x, u, s) of the slacked problem eq. (3), the
 * multipliers y of g = 0 and z of h + s = 0 in the Lagrangian eq. (4), the
 * bound multipliers (the paper's kappa, lambda, nu of eq. (4); here one per
 * finite side of each two-sided box, the paper having one-sided bounds only),
 * the barrier parameter mu of the smoothed complementarity X kappa = mu e of
 * eq. (5), and the line-search penalty rho and last inertia shift (state of
 * the rule set the paper leaves to MadNLP, §2.2).  Errors: IPM_ERR_ARG on a
 * NULL pointer, IPM_ERR_CUDA on a failed copy. */
ipm_status ipm_set_state(ipm_ctx *ctx, const double *state, int on_device, void *stream);
ipm_status ipm_get_state(ipm_ctx *ctx, double *state, int on_device, void *stream);

/* Evaluate f, g, h, the Jacobians G, H and the Lagrangian Hessian W of every
 * scenario at the current state (eq. (4) without bound terms). */
ipm_status ipm_eval_derivatives(ipm_ctx *ctx, void *stream);

/* Condense and reduce at the current state and barrier parameter mu:
 * Sigma's, K = W + Sigma_p + H^T Sigma_s H (Prop. 2.1/2.2), the static-pivot
 * LU of every G_x^i, Z_i = -(G_x^i)^{-1} G_u^i, Y_i = K_i [Z_i; I], and
 * K_hat = sum_i Z_i^T K_i Z_i + Sigma_u (Prop. 2.3), plus the reduced
 * right-hand side of eq. (11).  Requires ipm_eval_derivatives first.
 * Errors: IPM_ERR_SINGULAR_GX when a pivot |u_ii| < 1e-14 max|row|. */
ipm_status ipm_condense_scenarios(ipm_ctx *ctx, void *stream);

/* Factor K_hat + delta_w (sum_i Z_i^T Z_i + I) -- i.e. the reduced matrix of
 * K + delta_w I -- by dense FP64 Cholesky.  *is_pd = 1 on success, 0 when a
 * pivot is not positive.
 * K_hat = Z^T K Z of Prop. 2.3 (eq. (11)) is the Schur complement S_uu of the
 * block-angular condensed system (Prop. 2.4, with the A_i^{-1} of eq. (15));
 * once summed over scenarios (§3.2, "Global reduction"), it is factored
 * densely (§4.2: a LAPACK factorization on the GPU, a small share of the
 * time).  With every G_x^i invertible, the condensed matrix of eq. (8)
 * has inertia (N n_x + n_u, N n_x, 0) exactly when S_uu is positive definite
 * (Haynsworth's inertia additivity over the Schur complement; each A_i has
 * inertia (n_x, n_x, 0)), so a successful factorization is the inertia test.
 * The paper does not describe inertia correction: delta_w adds delta_w I to
 * the W block of eq. (6) (IPOPT's rule, the reading the library takes).
 * Errors: IPM_ERR_STATE before ipm_condense_scenarios. */
ipm_status ipm_factor_schur(ipm_ctx *ctx, double delta_w, int *is_pd, void *stream);

/* Solve the Newton system eq. (6) through eq. (11) and the recoveries of
 * Props. 2.1 and 2.3, then refine it on the residual of eq. (6) itself
 * (opt.aug_refine).  step: nullable device pointer receiving step_len
 * doubles.  refine_resid: nullable host pointer receiving the relative
 * residual max|rho| / max|r| of the augmented system eq. (6) at the returned
 * step (the CG residual of the reduced system on the mixed path when
 * aug_refine = 0). */
ipm_status ipm_solve_kkt(ipm_ctx *ctx, double *step, double *refine_resid, void *stream);

/* One full interior-point iteration (evaluate, test convergence, update mu,
 * condense, factor with inertia correction, solve, fraction to boundary,
 * backtracking line search, update).  *converged = 1 when the current point
 * already meets E_0 <= tol (no step is then taken); *kkt_err = E_0 there.
 * §2.2: one Newton step on the KKT conditions eq. (5) with the complementarity
 * smoothed by mu, its direction the solution of the augmented system eq. (6),
 * obtained here through the condensation of Prop. 2.1 and the reduction of
 * Prop. 2.3.  The paper delegates the step-length, barrier and stopping rules
 * to MadNLP (Nocedal & Wright ch. 19); the library takes fraction to the
 * boundary, an l1-merit backtracking line search and E_0 of Waechter and
 * Biegler as its reading.  Errors: IPM_ERR_NOT_PD, IPM_ERR_LINESEARCH,
 * IPM_ERR_SINGULAR_GX, IPM_ERR_TIMEOUT, IPM_ERR_CUDA. */
ipm_status ipm_step(ipm_ctx *ctx, int *converged, double *kkt_err, void *stream);

/* Run ipm_step until convergence or max_iter.  *iters = Newton steps taken.
 * §4.2 solves every instance "to a KKT residual" of the IPM of §2.2; the
 * library stops at E_0 <= opt.tol (1e-8), E_0 = max(scaled dual residual of
 * eq. (5a)-(5c), primal residual of eq. (5d)-(5e), scaled complementarity of
 * eq. (5f)-(5h)).  Errors: those of ipm_step, IPM_ERR_MAXITER. */
ipm_status ipm_solve(ipm_ctx *ctx, int *iters, double *kkt_err, void *stream);

/* Diagnostics for tests: copy an internal quantity to host memory.
 * which: IPM_Q_KHAT (n_u*n_u, row-major, before factorization, delta = 0),
 *        IPM_Q_ZTZ (n_u*n_u: sum_i Z_i^T Z_i of the inertia correction, after
 *        a factorization with delta_w > 0),
 *        IPM_Q_RHS_U (n_u), IPM_Q_Z (scenario scen, n_x*n_u row-major, rows in
 *        the x order of the state vector), IPM_Q_FGH (scen: f, g[n_x], h[m]),
 *        IPM_Q_JAC (scen: dense G_x, G_u, H_x, H_u row-major, concatenated),
 *        IPM_Q_HESS (scen: dense W_xx, W_xu, W_uu^i), IPM_Q_ERRS (6 doubles:
 *        dual, primal, compl max, compl min, s_d, s_c), IPM_Q_INFO (10 doubles:
 *        alpha, alpha_max, alpha_z, delta, trials, rho, mu_used, refinement
 *        iterations, refinement relative residual, 1 if the iteration fell back
 *        to the FP64 condensation; if cap allows, then the number of
 *        iterations since ipm_create that fell back to the FP64
 *        condensation, the number of emulated contractions redone on the
 *        FP64 units, for the last solve the refinement steps on the
 *        augmented system eq. (6), its relative residual before and after
 *        them, then 1 if K_hat is formed by the adjoint-solve reduction, and
 *        the autotuner's times (ms) of the dense and the adjoint reduction,
 *        and the number of times since ipm_create that the mixed path raised
 *        delta_w because CG met non-positive curvature of the exact
 *        operator),
 *        IPM_Q_TIMERS (2*IPM_N_PHASES doubles: accumulated device milliseconds
 *        and call counts per phase, see ipm_set_profiling; a further double,
 *        if cap allows, is the total number of kernels the library launched).
 * cap: capacity of host_out in doubles. */
enum { IPM_Q_KHAT = 0, IPM_Q_RHS_U = 1, IPM_Q_Z = 2, IPM_Q_FGH = 3, IPM_Q_JAC = 4,
       IPM_Q_HESS = 5, IPM_Q_ERRS = 6, IPM_Q_INFO = 7, IPM_Q_TIMERS = 8, IPM_Q_ZTZ = 9 };
ipm_status ipm_get_quantity(ipm_ctx *ctx, int which, int scen, double *host_out,
                            long long cap, void *stream);

/* Phase timers (tracing).  When on, CUDA events are recorded on the call's
 * stream around each phase of the path and the elapsed device time is
 * accumulated (a phase met several times in one iteration counts each
 * time); on = 2 also resets the accumulators.  Phases, in order:
 * eval, condense_K (Sigma, K, right-hand sides), lu, zsolve (Z and Y),
 * gemm (Z^T Y + scenario sum), reduced_rhs, cholesky, recover, linesearch,
 * split (the tensor-core operands of Z and Y: BF16 slices or planes),
 * fallback (mixed path: the whole FP64 condensation and solve of an
 * iteration condensed again; its inner phases are not added to the others),
 * solve1 (every solve of one vector per scenario with G_x or G_x^T on the
 * call's stream, counted each time; nested in the phases above).
 * Profiling serialises the host with the device at phase boundaries. */
enum { IPM_N_PHASES = 12 };
ipm_status ipm_set_profiling(ipm_ctx *ctx, int on);

/* Kernels this library has launched in the process so far (all contexts;
 * a replayed CUDA graph counts its kernel nodes). */
long long ipm_kernel_launches(void);

/* Self-test of the failure path of the bounded device waits: one thread
 * waits on an mbarrier that nothing arrives at, gives up after `polls` polls
 * (1 .. 2^22) and raises the timeout flag, exactly as the waits of the
 * tensor-core kernels do (there with 2^22 polls).  Returns IPM_ERR_TIMEOUT
 * when the wait gave up (the expected outcome) and leaves the device usable;
 * IPM_ERR_ARG for a poll count out of range. */
ipm_status ipm_selftest_bounded_wait(long long polls, void *stream);

/* Host-side symbolic analysis only (no GPU, no context): one of the integer
 * structures the kernels are driven by, for checks of the host logic (the
 * static-pivot LU pattern and the schedules built from it).
 *   IPM_SYM_DIMS: n_x, n_u, t0 (first position of the dense trailing block),
 *     nd, nnz(L+U), number of solve panels, number of trailing-block product
 *     lists;
 *   IPM_SYM_LU_COLPTR, IPM_SYM_LU_ROW: CSC pattern of L+U by elimination
 *     position (a slot is an index into lu_row);
 *   IPM_SYM_FR_PTR, _FR_COL, _FR_LSLOT: L by rows (columns k < i, their slots);
 *   IPM_SYM_GU_PTR, _GU_COL: G_u by rows (positions), u columns;
 *   IPM_SYM_ZP_*: the per-panel forward schedules of the multi-RHS solve
 *     (level offsets per panel, level pointers, rows, product pointers,
 *     product columns and slots, zero-row pointers and rows, trailing-row
 *     product pointers, columns and slots);
 *   IPM_SYM_TW_*: the products of the sparse pivots into the trailing block
 *     (list lengths; L slot, U slot and flushed entry slot or -1 per product,
 *     product q of list t at q * lists + t);
 *   IPM_SYM_LU_SLOT: the storage slot of every entry of the CSC pattern (the
 *     entries outside the trailing block in CSC order, then the trailing
 *     block column-major with leading dimension nd at dense_base).
 * IPM_SYM_DIMS then also gives dense_base and 1 if the trailing block is
 * handled by the large-block (global-memory) kernels.  which |
 * IPM_SYM_FORCE_BIG builds the structures of that mode whatever nd is (its
 * dense block also takes the sparse pivots just before it that reach a
 * sixth of it).
 * Writes min(cap, size) values to out (out may be NULL) and the size to *len.
 * Errors: IPM_ERR_ARG for an invalid network or structure id. */
enum {
  IPM_SYM_DIMS = 0, IPM_SYM_LU_COLPTR, IPM_SYM_LU_ROW, IPM_SYM_FR_PTR, IPM_SYM_FR_COL, IPM_SYM_FR_LSLOT,
  IPM_SYM_GU_PTR, IPM_SYM_GU_COL, IPM_SYM_ZP_LEV_OFF, IPM_SYM_ZP_LEV_PTR, IPM_SYM_ZP_ROWS, IPM_SYM_ZP_EPTR,
  IPM_SYM_ZP_COL, IPM_SYM_ZP_SLOT, IPM_SYM_ZP_ZPTR, IPM_SYM_ZP_ZROWS, IPM_SYM_ZP_TPTR, IPM_SYM_ZP_TCOL,
  IPM_SYM_ZP_TSLOT, IPM_SYM_TW_LEN, IPM_SYM_TW_L, IPM_SYM_TW_U, IPM_SYM_TW_E, IPM_SYM_LU_SLOT, IPM_SYM_COUNT
};
#define IPM_SYM_FORCE_BIG 0x100
ipm_status ipm_symbolic_export(const ipm_network *net, int which, int *out, long long cap, long long *len);

/* Replace the scenario loads of a context (same network and N) and reset the
 * cold-start state.  pd, qd: host [n_scen][n_bus].  Reuses every symbolic
 * structure and device workspace (no allocation).  Errors: IPM_ERR_ARG on
 * non-finite or negative loads. */
ipm_status ipm_set_loads(ipm_ctx *ctx, const double *pd, const double *qd, void *stream);

/* Line contingencies (§4.1.1: every scenario is assigned its own loads and
 * potential contingencies, line tripping).  trip: host [n_scen], the index
 * of the line out of service in that scenario, or -1 for none (NULL: every
 * line back in service).  A tripped line contributes zeros to that
 * scenario's injections, flows, Jacobians and Hessian; the sparsity
 * patterns stay those of the intact network, so the symbolic analysis, the
 * static-pivot LU order and every workspace are reused.  Resets the cold
 * start like ipm_set_loads.  Errors: IPM_ERR_ARG for an index out of range
 * or a line whose loss disconnects the network (G_x would be singular),
 * checked on the host before anything changes. */
ipm_status ipm_set_contingencies(ipm_ctx *ctx, const int *trip, void *stream);

/* ---- Multi-instance runner ------------------------------------------------
 * Many independent instances (networks of any size, any scenario counts) on
 * one GPU.  The paper solves one two-stage problem at a time; this runner
 * has no counterpart there.  Host worker threads each drive one instance at
 * a time through the ordinary IPM iteration on their own stream.  With
 * group_contraction, the FP64 reduced-Hessian contractions of the instances
 * that reach the condensation together run as ONE persistent launch over
 * their (instance, tile, scenario group) work items; an instance waits at
 * most window_us for the others before the launch goes ahead without them,
 * and converged instances drop out.  Results are bit-identical to solving
 * each context alone (the work items compute exactly the per-instance
 * partial tiles). */
typedef struct {
  int n_threads;          /* host worker threads (0 = 8) */
  int group_contraction;  /* 1 (default): grouped persistent contraction */
  double window_us;       /* longest rendezvous wait (2000) */
  int reserved[4];
} ipm_batch_options;

#define IPM_BATCH_N_STATS 8
/* stats (nullable, IPM_BATCH_N_STATS doubles): grouped launches, work items,
 * mean instances per grouped launch, most instances active at once, wall
 * time in ms of the whole call, then zeros. */

ipm_status ipm_batch_default_options(ipm_batch_options *opt);

/* Solve n existing contexts from their current states.  streams: NULL (the
 * runner creates one non-blocking stream per worker) or one stream per
 * context.  iters, kkt_err, status: [n] outputs.  Returns IPM_OK when every
 * instance converged, else the first failing status (all are attempted). */
ipm_status ipm_solve_batch(ipm_ctx **ctxs, int n, void **streams, const ipm_batch_options *opt, int *iters,
                           double *kkt_err, int *status, double *stats);

/* Create, solve and destroy n instances under a device-memory budget (bytes):
 * a worker creates its next context (symbolic analysis included) only while
 * the estimated footprints of the live contexts plus its own fit in
 * mem_budget (one context alone is always admitted); largest instances go
 * first.  nets[i], n_scen[i], pd[i], qd[i] as for ipm_create; opt applies to
 * all.  states_out: NULL, or per instance NULL or a host array of that
 * instance's state_len doubles that receives the final state. */
ipm_status ipm_run_instances(const ipm_network *nets, int n, const int *n_scen, const double *const *pd,
                             const double *const *qd, const ipm_options *opt, const ipm_batch_options *bopt,
                             long long mem_budget, double *const *states_out, int *iters, double *kkt_err,
                             int *status, double *stats);

/* ---- Learned warm start ---------------------------------------------------
 * Not in the paper.  A small MLP maps a scenario's load vector to a
 * primal-dual starting point of the IPM; the cold start stays the fallback.
 *   y = W3 GELU(W2 GELU(W1 xn + b1) + b2) + b3,   xn = (x - in_mean) / in_std,
 * prediction = out_mean + out_std * y, GELU(a) = a Phi(a) (Gauss error
 * function form).  Products run in BF16 on the tensor cores with FP32
 * accumulation; weights are FP32 masters trained by Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8) on the mean squared error of the normalised outputs,
 *   L = (1 / (B d_out)) sum_b sum_k (y_bk - (t_bk - out_mean_k) / out_std_k)^2.
 * Parameter vectors (host FP32) use the logical layout W1 [d_hidden][d_in],
 * b1, W2 [d_hidden][d_hidden], b2, W3 [d_out][d_hidden], b3. */
typedef struct ipm_mlp ipm_mlp;

/* d_hidden: a multiple of 128.  max_batch: rows per internal pass (forward
 * splits larger batches).  He-uniform weights from seed, zero biases, unit
 * normalisation.  Errors: IPM_ERR_ARG, IPM_ERR_OOM. */
ipm_status ipm_mlp_create(int d_in, int d_hidden, int d_out, int max_batch, unsigned long long seed,
                          ipm_mlp **out);
ipm_status ipm_mlp_destroy(ipm_mlp *mlp);
long long ipm_mlp_param_count(const ipm_mlp *mlp);
/* host FP32 params in the logical layout; resets the Adam moments */
ipm_status ipm_mlp_set_params(ipm_mlp *mlp, const float *params);
ipm_status ipm_mlp_get_params(ipm_mlp *mlp, float *params);
/* host FP32 [d_in], [d_in], [d_out], [d_out]; stds must be > 0 */
ipm_status ipm_mlp_set_normalization(ipm_mlp *mlp, const float *in_mean, const float *in_std,
                                     const float *out_mean, const float *out_std);
/* x: device FP32 [batch][d_in]; y: device FP32 [batch][d_out] (de-normalised) */
ipm_status ipm_mlp_forward(ipm_mlp *mlp, const float *x, int batch, float *y, void *stream);
/* loss and its gradient at the current weights (no update): x, target device
 * FP32 [batch][d_in], [batch][d_out] (targets in output units), batch <=
 * max_batch; grads: NULL or host FP32 in the logical layout; loss: host. */
ipm_status ipm_mlp_gradients(ipm_mlp *mlp, const float *x, const float *target, int batch, float *grads,
                             float *loss, void *stream);
/* one Adam step at learning rate lr on the minibatch; loss before the step */
ipm_status ipm_mlp_train_step(ipm_mlp *mlp, const float *x, const float *target, int batch, float lr,
                              float *loss, void *stream);

/* Warm-start vectors of a context, per scenario (FP32, device, [N][d]):
 *   [ x (n_x) | u (n_u) | s (m) | log zl_x | log zu_x | log zl_u | log zu_u |
 *     log zl_s | log zu_s ]
 * where each log-dual block lists only the components with a finite bound of
 * that side, in index order.  ipm_warm_dim gives d. */
ipm_status ipm_warm_dim(const ipm_ctx *ctx, int *d);
/* the current state (normally a converged one) as warm-start vectors */
ipm_status ipm_warm_target(ipm_ctx *ctx, float *out, void *stream);
/* Start the IPM from predicted vectors: x_i, s_i from each scenario's row,
 * u = mean over the rows; primal values pushed into their bounds as at a
 * cold start; bound duals exp(log dual) clipped to [1e-12, 1e12]; the slack
 * multipliers from their stationarity (z = zl_s - zu_s); y from the
 * stationarity of the Lagrangian in x, G_x^T y = -(grad_x f + H_x^T z -
 * zl_x + zu_x), one batched transposed LU solve; mu = max(1e-6, mean
 * complementarity).  Then ipm_solve continues from this point. */
ipm_status ipm_warm_start(ipm_ctx *ctx, const float *pred, void *stream);

/* The emulated FP64 contraction of IPM_PREC_FP64_TC on caller-owned device
 * matrices: Khat [n_u][n_u] = sum_s Z_s^T Y_s, with Z, Y device FP64
 * [n_scen][n_x][n_u] (row-major).  Allocates its scratch, synchronises the
 * stream before returning.  IPM_ERR_ARG also when the result is not finite.
 * For checking the kernel on
 * arbitrary data; the paper has no counterpart (it is GB300 specific). */
ipm_status ipm_schur_sum_tc(const double *Z, const double *Y, int n_scen, int n_x, int n_u, double *Khat,
                            void *stream);

/* Allocation-free reduced-Hessian sum.  The paper has no counterpart to this
 * entry point; it exists for callers that cannot call cudaMalloc (code that
 * runs while another memory pool owns the device, plug-ins that are only
 * handed device buffers by their host application, processes with a locked
 * allocator).  It needs no context and allocates nothing.
 *
 *   Khat = sum_s Z_s^T Y_s + sum_s Yu_s + diag(d)
 *
 * Z, Y: device [n_scen][n_x][n_u] row-major; Yu: device [n_scen][n_u][n_u]
 * or NULL; d: device [n_u] or NULL; Khat: device [n_u][n_u] output.  Only
 * the upper triangle of the sum is formed and mirrored (the result is taken
 * as symmetric, as K_hat is).  All pointers are caller-owned; work is
 * enqueued on "stream".
 *
 * Scratch: the split-K partial tiles live in one 4 MiB file-scope device
 * array that every GPU loading the library holds until exit; n_u above
 * IPM_SCHUR_NOALLOC_MAX_NU does not fit and returns IPM_ERR_ARG without
 * launching anything.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Under CUDA's default lazy module
 * loading the array (with the module's code) is committed to device memory
 * by that first lookup, not when the library is loaded: make the first call
 * before another pool claims the device's memory, or set
 * CUDA_MODULE_LOADING=EAGER so the array is committed at load time.  A CUDA
 * error already pending on the calling thread is reported as IPM_ERR_CUDA
 * before anything is launched (and left pending).  All calls share the array: calls
 * that overlap on the GPU race and must be serialised by the caller.
 * Errors: IPM_ERR_ARG (null pointer, non-positive size, n_u too large),
 * IPM_ERR_CUDA (symbol lookup or launch failed). */
#define IPM_SCHUR_NOALLOC_MAX_NU 960
ipm_status ipm_schur_sum_noalloc(const double *Z, const double *Y, const double *Yu,
                                 const double *d, int n_scen, int n_x, int n_u, double *Khat,
                                 void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IPM_H */
