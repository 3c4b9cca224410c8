/*
 * fil.h -- C ABI of the GB300 filament-suspension hot path.
 *
 * Method: Schoeller, Townsend, Westwood & Keaveny, "Methods for suspensions
 * of passive and active filaments". Each filament is N rigid spheres
 * ("segments") of radius a, spacing dL, with a unit quaternion per segment
 * (Sec. 2.9). One timestep solves f(X) = 0 (eqn RA-3d-system) for
 * X = (Y_1, u_1..u_N, Lambda_{3/2}..Lambda_{N-1/2}) per filament by the
 * limited-memory bad Broyden method (Algorithm 2) with the block-diagonal
 * approximate Jacobian J0 of App. B.2; every residual evaluation applies the
 * Rotne-Prager-Yamakawa mobility (Sec. 2.7.1) to all segment pairs.
 *
 * Conventions (all entry points):
 *  - Every entry point returns a fil_status; nothing aborts, exits or throws
 *    across the ABI. fil_last_error(ctx) holds a message for the last failure.
 *  - Pointers to arrays may be HOST or DEVICE memory (detected per call with
 *    cudaPointerGetAttributes); host buffers are staged through the context's
 *    device workspace with copies on the context stream. The caller owns
 *    every buffer it passes; the library never frees or retains them.
 *  - The library allocates device memory only in fil_create (and frees it in
 *    fil_destroy). Work is issued on the stream given at creation. Calls that
 *    return host scalars (finf, converged, iters) or read host arrays
 *    synchronise that stream before returning.
 *  - Segments of all filaments are concatenated filament-major: segment n
 *    (0-based) of filament i is row off[i] + n, off[i] = sum_{k<i} N_k.
 *    S = sum N_i. Per-segment arrays are row-major: Y, u are S x 3, q is
 *    S x 4 scalar-first (q0, q1, q2, q3), FT and VW are S x 6 (F then T,
 *    V then Omega). Lambda is sum(N_i - 1) x 3, filament-major, row n of a
 *    filament holding Lambda_{n+3/2}.
 *  - X and f are 6S long, per filament [Y_1 (3), u_1..u_N (3N),
 *    Lambda_{3/2}..Lambda_{N-1/2} (3(N-1))] and [f^1 (3), f^2_1..N (3N),
 *    f^3_2..N (3(N-1))] (eqn RA-3d-system).
 *  - Units are the caller's; a, eta, dL, KB, KT must be > 0.
 */
#ifndef FIL_H
#define FIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fil_ctx fil_ctx;

typedef enum {
    FIL_OK = 0,
    FIL_EINVAL = 1,   /* bad argument or size                                 */
    FIL_ENOMEM = 2,   /* device allocation failed in fil_create               */
    FIL_ECUDA = 3,    /* a CUDA call failed (message in fil_last_error)       */
    FIL_ENOCONV = 4,  /* Broyden reached max_iter without ||f||_inf <= tol*a  */
    FIL_ENAN = 5,     /* the residual became NaN or Inf                       */
    FIL_ESTALL = 6,   /* ||f(X_{k+1}) - f(X_k)||_2 = 0: no secant update      */
    FIL_ESTATE = 7,   /* call out of order (e.g. a Broyden step before begin) */
    FIL_EOVERFLOW = 8 /* a fixed-capacity table overflowed (steric cell grid:
                         more segments in one cell or within range of one
                         segment than it holds; the configuration has collapsed) */
} fil_status;

typedef enum {
    FIL_FP64 = 0,     /* every step in FP64, including the RPY pair sums       */
    FIL_MIXED = 1,    /* RPY pair sums in FP32 with per-target compensated
                         accumulation; J0 factors / inverse and their solves
                         and the Broyden history (c_i, d_i of Algorithm 2) in
                         FP32; state, residual, iterates and norms in FP64     */
    FIL_PAIR32 = 2    /* RPY pair sums in FP32 with per-target compensated
                         accumulation (as FIL_MIXED); everything else as
                         FIL_FP64: the Broyden history, its dot products and
                         rank-one updates, the J0 factors and solves (the
                         filament-RPY inverse with its FP64 refinement), the
                         quaternion exponential map, state and residual      */
} fil_precision;

typedef enum {
    FIL_J0_DRAG = 0,          /* J0 of App. B.2 as printed: diagonal (self) mobility
                                 in f_0; banded O(N) factorisation per filament     */
    FIL_J0_FILAMENT_RPY = 1   /* f_0 keeps every RPY block between segments of the
                                 same filament (inter-filament coupling and dM/dY
                                 dropped); a dense 6N x 6N block per filament,
                                 inverted in FP32 by Gauss-Jordan elimination (plus
                                 one FP64 refinement per solve in FP64 mode); N <= 38.
                                 Reduces to FIL_J0_DRAG when those blocks are cut to
                                 the self term; far fewer Broyden iterations in dense
                                 suspensions                                         */
} fil_j0_model;

typedef enum {
    FIL_EXTRAP_LINEAR = 1,     /* x_0 = 2 x^j - x^{j-1}                              */
    FIL_EXTRAP_QUADRATIC = 2,  /* x_0 = 3 x^j - 3 x^{j-1} + x^{j-2}                  */
    FIL_EXTRAP_ADAPTIVE = 3    /* per filament and per block of unknowns (Y_1, u,
                                  Lambda): the linear guess plus a fitted fraction
                                  (0..1) of the quadratic correction             */
} fil_extrapolation_order;

typedef struct {
    int32_t n_fil;                /* number of filaments M >= 1                    */
    const int32_t *seg_per_fil;   /* HOST array of M segment counts N_i >= 1; copied */
    double a;                     /* segment radius                                */
    double eta;                   /* viscosity                                     */
    double dL;                    /* segment spacing Delta L                       */
    double KB, KT;                /* bending and twist moduli (Sec. 2.2)           */
    double gamma0, kappa_mu, kappa_nu; /* preferred twist and curvatures (Sec. 2.2) */
    double dt;                    /* timestep                                      */
    double tol;                   /* Broyden stops when ||f||_inf <= tol * a       */
    int32_t max_iter;             /* Broyden iteration cap and history depth >= 1  */
    int32_t precision;            /* fil_precision                                 */
    int32_t j0_model;             /* fil_j0_model                                  */
    void *stream;                 /* cudaStream_t, or NULL for the legacy stream   */
} fil_params;
/* Limits: S = sum N_i <= 2^30 and N_i <= 4266 (a filament's right-hand side is
 * kept in shared memory by the J0 solves). */

/* Create a context: validates p, copies the layout, allocates every device
 * buffer the other calls use (state, workspace, Broyden history of depth
 * max_iter, J0 band factors, RPY partial sums). The state starts with all
 * segments at the origin and identity quaternions; call fil_set_state or
 * fil_init_straight before stepping. *out is NULL on failure. */
fil_status fil_create(const fil_params *p, fil_ctx **out);

/* Ensemble of n_sys independent systems in one context (batched suspensions):
 * the filaments of p are taken in consecutive groups of fil_per_sys[s] >= 1
 * (HOST array; sum = p->n_fil). The mobility couples segments of the same
 * system only (Sec. 2.7.1 per system) and every system has its own Broyden
 * scalars, norms and convergence test (Algorithm 2 per system): a system that
 * meets the tolerance keeps its iterate while the others continue. All systems
 * share one launch per kernel (the RPY apply stays one persistent launch over
 * all systems' work units). fil_create is the case n_sys = 1. */
fil_status fil_create_ensemble(const fil_params *p, int32_t n_sys, const int32_t *fil_per_sys,
                               fil_ctx **out);

/* Per system (host arrays of n_sys, nullable): Broyden iterations of the
 * current / last step and the last ||f||_inf that was read. */
fil_status fil_sys_stats(const fil_ctx *c, int32_t *iters, double *finf);

/* Autotuner of the RPY pair kernel: times the pair kernel (which also sums
 * each tile's partials) of `reps` mobility applies of the current state's
 * loads (CUDA events around it, so host launch gaps do not count) for every
 * candidate schedule -- tiles of 256 targets (2 per thread) or 128 targets
 * (1 per thread, with source split 1 or 2 on the FP32 path: see
 * fil_set_source_split), and 1..occupancy resident CTAs per SM for the
 * stream-K split of the (tile, source chunk) work units -- and keeps the fastest for all
 * later applies. The applies first run for 50 ms of wall time (an idle GPU's
 * clock is still rising then) and the candidates are swept twice, each
 * keeping its faster time. Reports the choice (nullable outputs) and its
 * pair-kernel time per apply in ms. Results change only in rounding (the
 * summation order of the pair terms). FIL_ESTATE inside a step. */
fil_status fil_autotune(fil_ctx *c, int32_t reps, int32_t *tile, int32_t *ctas_per_sm,
                        double *ms);

/* Set the pair schedule by hand (the autotuner's candidates): tile 256 with 2
 * targets per thread or tile 128 with 1, and ctas_per_sm from 1 to the
 * kernel's occupancy; the source split goes back to 1. FIL_EINVAL for another
 * combination, FIL_ESTATE inside a step. fil_pair_schedule reads the current
 * one (nullable outputs). */
fil_status fil_set_pair_schedule(fil_ctx *c, int32_t tile, int32_t targets_per_thread,
                                 int32_t ctas_per_sm);
fil_status fil_pair_schedule(const fil_ctx *c, int32_t *tile, int32_t *targets_per_thread,
                             int32_t *ctas_per_sm);

/* Source split of the FP32 pair kernel with one target per thread (128-target
 * tiles): split = 2 runs each CTA with twice the warps on the same targets, the
 * two halves taking alternate 32-source groups of every chunk (their sums are
 * added in float-float arithmetic, first half first), for problems whose few
 * work units leave the SMs short of warps. Applies to the current schedule;
 * fil_set_pair_schedule sets it back to 1, fil_autotune chooses it with the
 * rest. FIL_EINVAL for a split other than 1 or 2, for 2 with 256-target tiles
 * or the FP64 path, or when ctas_per_sm exceeds the split kernel's occupancy
 * (2 on GB300); FIL_ESTATE inside a step. Results change only in rounding. */
fil_status fil_set_source_split(fil_ctx *c, int32_t split);
fil_status fil_source_split(const fil_ctx *c, int32_t *split);

/* Run each Broyden iteration of fil_broyden_step / fil_step as one CUDA graph
 * launch (enable = 1) instead of separate kernel launches: the graph holds the
 * update of X, the residual of the new iterate, the dot products, the J0 solve
 * and the history update, captured once per buffer parity at the start of a
 * step (an ensemble's set of iterating systems and its list of RPY tiles are
 * read from device memory, so the graphs stay valid as systems converge).
 * Same results. Not with fil_profile on. FIL_ESTATE inside a step. */
fil_status fil_set_graph(fil_ctx *c, int32_t enable);

/* RPY pair interactions evaluated by this context's mobility applies so far
 * (sum over each apply of S_s^2 over the systems it evaluated; padding and
 * converged systems excluded). */
fil_status fil_pair_count(const fil_ctx *c, double *pairs);

/* Steric barrier between segments (Sec. 2.6): a repulsive force
 *   F^B_nm = FS ((4a^2 chi^2 - r^2) / (4a^2 (chi^2 - 1)))^4 (Y_n - Y_m) / (2a)
 * on segment n from every segment m of the same system with r = |Y_n - Y_m|
 * < 2 chi a, except n itself and its neighbours n +- 1 in the same filament,
 * added to the forces of every residual evaluation (fil_residual, the Broyden
 * iterations, fil_step). FS = 0 (the default) switches it off; chi > 1. The
 * first call with FS != 0 allocates a hashed cell grid (2^k >= 2S buckets of
 * 16 segments, on the device); a residual evaluation whose grid overflows
 * (more than 16 segments hashed to one bucket, or more than 48 within range
 * of one segment) returns FIL_EOVERFLOW. Forces are summed per segment in
 * increasing order of m, so results are reproducible run to run.
 * FIL_EINVAL for a negative or non-finite FS or chi <= 1; FIL_ESTATE inside
 * a step. */
fil_status fil_set_steric(fil_ctx *c, double FS, double chi);

/* Tethered and clamped filaments (Sec. 5.2.1; eqs. tethering_constraint,
 * tethered_rotation_constraint, tethering_constraint_force_and_torque).
 * mask [M] (nonzero: tethered; a null mask unties every filament), Y1 [M x 3]
 * the base position Y_1 each tethered filament must reach at the end of the
 * next step, u1 [M x 3] the rotation of its first segment over that step
 * (q_1 <- exp(u1) q_1^j); host or device arrays, rows of free filaments
 * ignored. The values persist until the next call: call once for a clamp
 * (Y1 fixed, u1 = 0), before every step for a moving base (a motor:
 * Y1 = delta_0 (cos jw dt, sin jw dt, 0), u1 = (0, 0, w dt)).
 * For a tethered filament the Y_1 slot of X (fil_residual, fil_get_iterate,
 * fil_j0_solve) holds the multiplier lambda_1, a force on segment 1, and the
 * u_1 slot lambda_2, which exerts the torque D^T lambda_2 on segment 1
 * (D v = dexpinv_{u1}(v)); the first segment's update equations are those of
 * a free filament with Y_1, u_1 substituted. The multipliers' initial guess
 * is extrapolated from the last two steps; a change of the mask (or
 * fil_set_state) restarts that history. J0 of a tethered filament is the free
 * J0 with the six slot columns replaced by the multiplier derivatives (same
 * mobility model), solved through the free J0 plus a rank-6 correction.
 * The first call allocates (M x 66 + 13 nX doubles) on the device.
 * FIL_ESTATE inside a step or with a warm-start network attached
 * (fil_warm_attach refuses a network while filaments are tethered);
 * FIL_EINVAL for null Y1 / u1 with a mask. */
fil_status fil_set_tether(fil_ctx *c, const int32_t *mask, const double *Y1, const double *u1);

/* Multipliers (lambda_1, lambda_2) of every filament from the last committed
 * step, [M x 6] (zero for free filaments or before any tethered step). */
fil_status fil_get_tether(fil_ctx *c, double *lam);

/* Release the context and its device memory (synchronises its stream). */
void fil_destroy(fil_ctx *c);

/* Message of the last failed call on this context ("" if none). */
const char *fil_last_error(const fil_ctx *c);

/* Sizes of the context: S segments, 6S unknowns, sum(N_i - 1) multipliers. */
fil_status fil_sizes(const fil_ctx *c, int64_t *n_seg, int64_t *n_unknowns, int64_t *n_lambda);

/* Set the time-integration state (Sec. 2.9.3): positions Y^j (S x 3) and
 * quaternions q^j (S x 4) are required; Yprev = Y^{j-1} (S x 3) and u^j
 * (S x 3, the Lie-algebra elements of the previous step) are optional and
 * must be given together: with them the next step is BDF2, without them the
 * next step is backward Euler (first step). Lambda (sum(N_i-1) x 3) is
 * optional (zero if NULL) and seeds the next step's initial guess. */
fil_status fil_set_state(fil_ctx *c, const double *Y, const double *q, const double *Yprev,
                         const double *u, const double *Lambda);

/* Read the state back; any pointer may be NULL to skip that array. Yprev and
 * u are zero before the first committed step. */
fil_status fil_get_state(fil_ctx *c, double *Y, double *q, double *Yprev, double *u,
                         double *Lambda);

/* Initialise straight filaments (App. A.1 and A.5): filament i starts at
 * base[i] (M x 3) with unit tangent t[i] and unit normal mu[i] (M x 3,
 * orthonormal); the quaternion of every segment is the one whose rotation
 * maps (e_x, e_y) to (t, mu) (App. A.1 steps 1-5); if xi (S x 3) is not NULL
 * each quaternion is then perturbed to exp(xi_n) q_n. Positions follow the
 * robot-arm construction Y_n = Y_1 + (dL/2) sum_{m=2}^n (t_{m-1} + t_m)
 * (eqn positionSubstitution-3d). History is cleared (next step is backward
 * Euler), Lambda is zero. */
fil_status fil_init_straight(fil_ctx *c, const double *base, const double *t, const double *mu,
                             const double *xi);

/* External loads (Sec. 2.5): a constant force Fext (S x 3) and torque Text
 * (S x 3) per segment, and a follower force -follower[i] * t_N on the last
 * segment of filament i (M entries). NULL clears the corresponding load. */
fil_status fil_set_external(fil_ctx *c, const double *Fext, const double *Text,
                            const double *follower);

/* Mobility apply (Sec. 2.7.1, eq. mobility-problem): VW = M(Y) FT over all
 * S^2 ordered segment pairs of the context, with the self term for n = m,
 * the far form for r >= 2a and the equal-radius overlapping form for r < 2a
 * (r = 0 between distinct segments takes the self values). Y is S x 3, FT and
 * VW are S x 6. Precision follows the context (FP64, or FP32 pair sums with
 * compensated per-target accumulation in FIL_MIXED and FIL_PAIR32). */
fil_status fil_mobility_apply(fil_ctx *c, const double *Y, const double *FT, double *VW);

/* Residual f(X) of eqn RA-3d-system at X (6S), using the context's state
 * and external loads: unpack (q = exp(u) q^j, robot-arm positions), forces
 * and torques (Sec. 2.5, eq. quaternionM), mobility, then the BDF2 rows
 * (backward Euler before the first committed step). Writes f (6S) and, if
 * finf is not NULL, ||f||_inf. */
fil_status fil_residual(fil_ctx *c, const double *X, double *f, double *finf);

/* Start a timestep (set-up of Algorithm 2): initial guess X_0 (each unknown
 * extrapolated linearly from the two previous steps, 2 x^j - x^{j-1}, where
 * both exist: Y_1 whenever Y^{j-1} is known, u and Lambda once two steps were
 * committed since the last fil_set_state / fil_init_straight; otherwise the
 * last value, with u = 0 on the first step), J0 at X_0 (App. B.2, or the
 * filament-RPY variant) assembled and factored per filament, f(X_0). Writes
 * ||f(X_0)||_inf to *finf if not NULL. */
fil_status fil_broyden_begin(fil_ctx *c, double *finf);

/* One pass of Algorithm 2's loop: dX_k = -H_k f(X_k), X_{k+1} = X_k + dX_k,
 * f(X_{k+1}), and the rank-one pair (c_{k+1}, d_{k+1}). *converged is set to 1
 * when ||f(X_{k+1})||_inf <= tol * a (the pair is then not formed). Returns
 * FIL_ESTATE before fil_broyden_begin, FIL_ENOCONV once max_iter iterations
 * were taken without convergence, FIL_ENAN / FIL_ESTALL as documented. */
fil_status fil_broyden_step(fil_ctx *c, int32_t *converged, double *finf);

/* Copy the current iterate X_k and f(X_k) (each 6S, either may be NULL). */
fil_status fil_get_iterate(fil_ctx *c, double *X, double *f);

/* Apply the factored J0^{-1} of the current step to b (6S) -> x (6S): exact to
 * FP64 rounding in FP64 mode (dense model: FP32 inverse plus one FP64
 * refinement step, ~1e-14 relative); FIL_PAIR32 solves as FIL_FP64. In
 * FIL_MIXED mode J0 is assembled and
 * factored or inverted in FP32 without refinement: the normwise backward
 * error per filament block is O(6N) FP32 roundings (~1e-6 measured on the
 * stiff blocks of a 32-segment suspension filament; the forward error scales
 * with the block's condition). J0 only shapes the Broyden iterates, so the
 * converged X is unaffected. */
fil_status fil_j0_solve(fil_ctx *c, const double *b, double *x);

/* Finish the timestep at the current iterate: q^{j+1} = exp(u) q^j,
 * Y^{j+1} from the robot arm, Y^{j-1} <- Y^j, u^j <- u, Lambda^j <- Lambda. */
fil_status fil_broyden_commit(fil_ctx *c);

/* One whole timestep: begin, Broyden steps until convergence, commit.
 * *iters (if not NULL) receives the number of Broyden iterations. On
 * FIL_ENOCONV / FIL_ENAN / FIL_ESTALL the state is left at the previous step
 * (the caller may retry with a smaller dt via fil_set_dt). */
fil_status fil_step(fil_ctx *c, int32_t *iters);

/* Change the timestep (takes effect at the next fil_broyden_begin). */
fil_status fil_set_dt(fil_ctx *c, double dt);

/* J0 reuse across timesteps. The paper builds J0 at the initial guess of every
 * step (Sec. 3.2.2 evaluates it once per timestep); J0 only shapes the Broyden
 * iterates (H_0 of Algorithm 2), not the converged solution, so its factors
 * may be kept for several steps. With max_age > 1, fil_broyden_begin / fil_step
 * keep the factors of the step that built them for at most max_age steps in
 * all, and build new ones earlier when the last committed step took more than
 * one Broyden iteration more than the step that built them, when the scheme
 * weight times dt changed (first step, fil_set_dt), after fil_set_state or
 * fil_init_straight, and after every fil_set_tether (tethered J0 columns follow
 * the prescribed motion; a prescription set once, such as a clamp, lets J0 be
 * kept). fil_step restarts a step that fails on reused factors
 * with factors built for it. max_age = 1 (the default) builds J0 every step.
 * FIL_EINVAL for max_age < 1, FIL_ESTATE inside a step. */
fil_status fil_set_j0_reuse(fil_ctx *c, int32_t max_age);

/* Steps whose J0 was built and steps that reused an earlier J0, since the
 * context was created (either pointer may be NULL). */
fil_status fil_j0_stats(const fil_ctx *c, int64_t *builds, int64_t *reuses);

/* Extrapolation that gives a step's initial guess X_0 (fil_extrapolation_order).
 * The paper starts Algorithm 2 from guesses extrapolated from the solutions of
 * past timesteps (Sec. 3.3) without stating the form. Each unknown takes the
 * value at the next step of the polynomial through its last committed values:
 * FIL_EXTRAP_LINEAR (the default) through two, x_0 = 2 x^j - x^{j-1};
 * FIL_EXTRAP_QUADRATIC through three, x_0 = 3 x^j - 3 x^{j-1} + x^{j-2}, which
 * is the linear guess plus the second difference d = x^j - 2 x^{j-1} + x^{j-2}.
 * The quadratic form has the smaller truncation error but weighs the past
 * solutions by 3, -3, 1 instead of 2, -1, so it carries more of their own
 * error (each is converged only to the tolerance): it wins when the motion
 * over a step is large compared with that, and loses when it is not.
 * FIL_EXTRAP_ADAPTIVE uses x_0 = 2 x^j - x^{j-1} + theta d, with theta fitted
 * for each filament and each of its blocks of unknowns (Y_1; u_1..u_N; Lambda)
 * by least squares over the past commits: at each commit, with x* the block's
 * solution and l, d the linear guess and second difference it was predicted
 * from, P <- 0.7 P + <x* - l, d> and Q <- 0.7 Q + <d, d>; theta = P / Q clipped
 * to [0, 1] (0, i.e. linear, until a block has been fitted); a step that took
 * no Broyden iteration (its solution is the guess itself) leaves the fit as it
 * was.
 * With fewer committed values the order drops to what they allow: Y_1 uses
 * Y^j, Y^{j-1} (held from the first committed step on, or given to
 * fil_set_state) and Y^{j-2}; u and Lambda use the values of committed steps
 * only, u = 0 and Lambda = Lambda^j before the first. Tether multipliers stay
 * linear. The converged solution does not depend on X_0 beyond the tolerance;
 * the iteration count does. A warm-start network (fil_warm_attach) predicts a
 * correction to this extrapolation, so use it with the choice it was trained
 * with. FIL_EINVAL for another value, FIL_ESTATE inside a step. */
fil_status fil_set_extrapolation(fil_ctx *c, int32_t order);

/* Broyden memory across timesteps. Algorithm 2 starts every step from
 * H_0 = J0^{-1}; its rank-one corrections, which learn the coupling between
 * filaments that the block-diagonal J0 leaves out, are discarded at the end of
 * the step. With keep > 0, a step whose J0 is the previous step's (see
 * fil_set_j0_reuse) starts instead from H_0 = J0^{-1} + sum_i c_i d_i^T over the
 * last min(keep, k) pairs (c_i, d_i) of the previous step's H_k, so that its
 * first iterate already uses them; the new step's updates are appended. A
 * step that converges on entry ends with H_k = H_0, so the pairs it carried
 * are the ones it passes on. The pairs are dropped whenever J0 is rebuilt (so also after every
 * fil_set_tether), after fil_set_state, fil_init_straight or a failed step. Like J0,
 * H_0 only shapes the iterates: every step still converges to ||f||_inf <= tol a.
 * keep = 0 (the default) is the paper's reset at every step. The call
 * allocates device memory for max_iter + keep history pairs when that is more
 * than the context holds (the pairs of the last step are then not carried);
 * besides fil_set_steric's cell grid it is the only allocation after
 * fil_create. In an ensemble each system keeps its own pairs
 * (a system that converged before the others has zero rows in the later
 * pairs). FIL_EINVAL for keep < 0 or keep > max_iter, FIL_ESTATE inside a
 * step, FIL_ENOMEM if the allocation fails. */
fil_status fil_set_broyden_memory(fil_ctx *c, int32_t keep);

/* The extrapolation in use (a fil_extrapolation_order value). */
fil_status fil_extrapolation(const fil_ctx *c, int32_t *order);

/* Counters since creation: RPY applies, Broyden iterations and kernels this
 * library launched (any pointer may be NULL). */
fil_status fil_counters(const fil_ctx *c, int64_t *mobility_applies, int64_t *broyden_iters,
                        int64_t *kernel_launches);

/* Kernel timing: while enabled, every RPY pair-kernel launch is bracketed by
 * two CUDA events recorded on the context stream (at most 4096 launches are
 * kept). fil_profile_read synchronises the stream, returns the number of
 * timed launches and their summed device time in milliseconds, and clears the
 * record. Enabling is cheap; the events add no synchronisation. Applies
 * captured into a CUDA graph record their events as event-record nodes: after
 * replays, fil_profile_read returns the times of the last replay. */
fil_status fil_profile(fil_ctx *c, int32_t enable);
fil_status fil_profile_read(fil_ctx *c, int64_t *launches, double *total_ms);

/* Measured FMA rate of the current device. A measurement helper with no
 * counterpart in the paper: the pair kernels' roofline fractions are reported
 * against the derived peak SMs x lanes x 2 flops x clock, and this call
 * measures what an FMA-only kernel actually reaches. It runs packed FP32x2
 * FMAs (fp64 = 0) or FP64 FMAs (fp64 = 1) in independent dependency chains on
 * every SM at full occupancy and returns the rate in flops/s (an FMA counts 2)
 * and the SM clock during the run in MHz, read from clock64 against the GPU's
 * nanosecond timer (either pointer may be NULL). Synchronous on the legacy
 * default stream; about 0.1 s (FP32) or 0.2 s (FP64); allocates nothing.
 * FIL_EINVAL for fp64 other than 0 or 1, FIL_ECUDA on a CUDA failure. */
fil_status fil_fma_peak(int32_t fp64, double *flops_per_s, double *sm_mhz);

/* Allocation-free mobility apply. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves --
 * code that runs where cudaMalloc is unavailable or not allowed, such as
 * inside another framework's memory pool or a host process whose device
 * allocations belong to someone else -- and so cannot hold a context.
 * It computes the same product as fil_mobility_apply of a FIL_MIXED context
 * (FP32 pair sums with compensated accumulation, FP64 results) for S =
 * n_seg segments with radius a and viscosity eta: Y (S x 3), FT (S x 6) and
 * VW (S x 6) must be DEVICE pointers of the current device (or managed
 * memory), owned by the caller. It allocates nothing: its scratch is a fixed
 * static device array of about 10.6 MB in the library (plus 128 per-tile
 * completion counters, zero between calls), which every GPU that loads the
 * library keeps until the process exits. Limits: 1 <= n_seg <=
 * 32768; larger sizes, host pointers, pointers to another GPU's memory or
 * non-positive a, eta return FIL_EINVAL; a failed launch returns FIL_ECUDA.
 * The scratch holds the stream-K partial sums of up to 4 x 152 CTAs (the
 * context path's grid on a 152-SM GB300); on a part with more SMs the grid is
 * capped there and the results differ from fil_mobility_apply's in rounding.
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress) and should come before any stream capture;
 * the address is kept for the life of the process, so the device's primary
 * context must stay the one in use (no cudaDeviceReset, no other driver
 * context on that device, between calls).
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the legacy stream)
 * without synchronising. All calls share the one array and leave their
 * contents in it; calls whose executions overlap on the GPU (different
 * streams, or different host threads) race on it and must be serialised by
 * the caller. */
fil_status fil_rpy_apply_noalloc(int64_t n_seg, const double *Y, const double *FT, double *VW,
                                 double a, double eta, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FIL_H */
