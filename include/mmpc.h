/*
 * mmpc.h -- C ABI of the GB300 (sm_103a) batch non-holonomic trajectory
 * optimizer of Adajania et al., "Multi-Modal Model Predictive Control through
 * Batch Non-Holonomic Trajectory Optimization" (arXiv 2109.10392).
 *
 * One scene (ego state, m constant-velocity obstacles, Sec. III assumption 3)
 * and a batch of B goals (end-of-horizon lateral position, speed,
 * acceleration; Sec. I "Main Idea") define B trajectory optimisation problems
 * that share every matrix (Remark 1).  mmpc_solve runs Algorithm 1 (Sec.
 * III-E) for all of them on one stream; mmpc_score evaluates the meta cost
 * of Sec. III-F and the batch argmin.
 *
 * Conventions
 *   - Road-attached frame (Sec. III assumption 1): x along the road, y to the
 *     left, heading psi from the centre line.  The ego starts at x = 0.
 *   - Every array is row-major and densely packed.
 *   - "device" pointers are CUDA device memory of the current device, owned
 *     by the caller; "host" pointers are host memory owned by the caller.
 *     The library owns only its mmpc_ctx (device constants and a few bytes
 *     of device scratch, allocated in mmpc_setup, freed in mmpc_destroy).
 *   - Calls taking a stream are asynchronous on that stream (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  Argument errors are
 *     detected on the host before anything is enqueued.
 *   - Return codes: MMPC_OK or a negative MMPC_ERR_*.  mmpc_last_error()
 *     gives a message for the last failing call on a context.  Non-convergence
 *     is not an error: it is reported through the residual outputs.
 *   - One context may be used from one host thread at a time, and its calls
 *     must be ordered on the GPU (one stream, or streams joined by events):
 *     mmpc_score uses the context's device scratch.
 */
#ifndef MMPC_H
#define MMPC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMPC_OK 0
#define MMPC_ERR_INVALID_ARG (-1) /* bad pointer, NaN or out-of-range scalar */
#define MMPC_ERR_SHAPE (-2)       /* size outside the supported range, or m != the m of setup */
#define MMPC_ERR_CUDA (-3)        /* a CUDA runtime call failed (message in mmpc_last_error) */
#define MMPC_ERR_TIMEOUT (-4)     /* a bounded device wait expired (reported by mmpc_status) */
#define MMPC_ERR_NOT_SETUP (-5)   /* NULL or destroyed context */

/* Boundary rows per axis (the boundary set C_b,l of Eq. boundary):
 *   x:   x(0), xdot(0), xddot(0), xdot(T), xddot(T)        (terminal x free)
 *   y:   y(0), ydot(0), yddot(0), y(T), ydot(T), yddot(T)
 *   psi: psi(0), psidot(0), psi(T), psidot(T)
 * with values x(0) = 0, xdot(0) = v0 cos psi0, xddot(0) = acc0 cos psi0,
 * xdot(T) = v_g, xddot(T) = a_g; y(0) = y0, ydot(0) = v0 sin psi0,
 * yddot(0) = acc0 sin psi0, y(T) = y_g, ydot(T) = yddot(T) = 0;
 * psi(0) = psi0 and zero heading rate at both ends and heading at T. */
#define MMPC_NEQ_X 5
#define MMPC_NEQ_Y 6
#define MMPC_NEQ_PSI 4

/* Supported sizes of this build. */
#define MMPC_MIN_N 8
#define MMPC_MAX_N 512      /* time samples (one GPU thread per sample) */
#define MMPC_MIN_COEF 7     /* six y boundary rows need at least 7 coefficients */
#define MMPC_MAX_COEF 16    /* coefficients per axis */
#define MMPC_MAX_OBST 1024  /* obstacles per scene */

/* Meta-cost kinds (Sec. III-F). */
#define MMPC_META_CRUISE 0 /* Eq. cruise_cost: sum_t (v(t) - v_ref)^2 */
#define MMPC_META_HSRL 1   /* Eq. hsrl_cost:  sum_t w1 (v(t) - v_ref)^2 + w2 (y(t) - y_ref)^2 */
#define MMPC_META_ABS 2    /* sum_t w1 |v(t) - v_ref| + w2 |y(t) - y_ref| */

typedef struct {
    double T;        /* horizon [s] > 0 */
    int N;           /* time samples t_i = i T / (N - 1), MMPC_MIN_N..MMPC_MAX_N */
    int n;           /* basis functions per axis, MMPC_MIN_COEF..MMPC_MAX_COEF */
    double rho;      /* penalty rho_xy of Eq. aug_cost, > 0 (one value for every block) */
    double a, b;     /* obstacle ellipse semi-axes incl. inflation [m], Eq. coll_nonhol_standar */
    double v_min;    /* speed bounds of Eq. v_bound, 0 < v_min <= v_max [m/s] */
    double v_max;
    double a_max;    /* acceleration bound of Eq. v_bound, > 0 [m/s^2] */
    int iters;       /* maximum AM iterations of Algorithm 1, >= 0 */
    float tol;       /* early exit: a trajectory stops once max(r_obs, r_acc, r_nh) <= tol
                        (residual definitions at mmpc_solve); <= 0 disables */
    int check_every; /* residuals are formed after iterations k with k % check_every == 0
                        and after the last one; >= 1 */
    int cull;        /* 1: skip the obstacle-sample pairs of Eq. split_alpha_o that are
                        provably outside the ellipse (each skipped pair contributes exactly
                        zero, so results are bit-identical to 0 = evaluate every pair) */
    int variant;     /* kernel: 1 = one time sample per thread (N <= 256), 2 = two
                        samples per thread; 0 = automatic (1 for batches of at most one
                        trajectory per SM, else 2).  Results agree to rounding. */
    float stall_tol;   /* stall stop (opt-in, <= 0 disables): at a residual check k >= 2
                          check_every, a trajectory also stops when its convergence
                          residual is above stall_tol and above stall_ratio times the
                          residual of two checks earlier (it is far from the target and
                          no longer closing in).  Not in the paper: a serving option for
                          scenes whose infeasible goals would spend the whole budget. */
    float stall_ratio; /* in (0, 1] when stall_tol > 0 */
    int precision;     /* operands of the basis products (the evaluations P c and the
                          contractions P^T e of Algorithm 1, both operands) as the
                          tensor cores would take them, FP32 accumulation:
                          MMPC_PREC_FP32 (0, the default: full FP32), MMPC_PREC_TF32 /
                          MMPC_PREC_BF16 (both operands rounded to TF32 -- 10-bit
                          significand, round to nearest, ties away -- or to BF16 --
                          7-bit, round to nearest even), MMPC_PREC_TF32_SPLIT /
                          MMPC_PREC_BF16_SPLIT (each operand as hi + lo of that type,
                          a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi).  The projections, the
                          QP steps (K11 applied as FP32 hi + lo) and the multipliers stay
                          FP32; the KKT inverse is FP64 from mmpc_build.  A study of the
                          accuracy each dtype would give (the error table of the
                          precision workload), not a faster path: the rounding runs on
                          the CUDA cores.  Other than 0 it needs the pair kernel with 128
                          threads (N in 129..256), n in 13..16 and variant 0 or 2;
                          otherwise mmpc_setup returns MMPC_ERR_INVALID_ARG. */
} mmpc_params;

#define MMPC_PREC_FP32 0
#define MMPC_PREC_TF32 1
#define MMPC_PREC_TF32_SPLIT 2
#define MMPC_PREC_BF16 3
#define MMPC_PREC_BF16_SPLIT 4

typedef struct mmpc_ctx mmpc_ctx;

/* Number of doubles of the problem buffer for N samples and n coefficients:
 *   N + 3 N n + n + 4 n^2 + 30 n.  Returns 0 for sizes out of range. */
size_t mmpc_problem_size(int N, int n);

/* Host FP64 builder of the shared matrices (Sec. III-C, Remark 1), written
 * into `buf` (host, mmpc_problem_size(N, n) doubles), in this order:
 *   t      [N]     sample times t_i = i T / (N - 1)
 *   P      [N][n]  basis (Eq. param): Bernstein polynomials of degree n - 1 on t/T
 *   Pd     [N][n]  first time derivative of the basis
 *   Pdd    [N][n]  second time derivative
 *   lin    [n]     coefficients of the function f(t) = t (P lin = t)
 *   Q      [n][n]  Pdd^T Pdd (Eq. cost_reform)
 *   K11_x  [n][n]  top-left block of Q_xy^-1 for the x axis (Eq. lin_solve_xy_1;
 *                  Q_xy is block diagonal in x and y with blocks
 *                  [[Q + rho (m P^T P + Pdd^T Pdd + Pd^T Pd), A_x^T], [A_x, 0]])
 *   K11_y  [n][n]  same for y
 *   K11_psi[n][n]  top-left block of Q_psi^-1 (Eq. lin_solve_psi_1)
 *   K12_psi[n][4]  top-right block of Q_psi^-1
 *   K12_x  [n][5]  top-right block of the x block of Q_xy^-1
 *   K12_y  [n][6]  top-right block of the y block of Q_xy^-1
 *   C0_x   [n][5]  top-right blocks of the boundary-only KKT inverses
 *   C0_y   [n][6]  (rho = 0): the cold start c0 = C0 b solves
 *   C0_psi [n][4]  min 1/2 c^T Q c s.t. A c = b
 * for a scene with m obstacles (the xy blocks depend on m through F^T F).
 * Returns MMPC_OK, MMPC_ERR_INVALID_ARG or MMPC_ERR_SHAPE; on a singular KKT
 * matrix MMPC_ERR_INVALID_ARG. */
int mmpc_build(const mmpc_params* p, int m, double* buf, size_t buf_len);

/* Stages a problem buffer (layout of mmpc_build; a caller may supply its own
 * basis and inverses in that layout) for scenes with exactly m obstacles:
 * converts to FP32 (the K11_x and K11_y blocks as hi + lo FP32 pairs) and
 * copies to device memory owned by the new context.  Synchronous.
 * *out is NULL on failure. */
int mmpc_setup(const mmpc_params* p, int m, const double* buf, size_t buf_len, mmpc_ctx** out);

/* Algorithm 1 (Sec. III-E) for a batch of B goals in one scene, K iterations
 * (p->iters) or fewer with early exit:
 *   ego      device float[4]      y0, v0, psi0, acc0 (x0 = 0); v0 > 0
 *   obst     device float[m][4]   x0, y0, vx, vy of each obstacle at t = 0;
 *                                 predicted at constant velocity (m must equal
 *                                 the m of mmpc_setup; may be NULL when m = 0)
 *   goals    device float[B][3]   y_g, v_g, a_g at t = T
 *   warm_coef device float[B][3n] or NULL: initial c_x, c_y, c_psi; NULL =
 *                                 cold start (boundary-only QP, C0 above)
 *   warm_lam device float[B][3n] or NULL: initial multipliers (NULL = 0)
 *   coef_out device float[B][3n]  final c_x, c_y, c_psi
 *   lam_out  device float[B][3n] or NULL: final lambda_x, lambda_y, lambda_psi
 *   resid_out device float[B][4] or NULL: residual norms after the last
 *                                 iteration, Euclidean norms of the blocks of
 *                                 F c - g (Eq. nonconvex_reform):
 *                                 [0] obstacle rows [m], [1] acceleration rows
 *                                 [m/s^2], [2] non-holonomic rows [m/s], and
 *                                 [3] the heading surrogate atan2(ydot, xdot) -
 *                                 P c_psi [rad]
 *   iters_out device int[B] or NULL: iterations run per trajectory
 *   stream   cudaStream_t or NULL
 * B = 0 enqueues nothing.  Output buffers must not alias inputs. */
int mmpc_solve(mmpc_ctx* ctx, const float* ego, const float* obst, int m, const float* goals, int B,
               const float* warm_coef, const float* warm_lam, float* coef_out, float* lam_out,
               float* resid_out, int* iters_out, void* stream);

typedef struct {
    int kind;          /* MMPC_META_* */
    float w1, w2;      /* weights >= 0 (w1 unused by MMPC_META_CRUISE) */
    float v_ref;       /* cruise speed (CRUISE, ABS) or maximum speed (HSRL) [m/s] */
    float y_ref;       /* lateral reference, e.g. the right lane centre [m] */
    float psi_max;     /* heading restriction (Sec. III assumption 2) [rad]: a
                          trajectory with |P c_psi| > psi_max at any sample gets
                          cost +inf; <= 0 disables */
} mmpc_meta;

/* Meta cost of every trajectory (Sec. III-F) on the N samples, with
 * v(t) = |(Pd c_x, Pd c_y)| and y(t) = P c_y, and the batch argmin:
 *   meta       host mmpc_meta
 *   coef       device float[B][3n] (as written by mmpc_solve)
 *   cost_out   device float[B]; NaN costs are written as +inf
 *   argmin_out device int[1]: lowest cost, lowest index on ties; -1 if every
 *              cost is +inf or B = 0 */
int mmpc_score(mmpc_ctx* ctx, const mmpc_meta* meta, const float* coef, int B, float* cost_out,
               int* argmin_out, void* stream);

/* One MPC step through host memory (Sec. III: solve the batch, score it,
 * take the best): copies ego [4], obst [m][4] and goals [B][3] from host
 * buffers into device buffers the context owns, runs mmpc_solve (cold start)
 * and mmpc_score on `stream`, copies coef [B][3n], resid [B][4] (may be
 * NULL), cost [B] and argmin [1] back to host buffers, and waits for the
 * stream.  Host buffers should be page-locked for the copies to run
 * asynchronously; when ego, obst and goals are contiguous in that order in
 * host memory the inputs go in one copy, and when coef, resid and cost are
 * contiguous in that order the outputs come back in one copy.  The device buffers grow on demand: the first call with a
 * larger B allocates (after synchronising the stream), later calls allocate
 * nothing.  m must be the m of mmpc_setup.  Errors as mmpc_solve / mmpc_score,
 * and MMPC_ERR_TIMEOUT (read and cleared as by mmpc_status) when a bounded
 * device wait of the step expired: the outputs are then not valid. */
int mmpc_step_host(mmpc_ctx* ctx, const mmpc_meta* meta, const float* ego, const float* obst, int m,
                   const float* goals, int B, float* coef_out, float* resid_out, float* cost_out, int* argmin_out,
                   void* stream);

/* ---- Batches of scenes ---------------------------------------------------
 * Many independent scenes (MPC problems of different vehicles, or of one
 * vehicle at different times) solved and scored together: one persistent
 * launch of the solve kernel over all (scene, trajectory) items, one scoring
 * launch and a per-scene argmin.  Each scene has its own context, so scenes
 * may differ in N and m (and in the other parameters); all contexts must have
 * n <= 12, or all n > 12. */
typedef struct {
    mmpc_ctx* ctx;       /* the scene's problem; ctx->m obstacles */
    const float* ego;    /* device float[4], as for mmpc_solve */
    const float* obst;   /* device float[m][4] */
    const float* goals;  /* device float[B][3] */
    int B;               /* goals of this scene, >= 0 */
    float* coef_out;     /* device float[B][3n] */
    float* lam_out;      /* device float[B][3n] or NULL */
    float* resid_out;    /* device float[B][4] or NULL */
    int* iters_out;      /* device int[B] or NULL */
    float* cost_out;     /* device float[B]: meta costs */
    int* argmin_out;     /* device int[1]: argmin as mmpc_score */
    const float* warm_coef;  /* device float[B][3n] initial c, or NULL (cold start), as mmpc_solve */
    const float* warm_lam;   /* device float[B][3n] initial lambda, or NULL (zero) */
} mmpc_scene;

typedef struct mmpc_batch mmpc_batch;

/* Creates a batch over S scene descriptors (copied; the device buffers they
 * point to must stay valid) scored with one meta cost.  Allocates the
 * batch's device tables once; mmpc_batch_run then allocates nothing and can
 * be captured in a CUDA graph.  Synchronous. */
int mmpc_batch_create(const mmpc_scene* scenes, int S, const mmpc_meta* meta, mmpc_batch** out);

/* Schedule of the solve: 1-3 are one persistent launch sized for the
 * longest horizon, taking (scene, trajectory) items scene by scene as given
 * (1), scenes by decreasing work per trajectory N (m + 32) (2), or
 * round-robin over the scenes of 2, one trajectory of each at a time (3);
 * 4 groups the scenes by horizon (the CTA size ceil(N / 2) rounded up to
 * whole warps) and runs one right-sized persistent launch per group, on
 * streams forked from and joined back to the run's stream, so that no warp
 * idles through a shorter horizon.  5 runs the tensor-core kernel (one
 * persistent launch over 32-goal items of every scene; also the fallback) and
 * needs one context of variant 3 for every scene; such a batch starts with 5,
 * any other with 1.  Schedules 1-4 run the FP32 kernel (for a variant 3
 * context its rows are FP32).  Other values -> MMPC_ERR_INVALID_ARG.
 * Synchronous. */
int mmpc_batch_set_schedule(mmpc_batch* b, int schedule);

/* Times the schedules the batch can run (1-4, and 5 when it can run on the
 * tensor cores; a warm-up and two timed runs each, on `stream`), keeps the
 * fastest and writes it to *chosen (may be NULL).  The choice is cached per
 * batch signature (each scene's goal count, N, n, m and warm start, in
 * order, and the kernel family) for the life of the process: a later batch
 * of the same signature takes it without timing.  Synchronous. */
int mmpc_batch_autotune(mmpc_batch* b, void* stream, int* chosen);

/* One persistent solve launch of a batch's current schedule (what
 * mmpc_batch_autotune chose, or mmpc_batch_set_schedule set). */
typedef struct {
    int kernel;        /* 0 the FP32 pair kernel (one CTA per trajectory), 1 the tensor-core kernel */
    int threads;       /* threads per CTA */
    int grid;          /* persistent CTAs */
    int smem_bytes;    /* dynamic shared memory per CTA */
    int trajectories;  /* goals the launch solves */
} mmpc_launch_shape;

/* The solve launches mmpc_batch_run enqueues in the current schedule: one
 * for schedules 1-3 and 5, one per horizon group for schedule 4 (CTA size
 * ceil(N / 2) rounded up to whole warps).  *schedule receives the schedule
 * and *launches the count (either may be NULL); the first min(count, max)
 * shapes go to out (may be NULL when max is 0).  Host-side, no device call
 * except a device attribute query. */
int mmpc_batch_describe(mmpc_batch* b, int* schedule, int* launches, mmpc_launch_shape* out, int max);

/* Solves and scores every scene of the batch on `stream` (asynchronous).
 * With the fallback on, the trajectories of warm-started scenes whose
 * convergence residual (largest of resid_out[0..2]) missed the scene's
 * tol > 0 are solved again from the cold start, in a second persistent
 * launch over a list built on the device, before scoring; their outputs
 * (coef, lam, resid, iters) are those of the cold solve. */
int mmpc_batch_run(mmpc_batch* b, void* stream);

/* Fallback to the cold start (see mmpc_batch_run): mode 0 off (the
 * default), 1 every warm-started trajectory that missed tol, 2 only the
 * misses that ran the whole iteration budget -- a miss that the opt-in stall
 * rule (mmpc_params.stall_tol / stall_ratio) stopped earlier is kept as it
 * is, because its residual trace showed it far from the target and no longer
 * closing in (without the stall rule mode 2 equals mode 1) -- and 3 only the
 * near misses among those of mode 2: convergence residual at most near x
 * tol (mmpc_batch_set_fallback_near, default 5), re-solved on the FP32
 * pair kernel also in a tensor-core batch (one CTA per trajectory suits a
 * few misses per scene).  A NaN residual always falls back.  Modes 2 and 3 are not in the paper.  Needs resid_out (and,
 * for modes 2 and 3, iters_out) of the warm-started scenes.  Other modes ->
 * MMPC_ERR_INVALID_ARG. */
int mmpc_batch_set_fallback(mmpc_batch* b, int on);

/* The near-miss factor of fallback mode 3 (finite, >= 1; default 5):
 * MMPC_ERR_INVALID_ARG otherwise. */
int mmpc_batch_set_fallback_near(mmpc_batch* b, float near);

/* Optional timing of the solve launches inside mmpc_batch_run: events[0..3]
 * (cudaEvent_t, created by the caller with timing enabled) are recorded on
 * the run's stream before and after the persistent solve launch(es) (with
 * schedule 4: before the fork and after the join of the horizon-group
 * streams) and before and after the fallback solve launch.  NULL turns
 * timing off (the default).  The events are the caller's; set NULL before
 * destroying them.  Recording inside a graph capture is not supported:
 * turn timing off before capturing. */
int mmpc_batch_set_timing(mmpc_batch* b, void* const* events);

/* After a run (synchronises the device): the number of trajectories the
 * last run solved again from the cold start. */
int mmpc_batch_fallbacks(mmpc_batch* b, int* count);

/* After a run (synchronises the device): each scene's completion time in ms
 * since the run's first CTA started (host float[S], may be NULL), and the
 * largest of them. */
int mmpc_batch_times(mmpc_batch* b, float* scene_ms, float* makespan_ms);

/* Frees the batch (synchronises the device first).  NULL is a no-op. */
void mmpc_batch_destroy(mmpc_batch* b);

/* Number of obstacle-sample pairs (Eq. split_alpha_o) the solve kernels of
 * this context evaluated since the last call, summed over iterations and
 * trajectories (m N per trajectory-iteration without culling).  Synchronises
 * the device, writes the count to *elements (host) and resets it. */
int mmpc_take_work_count(mmpc_ctx* ctx, unsigned long long* elements);

/* Device-side failures of the solves on this context since the last call.
 * Every wait of the solve kernels is bounded: the staging of the constants
 * (a TMA bulk copy completing an mbarrier) gives up after about 0.2 s,
 * records the expiry in the context's error word, waits once more (again
 * bounded) so that no copy is left in flight, and the CTA then returns
 * without writing its trajectory's outputs.  mmpc_status synchronises
 * `stream` (a cudaStream_t as void*, NULL = the legacy default stream),
 * reads and clears the word, and returns MMPC_ERR_TIMEOUT if a wait expired,
 * else MMPC_OK (MMPC_ERR_NOT_SETUP for a NULL context, MMPC_ERR_CUDA if the
 * synchronisation or the copy fails).  The context stays usable. */
int mmpc_status(mmpc_ctx* ctx, void* stream);

/* The same for a batch: the error words of every context its scenes use. */
int mmpc_batch_status(mmpc_batch* b, void* stream);

/* Test hook of the failure path.  With on != 0 the solves launched on this
 * context afterwards (mmpc_solve, mmpc_step_host, and batches created
 * afterwards from it) have their staging wait expect 16 bytes that no copy
 * delivers, so every CTA's wait runs out after its time limit -- a wait on
 * something nothing completes: no fault, no hang -- and mmpc_status reports
 * MMPC_ERR_TIMEOUT.  on = 0 restores normal operation.  Returns MMPC_OK, or
 * MMPC_ERR_NOT_SETUP for a NULL context. */
int mmpc_debug_expire_wait(mmpc_ctx* ctx, int on);

/* Frees the context's device memory (synchronises the device first).  NULL is a no-op. */
void mmpc_destroy(mmpc_ctx* ctx);

/* Message of the last failing call on ctx (or, when ctx is NULL, of the last
 * failing call that takes no context: mmpc_setup, mmpc_build and
 * mmpc_score_static).  Never NULL. */
const char* mmpc_last_error(const mmpc_ctx* ctx);

/* Allocation-free scoring, for callers that cannot allocate device memory
 * once they run: a hard real-time control loop that reserves all its memory at
 * start-up, or a host framework that hands out device memory only from its
 * own pool.  The paper has no counterpart; this is the computation of
 * mmpc_score without a context:
 *   meta       host mmpc_meta
 *   N, n       samples and coefficients per axis (same ranges as mmpc_params)
 *   P, Pd      device float[N][n]: the basis and its first derivative (e.g. the
 *              P and Pd sections of an mmpc_build buffer cast to float)
 *   coef, B, cost_out, argmin_out: as in mmpc_score; 0 <= B <= MMPC_STATIC_SCORE_MAX_B,
 *              larger B -> MMPC_ERR_SHAPE
 * Its scratch (8 bytes per 8 trajectories plus 8, at most 64 KiB) is a
 * file-scope device array of the library, held by every GPU that loads it
 * until the process exits, and shared by all calls: calls whose work overlaps
 * on the GPU race and must be serialised by the caller.  It calls no
 * cudaMalloc or cudaFree.  The first call on a device looks up the array's
 * address (cudaGetSymbolAddress, with that device current) and keeps it for
 * the life of the process; make that first call before any stream capture.
 * The kept address belongs to the device's primary context: after
 * cudaDeviceReset (or anything else that destroys that context) the library
 * must not be called through this entry point again in the same process. */
#define MMPC_STATIC_SCORE_MAX_B 65536
int mmpc_score_static(const mmpc_meta* meta, int N, int n, const float* P, const float* Pd, const float* coef,
                      int B, float* cost_out, int* argmin_out, void* stream);

/* ABI version of this header (2: mmpc_params.precision). */
int mmpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MMPC_H */
