/*
 * FP64 CPU oracle of the batch non-holonomic trajectory optimizer of
 * Adajania et al., "Multi-Modal Model Predictive Control through Batch
 * Non-Holonomic Trajectory Optimization" (arXiv 2109.10392).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The product
 * (the CUDA path behind include/mmpc.h) never loads, links or imports it, and
 * the two share no code: this file builds its own basis, its own matrices and
 * its own inverses.
 *
 * What it computes, in the paper's order and notation:
 *   - basis matrices P, Pdot, Pddot (Eq. param, Sec. III-B), Bernstein
 *     polynomials of degree n-1 on tau = t/T (the paper only says "e.g.
 *     polynomials");
 *   - the matrices of the multi-convex reformulation (Sec. III-C): Q, A, the
 *     stacked F = blockdiag([F_o; Pddot; Pdot], [F_o; Pddot; Pdot]) with F_o =
 *     P stacked m times, all MATERIALISED, as printed;
 *   - the KKT matrices Q_xy (Eq. lin_solve_xy_1) and Q_psi (Eq.
 *     lin_solve_psi_1), inverted once by Gauss-Jordan elimination with
 *     partial pivoting;
 *   - Algorithm 1 for every trajectory l of the batch: the c_xy QP (Eq.
 *     split_xy / lin_solve_xy_2), the c_psi QP with the atan2 surrogate (Eq.
 *     split_psi / lin_solve_psi_2), the velocity closed form (Eq. v_update),
 *     alpha and d (Eq. split_alpha_o), alpha_a and d_a (Eq. split_alpha_a),
 *     and the multiplier update (Sec. III-E, "Multiplier Update");
 *   - the meta costs of Sec. III-F (Eq. cruise_cost, Eq. hsrl_cost) with the
 *     heading restriction of Sec. III (assumption 2) and the batch argmin.
 *
 * Every auxiliary variable (alpha, d, alpha_a, d_a, v) is stored explicitly
 * and every trigonometric function is called as written.  Readings of points
 * the paper leaves open are marked "READING:" where they are used.
 *
 * Parity status per function (what pins it, in tests/test_oracle_*.py):
 *   orc_bernstein       pinned: partition of unity, endpoint interpolation,
 *                       polynomial reproduction, finite differences.
 *   orc_invert          pinned: A * inv(A) = I on random and KKT matrices.
 *   orc_qp_xy/psi       pinned: A c = b to 1e-9; equal to a null-space
 *                       least-squares solve built from the cost itself.
 *   orc_project_*       pinned: brute-force sampling on tiny inputs.
 *   orc_solve           pinned by invariants (fixed point, mirror,
 *                       translation, permutation, far obstacles, residual
 *                       decrease on obstacle-free scenes); the exact
 *                       trajectories on obstacle-dense scenes are parity
 *                       unpinned (the paper prints no worked example).
 *   orc_meta_cost       pinned: brute-force evaluation from coefficients.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_SINGULAR (-2)
#define ORC_ERR_NOMEM (-3)

/* Number of boundary rows per axis (READING of the boundary set C_b,l, which
 * the paper does not spell out, Eq. boundary):
 *   x:   x(0), xdot(0), xddot(0), xdot(T), xddot(T)          (x(T) free)
 *   y:   y(0), ydot(0), yddot(0), y(T), ydot(T), yddot(T)
 *   psi: psi(0), psidot(0), psi(T), psidot(T)                                */
#define NEQ_X 5
#define NEQ_Y 6
#define NEQ_XY (NEQ_X + NEQ_Y)
#define NEQ_PSI 4

typedef struct {
    double T;      /* horizon [s] */
    int N;         /* time samples */
    int n;         /* basis functions per axis */
    double rho;    /* penalty rho_xy (one value for every block) */
    double a, b;   /* ellipse semi-axes (inflated), Eq. coll_nonhol_standar */
    double v_min, v_max, a_max;
    int iters;     /* maximum AM iterations ("maxiter" of Algorithm 1) */
    double tol;    /* early-exit tolerance on the residual; <= 0: none */
    int check_every;      /* residual checked after iterations k*check_every */
    int psi_sign_printed; /* 1: lambda_psi update with the printed sign */
    int basis_bits;       /* > 0: the basis operands (P, Pdot, Pddot and F) are rounded to this
                             many significant bits (8: bfloat16, 11: TF32, 24: float32) after the
                             KKT inverses are formed, to emulate reduced-precision operands of
                             the contractions; 0: exact (the default) */
    int basis_split;      /* 1: operands held as hi + lo, each rounded to basis_bits */
} orc_params;

/* ------------------------------------------------------------------------ */
/* small dense linear algebra, row-major                                    */
/* ------------------------------------------------------------------------ */

/* y = A x, A is r x c */
static void matvec(const double* A, int r, int c, const double* x, double* y)
{
    for (int i = 0; i < r; ++i) {
        double s = 0.0;
        for (int j = 0; j < c; ++j) s += A[(size_t)i * c + j] * x[j];
        y[i] = s;
    }
}

/* y = A^T x, A is r x c */
static void mattvec(const double* A, int r, int c, const double* x, double* y)
{
    for (int j = 0; j < c; ++j) y[j] = 0.0;
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) y[j] += A[(size_t)i * c + j] * x[i];
}

/* C = A^T B, A is r x p, B is r x q, C is p x q */
static void mattmat(const double* A, const double* B, int r, int p, int q, double* C)
{
    for (int i = 0; i < p * q; ++i) C[i] = 0.0;
    for (int k = 0; k < r; ++k)
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < q; ++j) C[i * q + j] += A[(size_t)k * p + i] * B[(size_t)k * q + j];
}

/* Gauss-Jordan elimination with partial pivoting: Ainv = A^-1 (dim x dim). */
int orc_invert(int dim, const double* A, double* Ainv)
{
    if (dim <= 0 || !A || !Ainv) return ORC_ERR_ARG;
    int w = 2 * dim;
    double* M = (double*)malloc(sizeof(double) * dim * w);
    if (!M) return ORC_ERR_NOMEM;
    for (int i = 0; i < dim; ++i) {
        for (int j = 0; j < dim; ++j) M[i * w + j] = A[i * dim + j];
        for (int j = 0; j < dim; ++j) M[i * w + dim + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int col = 0; col < dim; ++col) {
        int piv = col;
        double best = fabs(M[col * w + col]);
        for (int r = col + 1; r < dim; ++r)
            if (fabs(M[r * w + col]) > best) { best = fabs(M[r * w + col]); piv = r; }
        if (best == 0.0) { free(M); return ORC_ERR_SINGULAR; }
        if (piv != col)
            for (int j = 0; j < w; ++j) { double t = M[col * w + j]; M[col * w + j] = M[piv * w + j]; M[piv * w + j] = t; }
        double inv = 1.0 / M[col * w + col];
        for (int j = 0; j < w; ++j) M[col * w + j] *= inv;
        for (int r = 0; r < dim; ++r) {
            if (r == col) continue;
            double f = M[r * w + col];
            if (f == 0.0) continue;
            for (int j = 0; j < w; ++j) M[r * w + j] -= f * M[col * w + j];
        }
    }
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) Ainv[i * dim + j] = M[i * w + dim + j];
    free(M);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. param: trajectory parameterisation                                   */
/* ------------------------------------------------------------------------ */

static double binom(int p, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(p - k + i) / (double)i;
    return r;
}

/* Bernstein polynomial B_{k,p}(tau); zero outside 0 <= k <= p. */
static double bern(int k, int p, double tau)
{
    if (k < 0 || k > p || p < 0) return 0.0;
    return binom(p, k) * pow(tau, (double)k) * pow(1.0 - tau, (double)(p - k));
}

/* READING: time grid t_i = i T / (N-1), i = 0..N-1 (endpoints included),
 * and a Bernstein basis of degree p = n-1 on tau = t/T.  Row i of P holds the
 * n basis functions at t_i; Pd and Pdd hold their first and second time
 * derivatives (textbook Bernstein derivative identities). */
int orc_bernstein(int N, int n, double T, double* P, double* Pd, double* Pdd)
{
    if (N < 2 || n < 3 || !(T > 0.0) || !P || !Pd || !Pdd) return ORC_ERR_ARG;
    int p = n - 1;
    for (int i = 0; i < N; ++i) {
        double tau = (double)i / (double)(N - 1);
        for (int k = 0; k < n; ++k) {
            P[i * n + k] = bern(k, p, tau);
            Pd[i * n + k] = (double)p / T * (bern(k - 1, p - 1, tau) - bern(k, p - 1, tau));
            Pdd[i * n + k] = (double)p * (double)(p - 1) / (T * T) *
                             (bern(k - 2, p - 2, tau) - 2.0 * bern(k - 1, p - 2, tau) + bern(k, p - 2, tau));
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-C: matrices of the multi-convex reformulation                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_params p;
    int m;               /* obstacles */
    int N, n;
    int rows_axis;       /* (m+2) N: rows of [F_o; Pddot; Pdot] */
    int dim_xy, dim_psi; /* KKT sizes */
    double *t, *P, *Pd, *Pdd;
    double* Q;           /* n x n: Pddot^T Pddot */
    double* F;           /* 2 rows_axis x 2n, block diagonal (as printed) */
    double* Axy;         /* NEQ_XY x 2n, block diagonal */
    double* Apsi;        /* NEQ_PSI x n */
    double* Kxy_inv;     /* Q_xy^-1, Eq. lin_solve_xy_1 */
    double* Kpsi_inv;    /* Q_psi^-1, Eq. lin_solve_psi_1 */
    double* K0xy_inv;    /* cold-start (boundary-only) KKT inverses */
    double* K0psi_inv;
} orc_problem;

static void prob_free(orc_problem* pr)
{
    free(pr->t); free(pr->P); free(pr->Pd); free(pr->Pdd); free(pr->Q); free(pr->F);
    free(pr->Axy); free(pr->Apsi); free(pr->Kxy_inv); free(pr->Kpsi_inv);
    free(pr->K0xy_inv); free(pr->K0psi_inv);
    memset(pr, 0, sizeof(*pr));
}

static int params_ok(const orc_params* p)
{
    if (!p) return 0;
    if (p->N < 2 || p->n < 7 || !(p->T > 0.0)) return 0; /* 6 y boundary rows need n >= 7 */
    if (!(p->rho > 0.0) || !(p->a > 0.0) || !(p->b > 0.0)) return 0;
    if (!(p->v_min > 0.0) || !(p->v_max >= p->v_min) || !(p->a_max > 0.0)) return 0;
    if (p->iters < 0) return 0;
    return 1;
}

/* x rounded to k significant bits, ties to even (the rounding of a float
 * with a k-bit significand: 8 for bfloat16, 11 for TF32, 24 for float32;
 * exponent range unlimited). */
double orc_round_bits(double x, int k)
{
    if (x == 0.0 || !isfinite(x) || k <= 0) return x;
    int e;
    const double m = frexp(x, &e); /* x = m 2^e, 0.5 <= |m| < 1 */
    return ldexp(nearbyint(ldexp(m, k)), e - k);
}

static double round_operand(double x, int k, int split)
{
    const double hi = orc_round_bits(x, k);
    return split ? hi + orc_round_bits(x - hi, k) : hi;
}

static int prob_build(const orc_params* p, int m, orc_problem* pr)
{
    memset(pr, 0, sizeof(*pr));
    if (!params_ok(p) || m < 0) return ORC_ERR_ARG;
    pr->p = *p;
    pr->m = m;
    int N = p->N, n = p->n;
    pr->N = N; pr->n = n;
    pr->rows_axis = (m + 2) * N;
    pr->dim_xy = 2 * n + NEQ_XY;
    pr->dim_psi = n + NEQ_PSI;
    size_t Nn = (size_t)N * n;
    pr->t = (double*)malloc(sizeof(double) * N);
    pr->P = (double*)malloc(sizeof(double) * Nn);
    pr->Pd = (double*)malloc(sizeof(double) * Nn);
    pr->Pdd = (double*)malloc(sizeof(double) * Nn);
    pr->Q = (double*)malloc(sizeof(double) * n * n);
    pr->F = (double*)calloc((size_t)2 * pr->rows_axis * 2 * n, sizeof(double));
    pr->Axy = (double*)calloc((size_t)NEQ_XY * 2 * n, sizeof(double));
    pr->Apsi = (double*)calloc((size_t)NEQ_PSI * n, sizeof(double));
    pr->Kxy_inv = (double*)malloc(sizeof(double) * pr->dim_xy * pr->dim_xy);
    pr->Kpsi_inv = (double*)malloc(sizeof(double) * pr->dim_psi * pr->dim_psi);
    pr->K0xy_inv = (double*)malloc(sizeof(double) * pr->dim_xy * pr->dim_xy);
    pr->K0psi_inv = (double*)malloc(sizeof(double) * pr->dim_psi * pr->dim_psi);
    if (!pr->t || !pr->P || !pr->Pd || !pr->Pdd || !pr->Q || !pr->F || !pr->Axy || !pr->Apsi ||
        !pr->Kxy_inv || !pr->Kpsi_inv || !pr->K0xy_inv || !pr->K0psi_inv) {
        prob_free(pr);
        return ORC_ERR_NOMEM;
    }
    for (int i = 0; i < N; ++i) pr->t[i] = p->T * (double)i / (double)(N - 1);
    orc_bernstein(N, n, p->T, pr->P, pr->Pd, pr->Pdd);

    /* Eq. cost_reform: sum_t xddot^2 = c^T (Pddot^T Pddot) c, for x, y and psi. */
    mattmat(pr->Pdd, pr->Pdd, N, n, n, pr->Q);

    /* F = blockdiag([F_o; Pddot; Pdot], same), F_o = P stacked m times
     * (Sec. III-C and the matrix-representation paragraph of Sec. III-B). */
    int W = 2 * n;
    for (int blk = 0; blk < 2; ++blk) {
        int r0 = blk * pr->rows_axis, c0 = blk * n;
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < N; ++i)
                for (int k = 0; k < n; ++k)
                    pr->F[(size_t)(r0 + j * N + i) * W + c0 + k] = pr->P[i * n + k];
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < n; ++k) {
                pr->F[(size_t)(r0 + m * N + i) * W + c0 + k] = pr->Pdd[i * n + k];
                pr->F[(size_t)(r0 + (m + 1) * N + i) * W + c0 + k] = pr->Pd[i * n + k];
            }
    }

    /* Boundary rows (READING above), Eq. eq_reform. */
    const double* P0 = pr->P;              const double* PT = pr->P + (size_t)(N - 1) * n;
    const double* Pd0 = pr->Pd;            const double* PdT = pr->Pd + (size_t)(N - 1) * n;
    const double* Pdd0 = pr->Pdd;          const double* PddT = pr->Pdd + (size_t)(N - 1) * n;
    const double* rx[NEQ_X] = {P0, Pd0, Pdd0, PdT, PddT};
    const double* ry[NEQ_Y] = {P0, Pd0, Pdd0, PT, PdT, PddT};
    const double* rp[NEQ_PSI] = {P0, Pd0, PT, PdT};
    for (int r = 0; r < NEQ_X; ++r)
        for (int k = 0; k < n; ++k) pr->Axy[r * W + k] = rx[r][k];
    for (int r = 0; r < NEQ_Y; ++r)
        for (int k = 0; k < n; ++k) pr->Axy[(NEQ_X + r) * W + n + k] = ry[r][k];
    for (int r = 0; r < NEQ_PSI; ++r)
        for (int k = 0; k < n; ++k) pr->Apsi[r * n + k] = rp[r][k];

    /* Q_xy = [[Qxy + rho F^T F, A^T], [A, 0]]   (Eq. lin_solve_xy_1)
     * Q_psi = [[Q + rho P^T P, A^T], [A, 0]]     (Eq. lin_solve_psi_1)
     * and the same two with rho = 0 for the cold start. */
    int Dx = pr->dim_xy, Dp = pr->dim_psi;
    double* FtF = (double*)malloc(sizeof(double) * W * W);
    double* PtP = (double*)malloc(sizeof(double) * n * n);
    double* Kx = (double*)calloc((size_t)Dx * Dx, sizeof(double));
    double* Kp = (double*)calloc((size_t)Dp * Dp, sizeof(double));
    if (!FtF || !PtP || !Kx || !Kp) { free(FtF); free(PtP); free(Kx); free(Kp); prob_free(pr); return ORC_ERR_NOMEM; }
    mattmat(pr->F, pr->F, 2 * pr->rows_axis, W, W, FtF);
    mattmat(pr->P, pr->P, N, n, n, PtP);
    int rc = ORC_OK;
    for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
        double rho = (pass == 0) ? p->rho : 0.0;
        memset(Kx, 0, sizeof(double) * Dx * Dx);
        memset(Kp, 0, sizeof(double) * Dp * Dp);
        for (int i = 0; i < W; ++i)
            for (int j = 0; j < W; ++j) {
                double q = 0.0;
                if (i / n == j / n) q = pr->Q[(i % n) * n + (j % n)]; /* blockdiag(Q, Q) */
                Kx[i * Dx + j] = q + rho * FtF[i * W + j];
            }
        for (int r = 0; r < NEQ_XY; ++r)
            for (int k = 0; k < W; ++k) {
                Kx[(W + r) * Dx + k] = pr->Axy[r * W + k];
                Kx[k * Dx + W + r] = pr->Axy[r * W + k];
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Kp[i * Dp + j] = pr->Q[i * n + j] + rho * PtP[i * n + j];
        for (int r = 0; r < NEQ_PSI; ++r)
            for (int k = 0; k < n; ++k) {
                Kp[(n + r) * Dp + k] = pr->Apsi[r * n + k];
                Kp[k * Dp + n + r] = pr->Apsi[r * n + k];
            }
        rc = orc_invert(Dx, Kx, pass == 0 ? pr->Kxy_inv : pr->K0xy_inv);
        if (rc == ORC_OK) rc = orc_invert(Dp, Kp, pass == 0 ? pr->Kpsi_inv : pr->K0psi_inv);
    }
    free(FtF); free(PtP); free(Kx); free(Kp);
    if (rc == ORC_OK && p->basis_bits > 0) {
        /* reduced-precision operands of the contractions (evaluations and
         * transposed products); the KKT inverses stay exact */
        const size_t Nn = (size_t)N * n, nf = (size_t)2 * pr->rows_axis * 2 * n;
        for (size_t q = 0; q < Nn; ++q) {
            pr->P[q] = round_operand(pr->P[q], p->basis_bits, p->basis_split);
            pr->Pd[q] = round_operand(pr->Pd[q], p->basis_bits, p->basis_split);
            pr->Pdd[q] = round_operand(pr->Pdd[q], p->basis_bits, p->basis_split);
        }
        for (size_t q = 0; q < nf; ++q) pr->F[q] = round_operand(pr->F[q], p->basis_bits, p->basis_split);
    }
    if (rc != ORC_OK) prob_free(pr);
    return rc;
}

/* READING of the boundary values: ego = (y0, v0, psi0, acc0) with x0 = 0 and
 * the initial heading rate taken as 0; goal = (y_g, v_g, a_g) at t = T with
 * heading 0 (Sec. I: goals are end-of-horizon position / velocity /
 * acceleration tuples).  The scalar acceleration acc0 acts along psi0. */
static void boundary_values(const double* ego, const double* goal, double* bxy, double* bpsi)
{
    double y0 = ego[0], v0 = ego[1], psi0 = ego[2], acc0 = ego[3];
    double yg = goal[0], vg = goal[1], ag = goal[2];
    /* x */
    bxy[0] = 0.0;
    bxy[1] = v0 * cos(psi0);
    bxy[2] = acc0 * cos(psi0);
    bxy[3] = vg;
    bxy[4] = ag;
    /* y */
    bxy[5] = y0;
    bxy[6] = v0 * sin(psi0);
    bxy[7] = acc0 * sin(psi0);
    bxy[8] = yg;
    bxy[9] = 0.0;
    bxy[10] = 0.0;
    /* psi */
    bpsi[0] = psi0;
    bpsi[1] = 0.0;
    bpsi[2] = 0.0;
    bpsi[3] = 0.0;
}

int orc_boundary(const double* ego, const double* goal, double* bxy, double* bpsi)
{
    if (!ego || !goal || !bxy || !bpsi) return ORC_ERR_ARG;
    boundary_values(ego, goal, bxy, bpsi);
    return ORC_OK;
}

/* Copies of the oracle's own matrices, for the tests. */
int orc_matrices(const orc_params* p, int m, double* P, double* Pd, double* Pdd, double* Q,
                 double* F, double* Axy, double* Apsi, double* Kxy_inv, double* Kpsi_inv,
                 double* K0xy_inv, double* K0psi_inv)
{
    orc_problem pr;
    int rc = prob_build(p, m, &pr);
    if (rc != ORC_OK) return rc;
    size_t Nn = (size_t)pr.N * pr.n;
    if (P) memcpy(P, pr.P, sizeof(double) * Nn);
    if (Pd) memcpy(Pd, pr.Pd, sizeof(double) * Nn);
    if (Pdd) memcpy(Pdd, pr.Pdd, sizeof(double) * Nn);
    if (Q) memcpy(Q, pr.Q, sizeof(double) * pr.n * pr.n);
    if (F) memcpy(F, pr.F, sizeof(double) * (size_t)2 * pr.rows_axis * 2 * pr.n);
    if (Axy) memcpy(Axy, pr.Axy, sizeof(double) * NEQ_XY * 2 * pr.n);
    if (Apsi) memcpy(Apsi, pr.Apsi, sizeof(double) * NEQ_PSI * pr.n);
    if (Kxy_inv) memcpy(Kxy_inv, pr.Kxy_inv, sizeof(double) * pr.dim_xy * pr.dim_xy);
    if (Kpsi_inv) memcpy(Kpsi_inv, pr.Kpsi_inv, sizeof(double) * pr.dim_psi * pr.dim_psi);
    if (K0xy_inv) memcpy(K0xy_inv, pr.K0xy_inv, sizeof(double) * pr.dim_xy * pr.dim_xy);
    if (K0psi_inv) memcpy(K0psi_inv, pr.K0psi_inv, sizeof(double) * pr.dim_psi * pr.dim_psi);
    prob_free(&pr);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-E: the steps of Algorithm 1                                     */
/* ------------------------------------------------------------------------ */

/* Step (split_xy), Eq. lin_solve_xy_1/2:
 *   [c_x; c_y; mu] = Q_xy^-1 [rho F^T g + lambda_xy; b]. */
static void step_xy(const orc_problem* pr, const double* g, const double* lam, const double* bxy,
                    double* Ftg, double* q, double* sol)
{
    int W = 2 * pr->n, D = pr->dim_xy;
    mattvec(pr->F, 2 * pr->rows_axis, W, g, Ftg);
    for (int i = 0; i < W; ++i) q[i] = pr->p.rho * Ftg[i] + lam[i];
    for (int r = 0; r < NEQ_XY; ++r) q[W + r] = bxy[r];
    matvec(pr->Kxy_inv, D, D, q, sol);
}

/* Step (split_psi), Eq. lin_solve_psi_1/2:
 *   [c_psi; mu] = Q_psi^-1 [rho P^T atan2(ydot, xdot) + lambda_psi; b_psi]. */
static void step_psi(const orc_problem* pr, const double* theta, const double* lam_psi,
                     const double* bpsi, double* Ptth, double* q, double* sol)
{
    int n = pr->n, D = pr->dim_psi;
    mattvec(pr->P, pr->N, n, theta, Ptth);
    for (int i = 0; i < n; ++i) q[i] = pr->p.rho * Ptth[i] + lam_psi[i];
    for (int r = 0; r < NEQ_PSI; ++r) q[n + r] = bpsi[r];
    matvec(pr->Kpsi_inv, D, D, q, sol);
}

/* Eq. v_update: v = clip(sqrt(xdot^2 + ydot^2), v_min, v_max). */
double orc_velocity(double xdot, double ydot, double v_min, double v_max)
{
    double v = sqrt(xdot * xdot + ydot * ydot);
    if (v < v_min) v = v_min;
    if (v > v_max) v = v_max;
    return v;
}

/* Eq. split_alpha_o.  First part: the printed closed form
 *   alpha = atan2(a (y - xi_y), b (x - xi_x)).
 * Second part: for that alpha, the unconstrained minimiser over d of
 *   (w_x - a d cos alpha)^2 + (w_y - b d sin alpha)^2
 * is d = (a w_x cos alpha + b w_y sin alpha) / (a^2 cos^2 alpha + b^2 sin^2 alpha);
 * READING: it is then clipped to d >= 1 (the paper's text says "[0 1]", which
 * contradicts the constraint d >= 1 of Eq. sphere_proposed and Eq.
 * split_alpha_o; the constraint wins).  At w = 0, atan2(0, 0) = 0 and d = 1. */
void orc_project_obstacle(double wx, double wy, double a, double b, double* alpha, double* d)
{
    double al = atan2(a * wy, b * wx);
    double ca = cos(al), sa = sin(al);
    double num = a * wx * ca + b * wy * sa;
    double den = a * a * ca * ca + b * b * sa * sa;
    double dd = num / den;
    if (dd < 1.0) dd = 1.0;
    *alpha = al;
    *d = dd;
}

/* Eq. split_alpha_a ("same structure"): alpha_a = atan2(yddot, xddot);
 * the unconstrained minimiser over d_a given alpha_a is
 * xddot cos alpha_a + yddot sin alpha_a, then clipped to d_a <= a_max. */
void orc_project_accel(double xdd, double ydd, double a_max, double* alpha_a, double* d_a)
{
    double al = atan2(ydd, xdd);
    double dd = xdd * cos(al) + ydd * sin(al);
    if (dd > a_max) dd = a_max;
    *alpha_a = al;
    *d_a = dd;
}

/* Public single steps, for the tests. */
int orc_qp_xy(const orc_params* p, int m, const double* g, const double* lam, const double* bxy,
              double* c, double* mu)
{
    orc_problem pr;
    int rc = prob_build(p, m, &pr);
    if (rc != ORC_OK) return rc;
    int W = 2 * pr.n;
    double* Ftg = (double*)malloc(sizeof(double) * W);
    double* q = (double*)malloc(sizeof(double) * pr.dim_xy);
    double* sol = (double*)malloc(sizeof(double) * pr.dim_xy);
    if (!Ftg || !q || !sol) { free(Ftg); free(q); free(sol); prob_free(&pr); return ORC_ERR_NOMEM; }
    step_xy(&pr, g, lam, bxy, Ftg, q, sol);
    memcpy(c, sol, sizeof(double) * W);
    if (mu) memcpy(mu, sol + W, sizeof(double) * NEQ_XY);
    free(Ftg); free(q); free(sol);
    prob_free(&pr);
    return ORC_OK;
}

int orc_qp_psi(const orc_params* p, const double* theta, const double* lam_psi, const double* bpsi,
               double* c, double* mu)
{
    orc_problem pr;
    int rc = prob_build(p, 0, &pr);
    if (rc != ORC_OK) return rc;
    double* Ptth = (double*)malloc(sizeof(double) * pr.n);
    double* q = (double*)malloc(sizeof(double) * pr.dim_psi);
    double* sol = (double*)malloc(sizeof(double) * pr.dim_psi);
    if (!Ptth || !q || !sol) { free(Ptth); free(q); free(sol); prob_free(&pr); return ORC_ERR_NOMEM; }
    step_psi(&pr, theta, lam_psi, bpsi, Ptth, q, sol);
    memcpy(c, sol, sizeof(double) * pr.n);
    if (mu) memcpy(mu, sol + pr.n, sizeof(double) * NEQ_PSI);
    free(Ptth); free(q); free(sol);
    prob_free(&pr);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 for one trajectory                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* trajectory-sized work arrays */
    double *cxy, *cpsi, *lam_xy, *lam_psi;          /* 2n, n, 2n, n */
    double *x, *y, *xd, *yd, *xdd, *ydd, *psi, *theta; /* N each */
    double *v, *alpha_a, *d_a;                      /* N each */
    double *alpha, *d;                              /* m N each */
    double *g, *Fc, *r, *Ftr;                       /* 2(m+2)N, 2(m+2)N, 2(m+2)N, 2n */
    double *Ftg, *qxy, *solxy, *Ptth, *qpsi, *solpsi, *tmp;
} orc_work;

static void work_free(orc_work* w)
{
    double** f = (double**)w;
    for (size_t i = 0; i < sizeof(orc_work) / sizeof(double*); ++i) free(f[i]);
    memset(w, 0, sizeof(*w));
}

static int work_alloc(const orc_problem* pr, orc_work* w)
{
    memset(w, 0, sizeof(*w));
    int N = pr->N, n = pr->n, m = pr->m;
    size_t G = (size_t)2 * pr->rows_axis;
    size_t mN = (size_t)m * N > 0 ? (size_t)m * N : 1;
    w->cxy = (double*)calloc(2 * n, sizeof(double));
    w->cpsi = (double*)calloc(n, sizeof(double));
    w->lam_xy = (double*)calloc(2 * n, sizeof(double));
    w->lam_psi = (double*)calloc(n, sizeof(double));
    w->x = (double*)calloc(N, sizeof(double));
    w->y = (double*)calloc(N, sizeof(double));
    w->xd = (double*)calloc(N, sizeof(double));
    w->yd = (double*)calloc(N, sizeof(double));
    w->xdd = (double*)calloc(N, sizeof(double));
    w->ydd = (double*)calloc(N, sizeof(double));
    w->psi = (double*)calloc(N, sizeof(double));
    w->theta = (double*)calloc(N, sizeof(double));
    w->v = (double*)calloc(N, sizeof(double));
    w->alpha_a = (double*)calloc(N, sizeof(double));
    w->d_a = (double*)calloc(N, sizeof(double));
    w->alpha = (double*)calloc(mN, sizeof(double));
    w->d = (double*)calloc(mN, sizeof(double));
    w->g = (double*)calloc(G, sizeof(double));
    w->Fc = (double*)calloc(G, sizeof(double));
    w->r = (double*)calloc(G, sizeof(double));
    w->Ftr = (double*)calloc(2 * n, sizeof(double));
    w->Ftg = (double*)calloc(2 * n, sizeof(double));
    w->qxy = (double*)calloc(pr->dim_xy, sizeof(double));
    w->solxy = (double*)calloc(pr->dim_xy, sizeof(double));
    w->Ptth = (double*)calloc(n, sizeof(double));
    w->qpsi = (double*)calloc(pr->dim_psi, sizeof(double));
    w->solpsi = (double*)calloc(pr->dim_psi, sizeof(double));
    w->tmp = (double*)calloc(N > 2 * n ? N : 2 * n, sizeof(double));
    double** f = (double**)w;
    for (size_t i = 0; i < sizeof(orc_work) / sizeof(double*); ++i)
        if (!f[i]) { work_free(w); return ORC_ERR_NOMEM; }
    return ORC_OK;
}

/* Trajectory samples from the coefficients (Eq. param and its derivatives). */
static void evaluate(const orc_problem* pr, orc_work* w)
{
    int N = pr->N, n = pr->n;
    const double* cx = w->cxy;
    const double* cy = w->cxy + n;
    matvec(pr->P, N, n, cx, w->x);
    matvec(pr->P, N, n, cy, w->y);
    matvec(pr->Pd, N, n, cx, w->xd);
    matvec(pr->Pd, N, n, cy, w->yd);
    matvec(pr->Pdd, N, n, cx, w->xdd);
    matvec(pr->Pdd, N, n, cy, w->ydd);
    matvec(pr->P, N, n, w->cpsi, w->psi);
}

/* Eqs. split_v, split_alpha_o, split_alpha_a for the current coefficients:
 * the velocity, obstacle and acceleration auxiliaries. */
static void update_aux(const orc_problem* pr, const double* obst, orc_work* w)
{
    const orc_params* p = &pr->p;
    int N = pr->N, m = pr->m;
    for (int i = 0; i < N; ++i) w->v[i] = orc_velocity(w->xd[i], w->yd[i], p->v_min, p->v_max);
    /* Sec. III assumption 3: constant-velocity obstacle prediction. */
    for (int j = 0; j < m; ++j) {
        const double* o = obst + 4 * j;
        for (int i = 0; i < N; ++i) {
            double xi_x = o[0] + o[2] * pr->t[i];
            double xi_y = o[1] + o[3] * pr->t[i];
            orc_project_obstacle(w->x[i] - xi_x, w->y[i] - xi_y, p->a, p->b,
                                 &w->alpha[j * N + i], &w->d[j * N + i]);
        }
    }
    for (int i = 0; i < N; ++i) orc_project_accel(w->xdd[i], w->ydd[i], p->a_max, &w->alpha_a[i], &w->d_a[i]);
}

/* g_l of Sec. III-C, stacked as printed:
 * [xi_x + a d cos alpha; d_a cos alpha_a; v cos(P c_psi);
 *  xi_y + b d sin alpha; d_a sin alpha_a; v sin(P c_psi)]. */
static void assemble_g(const orc_problem* pr, const double* obst, orc_work* w)
{
    const orc_params* p = &pr->p;
    int N = pr->N, m = pr->m, R = pr->rows_axis;
    for (int j = 0; j < m; ++j) {
        const double* o = obst + 4 * j;
        for (int i = 0; i < N; ++i) {
            double xi_x = o[0] + o[2] * pr->t[i];
            double xi_y = o[1] + o[3] * pr->t[i];
            double al = w->alpha[j * N + i], dd = w->d[j * N + i];
            w->g[j * N + i] = xi_x + p->a * dd * cos(al);
            w->g[R + j * N + i] = xi_y + p->b * dd * sin(al);
        }
    }
    for (int i = 0; i < N; ++i) {
        w->g[m * N + i] = w->d_a[i] * cos(w->alpha_a[i]);
        w->g[(m + 1) * N + i] = w->v[i] * cos(w->psi[i]);
        w->g[R + m * N + i] = w->d_a[i] * sin(w->alpha_a[i]);
        w->g[R + (m + 1) * N + i] = w->v[i] * sin(w->psi[i]);
    }
}

/* Residuals of the stacked constraint F c = g (Eq. nonconvex_reform), by
 * component, as Euclidean norms (READING: the paper plots the components but
 * states no norm):
 *   [0] obstacle rows  (m)      [1] acceleration rows (m/s^2)
 *   [2] non-holonomic rows (m/s)  [3] heading surrogate theta - P c_psi (rad) */
static void residuals(const orc_problem* pr, orc_work* w, double* res)
{
    int N = pr->N, m = pr->m, R = pr->rows_axis, W = 2 * pr->n;
    matvec(pr->F, 2 * R, W, w->cxy, w->Fc);
    double so = 0.0, sa = 0.0, sv = 0.0, sp = 0.0;
    for (int blk = 0; blk < 2; ++blk) {
        const double* Fc = w->Fc + blk * R;
        const double* g = w->g + blk * R;
        for (int k = 0; k < m * N; ++k) so += (Fc[k] - g[k]) * (Fc[k] - g[k]);
        for (int k = m * N; k < (m + 1) * N; ++k) sa += (Fc[k] - g[k]) * (Fc[k] - g[k]);
        for (int k = (m + 1) * N; k < (m + 2) * N; ++k) sv += (Fc[k] - g[k]) * (Fc[k] - g[k]);
    }
    for (int i = 0; i < N; ++i) sp += (w->theta[i] - w->psi[i]) * (w->theta[i] - w->psi[i]);
    res[0] = sqrt(so);
    res[1] = sqrt(sa);
    res[2] = sqrt(sv);
    res[3] = sqrt(sp);
}

/* READING: the convergence residual in metres is the largest of the
 * obstacle, acceleration (x 1 s^2) and non-holonomic (x 1 s) components. */
static double conv_residual(const double* res)
{
    double r = res[0];
    if (res[1] > r) r = res[1];
    if (res[2] > r) r = res[2];
    return r;
}

static void theta_from_velocity(const orc_problem* pr, orc_work* w)
{
    for (int i = 0; i < pr->N; ++i) w->theta[i] = atan2(w->yd[i], w->xd[i]);
}

/* Algorithm 1 for one trajectory.  init (3n: c_x, c_y, c_psi) and init_lam
 * (3n) replace the cold start when given. */
static int am_trajectory(const orc_problem* pr, const double* ego, const double* goal, const double* obst,
                         const double* init, const double* init_lam, double* coef, double* lam,
                         double* res_out, int* iters_out, double* trace)
{
    const orc_params* p = &pr->p;
    int n = pr->n, N = pr->N, W = 2 * n, R = pr->rows_axis;
    orc_work w;
    if (work_alloc(pr, &w) != ORC_OK) return ORC_ERR_NOMEM;
    double bxy[NEQ_XY], bpsi[NEQ_PSI], res[4];
    boundary_values(ego, goal, bxy, bpsi);

    if (init) {
        memcpy(w.cxy, init, sizeof(double) * W);
        memcpy(w.cpsi, init + W, sizeof(double) * n);
    } else {
        /* READING (cold start; the paper leaves the initialisation open):
         * the boundary-only QP min 1/2 c^T Q c s.t. A c = b, i.e. Q_xy and
         * Q_psi with rho = 0 and lambda = 0. */
        double* q0 = w.qxy;
        for (int i = 0; i < W; ++i) q0[i] = 0.0;
        for (int r = 0; r < NEQ_XY; ++r) q0[W + r] = bxy[r];
        matvec(pr->K0xy_inv, pr->dim_xy, pr->dim_xy, q0, w.solxy);
        memcpy(w.cxy, w.solxy, sizeof(double) * W);
        double* qp = w.qpsi;
        for (int i = 0; i < n; ++i) qp[i] = 0.0;
        for (int r = 0; r < NEQ_PSI; ++r) qp[n + r] = bpsi[r];
        matvec(pr->K0psi_inv, pr->dim_psi, pr->dim_psi, qp, w.solpsi);
        memcpy(w.cpsi, w.solpsi, sizeof(double) * n);
    }
    if (init_lam) {
        memcpy(w.lam_xy, init_lam, sizeof(double) * W);
        memcpy(w.lam_psi, init_lam + W, sizeof(double) * n);
    }
    /* auxiliaries of iterate 0 from c^0 */
    evaluate(pr, &w);
    theta_from_velocity(pr, &w);
    update_aux(pr, obst, &w);
    assemble_g(pr, obst, &w);
    residuals(pr, &w, res);
    if (trace) memcpy(trace, res, sizeof(res));

    int k = 0;
    while (k < p->iters) {
        /* Eq. split_xy via Eq. lin_solve_xy_2 (mu is discarded) */
        step_xy(pr, w.g, w.lam_xy, bxy, w.Ftg, w.qxy, w.solxy);
        memcpy(w.cxy, w.solxy, sizeof(double) * W);
        /* Eq. split_psi: surrogate target atan2(ydot, xdot), Eq. lin_solve_psi_2 */
        matvec(pr->Pd, N, n, w.cxy, w.xd);
        matvec(pr->Pd, N, n, w.cxy + n, w.yd);
        theta_from_velocity(pr, &w);
        step_psi(pr, w.theta, w.lam_psi, bpsi, w.Ptth, w.qpsi, w.solpsi);
        memcpy(w.cpsi, w.solpsi, sizeof(double) * n);
        /* Eqs. split_v, split_alpha_o, split_alpha_a */
        evaluate(pr, &w);
        update_aux(pr, obst, &w);
        assemble_g(pr, obst, &w);
        /* Multiplier update (Sec. III-E):
         * lambda_xy <- lambda_xy - rho F^T (F c - g^{k+1}). */
        matvec(pr->F, 2 * R, W, w.cxy, w.Fc);
        for (int i = 0; i < 2 * R; ++i) w.r[i] = w.Fc[i] - w.g[i];
        mattvec(pr->F, 2 * R, W, w.r, w.Ftr);
        for (int i = 0; i < W; ++i) w.lam_xy[i] -= p->rho * w.Ftr[i];
        /* READING of the heading multiplier: the printed update
         * lambda_psi - rho P^T (theta - P c_psi) has the opposite sign of the
         * xy update; by default the xy convention is used for both,
         * lambda_psi <- lambda_psi - rho P^T (P c_psi - theta). */
        for (int i = 0; i < N; ++i) w.tmp[i] = w.psi[i] - w.theta[i];
        if (p->psi_sign_printed)
            for (int i = 0; i < N; ++i) w.tmp[i] = -w.tmp[i];
        mattvec(pr->P, N, n, w.tmp, w.Ptth);
        for (int i = 0; i < n; ++i) w.lam_psi[i] -= p->rho * w.Ptth[i];
        ++k;
        residuals(pr, &w, res);
        if (trace) memcpy(trace + 4 * k, res, sizeof(res));
        if (p->tol > 0.0 && p->check_every > 0 && k % p->check_every == 0 && conv_residual(res) <= p->tol)
            break;
    }
    memcpy(coef, w.cxy, sizeof(double) * W);
    memcpy(coef + W, w.cpsi, sizeof(double) * n);
    if (lam) {
        memcpy(lam, w.lam_xy, sizeof(double) * W);
        memcpy(lam + W, w.lam_psi, sizeof(double) * n);
    }
    memcpy(res_out, res, sizeof(res));
    if (iters_out) *iters_out = k;
    work_free(&w);
    return ORC_OK;
}

/* Batch solve: every trajectory l of the batch shares the scene (Sec. II
 * note: same bounds and obstacles) and differs only in its goal.
 *   ego   [4]      y0, v0, psi0, acc0 (x0 = 0)
 *   obst  [m][4]   x0, y0, vx, vy at t = 0
 *   goals [B][3]   y_g, v_g, a_g at t = T
 *   init, init_lam [B][3n] or NULL (cold start)
 *   coef_out, lam_out [B][3n] (c_x, c_y, c_psi / lambda_x, lambda_y, lambda_psi)
 *   resid_out [B][4]; iters_out [B] or NULL; trace_out [B][iters+1][4] or NULL */
int orc_solve(const orc_params* p, const double* ego, const double* obst, int m, const double* goals, int B,
              const double* init, const double* init_lam, int nthreads, double* coef_out, double* lam_out,
              double* resid_out, int* iters_out, double* trace_out)
{
    if (!params_ok(p) || !ego || (m > 0 && !obst) || m < 0 || B < 0 || (B > 0 && (!goals || !coef_out || !resid_out)))
        return ORC_ERR_ARG;
    if (B == 0) return ORC_OK;
    orc_problem pr;
    int rc = prob_build(p, m, &pr);
    if (rc != ORC_OK) return rc;
    int n3 = 3 * p->n;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int l = 0; l < B; ++l) {
        int e = am_trajectory(&pr, ego, goals + 3 * l, obst, init ? init + (size_t)l * n3 : NULL,
                              init_lam ? init_lam + (size_t)l * n3 : NULL, coef_out + (size_t)l * n3,
                              lam_out ? lam_out + (size_t)l * n3 : NULL, resid_out + 4 * (size_t)l,
                              iters_out ? iters_out + l : NULL,
                              trace_out ? trace_out + (size_t)l * (p->iters + 1) * 4 : NULL);
        if (e != ORC_OK) err = e;
    }
    (void)nthreads;
    prob_free(&pr);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Sec. III-F: meta cost and batch argmin                                   */
/* ------------------------------------------------------------------------ */

#define ORC_META_CRUISE 0 /* Eq. cruise_cost: sum_t (v - v_ref)^2 */
#define ORC_META_HSRL 1   /* Eq. hsrl_cost: sum_t w1 (v - v_ref)^2 + w2 (y - y_ref)^2 */
#define ORC_META_ABS 2    /* sum_t w1 |v - v_ref| + w2 |y - y_ref| */

/* cost_out[l]: meta cost of trajectory l, evaluated on the N samples with
 * v(t) = |(xdot, ydot)| and y(t) = P c_y.  Sec. III assumption 2 (heading
 * restriction): a trajectory with |P c_psi| > psi_max at any sample is
 * discarded (cost +inf); psi_max <= 0 disables the filter.  A NaN cost counts
 * as +inf.  argmin_out: the lowest cost, lowest index on ties, -1 when every
 * cost is +inf or B = 0. */
int orc_meta_cost(const orc_params* p, const double* coef, int B, int kind, double w1, double w2,
                  double v_ref, double y_ref, double psi_max, double* cost_out, int* argmin_out)
{
    if (!p || p->N < 2 || p->n < 3 || B < 0 || (B > 0 && (!coef || !cost_out)) || kind < 0 || kind > 2)
        return ORC_ERR_ARG;
    int N = p->N, n = p->n;
    double* P = (double*)malloc(sizeof(double) * N * n);
    double* Pd = (double*)malloc(sizeof(double) * N * n);
    double* Pdd = (double*)malloc(sizeof(double) * N * n);
    if (!P || !Pd || !Pdd) { free(P); free(Pd); free(Pdd); return ORC_ERR_NOMEM; }
    orc_bernstein(N, n, p->T, P, Pd, Pdd);
    int best = -1;
    double best_cost = INFINITY;
    for (int l = 0; l < B; ++l) {
        const double* cx = coef + (size_t)l * 3 * n;
        const double* cy = cx + n;
        const double* cp = cy + n;
        double cost = 0.0;
        int discard = 0;
        for (int i = 0; i < N; ++i) {
            double xd = 0, yd = 0, y = 0, ps = 0;
            for (int k = 0; k < n; ++k) {
                xd += Pd[i * n + k] * cx[k];
                yd += Pd[i * n + k] * cy[k];
                y += P[i * n + k] * cy[k];
                ps += P[i * n + k] * cp[k];
            }
            double v = sqrt(xd * xd + yd * yd);
            if (psi_max > 0.0 && fabs(ps) > psi_max) discard = 1;
            if (kind == ORC_META_CRUISE) cost += (v - v_ref) * (v - v_ref);
            else if (kind == ORC_META_HSRL) cost += w1 * (v - v_ref) * (v - v_ref) + w2 * (y - y_ref) * (y - y_ref);
            else cost += w1 * fabs(v - v_ref) + w2 * fabs(y - y_ref);
        }
        if (discard || isnan(cost)) cost = INFINITY;
        cost_out[l] = cost;
        if (cost < best_cost) { best_cost = cost; best = l; }
    }
    if (argmin_out) *argmin_out = best;
    free(P); free(Pd); free(Pdd);
    return ORC_OK;
}

int orc_abi_version(void) { return 1; }
