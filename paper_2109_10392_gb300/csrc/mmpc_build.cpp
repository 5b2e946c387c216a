// Host FP64 builder of the shared matrices of the batch optimizer (Sec. III-B
// Eq. param, Sec. III-C, Remark 1, and the KKT systems of Sec. III-E Eqs.
// lin_solve_xy_1 and lin_solve_psi_1).  Everything here runs once per
// (T, N, n, rho, m) on the host; the GPU only ever multiplies by the results.
//
// The basis is the Bernstein basis of degree n-1 on tau = t/T, evaluated by
// the de Casteljau recurrence B_{k,q} = (1-tau) B_{k,q-1} + tau B_{k-1,q-1};
// its derivatives follow from d/dtau B_{k,q} = q (B_{k-1,q-1} - B_{k,q-1}).
// The KKT inverses come from an LU factorisation with partial pivoting.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mmpc.h"
#include "mmpc_internal.h"

namespace {

// Bernstein values B_{k,q}(tau) for all degrees q <= p, tab[q][k].
std::vector<std::vector<double>> bernstein_table(int p, double tau)
{
    std::vector<std::vector<double>> tab(p + 1);
    tab[0] = {1.0};
    for (int q = 1; q <= p; ++q) {
        tab[q].assign(q + 1, 0.0);
        for (int k = 0; k <= q; ++k) {
            double left = (k <= q - 1) ? tab[q - 1][k] : 0.0;
            double down = (k >= 1) ? tab[q - 1][k - 1] : 0.0;
            tab[q][k] = (1.0 - tau) * left + tau * down;
        }
    }
    return tab;
}

double get(const std::vector<double>& row, int k) { return (k >= 0 && k < (int)row.size()) ? row[k] : 0.0; }

// In-place LU factorisation with partial pivoting of the dim x dim matrix A.
bool lu_factor(std::vector<double>& A, int dim, std::vector<int>& piv)
{
    piv.resize(dim);
    for (int k = 0; k < dim; ++k) {
        int best = k;
        for (int r = k + 1; r < dim; ++r)
            if (std::fabs(A[r * dim + k]) > std::fabs(A[best * dim + k])) best = r;
        piv[k] = best;
        if (A[best * dim + k] == 0.0) return false;
        if (best != k)
            for (int c = 0; c < dim; ++c) std::swap(A[k * dim + c], A[best * dim + c]);
        for (int r = k + 1; r < dim; ++r) {
            double f = A[r * dim + k] / A[k * dim + k];
            A[r * dim + k] = f;
            for (int c = k + 1; c < dim; ++c) A[r * dim + c] -= f * A[k * dim + c];
        }
    }
    return true;
}

void lu_solve(const std::vector<double>& LU, int dim, const std::vector<int>& piv, std::vector<double>& x)
{
    for (int k = 0; k < dim; ++k) std::swap(x[k], x[piv[k]]);
    for (int r = 1; r < dim; ++r)
        for (int c = 0; c < r; ++c) x[r] -= LU[r * dim + c] * x[c];
    for (int r = dim - 1; r >= 0; --r) {
        for (int c = r + 1; c < dim; ++c) x[r] -= LU[r * dim + c] * x[c];
        x[r] /= LU[r * dim + r];
    }
}

// Inverse of the KKT matrix [[M, A^T], [A, 0]] (n + ne square); returns the
// top-left n x n block in K11 and the top-right n x ne block in K12.
bool kkt_blocks(const std::vector<double>& M, const std::vector<double>& A, int n, int ne, double* K11, double* K12)
{
    int dim = n + ne;
    std::vector<double> K(dim * dim, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) K[i * dim + j] = M[i * n + j];
    for (int r = 0; r < ne; ++r)
        for (int k = 0; k < n; ++k) {
            K[(n + r) * dim + k] = A[r * n + k];
            K[k * dim + n + r] = A[r * n + k];
        }
    std::vector<int> piv;
    if (!lu_factor(K, dim, piv)) return false;
    std::vector<double> col(dim);
    for (int j = 0; j < dim; ++j) {  // column j of the inverse
        std::fill(col.begin(), col.end(), 0.0);
        col[j] = 1.0;
        lu_solve(K, dim, piv, col);
        for (int i = 0; i < n; ++i) {
            if (j < n) K11[i * n + j] = col[i];
            else K12[i * ne + (j - n)] = col[i];
        }
    }
    return true;
}

// C = X^T Y for X, Y of N rows and n columns.
void gram(const double* X, const double* Y, int N, int n, std::vector<double>& C)
{
    C.assign(n * n, 0.0);
    for (int t = 0; t < N; ++t)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) C[i * n + j] += X[t * n + i] * Y[t * n + j];
}

}  // namespace

namespace mmpc {

bool sizes_ok(int N, int n)
{
    return N >= MMPC_MIN_N && N <= MMPC_MAX_N && n >= MMPC_MIN_COEF && n <= MMPC_MAX_COEF;
}

ProblemLayout layout(int N, int n)
{
    ProblemLayout L{};
    size_t o = 0;
    L.t = o; o += N;
    L.P = o; o += (size_t)N * n;
    L.Pd = o; o += (size_t)N * n;
    L.Pdd = o; o += (size_t)N * n;
    L.lin = o; o += n;
    L.Q = o; o += (size_t)n * n;
    L.K11x = o; o += (size_t)n * n;
    L.K11y = o; o += (size_t)n * n;
    L.K11p = o; o += (size_t)n * n;
    L.K12p = o; o += (size_t)n * MMPC_NEQ_PSI;
    L.K12x = o; o += (size_t)n * MMPC_NEQ_X;
    L.K12y = o; o += (size_t)n * MMPC_NEQ_Y;
    L.C0x = o; o += (size_t)n * MMPC_NEQ_X;
    L.C0y = o; o += (size_t)n * MMPC_NEQ_Y;
    L.C0p = o; o += (size_t)n * MMPC_NEQ_PSI;
    L.total = o;
    return L;
}

std::string check_params(const mmpc_params* p)
{
    if (!p) return "params is NULL";
    if (!sizes_ok(p->N, p->n)) return "N or n out of the supported range";
    if (!(p->T > 0.0) || !std::isfinite(p->T)) return "horizon T must be positive";
    if (!(p->rho > 0.0) || !std::isfinite(p->rho)) return "rho must be positive";
    if (!(p->a > 0.0) || !(p->b > 0.0) || !std::isfinite(p->a) || !std::isfinite(p->b))
        return "ellipse semi-axes must be positive";
    if (!(p->v_min > 0.0) || !(p->v_max >= p->v_min) || !std::isfinite(p->v_max)) return "need 0 < v_min <= v_max";
    if (!(p->a_max > 0.0) || !std::isfinite(p->a_max)) return "a_max must be positive";
    if (p->iters < 0) return "iters must be >= 0";
    if (p->check_every < 1) return "check_every must be >= 1";
    if (std::isnan(p->tol)) return "tol is NaN";
    if (p->variant < 0 || p->variant > 3) return "variant must be 0, 1, 2 or 3";
    if (std::isnan(p->stall_tol)) return "stall_tol is NaN";
    if (p->stall_tol > 0.f && !(p->stall_ratio > 0.f && p->stall_ratio <= 1.f)) return "stall_ratio must be in (0, 1]";
    if (p->precision < MMPC_PREC_FP32 || p->precision > MMPC_PREC_BF16_SPLIT) return "unknown precision";
    if (p->variant == 3) {
        if (p->precision == MMPC_PREC_FP32) return "variant 3 (tensor cores) needs a TF32 or BF16 precision";
        if (p->N > 256) return "variant 3 needs N <= 256";
    } else if (p->precision != MMPC_PREC_FP32 && (p->N < 129 || p->N > 256 || p->n < 13 || p->variant == 1)) {
        return "precision variants need N in 129..256, n in 13..16 and the pair kernel";
    }
    if (p->variant == 1 && p->N > 256) return "variant 1 needs N <= 256";
    return "";
}

}  // namespace mmpc

extern "C" size_t mmpc_problem_size(int N, int n)
{
    if (!mmpc::sizes_ok(N, n)) return 0;
    return mmpc::layout(N, n).total;
}

extern "C" int mmpc_build(const mmpc_params* p, int m, double* buf, size_t buf_len)
{
    std::string err = mmpc::check_params(p);
    if (!err.empty()) {
        mmpc::set_global_error(err);
        return (p && !mmpc::sizes_ok(p->N, p->n)) ? MMPC_ERR_SHAPE : MMPC_ERR_INVALID_ARG;
    }
    if (m < 0 || m > MMPC_MAX_OBST) { mmpc::set_global_error("m out of range"); return MMPC_ERR_SHAPE; }
    const int N = p->N, n = p->n, deg = n - 1;
    const mmpc::ProblemLayout L = mmpc::layout(N, n);
    if (!buf || buf_len < L.total) { mmpc::set_global_error("problem buffer missing or too small"); return MMPC_ERR_INVALID_ARG; }
    std::memset(buf, 0, sizeof(double) * L.total);
    const double T = p->T;
    double* t = buf + L.t;
    double* P = buf + L.P;
    double* Pd = buf + L.Pd;
    double* Pdd = buf + L.Pdd;
    for (int i = 0; i < N; ++i) {
        double tau = (double)i / (double)(N - 1);
        t[i] = T * tau;
        auto tab = bernstein_table(deg, tau);
        for (int k = 0; k < n; ++k) {
            P[i * n + k] = tab[deg][k];
            Pd[i * n + k] = deg / T * (get(tab[deg - 1], k - 1) - get(tab[deg - 1], k));
            Pdd[i * n + k] = deg * (deg - 1) / (T * T) *
                             (get(tab[deg - 2], k - 2) - 2.0 * get(tab[deg - 2], k - 1) + get(tab[deg - 2], k));
        }
    }
    for (int k = 0; k < n; ++k) buf[L.lin + k] = T * (double)k / (double)deg;

    std::vector<double> PtP, PdtPd, PddtPdd;
    gram(P, P, N, n, PtP);
    gram(Pd, Pd, N, n, PdtPd);
    gram(Pdd, Pdd, N, n, PddtPdd);
    for (int i = 0; i < n * n; ++i) buf[L.Q + i] = PddtPdd[i];

    // Boundary rows (the reading documented in mmpc.h).
    const double* P0 = P;       const double* PT = P + (size_t)(N - 1) * n;
    const double* Pd0 = Pd;     const double* PdT = Pd + (size_t)(N - 1) * n;
    const double* Pdd0 = Pdd;   const double* PddT = Pdd + (size_t)(N - 1) * n;
    std::vector<double> Ax, Ay, Ap;
    for (const double* r : {P0, Pd0, Pdd0, PdT, PddT}) Ax.insert(Ax.end(), r, r + n);
    for (const double* r : {P0, Pd0, Pdd0, PT, PdT, PddT}) Ay.insert(Ay.end(), r, r + n);
    for (const double* r : {P0, Pd0, PT, PdT}) Ap.insert(Ap.end(), r, r + n);

    // Per-axis block of Q + rho F^T F: F stacks P m times, Pdd and Pd (Sec. III-C).
    std::vector<double> Mxy(n * n), Mp(n * n), Q0(n * n);
    for (int i = 0; i < n * n; ++i) {
        Mxy[i] = PddtPdd[i] + p->rho * (m * PtP[i] + PddtPdd[i] + PdtPd[i]);
        Mp[i] = PddtPdd[i] + p->rho * PtP[i];
        Q0[i] = PddtPdd[i];
    }
    bool ok = kkt_blocks(Mxy, Ax, n, MMPC_NEQ_X, buf + L.K11x, buf + L.K12x) &&
              kkt_blocks(Mxy, Ay, n, MMPC_NEQ_Y, buf + L.K11y, buf + L.K12y) &&
              kkt_blocks(Mp, Ap, n, MMPC_NEQ_PSI, buf + L.K11p, buf + L.K12p);
    std::vector<double> scratch(n * n);
    ok = ok && kkt_blocks(Q0, Ax, n, MMPC_NEQ_X, scratch.data(), buf + L.C0x) &&
         kkt_blocks(Q0, Ay, n, MMPC_NEQ_Y, scratch.data(), buf + L.C0y) &&
         kkt_blocks(Q0, Ap, n, MMPC_NEQ_PSI, scratch.data(), buf + L.C0p);
    if (!ok) { mmpc::set_global_error("singular KKT matrix"); return MMPC_ERR_INVALID_ARG; }
    return MMPC_OK;
}
