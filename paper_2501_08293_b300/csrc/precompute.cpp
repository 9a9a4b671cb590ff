// FP64 precompute of the closed-form local operators (Eq. closed_2) with
// the row reduction of Section IV-B done by a rank-revealing factorization.
//
// For a component with rows A_s (m x n) and right-hand side b_s:
//   Householder QR with column pivoting of A_s^T:  A_s^T Pi = Q R.
//   The rank r is the number of pivots above 1e-10 * (largest row norm); the
//   rows Pi(0..r-1) are a maximal independent subset of A_s (the rows the
//   row reduction keeps) and Q1 = Q(:, 0..r-1) spans the row space.
//   Then A^T (A A^T)^{-1} A = Q1 Q1^T for the reduced rows, so
//       P_s    = I - Q1 Q1^T           (= -Abar_s, projector onto null(A_s))
//       bbar_s = Q1 R11^{-T} b_I       (= A^T (A A^T)^{-1} b, the minimum-norm
//                                        solution of A_s x = b_s)
//   and the dropped rows must be satisfied by bbar_s, otherwise the local
//   system is inconsistent (the paper's 0 = b, b != 0 row).
// This gives the same P_s and bbar_s as row reduction + Cholesky of
// A A^T (both are unique), with better conditioning for nearly dependent rows.
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace opf {

Operator make_operator(const Component& C) {
    const int n = C.n();
    const int m = C.m;
    Operator op;
    op.n = n;
    op.P.assign((size_t)n * n, 0.0);
    op.bbar.assign(n, 0.0);
    for (int i = 0; i < n; ++i) op.P[(size_t)i * n + i] = 1.0;
    if (m == 0) return op;

    // M = A^T, column-major n x m: M[i + j*n] = A[j*n + i]
    std::vector<double> M((size_t)n * m);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < n; ++i) M[i + (size_t)j * n] = C.A[(size_t)j * n + i];
    std::vector<int> perm(m);
    for (int j = 0; j < m; ++j) perm[j] = j;
    std::vector<double> cn(m);
    double cmax = 0.0;
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += M[i + (size_t)j * n] * M[i + (size_t)j * n];
        cn[j] = s;
        cmax = std::max(cmax, std::sqrt(s));
    }
    const double tol = 1e-10 * std::max(cmax, 1e-300);
    std::vector<double> tau;
    int r = 0;
    const int kmax = std::min(n, m);
    for (int k = 0; k < kmax; ++k) {
        // pivot: the remaining column with the largest norm (recomputed exactly)
        int best = k;
        double bn = -1.0;
        for (int j = k; j < m; ++j) {
            double s = 0.0;
            for (int i = k; i < n; ++i) s += M[i + (size_t)j * n] * M[i + (size_t)j * n];
            cn[j] = s;
            if (s > bn) { bn = s; best = j; }
        }
        if (std::sqrt(bn) <= tol) break;
        if (best != k) {
            for (int i = 0; i < n; ++i) std::swap(M[i + (size_t)k * n], M[i + (size_t)best * n]);
            std::swap(perm[k], perm[best]);
        }
        // Householder vector for column k, rows k..n-1
        double* col = &M[(size_t)k * n];
        double alpha = std::sqrt(bn);
        if (col[k] > 0) alpha = -alpha;
        double v0 = col[k] - alpha;
        // v = [1, col[k+1..]/v0], beta = -v0/alpha
        double t = -v0 / alpha;
        for (int i = k + 1; i < n; ++i) col[i] /= v0;
        col[k] = alpha;   // R_kk
        tau.push_back(t);
        // apply H = I - t v v^T to the remaining columns
        for (int j = k + 1; j < m; ++j) {
            double* cj = &M[(size_t)j * n];
            double s = cj[k];
            for (int i = k + 1; i < n; ++i) s += col[i] * cj[i];
            s *= t;
            cj[k] -= s;
            for (int i = k + 1; i < n; ++i) cj[i] -= s * col[i];
        }
        ++r;
    }
    op.m_reduced = r;
    if (r == 0) {
        for (int j = 0; j < m; ++j)
            if (std::fabs(C.b[j]) > 1e-9 * 1.0)
                throw Error(OPF_ERR_INCONSISTENT, "component " + std::to_string(C.index) + ": 0 = b with b != 0");
        return op;
    }
    // Q1 = H_0 ... H_{r-1} [I_r; 0]  (n x r, column-major)
    std::vector<double> Q((size_t)n * r, 0.0);
    for (int j = 0; j < r; ++j) Q[j + (size_t)j * n] = 1.0;
    for (int k = r - 1; k >= 0; --k) {
        const double* v = &M[(size_t)k * n];   // v[k] = 1 implicit, v[k+1..] stored
        for (int j = 0; j < r; ++j) {
            double* qj = &Q[(size_t)j * n];
            double s = qj[k];
            for (int i = k + 1; i < n; ++i) s += v[i] * qj[i];
            s *= tau[k];
            qj[k] -= s;
            for (int i = k + 1; i < n; ++i) qj[i] -= s * v[i];
        }
    }
    // P = I - Q1 Q1^T
    for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int j = 0; j < r; ++j) s += Q[a + (size_t)j * n] * Q[c + (size_t)j * n];
            op.P[(size_t)a * n + c] = (a == c ? 1.0 : 0.0) - s;
        }
    // symmetrize exactly (P is symmetric in exact arithmetic)
    for (int a = 0; a < n; ++a)
        for (int c = a + 1; c < n; ++c) {
            double s = 0.5 * (op.P[(size_t)a * n + c] + op.P[(size_t)c * n + a]);
            op.P[(size_t)a * n + c] = s;
            op.P[(size_t)c * n + a] = s;
        }
    // R11^T y = b_I  (R11 upper triangular r x r stored in M's upper part)
    std::vector<double> y(r);
    for (int i = 0; i < r; ++i) {
        double s = C.b[perm[i]];
        for (int j = 0; j < i; ++j) s -= M[j + (size_t)i * n] * y[j];   // R[j][i] = M[j + i*n]
        const double d = M[i + (size_t)i * n];
        if (d == 0.0 || !std::isfinite(d))
            throw Error(OPF_ERR_NUMERIC, "component " + std::to_string(C.index) + ": singular reduced rows");
        y[i] = s / d;
    }
    for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int j = 0; j < r; ++j) s += Q[a + (size_t)j * n] * y[j];
        op.bbar[a] = s;
    }
    // consistency of every row (kept rows to rounding, dropped rows = row reduction's 0 = b test)
    double bmax = 1.0;
    for (int j = 0; j < m; ++j) bmax = std::max(bmax, std::fabs(C.b[j]));
    for (int j = 0; j < m; ++j) {
        double s = -C.b[j];
        for (int i = 0; i < n; ++i) s += C.A[(size_t)j * n + i] * op.bbar[i];
        if (std::fabs(s) > 1e-9 * bmax)
            throw Error(OPF_ERR_INCONSISTENT, "component " + std::to_string(C.index) +
                                                  ": rows have no common solution (residual " + std::to_string(s) + ")");
    }
    return op;
}

}  // namespace opf
