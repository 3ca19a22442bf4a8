// eigen.cpp -- host FP64 symmetric eigendecomposition for the PCA of
// Section 3.2 (Eq. 11: W holds the eigenvectors of E[X X^T] ordered by
// descending eigenvalue).
//
// Method: Householder reduction to tridiagonal form, then implicit symmetric
// QR steps with a Wilkinson shift and deflation (the classical dense
// symmetric eigenvalue algorithm), accumulating every reflection and
// rotation into the eigenvector matrix.  O(n^3) for n <= 1024 dimensions;
// offline, runs once per index.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace dade {

namespace {

// Rotation acting on rows (or columns) i, i+1:  new_i = c a_i - s a_{i+1},
// new_{i+1} = s a_i + c a_{i+1}; chosen so that it maps (x, z) to (r, 0).
inline void givens(double x, double z, double &c, double &s) {
    if (z == 0.0) { c = 1.0; s = 0.0; return; }
    double r = std::hypot(x, z);
    c = x / r;
    s = -z / r;
}

} // namespace

bool sym_eig(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &Z) {
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    auto z = [&](int i, int j) -> double & { return Z[(size_t)i * n + j]; };
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) z(i, i) = 1.0;
    w.assign(n, 0.0);

    // ---- 1. Householder tridiagonalisation: A = Z T Z^T --------------------
    std::vector<double> v(n), p(n), ww(n);
    for (int k = 0; k + 2 < n; ++k) {
        int m = n - k - 1;                     // length of the column below the diagonal
        double xnorm = 0.0;
        for (int i = 0; i < m; ++i) xnorm += a(k + 1 + i, k) * a(k + 1 + i, k);
        xnorm = std::sqrt(xnorm);
        if (xnorm == 0.0) continue;
        double x0 = a(k + 1, k);
        double alpha = x0 >= 0.0 ? -xnorm : xnorm;    // reflect x onto alpha e_1
        for (int i = 0; i < m; ++i) v[i] = a(k + 1 + i, k);
        v[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < m; ++i) vn2 += v[i] * v[i];
        if (vn2 == 0.0) continue;
        double beta = 2.0 / vn2;               // H = I - beta v v^T
        // p = beta * A_sub v ; w = p - (beta/2)(v^T p) v ; A_sub -= v w^T + w v^T
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += a(k + 1 + i, k + 1 + j) * v[j];
            p[i] = beta * s;
        }
        double vp = 0.0;
        for (int i = 0; i < m; ++i) vp += v[i] * p[i];
        double K = 0.5 * beta * vp;
        for (int i = 0; i < m; ++i) ww[i] = p[i] - K * v[i];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) a(k + 1 + i, k + 1 + j) -= v[i] * ww[j] + ww[i] * v[j];
        a(k + 1, k) = alpha;
        a(k, k + 1) = alpha;
        for (int i = 1; i < m; ++i) { a(k + 1 + i, k) = 0.0; a(k, k + 1 + i) = 0.0; }
        // Z <- Z H (columns k+1 .. n-1)
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += z(r, k + 1 + j) * v[j];
            s *= beta;
            for (int j = 0; j < m; ++j) z(r, k + 1 + j) -= s * v[j];
        }
    }

    // ---- 2. implicit symmetric QR on the tridiagonal T (kept dense) ---------
    auto rot_rows = [&](int i, double c, double s, int j0, int j1) {
        for (int j = j0; j <= j1; ++j) {
            double x = a(i, j), y = a(i + 1, j);
            a(i, j) = c * x - s * y;
            a(i + 1, j) = s * x + c * y;
        }
    };
    auto rot_cols = [&](int i, double c, double s, int r0, int r1) {
        for (int r = r0; r <= r1; ++r) {
            double x = a(r, i), y = a(r, i + 1);
            a(r, i) = c * x - s * y;
            a(r, i + 1) = s * x + c * y;
        }
    };
    const double eps = 2.220446049250313e-16;
    // Deflation: an off-diagonal entry is negligible when it is small next to
    // its two diagonal neighbours, or at rounding level for the whole matrix
    // (the QR steps themselves reintroduce noise of size eps * ||T||).
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) {
        tnorm += a(i, i) * a(i, i);
        if (i + 1 < n) tnorm += 2.0 * a(i, i + 1) * a(i, i + 1);
    }
    const double floor_tol = 4.0 * eps * std::sqrt(tnorm);
    int hi = n - 1;
    long iters = 0;
    const long max_iters = 60L * n + 100;
    while (hi > 0) {
        // deflate negligible off-diagonal entries
        for (int i = 0; i < hi; ++i)
            if (std::fabs(a(i, i + 1)) <= eps * (std::fabs(a(i, i)) + std::fabs(a(i + 1, i + 1))) ||
                std::fabs(a(i, i + 1)) <= floor_tol) {
                a(i, i + 1) = 0.0;
                a(i + 1, i) = 0.0;
            }
        if (a(hi - 1, hi) == 0.0) { --hi; continue; }
        int lo = hi - 1;
        while (lo > 0 && a(lo - 1, lo) != 0.0) --lo;
        if (++iters > max_iters) return false;
        // Wilkinson shift from the trailing 2x2 block of T[lo..hi]
        double dd = 0.5 * (a(hi - 1, hi - 1) - a(hi, hi));
        double e = a(hi - 1, hi);
        double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * std::hypot(dd, e);
        double mu = a(hi, hi) - (den != 0.0 ? e * e / den : 0.0);
        double x = a(lo, lo) - mu, y = a(lo + 1, lo);
        for (int k = lo; k < hi; ++k) {
            double c, s;
            givens(x, y, c, s);
            int j0 = std::max(lo, k - 1), j1 = std::min(hi, k + 2);
            rot_rows(k, c, s, j0, j1);          // T <- R T
            rot_cols(k, c, s, j0, j1);          // T <- T R^T
            for (int r = 0; r < n; ++r) {       // Z <- Z R^T
                double zx = z(r, k), zy = z(r, k + 1);
                z(r, k) = c * zx - s * zy;
                z(r, k + 1) = s * zx + c * zy;
            }
            if (k + 1 < hi) { x = a(k + 1, k); y = a(k + 2, k); }
        }
    }
    // ---- 3. eigenvalues on the diagonal; sort descending ----------------------
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> diag(n);
    for (int i = 0; i < n; ++i) diag[i] = a(i, i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return diag[x] > diag[y]; });
    std::vector<double> Zs((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        w[k] = diag[order[k]];
        for (int r = 0; r < n; ++r) Zs[(size_t)r * n + k] = Z[(size_t)r * n + order[k]];
    }
    Z.swap(Zs);
    return true;
}

} // namespace dade
