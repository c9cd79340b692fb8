// Lowest eigenpair of the Lanczos tridiagonal T (Sec. 2.2, Eq. Tmatrix):
// bisection on the Sturm sequence for the eigenvalue, then inverse iteration
// for the eigenvector, whose last component gives the residual estimate
// rho = b_{m+1} |s_m|.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace hub {

namespace {

// Number of eigenvalues of T strictly below x (Sturm count via the LDL^T
// pivots of T - x I).
int sturm_count(const double* a, const double* b, int m, double x) {
    int cnt = 0;
    double q = a[0] - x;
    const double tiny = 1e-300;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        if (std::fabs(q) < tiny) q = (q < 0 ? -tiny : tiny);
        q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// Solve (T - x I) y = r by Gaussian elimination with partial pivoting on the
// tridiagonal band (r is overwritten by y).
void tridiag_solve(const double* a, const double* b, int m, double x, std::vector<double>& r) {
    // band storage after pivoting: up to two super-diagonals
    std::vector<double> d(m), u1(m, 0.0), u2(m, 0.0), l(m, 0.0);
    std::vector<int> swp(m, 0);
    for (int i = 0; i < m; ++i) d[i] = a[i] - x;
    for (int i = 0; i + 1 < m; ++i) u1[i] = b[i];
    std::vector<double> sub(m, 0.0);
    for (int i = 0; i + 1 < m; ++i) sub[i] = b[i];
    for (int i = 0; i + 1 < m; ++i) {
        // rows i and i+1: row i = (d[i], u1[i], u2[i]); row i+1 = (sub[i], d[i+1], u1[i+1])
        if (std::fabs(sub[i]) > std::fabs(d[i])) {
            std::swap(d[i], sub[i]);
            double t1 = u1[i];
            u1[i] = d[i + 1];
            d[i + 1] = t1;
            double t2 = u2[i];
            u2[i] = u1[i + 1];
            u1[i + 1] = t2;
            std::swap(r[i], r[i + 1]);
            swp[i] = 1;
        }
        if (d[i] == 0.0) d[i] = 1e-300;
        const double f = sub[i] / d[i];
        l[i] = f;
        d[i + 1] -= f * u1[i];
        u1[i + 1] -= f * u2[i];
        r[i + 1] -= f * r[i];
    }
    if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
    for (int i = m - 1; i >= 0; --i) {
        double s = r[i];
        if (i + 1 < m) s -= u1[i] * r[i + 1];
        if (i + 2 < m) s -= u2[i] * r[i + 2];
        r[i] = s / d[i];
    }
}

// Inverse iteration for the eigenvector of T at eigenvalue x (normalised,
// written to y[0..m)).
void inverse_iteration(const double* a, const double* b, int m, double x, std::vector<double>& y) {
    const double shift = x - 1e-14 * std::max(1.0, std::fabs(x));
    y.assign(m, 1.0 / std::sqrt((double)m));
    for (int it = 0; it < 4; ++it) {
        tridiag_solve(a, b, m, shift, y);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (double& v : y) v /= nrm;
    }
}

}  // namespace

double tridiag_gap_lower(const double* a, const double* b, int m, double b_next, double theta) {
    // the next Ritz value above theta that is not a copy of it (plain Lanczos
    // repeats a converged Ritz value), and the residual estimate of its Ritz
    // pair: an eigenvalue of H lies within rho_k of theta_k
    const double copy_tol = 1e-8 * std::max(1.0, std::fabs(theta));
    std::vector<double> y;
    for (int k = 1; k < std::min(m, 16); ++k) {
        const double tk = tridiag_kth(a, b, m, k);
        if (tk - theta <= copy_tol) continue;
        inverse_iteration(a, b, m, tk, y);
        const double rho_k = std::fabs(b_next) * std::fabs(y[m - 1]);
        return (tk - rho_k) - theta;
    }
    return 0.0;
}

double tridiag_kth(const double* a, const double* b, int m, int k) {
    // k-th smallest eigenvalue (k = 0 lowest) by bisection on the Sturm count
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, m, mid) >= k + 1) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

void tridiag_lowest_vector(const double* a, const double* b, int m, double* theta, double* s) {
    double th = 0.0, last = 0.0;
    tridiag_lowest(a, b, m, &th, &last);
    *theta = th;
    if (m == 1) {
        s[0] = 1.0;
        return;
    }
    const double shift = th - 1e-14 * std::max(1.0, std::fabs(th));
    std::vector<double> y(m, 1.0 / std::sqrt((double)m));
    for (int it = 0; it < 4; ++it) {
        tridiag_solve(a, b, m, shift, y);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (double& v : y) v /= nrm;
    }
    for (int i = 0; i < m; ++i) s[i] = y[i];
}

void tridiag_lowest(const double* a, const double* b, int m, double* theta, double* s_last) {
    if (m == 1) {
        *theta = a[0];
        *s_last = 1.0;
        return;
    }
    // Gershgorin interval
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    const double span = std::max(hi - lo, 1e-300);
    // bisection for the smallest eigenvalue: count(x) >= 1 <=> x > lambda_min
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, m, mid) >= 1) hi = mid; else lo = mid;
        if (hi - lo <= 4e-16 * std::max(std::fabs(lo), std::fabs(hi)) + 1e-300 * span) break;
    }
    const double x = 0.5 * (lo + hi);
    *theta = x;
    // inverse iteration with a slightly shifted eigenvalue estimate
    const double shift = x - 1e-14 * std::max(1.0, std::fabs(x));
    std::vector<double> y(m, 1.0 / std::sqrt((double)m));
    for (int it = 0; it < 4; ++it) {
        tridiag_solve(a, b, m, shift, y);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (double& v : y) v /= nrm;
    }
    *s_last = y[m - 1];
}

}  // namespace hub
