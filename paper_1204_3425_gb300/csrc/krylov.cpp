// Lanczos (Krylov) time propagation, host side: the eigendecomposition of
// the Lanczos tridiagonal T_m and the coefficients of exp(-i H tau) v in the
// Lanczos basis.  The paper names time propagation as the other main use of
// its H*v kernel (Sec. 6) without giving a scheme; this is the standard short
// iterative Lanczos propagator (Park & Light 1986):
//   exp(-i H tau) v ~ |v| V_m exp(-i T_m tau) e_1,
// V_m = [f_0 .. f_{m-1}] the Lanczos vectors of Algorithm 1 started from
// v / |v|, with the a-posteriori error estimate of Saad (1992)
//   |v| b_{m+1} |e_m^T exp(-i T_m tau) e_1|.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace hub {

// Symmetric tridiagonal QR iteration with implicit Wilkinson shifts (Golub &
// Van Loan, Matrix Computations, Sec. 8.3): each step applies the rotations
// G_lo .. G_{hi-1} of one shifted QR step to the unreduced block [lo, hi]
// (chasing the bulge down the band) and to the tracked rows of the
// eigenvector matrix; off-diagonals below eps (|d_i| + |d_{i+1}|) are set to
// zero and the block shrinks from the bottom.
bool tridiag_eigen(const double* a, const double* b, int m, double* lam, double* Z, int zrows, const int* rows) {
    std::vector<double> d(a, a + m), e(std::max(m - 1, 0));
    for (int i = 0; i + 1 < m; ++i) e[(size_t)i] = b[i];
    for (int r = 0; r < zrows; ++r)
        for (int k = 0; k < m; ++k) Z[(size_t)r * m + k] = (k == rows[r]) ? 1.0 : 0.0;
    const double eps = 0x1p-53;
    int hi = m - 1, iters = 0;
    while (hi > 0) {
        for (int i = 0; i < hi; ++i)
            if (std::fabs(e[(size_t)i]) <= eps * (std::fabs(d[(size_t)i]) + std::fabs(d[(size_t)i + 1])))
                e[(size_t)i] = 0.0;
        if (e[(size_t)hi - 1] == 0.0) {
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && e[(size_t)lo - 1] != 0.0) --lo;
        if (++iters > 60 * m) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2x2 block nearer d[hi]
        const double dd = 0.5 * (d[(size_t)hi - 1] - d[(size_t)hi]);
        const double eh = e[(size_t)hi - 1];
        const double mu = d[(size_t)hi] - eh * eh / (dd + std::copysign(std::hypot(dd, eh), dd == 0.0 ? 1.0 : dd));
        double x = d[(size_t)lo] - mu, z = e[(size_t)lo];
        double bulge = 0.0;
        for (int k = lo; k < hi; ++k) {
            // rotation G = [[c, s], [-s, c]] on (k, k+1) with G^T (x, z) = (r, 0)
            const double r = std::hypot(x, z);
            const double c = r == 0.0 ? 1.0 : x / r;
            const double s = r == 0.0 ? 0.0 : -z / r;
            if (k > lo) e[(size_t)k - 1] = r;             // (k-1, k); the bulge at (k-1, k+1) is gone
            const double dk = d[(size_t)k], dk1 = d[(size_t)k + 1], ek = e[(size_t)k];
            d[(size_t)k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
            d[(size_t)k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
            e[(size_t)k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
            if (k + 1 < hi) {
                const double ek1 = e[(size_t)k + 1];
                bulge = -s * ek1;                          // new (k, k+2)
                e[(size_t)k + 1] = c * ek1;
                x = e[(size_t)k];
                z = bulge;
            }
            for (int q = 0; q < zrows; ++q) {
                double* zr = Z + (size_t)q * m;
                const double zk = zr[k], zk1 = zr[k + 1];
                zr[k] = c * zk - s * zk1;
                zr[k + 1] = s * zk + c * zk1;
            }
        }
    }
    for (int i = 0; i < m; ++i) lam[i] = d[(size_t)i];
    return true;
}

bool krylov_exp_ends(const double* a, const double* b, int m, KrylovEnds& out) {
    out.m = m;
    out.lam.assign((size_t)m, 0.0);
    out.z0.assign((size_t)m, 0.0);
    out.zl.assign((size_t)m, 0.0);
    std::vector<double> Z(2 * (size_t)m);
    const int rows[2] = {0, m - 1};
    if (!tridiag_eigen(a, b, m, out.lam.data(), Z.data(), 2, rows)) return false;
    for (int k = 0; k < m; ++k) {
        out.z0[(size_t)k] = Z[(size_t)k];
        out.zl[(size_t)k] = Z[(size_t)m + k];
    }
    return true;
}

double krylov_last_coeff(const KrylovEnds& K, double tau) {
    std::complex<double> y(0.0, 0.0);
    for (int k = 0; k < K.m; ++k)
        y += K.zl[(size_t)k] * K.z0[(size_t)k] * std::polar(1.0, -K.lam[(size_t)k] * tau);
    return std::abs(y);
}

bool krylov_exp_coeffs(const double* a, const double* b, int m, double tau, double* yre, double* yim) {
    std::vector<double> lam((size_t)m), Z((size_t)m * m);
    std::vector<int> rows((size_t)m);
    for (int i = 0; i < m; ++i) rows[(size_t)i] = i;
    if (!tridiag_eigen(a, b, m, lam.data(), Z.data(), m, rows.data())) return false;
    // y_j = sum_k Z_jk Z_0k exp(-i lam_k tau)
    std::vector<std::complex<double>> w((size_t)m);
    for (int k = 0; k < m; ++k) w[(size_t)k] = Z[(size_t)k] * std::polar(1.0, -lam[(size_t)k] * tau);
    for (int j = 0; j < m; ++j) {
        std::complex<double> y(0.0, 0.0);
        for (int k = 0; k < m; ++k) y += Z[(size_t)j * m + k] * w[(size_t)k];
        yre[j] = y.real();
        yim[j] = y.imag();
    }
    return true;
}

}  // namespace hub

extern "C" int hubbard_host_krylov_exp(const double* a, const double* b, int m, double tau, double* y_re,
                                       double* y_im) {
    if (a == nullptr || y_re == nullptr || y_im == nullptr || m < 1 || (m > 1 && b == nullptr) || m > 4096 ||
        !std::isfinite(tau))
        return HUB_EINVAL;
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(a[i]) || (i + 1 < m && !std::isfinite(b[i]))) return HUB_EINVAL;
    return hub::krylov_exp_coeffs(a, b, m, tau, y_re, y_im) ? HUB_OK : HUB_ENOTCONV;
}
