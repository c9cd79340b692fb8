/* Kronecker-sum Hamiltonian-vector product for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: built and called by the oracle package, never by
 * the product library.
 *
 * H = H_up (x) I_dn + I_up (x) H_dn + H_int  (Eq. H-Kroneckersum plus the
 * diagonal interaction of Eq. 1).  The vector is viewed as D_up subvectors
 * of length D_dn (Fig. 2): H_up acts on the subvectors as whole units and
 * H_dn acts inside each subvector; H_int multiplies element J = (u, d) by
 * U * popcount(s_up[u] & s_dn[d]).  H_up and H_dn are given in CSR (rows =
 * output index), as the paper's CPU program stores them (Sec. 5).
 *
 * kron_hv_acc computes y <- y + H x, the second half of Eqs. (split1).
 * Plain loops, parallelised over subvectors with OpenMP; double throughout.
 */
#include <stdint.h>
#include <omp.h>

static int popcount32(uint32_t w) {
    int n = 0;
    while (w) { n += (int)(w & 1u); w >>= 1; }
    return n;
}

void kron_hv_acc(int64_t Dup, int64_t Ddn,
                 const int32_t* up_rowptr, const int32_t* up_col, const double* up_val,
                 const int32_t* dn_rowptr, const int32_t* dn_col, const double* dn_val,
                 const uint32_t* up_states, const uint32_t* dn_states, double U,
                 const double* x, double* y)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t u = 0; u < Dup; ++u) {
        double* yu = y + u * Ddn;
        const double* xu = x + u * Ddn;
        /* (H_up (x) I) x: subvector u gets sum_k H_up[u, u'] * x^(u') */
        for (int32_t k = up_rowptr[u]; k < up_rowptr[u + 1]; ++k) {
            const double h = up_val[k];
            const double* xs = x + (int64_t)up_col[k] * Ddn;
            for (int64_t d = 0; d < Ddn; ++d) yu[d] += h * xs[d];
        }
        /* (I (x) H_dn) x and H_int x, element by element inside subvector u */
        for (int64_t d = 0; d < Ddn; ++d) {
            double acc = U * (double)popcount32(up_states[u] & dn_states[d]) * xu[d];
            for (int32_t k = dn_rowptr[d]; k < dn_rowptr[d + 1]; ++k)
                acc += dn_val[k] * xu[dn_col[k]];
            yu[d] += acc;
        }
    }
}

/* y <- a*y (the first half of Eqs. split1), parallel over elements. */
void kron_scale(int64_t n, double a, double* y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] *= a;
}

/* sum_i x_i * y_i, parallel, summed per thread then over threads. */
double kron_dot(int64_t n, const double* x, const double* y)
{
    double s = 0.0;
    #pragma omp parallel for reduction(+:s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

/* y <- y + a*x */
void kron_axpy(int64_t n, double a, const double* x, double* y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) y[i] += a * x[i];
}

/* OpenMP threads for the calls above (n > 0); returns the previous maximum. */
int kron_set_threads(int n)
{
    const int prev = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return prev;
}
