// H*v and Lanczos vector kernels for sm_103a.
//
// Vector layout (Fig. 2): element J = u * D_dn + d, i.e. a row-major
// D_up x D_dn matrix V.  Up-hops combine whole rows of V (Algorithm 2),
// down-hops gather inside a row (Algorithm 3), the interaction is diagonal
// (Algorithm 4).
//
// Packed hop entry: (target << 1) | (sign < 0); <target|H_sigma|src> = -t*sign.
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "internal.h"
#include "splitmix.cuh"

namespace hub {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// thread-safe (static initialisation runs once; callers on other threads wait)
int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// ---------------------------------------------------------------------------
// Reference H*v: one thread per output element, native arithmetic of T.
// Rows u are taken block-stride, columns d thread-stride.
template <typename T>
__global__ void k_hv_reference(const T* __restrict__ v, T* __restrict__ w, int64_t Dup, int64_t Ddn,
                               const int32_t* __restrict__ up_ptr, const uint32_t* __restrict__ up_ent,
                               const int32_t* __restrict__ dn_ptr, const uint32_t* __restrict__ dn_ent,
                               const uint32_t* __restrict__ su, const uint32_t* __restrict__ sd,
                               T mt, T U) {
    for (int64_t u = blockIdx.x; u < Dup; u += gridDim.x) {
        const int32_t ub = up_ptr[u], ue = up_ptr[u + 1];
        const uint32_t su_u = su[u];
        const T* vrow = v + u * Ddn;
        for (int64_t d = threadIdx.x; d < Ddn; d += blockDim.x) {
            T hop = T(0);
            for (int32_t k = ub; k < ue; ++k) {          // H_up (x) I  (Algorithm 2)
                const uint32_t e = up_ent[k];
                const T x = v[(int64_t)(e >> 1) * Ddn + d];
                hop += (e & 1u) ? -x : x;
            }
            const int32_t db = dn_ptr[d], de = dn_ptr[d + 1];
            for (int32_t k = db; k < de; ++k) {          // I (x) H_dn  (Algorithm 3)
                const uint32_t e = dn_ent[k];
                const T x = vrow[e >> 1];
                hop += (e & 1u) ? -x : x;
            }
            const int nd = __popc(su_u & sd[d]);         // H_int  (Algorithm 4)
            w[u * Ddn + d] = mt * hop + U * T(nd) * vrow[d];
        }
    }
}

// ---------------------------------------------------------------------------
// Binary64 path in exact fixed point.
//
// Every element of v is rounded once to the grid 2^-k, with k chosen so that
// max|v| * 2^k < 2^48, and stored as X = hi * 2^24 + lo (lo in [0, 2^24),
// |hi| <= 2^24).  A hop sum of up to 2^6 signed terms then fits two int32
// accumulators without carries, and is exact.

// max biased exponent of |v| -> *emax (atomicMax; *emax must start at 0)
__global__ void k_max_exponent(const double* __restrict__ v, int64_t n, int* emax) {
    int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[i]);
        m = max(m, (int)((b >> 52) & 0x7FF));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(emax, m);
}

// rounding of one binary64 to the fixed-point grid given the exponent bound
__device__ __forceinline__ int2 to_fixed(double x, int emax) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & ((1ull << 52) - 1);
    if (e != 0) mant |= (1ull << 52);
    const int ee = e > 0 ? e : 1;
    // value = mant * 2^(ee-1075); X = value * 2^k, k = 1070 - emax  => right shift
    const int rs = emax - ee + 5;                     // >= 5 because ee <= emax
    long long X;
    if (rs >= 60) X = 0;
    else X = (long long)((mant + (1ull << (rs - 1))) >> rs);
    if (b >> 63) X = -X;
    int2 r;
    r.x = (int)(X & 0xFFFFFF);                        // lo, [0, 2^24)
    r.y = (int)(X >> 24);                             // hi, arithmetic shift
    return r;
}

__global__ void k_to_fixed(const double* __restrict__ v, int2* __restrict__ X, int64_t n,
                           const int* __restrict__ emax_p) {
    const int emax = max(*emax_p, 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[i] = to_fixed(v[i], emax);
}

// (-t * S) * 2^-k: the product -t * S is rounded once in the normal range and
// the power of two is applied to its exponent field; only a result that is
// itself subnormal is rounded a second time (by ldexp).  Scaling -t by 2^-k
// first would round -t to a few bits whenever 2^-k is below the normal range
// (inputs below about 2^-975).
__device__ __forceinline__ double scaled_hop_sum(long long S, double mt, int k) {
    if (S == 0) return 0.0;
    const double p = mt * (double)S;
    const long long bits = __double_as_longlong(p);
    const int be = (int)((bits >> 52) & 0x7FF) - k;
    if (be <= 0 || be >= 2047) return ldexp(p, -k);
    return __longlong_as_double(bits - ((long long)k << 52));
}

// w = -t * S * 2^-k + U * n_d * v  [ - beta * w_old ]
__global__ void k_hv_fixed(const int2* __restrict__ X, const double* __restrict__ v, double* w,
                           const double* w_old, double beta, int64_t Dup, int64_t Ddn,
                           const int32_t* __restrict__ up_ptr, const uint32_t* __restrict__ up_ent,
                           const int32_t* __restrict__ dn_ptr, const uint32_t* __restrict__ dn_ent,
                           const uint32_t* __restrict__ su, const uint32_t* __restrict__ sd,
                           double mt, double U, const int* __restrict__ emax_p) {
    const int emax = max(*emax_p, 1);
    const int kg = 1070 - emax;                       // grid 2^-kg
    for (int64_t u = blockIdx.x; u < Dup; u += gridDim.x) {
        const int32_t ub = up_ptr[u], ue = up_ptr[u + 1];
        const uint32_t su_u = su[u];
        const int2* xrow = X + u * Ddn;
        for (int64_t d = threadIdx.x; d < Ddn; d += blockDim.x) {
            int lo = 0, hi = 0;
            for (int32_t k = ub; k < ue; ++k) {
                const uint32_t e = up_ent[k];
                const int2 x = X[(int64_t)(e >> 1) * Ddn + d];
                if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
            }
            const int32_t db = dn_ptr[d], de = dn_ptr[d + 1];
            for (int32_t k = db; k < de; ++k) {
                const uint32_t e = dn_ent[k];
                const int2 x = xrow[e >> 1];
                if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
            }
            const long long S = ((long long)hi << 24) + (long long)lo;
            const int64_t J = u * Ddn + d;
            const int nd = __popc(su_u & sd[d]);
            double r = fma(U * (double)nd, v[J], scaled_hop_sum(S, mt, kg));
            if (w_old != nullptr) r = fma(-beta, w_old[J], r);
            w[J] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// Reductions: per-thread binary64 sums, warp shuffles, block tree, then one
// block sums the per-block partials in a fixed order (deterministic).
__device__ __forceinline__ double block_sum(double s) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = s;
    __syncthreads();
    s = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        s = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// Per-thread float-float accumulator for binary32 vectors: each product x*y
// is split exactly (p + e with e = fma(x, y, -p)) and added with Knuth's
// TwoSum, so the FP32 pipe carries ~48 bits and the binary64 pipe (1.7
// op/clk/SM here) is touched once per thread, not per element.
struct FF {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add_product(float x, float y) {
        const float p = x * y;
        const float e = fmaf(x, y, -p);
        const float s = hi + p;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (p - bb)) + e;
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__global__ void k_dot_f64(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* partials) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[i], y[i], s);
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_dot_f32(const float* __restrict__ x, const float* __restrict__ y, int64_t n, double* partials) {
    FF acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add_product(x[i], y[i]);
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// y <- y + a x ; partial sums of y^2
__global__ void k_axpy_nrm2_f64(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n,
                                double* partials) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = fma(a, x[i], y[i]);
        y[i] = r;
        s = fma(r, r, s);
    }
    s = block_sum(s);
    if (threadIdx.x == 0 && partials != nullptr) partials[blockIdx.x] = s;
}

__global__ void k_axpy_nrm2_f32(float a, const float* __restrict__ x, float* __restrict__ y, int64_t n,
                                double* partials) {
    FF acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = fmaf(a, x[i], y[i]);
        y[i] = r;
        acc.add_product(r, r);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0 && partials != nullptr) partials[blockIdx.x] = s;
}

template <typename T>
__global__ void k_axpy(T a, const T* __restrict__ x, T* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

template <typename T>
__global__ void k_scale(T a, T* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] *= a;
}

// y <- (y + a x) * inv with the roundings of k_axpy_nrm2 then k_scale
// (dv: a, inv from the device-resident step control)
__global__ void k_axpy_scale_f64(double a, double inv, const double* __restrict__ x, double* __restrict__ y,
                                 int64_t n, const LzDev* __restrict__ dv) {
    if (dv != nullptr) {
        a = dv->ua;
        inv = dv->uinv;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]) * inv;
}
__global__ void k_axpy_scale_f32(float a, float inv, const float* __restrict__ x, float* __restrict__ y, int64_t n,
                                 const LzDev* __restrict__ dv) {
    if (dv != nullptr) {
        a = (float)dv->ua;
        inv = (float)dv->uinv;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]) * inv;
}

// Device-resident Lanczos step control (Algorithm 1): the step in progress is
// closed with beta_{j+1}; the next step's H*v then reads beta = beta_{j+1} and
// completes f_{j+1} = (g + ua f_j) * uinv while staging its rows: ua = -a_j
// when g still holds H f_j - beta_j f_{j-1} (fused sums), 0 when the explicit
// branch already subtracted a_j f_j.  The roundings are those of the host-driven
// step (sqrt and the division are correctly rounded on both sides).
__device__ __forceinline__ void lz_close_step(LzDev* dv, double* hb, double bn, bool fused) {
    const int j = dv->j;
    hb[j] = bn;
    dv->ua = fused ? -dv->a : 0.0;
    dv->uinv = 1.0 / bn;
    dv->beta = bn;
    dv->j = j + 1;
}

// the three fused sums in the order of k_finish_sum3, then a_j and, unless the
// difference <w,w> - 2a^2 + a^2 <f,f> cancels more than six digits, beta_{j+1}
__global__ void k_lz_finish(double* partials, int nb, LzDev* dv, double* ha, double* hb) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += partials[i];
        b += partials[kPartStride + i];
        c += partials[2 * kPartStride + i];
    }
    a = block_sum(a);
    b = block_sum(b);
    c = block_sum(c);
    if (threadIdx.x == 0) {
        partials[kRedSlots - 1] = a;
        partials[kRedSlots - 2] = b;
        partials[kRedSlots - 3] = c;
        const double b2 = b - 2.0 * a * a + a * a * c;
        const int fused = b2 > 1e-6 * b;
        dv->a = a;
        dv->fused = fused;
        ha[dv->j] = a;
        if (fused) lz_close_step(dv, hb, sqrt(fmax(b2, 0.0)), true);
    }
}

// explicit branch: y <- y - a x and partial sums of y^2, as k_axpy_nrm2_*
__global__ void k_lz_axpy_nrm2_f64(const LzDev* __restrict__ dv, const double* __restrict__ x, double* __restrict__ y,
                                   int64_t n, double* partials) {
    if (dv->fused) return;
    const double a = -dv->a;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = fma(a, x[i], y[i]);
        y[i] = r;
        s = fma(r, r, s);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
__global__ void k_lz_axpy_nrm2_f32(const LzDev* __restrict__ dv, const float* __restrict__ x, float* __restrict__ y,
                                   int64_t n, double* partials) {
    if (dv->fused) return;
    const float a = (float)(-dv->a);
    FF acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = fmaf(a, x[i], y[i]);
        y[i] = r;
        acc.add_product(r, r);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
// sums the explicit branch's partials in the order of k_finish_sum, closes the step
__global__ void k_lz_finish2(double* partials, int nb, LzDev* dv, double* hb) {
    if (dv->fused) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        partials[kRedSlots - 1] = s;
        lz_close_step(dv, hb, sqrt(fmax(s, 0.0)), false);
    }
}

template <typename T>
__global__ void k_copy_scale(const T* __restrict__ x, T* __restrict__ y, int64_t n, T a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

__global__ void k_f64_to_f32_scaled(const double* __restrict__ x, float* __restrict__ y, int64_t n, double a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)(a * x[i]);
}

// psi <- (init ? 0 : psi) + s * f  (binary32 f, binary64 psi)
__global__ void k_psi_acc(const float* __restrict__ f, double* __restrict__ psi, int64_t n, double s, int init) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        psi[i] = init ? s * (double)f[i] : fma(s, (double)f[i], psi[i]);
}

// psi <- (init ? 0 : psi) + s * f  (binary64 f)
__global__ void k_psi_acc_f64(const double* __restrict__ f, double* __restrict__ psi, int64_t n, double s, int init) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        psi[i] = init ? s * f[i] : fma(s, f[i], psi[i]);
}

// psi = sum_j s_j f_j over m stored binary32 vectors f_j = base + j * stride,
// accumulated per element in j order with the same operations as successive
// k_psi_acc launches (so the result is bit-identical to that sequence).  Two
// elements per thread and eight vectors' loads issued before their
// multiply-adds (the loop is bound by the latency of m scattered streams);
// base and stride must keep f_j 8-byte aligned, psi 16-byte aligned.
__global__ void k_psi_multi(const float* __restrict__ base, int64_t stride, int m, const double* __restrict__ s,
                            double* __restrict__ psi, int64_t n) {
    constexpr int U = 8;
    const int64_t n2 = n / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const float* p = base + 2 * i;
        const float2 x0 = *reinterpret_cast<const float2*>(p);
        double ax = s[0] * (double)x0.x, ay = s[0] * (double)x0.y;
        int j = 1;
        for (; j + U <= m; j += U) {
            float2 x[U];
#pragma unroll
            for (int q = 0; q < U; ++q) x[q] = __ldcs(reinterpret_cast<const float2*>(p + (int64_t)(j + q) * stride));
#pragma unroll
            for (int q = 0; q < U; ++q) {
                ax = fma(s[j + q], (double)x[q].x, ax);
                ay = fma(s[j + q], (double)x[q].y, ay);
            }
        }
        for (; j < m; ++j) {
            const float2 x = __ldcs(reinterpret_cast<const float2*>(p + (int64_t)j * stride));
            ax = fma(s[j], (double)x.x, ax);
            ay = fma(s[j], (double)x.y, ay);
        }
        reinterpret_cast<double2*>(psi)[i] = make_double2(ax, ay);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t i = n - 1;
        double acc = s[0] * (double)base[i];
        for (int j = 1; j < m; ++j) acc = fma(s[j], (double)__ldcs(base + (int64_t)j * stride + i), acc);
        psi[i] = acc;
    }
}

// A <- A + ca f, B <- B + cb f (binary64): one Lanczos vector's share of the
// real and imaginary parts of a Krylov propagation
__global__ void k_acc2_f64(const double* __restrict__ f, double* __restrict__ A, double* __restrict__ B, int64_t n,
                           double ca, double cb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = __ldcs(f + i);
        A[i] = fma(ca, x, A[i]);
        B[i] = fma(cb, x, B[i]);
    }
}

// A <- A + sum_j c[j] f_j, B <- B + sum_j c[m + j] f_j over m stored binary64
// vectors f_j = base + j * stride, per element in j order with the operations
// of m successive k_acc2_f64 launches (so the result is bit-identical to them).
// Two elements per thread, four vectors' loads issued before their
// multiply-adds; base, stride, A and B must keep 16-byte alignment.
__global__ void k_combine2_f64(const double* __restrict__ base, int64_t stride, int m, const double* __restrict__ c,
                               double* __restrict__ A, double* __restrict__ B, int64_t n) {
    constexpr int U = 4;
    const int64_t n2 = n / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const double* p = base + 2 * i;
        double2 a = reinterpret_cast<const double2*>(A)[i];
        double2 b = reinterpret_cast<const double2*>(B)[i];
        int j = 0;
        for (; j + U <= m; j += U) {
            double2 x[U];
#pragma unroll
            for (int q = 0; q < U; ++q) x[q] = __ldcs(reinterpret_cast<const double2*>(p + (int64_t)(j + q) * stride));
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const double ca = c[j + q], cb = c[m + j + q];
                a.x = fma(ca, x[q].x, a.x);
                a.y = fma(ca, x[q].y, a.y);
                b.x = fma(cb, x[q].x, b.x);
                b.y = fma(cb, x[q].y, b.y);
            }
        }
        for (; j < m; ++j) {
            const double2 x = __ldcs(reinterpret_cast<const double2*>(p + (int64_t)j * stride));
            a.x = fma(c[j], x.x, a.x);
            a.y = fma(c[j], x.y, a.y);
            b.x = fma(c[m + j], x.x, b.x);
            b.y = fma(c[m + j], x.y, b.y);
        }
        reinterpret_cast<double2*>(A)[i] = a;
        reinterpret_cast<double2*>(B)[i] = b;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t i = n - 1;
        double a = A[i], b = B[i];
        for (int j = 0; j < m; ++j) {
            const double x = __ldcs(base + (int64_t)j * stride + i);
            a = fma(c[j], x, a);
            b = fma(c[m + j], x, b);
        }
        A[i] = a;
        B[i] = b;
    }
}

// Seeded uniform [-1, 1) start vector (splitmix.cuh), elements start .. start + n
__global__ void k_fill_splitmix(void* v, int64_t n, unsigned long long seed, int64_t start, int dtype) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double val = splitmix_uniform(seed, start + i);
        if (dtype == HUB_F64) ((double*)v)[i] = val;
        else ((float*)v)[i] = (float)val;
    }
}

// sums partials[0..nb) in index order into partials[kRedSlots-1]
__global__ void k_finish_sum(double* partials, int nb) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) partials[kRedSlots - 1] = s;
}

// the three arrays of a fused reduction (part[q kPartStride .. + nb)), each
// summed in a fixed order, into part[kRedSlots-1-q]
__global__ void k_finish_sum3(double* partials, int nb) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += partials[i];
        b += partials[kPartStride + i];
        c += partials[2 * kPartStride + i];
    }
    a = block_sum(a);
    b = block_sum(b);
    c = block_sum(c);
    if (threadIdx.x == 0) {
        partials[kRedSlots - 1] = a;
        partials[kRedSlots - 2] = b;
        partials[kRedSlots - 3] = c;
    }
}

int red_grid(int64_t n) { return grid_for(n, kThreads * 4, kRedBlocks); }

}  // namespace

// ---------------------------------------------------------------------------
int launch_hv_reference(const hubbard_sector* H, const void* v, void* w, int dtype, cudaStream_t s) {
    const int grid = grid_for(H->Dup, 1, sm_count() * 16);
    const DevSpin& up = H->dev[0];
    const DevSpin& dn = H->dev[1];
    if (dtype == HUB_F64) {
        k_hv_reference<double><<<grid, kThreads, 0, s>>>((const double*)v, (double*)w, H->Dup, H->Ddn,
            up.rowptr, up.ent, dn.rowptr, dn.ent, up.states, dn.states, -H->t, H->U);
    } else {
        k_hv_reference<float><<<grid, kThreads, 0, s>>>((const float*)v, (float*)w, H->Dup, H->Ddn,
            up.rowptr, up.ent, dn.rowptr, dn.ent, up.states, dn.states, (float)-H->t, (float)H->U);
    }
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

void launch_to_fixed(const double* v, int64_t n, void* X, const int* emax, cudaStream_t s) {
    const int g2 = grid_for(n, kThreads * 8, sm_count() * 8);
    k_to_fixed<<<g2, kThreads, 0, s>>>(v, (int2*)X, n, emax);
}

void launch_max_exponent(const double* v, int64_t n, int* emax, cudaStream_t s) {
    const int g2 = grid_for(n, kThreads * 8, sm_count() * 8);
    k_max_exponent<<<g2, kThreads, 0, s>>>(v, n, emax);
}

int launch_hv_fast(hubbard_sector* H, const void* v, void* w, int dtype, double beta, const void* w_old,
                   int fixed_emax, cudaStream_t s, double* part, bool* fused, const RowUpdate* upd, LzDev* dv,
                   double* ha, double* hb) {
    const DevSpin& up = H->dev[0];
    const DevSpin& dn = H->dev[1];
    const int grid = grid_for(H->Dup, 1, sm_count() * 16);
    if (fused != nullptr) *fused = false;
    if (H->fx_bytes >= (size_t)H->D * 16) {
        int np = 0;
        int rc = launch_hv_phases(H, v, w, dtype, beta, w_old, H->fx_scratch, fixed_emax, s, part, &np, upd, dv);
        if (rc != -1) {
            if (rc == HUB_OK && part != nullptr && np > 0) {
                if (dv != nullptr) {
                    if ((rc = launch_lz_finish(part, np, dv, ha, hb, s))) return rc;
                } else {
                    k_finish_sum3<<<1, 1024, 0, s>>>(part, np);
                    HUB_CUDA(cudaGetLastError());
                    count_launches(1);
                }
                if (fused != nullptr) *fused = true;
            } else if (rc == HUB_OK && dv != nullptr) {
                return fail(HUB_EINVAL, "device-resident Lanczos step without fused reductions");
            }
            return rc;
        }
    }
    if (dv != nullptr) return fail(HUB_EINVAL, "device-resident Lanczos step without fused reductions");
    if (upd != nullptr) {
        if (int rc = launch_axpy_scale(upd->a, upd->inv, upd->fo, const_cast<void*>(v), H->D, dtype, s, upd->dv))
            return rc;
    }
    if (dtype == HUB_F32) {
        if (w_old != nullptr || beta != 0.0) return fail(HUB_EINVAL, "f32 fused step not available");
        k_hv_reference<float><<<grid, kThreads, 0, s>>>((const float*)v, (float*)w, H->Dup, H->Ddn,
            up.rowptr, up.ent, dn.rowptr, dn.ent, up.states, dn.states, (float)-H->t, (float)H->U);
        HUB_CUDA(cudaGetLastError());
        count_launches(1);
        return HUB_OK;
    }
    const size_t need = (size_t)H->D * sizeof(int2);
    if (H->fx_bytes < need) return fail(HUB_ENOMEM, "fixed-point scratch not allocated");
    int* emax = H->status;
    HUB_CUDA(cudaMemsetAsync(emax, 0, sizeof(int), s));
    const int g2 = grid_for(H->D, kThreads * 8, sm_count() * 8);
    k_max_exponent<<<g2, kThreads, 0, s>>>((const double*)v, H->D, emax);
    k_to_fixed<<<g2, kThreads, 0, s>>>((const double*)v, (int2*)H->fx_scratch, H->D, emax);
    k_hv_fixed<<<grid, kThreads, 0, s>>>((const int2*)H->fx_scratch, (const double*)v, (double*)w,
        (const double*)w_old, beta, H->Dup, H->Ddn, up.rowptr, up.ent, dn.rowptr, dn.ent,
        up.states, dn.states, -H->t, H->U, emax);
    HUB_CUDA(cudaGetLastError());
    count_launches(3);
    return HUB_OK;
}

int launch_dot(const hubbard_sector*, const void* x, const void* y, int64_t n, int dtype, double* partials,
               cudaStream_t s) {
    const int g = red_grid(n);
    if (dtype == HUB_F64) k_dot_f64<<<g, kThreads, 0, s>>>((const double*)x, (const double*)y, n, partials);
    else k_dot_f32<<<g, kThreads, 0, s>>>((const float*)x, (const float*)y, n, partials);
    k_finish_sum<<<1, 1024, 0, s>>>(partials, g);
    HUB_CUDA(cudaGetLastError());
    count_launches(2);
    return HUB_OK;
}

int reduce_partials_host(double* partials, cudaStream_t s, double* out) {
    HUB_CUDA(cudaMemcpyAsync(out, partials + (kRedSlots - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    return HUB_OK;
}

int launch_axpy(double a, const void* x, void* y, int64_t n, int dtype, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    if (dtype == HUB_F64) k_axpy<double><<<g, kThreads, 0, s>>>(a, (const double*)x, (double*)y, n);
    else k_axpy<float><<<g, kThreads, 0, s>>>((float)a, (const float*)x, (float*)y, n);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_axpy_nrm2(double a, const void* x, void* y, int64_t n, int dtype, double* partials, cudaStream_t s) {
    const int g = red_grid(n);
    if (dtype == HUB_F64) k_axpy_nrm2_f64<<<g, kThreads, 0, s>>>(a, (const double*)x, (double*)y, n, partials);
    else k_axpy_nrm2_f32<<<g, kThreads, 0, s>>>((float)a, (const float*)x, (float*)y, n, partials);
    k_finish_sum<<<1, 1024, 0, s>>>(partials, g);
    HUB_CUDA(cudaGetLastError());
    count_launches(2);
    return HUB_OK;
}

int reduce_partials3_host(double* partials, cudaStream_t s, double out[3]) {
    double t[3];
    HUB_CUDA(cudaMemcpyAsync(t, partials + (kRedSlots - 3), 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    out[0] = t[2];
    out[1] = t[1];
    out[2] = t[0];
    return HUB_OK;
}

int launch_axpy_scale(double a, double inv, const void* x, void* y, int64_t n, int dtype, cudaStream_t s,
                      const LzDev* dv) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    if (dtype == HUB_F64) k_axpy_scale_f64<<<g, kThreads, 0, s>>>(a, inv, (const double*)x, (double*)y, n, dv);
    else k_axpy_scale_f32<<<g, kThreads, 0, s>>>((float)a, (float)inv, (const float*)x, (float*)y, n, dv);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_lz_explicit(LzDev* dv, const void* x, void* y, int64_t n, int dtype, double* partials, double* hb,
                       cudaStream_t s) {
    const int g = red_grid(n);
    if (dtype == HUB_F64) k_lz_axpy_nrm2_f64<<<g, kThreads, 0, s>>>(dv, (const double*)x, (double*)y, n, partials);
    else k_lz_axpy_nrm2_f32<<<g, kThreads, 0, s>>>(dv, (const float*)x, (float*)y, n, partials);
    k_lz_finish2<<<1, 1024, 0, s>>>(partials, g, dv, hb);
    HUB_CUDA(cudaGetLastError());
    count_launches(2);
    return HUB_OK;
}

int launch_lz_finish(double* part, int np, LzDev* dv, double* ha, double* hb, cudaStream_t s) {
    k_lz_finish<<<1, 1024, 0, s>>>(part, np, dv, ha, hb);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_scale(double a, void* y, int64_t n, int dtype, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    if (dtype == HUB_F64) k_scale<double><<<g, kThreads, 0, s>>>(a, (double*)y, n);
    else k_scale<float><<<g, kThreads, 0, s>>>((float)a, (float*)y, n);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_fill_splitmix(void* v, int64_t n, unsigned long long seed, int64_t start, int dtype, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_fill_splitmix<<<g, kThreads, 0, s>>>(v, n, seed, start, dtype);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_f64_to_f32_scaled(const double* x, float* y, int64_t n, double a, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_f64_to_f32_scaled<<<g, kThreads, 0, s>>>(x, y, n, a);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_psi_accumulate(const float* f, double* psi, int64_t n, double sj, bool init, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_psi_acc<<<g, kThreads, 0, s>>>(f, psi, n, sj, init ? 1 : 0);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_psi_accumulate_f64(const double* f, double* psi, int64_t n, double sj, bool init, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_psi_acc_f64<<<g, kThreads, 0, s>>>(f, psi, n, sj, init ? 1 : 0);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_psi_multi(const float* base, int64_t stride, int m, const double* s_dev, double* psi, int64_t n,
                     cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_psi_multi<<<g, kThreads, 0, s>>>(base, stride, m, s_dev, psi, n);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_acc2_f64(const double* f, double* A, double* B, int64_t n, double ca, double cb, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_acc2_f64<<<g, kThreads, 0, s>>>(f, A, B, n, ca, cb);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_combine2_f64(const double* base, int64_t stride, int m, const double* c_dev, double* A, double* B,
                        int64_t n, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    k_combine2_f64<<<g, kThreads, 0, s>>>(base, stride, m, c_dev, A, B, n);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

int launch_copy_normalise(const void* x, void* y, int64_t n, int dtype, double inv_norm, cudaStream_t s) {
    const int g = grid_for(n, kThreads * 8, sm_count() * 8);
    if (dtype == HUB_F64) k_copy_scale<double><<<g, kThreads, 0, s>>>((const double*)x, (double*)y, n, inv_norm);
    else k_copy_scale<float><<<g, kThreads, 0, s>>>((const float*)x, (float*)y, n, (float)inv_norm);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    return HUB_OK;
}

}  // namespace hub

// ---------------------------------------------------------------------------
// hubbard_apply_noalloc: binary64 H*v with its scratch in a file-scope device
// array, for callers that cannot allocate device memory at call time.
namespace hub {

static __device__ __align__(256) int2 g_noalloc_fixed[HUBBARD_NOALLOC_MAX_ELEMS];
static __device__ __align__(256) int g_noalloc_emax[64];

namespace {

constexpr int kMaxDevices = 64;
struct NoAllocAddr {
    std::once_flag once;
    int rc = HUB_OK;
    int2* fixed = nullptr;
    int* emax = nullptr;
};
NoAllocAddr g_noalloc_addr[kMaxDevices];

// Looks up, once per device with that device current, the device addresses
// of the scratch arrays.  In host code the array names are host-side stand-
// ins, so kernels must be given these looked-up addresses instead.
int noalloc_addresses(int dev, int2** fixed, int** emax) {
    if (dev < 0 || dev >= kMaxDevices) return fail(HUB_EINVAL, "device index out of range for the no-allocation path");
    NoAllocAddr& a = g_noalloc_addr[dev];
    std::call_once(a.once, [&a]() {
        cudaError_t e = cudaGetSymbolAddress((void**)&a.fixed, g_noalloc_fixed);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&a.emax, g_noalloc_emax);
        if (e != cudaSuccess) {
            a.rc = cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
            a.fixed = nullptr;
            a.emax = nullptr;
        }
    });
    if (a.rc != HUB_OK) return fail(a.rc, "no-allocation scratch address lookup failed on this device");
    *fixed = a.fixed;
    *emax = a.emax;
    return HUB_OK;
}

}  // namespace
}  // namespace hub

extern "C" int hubbard_apply_noalloc(hubbard_t H, const void* v, void* w, void* stream) {
    using namespace hub;
    clear_error();
    if (H == nullptr) return fail(HUB_EINVAL, "null handle");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != H->device)
        return fail(HUB_EINVAL, "handle was created on another device");
    if (v == nullptr || w == nullptr) return fail(HUB_EINVAL, "null vector");
    if ((reinterpret_cast<uintptr_t>(v) & 15u) || (reinterpret_cast<uintptr_t>(w) & 15u))
        return fail(HUB_EINVAL, "vectors must be 16-byte aligned");
    const size_t bytes = (size_t)H->D * sizeof(double);
    const char* a = (const char*)v;
    const char* b = (const char*)w;
    if (a < b + bytes && b < a + bytes) return fail(HUB_EINVAL, "v and w overlap");
    if (H->D > (int64_t)HUBBARD_NOALLOC_MAX_ELEMS)
        return fail(HUB_EINVAL, "sector dimension exceeds HUBBARD_NOALLOC_MAX_ELEMS (2^21) of the no-allocation path");
    // more than 127 hops per state overflow the two int32 fixed-point
    // accumulators: the native binary64 kernel needs no scratch at all
    if (H->host[0].W + H->host[1].W > 127) return launch_hv_reference(H, v, w, HUB_F64, (cudaStream_t)stream);
    int2* fixed = nullptr;
    int* emax = nullptr;
    int rc = noalloc_addresses(dev, &fixed, &emax);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const DevSpin& up = H->dev[0];
    const DevSpin& dn = H->dev[1];
    // the exponent word keeps the previous call's value: it must restart at 0
    HUB_CUDA(cudaMemsetAsync(emax, 0, sizeof(int), s));
    const int g2 = grid_for(H->D, kThreads * 8, sm_count() * 8);
    const int grid = grid_for(H->Dup, 1, sm_count() * 16);
    k_max_exponent<<<g2, kThreads, 0, s>>>((const double*)v, H->D, emax);
    k_to_fixed<<<g2, kThreads, 0, s>>>((const double*)v, fixed, H->D, emax);
    k_hv_fixed<<<grid, kThreads, 0, s>>>(fixed, (const double*)v, (double*)w, nullptr, 0.0, H->Dup, H->Ddn,
        up.rowptr, up.ent, dn.rowptr, dn.ent, up.states, dn.states, -H->t, H->U, emax);
    HUB_CUDA(cudaGetLastError());
    count_launches(3);
    return HUB_OK;
}
