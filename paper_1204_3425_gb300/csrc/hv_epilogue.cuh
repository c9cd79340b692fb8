// Device helpers of the binary64 fixed-point H*v (hv_phases.cu): the
// binary64 <-> fixed-point conversions, the epilogue parameters, and the fused
// Lanczos reductions.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace hub {

// ---------------------------------------------------------------------------
// binary64 <-> fixed point
__device__ __forceinline__ void fx_split(double x, int emax, int& lo, int& hi) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & ((1ull << 52) - 1);
    if (e != 0) mant |= (1ull << 52);
    const int ee = e > 0 ? e : 1;
    const int rs = max(emax - ee + 5, 1);             // >= 5 whenever |x| < 2^(emax-1022)
    long long X = (rs >= 60) ? 0 : (long long)((mant + (1ull << (rs - 1))) >> rs);
    if (b >> 63) X = -X;
    lo = (int)(X & 0xFFFFFF);
    hi = (int)(X >> 24);
}

__device__ __forceinline__ long long fx_join(int lo, int hi) { return ((long long)hi << 24) + (long long)lo; }

struct I128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ void mac128(I128& acc, long long a, long long b) {
    const unsigned long long plo = (unsigned long long)a * (unsigned long long)b;
    const long long phi = __mul64hi(a, b);
    const unsigned long long nlo = acc.lo + plo;
    acc.hi += phi + (nlo < plo ? 1 : 0);
    acc.lo = nlo;
}

// (hi * 2^64 + lo) * 2^e2, rounded to nearest (ties to even)
__device__ __forceinline__ double i128_to_double(I128 v, int e2) {
    unsigned long long lo = v.lo;
    unsigned long long hi = (unsigned long long)v.hi;
    const bool neg = v.hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0 ? 1ull : 0ull);
    }
    if (hi == 0 && lo == 0) return 0.0;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    unsigned long long nh, nl;
    if (lz == 0) {
        nh = hi;
        nl = lo;
    } else if (lz < 64) {
        nh = (hi << lz) | (lo >> (64 - lz));
        nl = lo << lz;
    } else {
        nh = lo << (lz - 64);
        nl = 0;
    }
    unsigned long long mant = nh >> 11;               // 53 bits, leading one at bit 52
    const unsigned long long rem = nh & 0x7FFull;
    const bool up = (rem > 0x400ull) || (rem == 0x400ull && (nl != 0 || (mant & 1ull)));
    mant += up ? 1ull : 0ull;
    int ex = 127 - lz + e2;
    if (mant == (1ull << 53)) {
        mant >>= 1;
        ++ex;
    }
    const int be = ex + 1023;
    if (be <= 0 || be >= 2047) {
        const double m = (double)mant;                // exact
        return ldexp(neg ? -m : m, ex - 52);
    }
    unsigned long long bits = ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1));
    if (neg) bits |= (1ull << 63);
    return __longlong_as_double((long long)bits);
}

// P * 2^e2, correctly rounded: I2F.F64 rounds once, the power of two is
// applied exactly to the exponent field (ldexp only off the normal range)
__device__ __forceinline__ double i64_scaled_to_double(long long P, int e2) {
    if (P == 0) return 0.0;
    const double d = __ll2double_rn(P);
    const long long bits = __double_as_longlong(d);
    const int be = (int)((bits >> 52) & 0x7FF) + e2;
    if (be <= 0 || be >= 2047) return ldexp(d, e2);
    return __longlong_as_double(bits + ((long long)e2 << 52));
}


struct EpiParams {
    long long A;          // round(-t * 2^m)
    long long Bbeta;      // round(-beta * 2^m)
    long long B[33];      // round(U * n * 2^m), n = 0..32
    int m;
    int nB;
    // exact int64 path, valid when t = +-2^et and U * 2^ju is a small integer:
    //   value = (sgn_t * T * 2^(et+ju) + Uint * n * X) * 2^-(k+ju)
    int fast;
    int tshift;           // et + ju >= 0
    int tneg;             // t < 0
    int ju;
    long long Uint;       // U * 2^ju
    double mbeta;         // -beta, applied after the exact part in the int64 path
};

__device__ __forceinline__ void add4(int4& A, int4 a, int4 b, int4 c, int4 d) {
    A.x += a.x + b.x + c.x + d.x;
    A.y += a.y + b.y + c.y + d.y;
    A.z += a.z + b.z + c.z + d.z;
    A.w += a.w + b.w + c.w + d.w;
}
__device__ __forceinline__ void add4(int4& A, int4 a) {
    A.x += a.x; A.y += a.y; A.z += a.z; A.w += a.w;
}
__device__ __forceinline__ void add4(int2& A, int2 a, int2 b, int2 c, int2 d) {
    A.x += a.x + b.x + c.x + d.x;
    A.y += a.y + b.y + c.y + d.y;
}
__device__ __forceinline__ void add4(int2& A, int2 a) { A.x += a.x; A.y += a.y; }


// Lanczos reductions fused into the up-phase epilogue (Algorithm 1): the CTA
// sums its threads' <w, f>, <w, w>, <f, f> in a fixed tree and stores the
// per-CTA partials at part[b], part[kPartStride + b], part[2 kPartStride + b].
__device__ __forceinline__ void block_sum3_store(double a, double b, double c, double* part) {
    __shared__ double red[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
        red[2][wid] = c;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? red[0][lane] : 0.0;
        b = lane < nw ? red[1][lane] : 0.0;
        c = lane < nw ? red[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            part[blockIdx.x] = a;
            part[kPartStride + blockIdx.x] = b;
            part[2 * kPartStride + blockIdx.x] = c;
        }
    }
}


// m such that M * 2^m <= 2^61, M = max(|t|, |U| Ns, |beta|, 2 (W |t| + |U| Ns)):
// the last term bounds every Lanczos beta (beta_{j+1} <= |H| <= W |t| + |U| Ns
// by Gershgorin, W = W_up + W_dn), so m does not depend on beta and a device-
// resident step can form round(-beta 2^m) itself with the host's m
inline EpiParams make_epilogue(double t, double U, int ns, double beta, int W) {
    EpiParams p{};
    const double gersh = 2.0 * ((double)W * std::fabs(t) + std::fabs(U) * ns);
    double M = std::max(std::max(std::fabs(t), std::fabs(U) * ns), std::max(std::fabs(beta), gersh));
    int m = 0;
    if (M > 0) {
        int ex = 0;
        std::frexp(M, &ex);                           // M < 2^ex
        m = 61 - ex;
    }
    p.m = m;
    p.A = (long long)std::llround(std::ldexp(-t, m));
    p.Bbeta = (long long)std::llround(std::ldexp(-beta, m));
    p.nB = std::min(ns, 32) + 1;
    for (int n = 0; n < 33; ++n) p.B[n] = n < p.nB ? (long long)std::llround(std::ldexp(U * n, m)) : 0;
    // int64 path: t = +-2^et and U * 2^ju an integer with |U 2^ju| Ns < 2^14 for some ju in [0, 8],
    // et + ju in [0, 6].  Then |T 2^(et+ju)| < 2^55 * 2^6 and |U 2^ju n X| < 2^14 * 2^48, so
    // H v is formed exactly in int64 and rounded once; a -beta w_old term is then added with
    // one fused multiply-add (a second rounding)
    p.fast = 0;
    p.mbeta = -beta;
    if (t != 0.0) {
        int et = 0;
        const double mt = std::frexp(std::fabs(t), &et);   // |t| = mt * 2^et, mt in [0.5, 1)
        if (mt == 0.5) {
            et -= 1;                                        // |t| = 2^et
            for (int ju = 0; ju <= 8; ++ju) {
                const double us = std::ldexp(U, ju);
                if (us == std::floor(us) && std::fabs(us) * ns < 16384.0 && et + ju >= 0 && et + ju <= 6) {
                    p.fast = 1;
                    p.tshift = et + ju;
                    p.tneg = t < 0 ? 1 : 0;
                    p.ju = ju;
                    p.Uint = (long long)us;
                    break;
                }
            }
        }
    }
    return p;
}


}  // namespace hub
