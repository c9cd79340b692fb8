// Two-phase H*v with shared-memory staging (Sec. 4.3 restated for sm_103a).
//
// V is the row-major D_up x D_dn matrix of Fig. 2.  The Kronecker sum of
// Eq. (H-Kroneckersum) splits H*v into
//   row phase  Y[u, :] = sum over down-hops inside row u          (Algorithm 3)
//   up phase   W[u, :] = sum over up-hops u -> u' of rows V[u', :] + Y[u, :]
//                        + U * popcount(s_up & s_dn) * V[u, :]     (Algorithms 2, 4)
// The row phase stages VEC whole rows of V in shared memory and gathers with a
// warp-sliced, bank-coloured hop table (one 16-byte shared load feeds VEC
// outputs).  The up phase combines whole row segments: a warp-uniform hop
// list, lanes over columns, coalesced loads of a column chunk that stays
// resident in L2 while every row of it is formed.
//
// Binary64 path: every element is rounded once to the fixed-point grid 2^-k
// (k = 1070 - emax, emax = biased exponent bound of max|v|) and held as
// (lo, hi) int32 words, X = hi * 2^24 + lo; hop sums are exact integer sums.
// The up phase forms, exactly in 128-bit integers,
//   T*A + X_own*B[n] + G*Bbeta,   A = -t 2^m, B[n] = U n 2^m, Bbeta = -beta 2^m
// (T = hop sum, G = fixed-point w_old) and rounds it once to binary64: the
// FP64 pipe (1.7 op/clk/SM on this part) is not used per element.  When t is
// a power of two and U a small dyadic number (the usual t = 1, integer U),
// the H v part fits int64 exactly and is rounded once; a Lanczos -beta w_old
// term is then one fused multiply-add.
#include <cstdint>
#include <cmath>
#include <type_traits>
#include <cuda_runtime.h>

#include "internal.h"
#include "row_blocks.cuh"
#include "hv_epilogue.cuh"

namespace hub {

namespace {

template <int VEC> struct FxVec;
template <> struct FxVec<1> { using T = int2; };
template <> struct FxVec<2> { using T = int4; };

template <int VEC> struct F32Vec;
template <> struct F32Vec<1> { using T = float; };
template <> struct F32Vec<2> { using T = float2; };
template <> struct F32Vec<4> { using T = float4; };

__device__ __forceinline__ float comp(float x, int) { return x; }
__device__ __forceinline__ float comp(float2 x, int i) { return i == 0 ? x.x : x.y; }
__device__ __forceinline__ float comp(float4 x, int i) { return i == 0 ? x.x : (i == 1 ? x.y : (i == 2 ? x.z : x.w)); }

// Row phase, binary64 fixed point: Y[u, d] = sum_{(d', s) in hops_dn(d)} s X[u, d'];
// also writes the fixed-point copy of V to Xg for the up phase.
// UPD: the previous Lanczos step's update is applied on the way in,
// v <- (v + ua fo) * uinv, rounded as k_axpy_scale_f64, and written back to v.
template <int VEC, typename EntT, bool UPD>
__global__ void __launch_bounds__(1024, 1) k_rows_f64x(std::conditional_t<UPD, double*, const double*> __restrict__ v,
                                                     long long* __restrict__ Y,
                                                     int2* __restrict__ Xg, int64_t Dup, int64_t Ddn,
                                                     const int64_t* __restrict__ boff,
                                                     const int32_t* __restrict__ bcnt,
                                                     const EntT* __restrict__ ent,
                                                     const int* __restrict__ emax_p, int fixed_emax,
                                                     const double* __restrict__ fo, double ua, double uinv,
                                                     const LzDev* __restrict__ dv) {
    using S = typename FxVec<VEC>::T;
    if constexpr (UPD) {
        if (dv != nullptr) {                              // device-resident step: the update's scalars
            ua = dv->ua;
            uinv = dv->uinv;
        }
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* X = reinterpret_cast<S*>(smem_raw);
    const int emax = fixed_emax > 0 ? fixed_emax : max(*emax_p, 1);
    const int lane = threadIdx.x & 31;
    const int64_t nblk = (Dup + VEC - 1) / VEC;
    const int64_t step = blockDim.x;
    constexpr int NL = UPD ? 2 : 4;                       // row elements per thread in flight
    {
        const int64_t z0 = staged_slots(Ddn) - 32;
        for (int i = threadIdx.x; i < 32; i += blockDim.x) {
            if constexpr (VEC == 1) X[z0 + i] = make_int2(0, 0);
            else X[z0 + i] = make_int4(0, 0, 0, 0);
        }
    }
    for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int64_t u0 = b * VEC;
        const int nrow = (int)((Dup - u0) < VEC ? (Dup - u0) : VEC);
        // stage rows u0 .. u0+nrow-1 as fixed point, NL loads per row in flight
        // (with UPD every load of a group is issued before the first store)
        for (int64_t d0 = threadIdx.x; d0 < Ddn; d0 += NL * step) {
            double xv[NL][VEC];
            [[maybe_unused]] double fv[NL][VEC];
#pragma unroll
            for (int i = 0; i < NL; ++i)
#pragma unroll
                for (int r = 0; r < VEC; ++r) {
                    const int64_t d = d0 + i * step;
                    const bool in = d < Ddn && r < nrow;
                    xv[i][r] = in ? v[(u0 + r) * Ddn + d] : 0.0;
                    if constexpr (UPD) fv[i][r] = in ? fo[(u0 + r) * Ddn + d] : 0.0;
                }
            if constexpr (UPD) {
#pragma unroll
                for (int i = 0; i < NL; ++i)
#pragma unroll
                    for (int r = 0; r < VEC; ++r) {
                        const int64_t d = d0 + i * step;
                        if (d < Ddn && r < nrow) {
                            xv[i][r] = fma(ua, fv[i][r], xv[i][r]) * uinv;
                            __stcs(v + (u0 + r) * Ddn + d, xv[i][r]);
                        }
                    }
            }
#pragma unroll
            for (int i = 0; i < NL; ++i) {
                const int64_t d = d0 + i * step;
                if (d >= Ddn) break;
                int w[2 * VEC];
#pragma unroll
                for (int r = 0; r < VEC; ++r) {
                    fx_split(xv[i][r], emax, w[2 * r], w[2 * r + 1]);
                    if (r < nrow) __stcg(Xg + (u0 + r) * Ddn + d, make_int2(w[2 * r], w[2 * r + 1]));
                }
                if constexpr (VEC == 1) X[d] = make_int2(w[0], w[1]);
                else X[d] = make_int4(w[0], w[1], w[2], w[3]);
            }
        }
        __syncthreads();
        for (int64_t d0 = threadIdx.x & ~31; d0 < Ddn; d0 += step) {
            const int64_t g = d0 >> 5;
            const int64_t d = d0 + lane;
            int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            for_each_hop<EntT>(ent + boff[g], bcnt[g], lane, [&](uint32_t e) {
                const int s = RowEnt<EntT>::sgn(e);           // padding reads a zero slot
                const S x = X[RowEnt<EntT>::idx(e)];
                a0 += s * x.x;
                a1 += s * x.y;
                if constexpr (VEC == 2) {
                    a2 += s * x.z;
                    a3 += s * x.w;
                }
            });
            if (d < Ddn) {
                Y[u0 * Ddn + d] = fx_join(a0, a1);
                if (VEC == 2 && nrow > 1) Y[(u0 + 1) * Ddn + d] = fx_join(a2, a3);
            }
        }
        __syncthreads();
    }
}

// Row phase for binary64 rows too long for shared memory: the fixed-point
// copy X is already in global memory (k_to_fixed) and the down-hop gathers
// read row u of it through L1/L2.
template <typename EntT>
__global__ void __launch_bounds__(512) k_rows_global_f64x(const int2* __restrict__ Xg, long long* __restrict__ Y,
                                                           int64_t Dup, int64_t Ddn,
                                                           const int64_t* __restrict__ boff,
                                                           const int32_t* __restrict__ bcnt,
                                                           const EntT* __restrict__ ent) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = blockIdx.x; u < Dup; u += gridDim.x) {
        const int2* X = Xg + u * Ddn;
        for (int64_t d0 = threadIdx.x & ~31; d0 < Ddn; d0 += blockDim.x) {
            const int64_t g = d0 >> 5;
            const int64_t d = d0 + lane;
            int a0 = 0, a1 = 0;
            for_each_hop<EntT>(ent + boff[g], bcnt[g], lane, [&](uint32_t e) {
                const uint32_t i = RowEnt<EntT>::idx(e);
                if (i < Ddn) {                                // padding: no zero slots in global rows
                    const int s = RowEnt<EntT>::sgn(e);
                    const int2 x = __ldg(X + i);
                    a0 += s * x.x;
                    a1 += s * x.y;
                }
            });
            if (d < Ddn) Y[u * Ddn + d] = fx_join(a0, a1);
        }
    }
}


// Up phase, binary64 fixed point (Algorithms 2 and 4):
//   W[u, c] = -t (sum_{(u', s) in hops_up(u)} s X[u', c] + Y[u, c]) + U n(u, c) X[u, c]  [- beta w_old]
// Row u of W is a signed combination of whole rows u' of X (Eq. H-Kroneckersum),
// so a warp builds one row segment of CC = 32 * VPL columns with lanes over
// columns: the hop list is warp-uniform and every access is coalesced.  Work
// items are (column chunk, block of RB rows); consecutive items share a chunk,
// which keeps that chunk of X resident in L2 while all rows are combined, and
// consecutive rows share part of their neighbours (reuse in L1).
constexpr int kUpRows = 16;

// Signed sum over the warp-uniform hop list of row u: targets t in
// list[kb .. kb+n), the first np with sign +1.  load(t) returns this lane's
// operand from row t; four independent loads are issued before they are
// added.  Loop bounds are warp-uniform, so the sign split costs no divergence.
template <typename Val, typename Load, typename Add>
__device__ __forceinline__ void uniform_hops(const uint32_t* __restrict__ list, int32_t kb, int n, int np, int lane,
                                             Val& P, Val& N, Load&& load, Add&& add) {
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int nk = min(32, n - k0);
        const uint32_t mine = lane < nk ? __ldg(list + kb + k0 + lane) : 0u;
        const int pend = max(0, min(nk, np - k0));
        int q = 0;
        for (; q + 4 <= pend; q += 4) {
            const Val a = load(__shfl_sync(0xffffffffu, mine, q));
            const Val b = load(__shfl_sync(0xffffffffu, mine, q + 1));
            const Val c = load(__shfl_sync(0xffffffffu, mine, q + 2));
            const Val d = load(__shfl_sync(0xffffffffu, mine, q + 3));
            add(P, a, b, c, d);
        }
        for (; q < pend; ++q) add(P, load(__shfl_sync(0xffffffffu, mine, q)));
        for (; q + 4 <= nk; q += 4) {
            const Val a = load(__shfl_sync(0xffffffffu, mine, q));
            const Val b = load(__shfl_sync(0xffffffffu, mine, q + 1));
            const Val c = load(__shfl_sync(0xffffffffu, mine, q + 2));
            const Val d = load(__shfl_sync(0xffffffffu, mine, q + 3));
            add(N, a, b, c, d);
        }
        for (; q < nk; ++q) add(N, load(__shfl_sync(0xffffffffu, mine, q)));
    }
}

// Lanczos reductions fused into the up-phase epilogue (Algorithm 1): each
// thread accumulates <w, f>, <w, w> and <f, f> over its outputs in a fixed
// order, the CTA sums its threads in a fixed tree, and the per-CTA partials
// (part[b], part[kPartStride + b], part[2 kPartStride + b]) are summed in
// index order afterwards, so the result is deterministic.  binary32 outputs
// use a float-float accumulator (exact product split + TwoSum), as the
// stand-alone dot kernel does.
struct FFAcc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add_product(float x, float y) {
        const float p = x * y;
        const float e = fmaf(x, y, -p);
        const float t = hi + p;
        const float bb = t - hi;
        lo += ((hi - (t - bb)) + (p - bb)) + e;
        hi = t;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Up phase, binary64 fixed point (Algorithms 2 and 4):
//   W[u, c] = -t (sum_{(u', s) in hops_up(u)} s X[u', c] + Y[u, c]) + U n(u, c) X[u, c]  [- beta w_old]
// Row u of W is a signed combination of whole rows u' of X (Eq. H-Kroneckersum),
// so a warp builds one row segment of CC = 32 * VPL columns with lanes over
// columns: the hop list is warp-uniform and every access is coalesced.  Work
// items are (column chunk, block of kUpRows rows); consecutive items share a
// chunk, which keeps that chunk of X resident in L2 while all rows are
// combined, and consecutive rows share part of their neighbours (L1 reuse).
// RED: also accumulate <W, fv>, <W, W> and <fv, fv> into part (block_sum3_store).
// PRE: the epilogue's own element and Y are requested before the gathers (their
// HBM latency then overlaps the hop sum); CT: CTAs per SM the launch bounds keep
template <int VPL, bool FAST, bool PRE = false, int CT = 4>
__global__ void __launch_bounds__(256, CT) k_up_f64x(const int2* __restrict__ X, const long long* __restrict__ Y,
                                                     double* w, const double* w_old, int64_t Dup, int64_t Ddn,
                                                     const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ npos,
                                                     const uint32_t* __restrict__ list,
                                                     const uint32_t* __restrict__ su,
                                                     const uint32_t* __restrict__ sd, EpiParams ep,
                                                     const int* __restrict__ emax_p, int fixed_emax) {
    using IV = typename FxVec<VPL>::T;
    __shared__ long long Bs[33];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) Bs[i] = i < ep.nB ? ep.B[i] : 0;
    __syncthreads();
    const int emax = fixed_emax > 0 ? fixed_emax : max(*emax_p, 1);
    const int k = 1070 - emax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int CC = 32 * VPL;
    const int64_t nchunk = (Ddn + CC - 1) / CC;
    const int64_t nrb = (Dup + kUpRows - 1) / kUpRows;
    // item = chunk * nrb + rb, advanced by gridDim.x without division
    int64_t chunk = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int64_t dch = gridDim.x / nrb, drb = gridDim.x % nrb;
    for (; chunk < nchunk; chunk += dch, rb += drb) {
        if (rb >= nrb) {
            rb -= nrb;
            ++chunk;
            if (chunk >= nchunk) break;
        }
        const int64_t c_raw = chunk * CC + (int64_t)lane * VPL;
        const bool act = c_raw < Ddn;
        const int64_t c = act ? c_raw : Ddn - VPL;     // tail lanes read a valid column, store nothing
        uint32_t sdc[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) sdc[j] = sd[c + j];
        const IV* base = reinterpret_cast<const IV*>(X + c);
        const int64_t uend = min(rb * kUpRows + kUpRows, Dup);
        for (int64_t u = rb * kUpRows + warp; u < uend; u += nw) {
            const int32_t kb = ptr[u];
            [[maybe_unused]] int4 t4p;
            [[maybe_unused]] longlong2 y2p;
            if constexpr (PRE && VPL == 2) {
                const int64_t J = u * Ddn + c;
                t4p = __ldg(reinterpret_cast<const int4*>(X + J));
                y2p = __ldcs(reinterpret_cast<const longlong2*>(Y + J));
            }
            IV P{}, N{};
            uniform_hops<IV>(list, kb, ptr[u + 1] - kb, npos[u], lane, P, N,
                [&](uint32_t t) { return __ldg(reinterpret_cast<const IV*>(reinterpret_cast<const int2*>(base) + (int64_t)t * Ddn)); },
                [](IV& A, auto... xs) { add4(A, xs...); });
            if (act) {
                const uint32_t su_u = su[u];
                const int64_t J = u * Ddn + c;
                int lo[VPL], hi[VPL];
                int2 xo[VPL];
                long long yv[VPL];
                if constexpr (VPL == 2) {
                    lo[0] = P.x - N.x; hi[0] = P.y - N.y; lo[1] = P.z - N.z; hi[1] = P.w - N.w;
                    int4 t4;
                    longlong2 y2;
                    if constexpr (PRE) {
                        t4 = t4p;
                        y2 = y2p;
                    } else {
                        t4 = __ldg(reinterpret_cast<const int4*>(X + J));
                        y2 = __ldcs(reinterpret_cast<const longlong2*>(Y + J));
                    }
                    xo[0] = make_int2(t4.x, t4.y);
                    xo[1] = make_int2(t4.z, t4.w);
                    yv[0] = y2.x;
                    yv[1] = y2.y;
                } else {
                    lo[0] = P.x - N.x; hi[0] = P.y - N.y;
                    xo[0] = __ldg(X + J);
                    yv[0] = __ldcs(Y + J);
                }
                double r[VPL];
#pragma unroll
                for (int j = 0; j < VPL; ++j) {
                    if constexpr (FAST) {
                        // exact: |T| < 2^55, |X| <= 2^48, |Uint * n| < 2^14 and tshift <= 6
                        long long Pv = (fx_join(lo[j], hi[j]) + yv[j]) << ep.tshift;
                        if (ep.tneg == 0) Pv = -Pv;
                        Pv += ep.Uint * (long long)__popc(su_u & sdc[j]) * fx_join(xo[j].x, xo[j].y);
                        r[j] = i64_scaled_to_double(Pv, -(k + ep.ju));
                        if (w_old != nullptr) r[j] = fma(ep.mbeta, w_old[J + j], r[j]);
                    } else {
                        I128 acc{0ull, 0ll};
                        mac128(acc, fx_join(lo[j], hi[j]) + yv[j], ep.A);
                        mac128(acc, fx_join(xo[j].x, xo[j].y), Bs[__popc(su_u & sdc[j])]);
                        if (w_old != nullptr) {
                            int glo, ghi;
                            fx_split(w_old[J + j], emax, glo, ghi);
                            mac128(acc, fx_join(glo, ghi), ep.Bbeta);
                        }
                        r[j] = i128_to_double(acc, -(k + ep.m));
                    }
                }
                if constexpr (VPL == 2) __stcs(reinterpret_cast<double2*>(w + J), make_double2(r[0], r[1]));
                else __stcs(w + J, r[0]);
            }
        }
    }
}

// Lanczos-step variant of k_up_f64x (Algorithm 1 fused with Algorithms 2, 4):
// W = H f - beta w_old and, per CTA, the partials of <W, f>, <W, W> and
// <f, f> (block_sum3_store).  Its epilogue streams four arrays (own element,
// Y, w_old, f), so with 16-byte vectors their loads are issued before the
// gathers; the extra live registers cost one CTA per SM (3 instead of 4).
template <int VPL, bool FAST>
__global__ void __launch_bounds__(256, 3) k_up_step_f64x(const int2* __restrict__ X, const long long* __restrict__ Y,
                                                     double* w, const double* w_old, int64_t Dup, int64_t Ddn,
                                                     const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ npos,
                                                     const uint32_t* __restrict__ list,
                                                     const uint32_t* __restrict__ su,
                                                     const uint32_t* __restrict__ sd, EpiParams ep,
                                                     const int* __restrict__ emax_p, int fixed_emax,
                                                     const double* __restrict__ fv, double* part,
                                                     const LzDev* __restrict__ dv) {
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    using IV = typename FxVec<VPL>::T;
    __shared__ long long Bs[33];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) Bs[i] = i < ep.nB ? ep.B[i] : 0;
    __syncthreads();
    if (dv != nullptr) {                                  // device-resident step: beta_j on the device
        const double b = dv->beta;
        ep.mbeta = -b;
        ep.Bbeta = llround(ldexp(-b, ep.m));
    }
    const int emax = fixed_emax > 0 ? fixed_emax : max(*emax_p, 1);
    const int k = 1070 - emax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int CC = 32 * VPL;
    const int64_t nchunk = (Ddn + CC - 1) / CC;
    const int64_t nrb = (Dup + kUpRows - 1) / kUpRows;
    // item = chunk * nrb + rb, advanced by gridDim.x without division
    int64_t chunk = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int64_t dch = gridDim.x / nrb, drb = gridDim.x % nrb;
    for (; chunk < nchunk; chunk += dch, rb += drb) {
        if (rb >= nrb) {
            rb -= nrb;
            ++chunk;
            if (chunk >= nchunk) break;
        }
        const int64_t c_raw = chunk * CC + (int64_t)lane * VPL;
        const bool act = c_raw < Ddn;
        const int64_t c = act ? c_raw : Ddn - VPL;     // tail lanes read a valid column, store nothing
        uint32_t sdc[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) sdc[j] = sd[c + j];
        const IV* base = reinterpret_cast<const IV*>(X + c);
        const int64_t uend = min(rb * kUpRows + kUpRows, Dup);
        for (int64_t u = rb * kUpRows + warp; u < uend; u += nw) {
            const int32_t kb = ptr[u];
            const int64_t J = u * Ddn + c;
            // streamed operands of the epilogue, requested before the gathers
            double wpre[VPL], fpre[VPL];
            int4 t4p;
            longlong2 y2p;
            if constexpr (VPL == 2) {
                t4p = __ldg(reinterpret_cast<const int4*>(X + J));
                y2p = __ldcs(reinterpret_cast<const longlong2*>(Y + J));
                if (w_old != nullptr) {
                    const double2 q = __ldcs(reinterpret_cast<const double2*>(w_old + J));
                    wpre[0] = q.x; wpre[1] = q.y;
                }
                {
                    const double2 q = __ldcs(reinterpret_cast<const double2*>(fv + J));
                    fpre[0] = q.x; fpre[1] = q.y;
                }
            }
            IV P{}, N{};
            uniform_hops<IV>(list, kb, ptr[u + 1] - kb, npos[u], lane, P, N,
                [&](uint32_t t) { return __ldg(reinterpret_cast<const IV*>(reinterpret_cast<const int2*>(base) + (int64_t)t * Ddn)); },
                [](IV& A, auto... xs) { add4(A, xs...); });
            if (act) {
                const uint32_t su_u = su[u];
                int lo[VPL], hi[VPL];
                int2 xo[VPL];
                long long yv[VPL];
                if constexpr (VPL == 2) {
                    lo[0] = P.x - N.x; hi[0] = P.y - N.y; lo[1] = P.z - N.z; hi[1] = P.w - N.w;
                    const int4 t4 = t4p;
                    xo[0] = make_int2(t4.x, t4.y);
                    xo[1] = make_int2(t4.z, t4.w);
                    const longlong2 y2 = y2p;
                    yv[0] = y2.x;
                    yv[1] = y2.y;
                } else {
                    lo[0] = P.x - N.x; hi[0] = P.y - N.y;
                    xo[0] = __ldg(X + J);
                    yv[0] = __ldcs(Y + J);
                }
                double r[VPL];
#pragma unroll
                for (int j = 0; j < VPL; ++j) {
                    if constexpr (FAST) {
                        // exact: |T| < 2^55, |X| <= 2^48, |Uint * n| < 2^14 and tshift <= 6
                        long long Pv = (fx_join(lo[j], hi[j]) + yv[j]) << ep.tshift;
                        if (ep.tneg == 0) Pv = -Pv;
                        Pv += ep.Uint * (long long)__popc(su_u & sdc[j]) * fx_join(xo[j].x, xo[j].y);
                        r[j] = i64_scaled_to_double(Pv, -(k + ep.ju));
                        if (w_old != nullptr) r[j] = fma(ep.mbeta, VPL == 2 ? wpre[j] : w_old[J + j], r[j]);
                    } else {
                        I128 acc{0ull, 0ll};
                        mac128(acc, fx_join(lo[j], hi[j]) + yv[j], ep.A);
                        mac128(acc, fx_join(xo[j].x, xo[j].y), Bs[__popc(su_u & sdc[j])]);
                        if (w_old != nullptr) {
                            int glo, ghi;
                            fx_split(w_old[J + j], emax, glo, ghi);
                            mac128(acc, fx_join(glo, ghi), ep.Bbeta);
                        }
                        r[j] = i128_to_double(acc, -(k + ep.m));
                    }
                }
                if constexpr (VPL == 2) __stcs(reinterpret_cast<double2*>(w + J), make_double2(r[0], r[1]));
                else __stcs(w + J, r[0]);
                {
                    double fj[VPL];
                    if constexpr (VPL == 2) {
                        fj[0] = fpre[0];
                        fj[1] = fpre[1];
                    } else {
                        fj[0] = __ldcs(fv + J);
                    }
#pragma unroll
                    for (int j = 0; j < VPL; ++j) {
                        s1 = fma(r[j], fj[j], s1);
                        s2 = fma(r[j], r[j], s2);
                        s3 = fma(fj[j], fj[j], s3);
                    }
                }
            }
        }
    }
    block_sum3_store(s1, s2, s3, part);
}

__device__ __forceinline__ void addf(float& A, float a, float b, float c, float d) { A += (a + b) + (c + d); }
__device__ __forceinline__ void addf(float& A, float a) { A += a; }
__device__ __forceinline__ void addf(float2& A, float2 a, float2 b, float2 c, float2 d) {
    A.x += (a.x + b.x) + (c.x + d.x);
    A.y += (a.y + b.y) + (c.y + d.y);
}
__device__ __forceinline__ void addf(float2& A, float2 a) { A.x += a.x; A.y += a.y; }
__device__ __forceinline__ void addf(float4& A, float4 a, float4 b, float4 c, float4 d) {
    A.x += (a.x + b.x) + (c.x + d.x);
    A.y += (a.y + b.y) + (c.y + d.y);
    A.z += (a.z + b.z) + (c.z + d.z);
    A.w += (a.w + b.w) + (c.w + d.w);
}
__device__ __forceinline__ void addf(float4& A, float4 a) { A.x += a.x; A.y += a.y; A.z += a.z; A.w += a.w; }

// Up phase, binary32: same decomposition, float arithmetic
// CTAs per SM of the binary32 up phase: 5 at <= 51 registers, 4 where 4
// columns per lane or the Lanczos variant's prefetched operands need more
template <int VPL, bool RED = false>
constexpr int up32_ctas() { return (RED || VPL == 4) ? 4 : 5; }

template <int VPL, bool RED>
__global__ void __launch_bounds__(256, up32_ctas<VPL, RED>()) k_up_f32(const float* __restrict__ v, const float* __restrict__ Y, float* w,
                                                    const float* w_old, int64_t Dup, int64_t Ddn,
                                                    const int32_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ npos,
                                                    const uint32_t* __restrict__ list,
                                                    const uint32_t* __restrict__ su,
                                                    const uint32_t* __restrict__ sd, float mt, float U, float mbeta,
                                                    double* part, const LzDev* __restrict__ dv) {
    FFAcc s1, s2, s3;
    if (dv != nullptr) mbeta = (float)-dv->beta;          // device-resident step: beta_j on the device
    using V = typename F32Vec<VPL>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int CC = 32 * VPL;
    const int64_t nchunk = (Ddn + CC - 1) / CC;
    const int64_t nrb = (Dup + kUpRows - 1) / kUpRows;
    int64_t chunk = blockIdx.x / nrb, rb = blockIdx.x % nrb;
    const int64_t dch = gridDim.x / nrb, drb = gridDim.x % nrb;
    for (; chunk < nchunk; chunk += dch, rb += drb) {
        if (rb >= nrb) {
            rb -= nrb;
            ++chunk;
            if (chunk >= nchunk) break;
        }
        const int64_t c_raw = chunk * CC + (int64_t)lane * VPL;
        const bool act = c_raw < Ddn;
        const int64_t c = act ? c_raw : Ddn - VPL;
        uint32_t sdc[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) sdc[j] = sd[c + j];
        const float* base = v + c;
        const int64_t uend = min(rb * kUpRows + kUpRows, Dup);
        for (int64_t u = rb * kUpRows + warp; u < uend; u += nw) {
            const int32_t kb = ptr[u];
            const int64_t J = u * Ddn + c;
            V xpre{}, ypre{}, wpre{};
            if constexpr (RED) {                      // Lanczos step: epilogue operands before the gathers
                xpre = __ldg(reinterpret_cast<const V*>(v + J));
                ypre = __ldcs(reinterpret_cast<const V*>(Y + J));
                if (w_old != nullptr) wpre = __ldcs(reinterpret_cast<const V*>(w_old + J));
            }
            V P{}, N{};
            uniform_hops<V>(list, kb, ptr[u + 1] - kb, npos[u], lane, P, N,
                [&](uint32_t t) { return __ldg(reinterpret_cast<const V*>(base + (int64_t)t * Ddn)); },
                [](V& A, auto... xs) { addf(A, xs...); });
            if (act) {
                const uint32_t su_u = su[u];
                const V xo = RED ? xpre : __ldg(reinterpret_cast<const V*>(v + J));
                const V yv = RED ? ypre : __ldcs(reinterpret_cast<const V*>(Y + J));
                float r[VPL];
#pragma unroll
                for (int j = 0; j < VPL; ++j) {
                    const float nd = (float)__popc(su_u & sdc[j]);
                    r[j] = fmaf(mt, (comp(P, j) - comp(N, j)) + comp(yv, j), U * nd * comp(xo, j));
                    if (w_old != nullptr) r[j] = fmaf(mbeta, RED ? comp(wpre, j) : w_old[J + j], r[j]);
                }
                if constexpr (VPL == 4) __stcs(reinterpret_cast<float4*>(w + J), make_float4(r[0], r[1], r[2], r[3]));
                else if constexpr (VPL == 2) __stcs(reinterpret_cast<float2*>(w + J), make_float2(r[0], r[1]));
                else __stcs(w + J, r[0]);
                if constexpr (RED) {
#pragma unroll
                    for (int j = 0; j < VPL; ++j) {
                        s1.add_product(r[j], comp(xo, j));
                        s2.add_product(r[j], r[j]);
                        s3.add_product(comp(xo, j), comp(xo, j));
                    }
                }
            }
        }
    }
    if constexpr (RED) block_sum3_store(s1.value(), s2.value(), s3.value(), part);
}

// ---------------------------------------------------------------------------
// binary32 variants: same structure, float arithmetic (UPD: the deferred
// Lanczos update, rounded as k_axpy_scale_f32)
template <int VEC, typename EntT, bool UPD>
__global__ void __launch_bounds__(1024, 1) k_rows_f32(std::conditional_t<UPD, float*, const float*> __restrict__ v,
                                                    float* __restrict__ Y, int64_t Dup,
                                                    int64_t Ddn, const int64_t* __restrict__ boff,
                                                    const int32_t* __restrict__ bcnt,
                                                    const EntT* __restrict__ ent,
                                                    const float* __restrict__ fo, float ua, float uinv,
                                                    const LzDev* __restrict__ dv) {
    using S = typename F32Vec<VEC>::T;
    if constexpr (UPD) {
        if (dv != nullptr) {
            ua = (float)dv->ua;
            uinv = (float)dv->uinv;
        }
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* X = reinterpret_cast<S*>(smem_raw);
    float* Xf = reinterpret_cast<float*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int64_t nblk = (Dup + VEC - 1) / VEC;
    const int64_t step = blockDim.x;
    constexpr int NL = UPD ? 2 : 4;                       // row elements per thread in flight
    {
        const int64_t z0 = staged_slots(Ddn) - 32;
        for (int i = threadIdx.x; i < 32 * VEC; i += blockDim.x) Xf[z0 * VEC + i] = 0.0f;
    }
    for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int64_t u0 = b * VEC;
        const int nrow = (int)((Dup - u0) < VEC ? (Dup - u0) : VEC);
        // NL loads per row in flight (with UPD all issued before the first store)
        for (int64_t d0 = threadIdx.x; d0 < Ddn; d0 += NL * step) {
            float xv[NL][VEC];
            [[maybe_unused]] float fv[NL][VEC];
#pragma unroll
            for (int i = 0; i < NL; ++i)
#pragma unroll
                for (int r = 0; r < VEC; ++r) {
                    const int64_t d = d0 + i * step;
                    const bool in = d < Ddn && r < nrow;
                    xv[i][r] = in ? v[(u0 + r) * Ddn + d] : 0.0f;
                    if constexpr (UPD) fv[i][r] = in ? fo[(u0 + r) * Ddn + d] : 0.0f;
                }
            if constexpr (UPD) {
#pragma unroll
                for (int i = 0; i < NL; ++i)
#pragma unroll
                    for (int r = 0; r < VEC; ++r) {
                        const int64_t d = d0 + i * step;
                        if (d < Ddn && r < nrow) {
                            xv[i][r] = fmaf(ua, fv[i][r], xv[i][r]) * uinv;
                            __stcs(v + (u0 + r) * Ddn + d, xv[i][r]);
                        }
                    }
            }
#pragma unroll
            for (int i = 0; i < NL; ++i) {
                const int64_t d = d0 + i * step;
                if (d >= Ddn) break;
#pragma unroll
                for (int r = 0; r < VEC; ++r) Xf[d * VEC + r] = xv[i][r];
            }
        }
        __syncthreads();
        for (int64_t d0 = threadIdx.x & ~31; d0 < Ddn; d0 += step) {
            const int64_t g = d0 >> 5;
            const int64_t d = d0 + lane;
            float acc[VEC];
#pragma unroll
            for (int r = 0; r < VEC; ++r) acc[r] = 0.0f;
            for_each_hop<EntT>(ent + boff[g], bcnt[g], lane, [&](uint32_t e) {
                const float s = (float)RowEnt<EntT>::sgn(e);  // padding reads a zero slot
                const S x = X[RowEnt<EntT>::idx(e)];
#pragma unroll
                for (int r = 0; r < VEC; ++r) acc[r] = fmaf(s, comp(x, r), acc[r]);
            });
            if (d < Ddn) {
#pragma unroll
                for (int r = 0; r < VEC; ++r)
                    if (r < nrow) Y[(u0 + r) * Ddn + d] = acc[r];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// thread-safe (static initialisation runs once; callers on other threads wait)
int smem_optin() {
    static const int v = [] {
        int dev = 0, x = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return x > 0 ? x : 48 * 1024;
    }();
    return v;
}

int sms() {
    static const int n = [] {
        int dev = 0, x = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, dev);
        return x > 0 ? x : 1;
    }();
    return n;
}

// largest VEC in {4,2,1} (capped by vmax) whose staging buffer (with the
// zero slots) fits
int pick_vec(int64_t len, int elem_bytes, int vmax, int reserve) {
    for (int v = vmax; v >= 1; v >>= 1)
        if (staged_slots(len) * elem_bytes * v + reserve <= smem_optin()) return v;
    return 0;
}

struct Launch {
    int blocks, threads;
    size_t smem;
};

// ctas = 0: two CTAs per SM when both fit, else one
Launch shape(size_t smem, int ctas) {
    const size_t per_sm = 228 * 1024;
    const int fit = (int)std::max<size_t>(1, std::min<size_t>(2, per_sm / (smem + 2048)));
    if (ctas <= 0 || ctas > fit) ctas = fit;
    Launch L;
    L.smem = smem;
    L.threads = ctas == 1 ? 1024 : 512;
    L.blocks = sms() * ctas;
    return L;
}

// The dynamic shared-memory limit is a per-kernel attribute shared by every
// host thread: raise it once per kernel (the template parameter is the kernel
// itself, so each instantiation has its own flag), to the device maximum, so
// that a concurrent launch of the same kernel can never see a lower limit.
// The limit is what the opt-in maximum leaves next to the kernel's static
// shared memory.
template <auto Kern>
void allow_smem() {
    static const bool once = [] {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, Kern) != cudaSuccess) return false;
        const int dyn = smem_optin() - (int)fa.sharedSizeBytes;
        return cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess;
    }();
    (void)once;
}

// a grid of at most `full` CTAs and no more than the work items
int grid_cap(int full, int64_t items) { return (int)std::max<int64_t>(1, std::min<int64_t>(full, items)); }

// requested vec (0 = largest that fits), capped to what fits
int choose_vec(int req, int64_t len, int elem_bytes, int vmax, int reserve) {
    const int fit = pick_vec(len, elem_bytes, vmax, reserve);
    if (req <= 0 || req > fit) return fit;
    return req;
}

}  // namespace

// Returns HUB_OK and launches, or returns -1 when the staging buffers do not fit
// (the caller then uses the single-pass gather kernel).
bool hv_phases_fuse(const hubbard_sector* H, int dtype) {
    if (sms() * 5 > kPartStride) return false;
    return dtype == HUB_F64 || choose_vec(H->vec_rows, H->Ddn, 4, 4, 0) != 0;
}

bool hv_phases_capturable(const hubbard_sector* H, int dtype) {
    // the binary64 path for rows longer than shared memory uploads its fixed
    // exponent word from host memory on each call
    return hv_phases_fuse(H, dtype) && (dtype == HUB_F32 || choose_vec(H->vec_rows, H->Ddn, 8, 2, 0) != 0);
}

int launch_hv_phases(hubbard_sector* H, const void* v, void* w, int dtype, double beta, const void* w_old,
                     void* ybuf, int fixed_emax, cudaStream_t s, double* part, int* nparts,
                     const RowUpdate* upd, const LzDev* dv) {
    if (nparts != nullptr) *nparts = 0;
    if (sms() * 5 > kPartStride) part = nullptr;        // partial arrays too short: no fused reduction
    const DevSpin& up = H->dev[0];
    const DevSpin& dn = H->dev[1];
    const int64_t Dup = H->Dup, Ddn = H->Ddn;
    const bool dn16 = dn.ent16 != nullptr;
    // up-phase CTAs: as many as the launch bounds keep resident (the phase is
    // bound by L2 latency, so occupancy is what counts: 4 per SM at <= 64
    // registers for binary64 (3 for the Lanczos variant, whose prefetched
    // epilogue operands need the registers), 5 at <= 51 for binary32 with up
    // to 2 columns per lane; measured best)
    if (dtype == HUB_F64) {
        const int va = choose_vec(H->vec_rows, Ddn, 8, 2, 0);
        int* emax = H->status;
        // the deferred update goes into the row phase when it stages rows in
        // shared memory with a fixed exponent bound; otherwise it is one pass first
        if (upd != nullptr && (va == 0 || fixed_emax <= 0)) {
            if (int rc = launch_axpy_scale(upd->a, upd->inv, upd->fo, const_cast<void*>(v), H->D, dtype, s, upd->dv))
                return rc;
            upd = nullptr;
        }
        if (fixed_emax <= 0) {
            HUB_CUDA(cudaMemsetAsync(emax, 0, sizeof(int), s));
            launch_max_exponent((const double*)v, H->D, emax, s);
            if (w_old != nullptr) launch_max_exponent((const double*)w_old, H->D, emax, s);
        }
        Launch LA = shape((size_t)staged_slots(Ddn) * 8 * std::max(va, 1), H->ctas_rows);
        LA.blocks = grid_cap(LA.blocks, (Dup + std::max(va, 1) - 1) / std::max(va, 1));   // no idle CTAs
        long long* Y = (long long*)ybuf;
        int2* Xg = (int2*)((char*)ybuf + (size_t)H->D * 8);
        int extra = 0;
        if (va == 0) {
            // rows longer than shared memory: fixed-point copy first, then gathers through L1/L2
            int* em = emax;
            int* fixed_word = H->status + 1;
            if (fixed_emax > 0) {
                H->fixed_emax_host = fixed_emax;
                HUB_CUDA(cudaMemcpyAsync(fixed_word, &H->fixed_emax_host, sizeof(int), cudaMemcpyHostToDevice, s));
                em = fixed_word;
            }
            launch_to_fixed((const double*)v, H->D, Xg, em, s);
            if (dn16) {
                k_rows_global_f64x<uint16_t><<<grid_cap(sms() * 4, Dup), 512, 0, s>>>(Xg, Y, Dup, Ddn, dn.blk_off,
                                                                                         dn.blk_cnt, dn.ent16);
            } else {
                k_rows_global_f64x<uint32_t><<<grid_cap(sms() * 4, Dup), 512, 0, s>>>(Xg, Y, Dup, Ddn, dn.blk_off,
                                                                                         dn.blk_cnt, dn.ent32);
            }
            extra = 2;
        } else {
#define ROWS64_U(V, E, P, U)                                                                                \
    allow_smem<k_rows_f64x<V, E, U>>();                                                                      \
    k_rows_f64x<V, E, U><<<LA.blocks, LA.threads, LA.smem, s>>>((double*)const_cast<void*>(v), Y, Xg, Dup,   \
        Ddn, dn.blk_off, dn.blk_cnt, P, emax, fixed_emax, upd ? (const double*)upd->fo : nullptr,            \
        upd ? upd->a : 0.0, upd ? upd->inv : 1.0, upd ? upd->dv : nullptr)
#define ROWS64(V, E, P) if (upd) { ROWS64_U(V, E, P, true); } else { ROWS64_U(V, E, P, false); }
        if (va == 2) {
            if (dn16) { ROWS64(2, uint16_t, dn.ent16); } else { ROWS64(2, uint32_t, dn.ent32); }
        } else {
            if (dn16) { ROWS64(1, uint16_t, dn.ent16); } else { ROWS64(1, uint32_t, dn.ent32); }
        }
        extra = 1;
        }
#undef ROWS64
#undef ROWS64_U
        const EpiParams ep = make_epilogue(H->t, H->U, H->ns, w_old ? beta : 0.0, H->host[0].W + H->host[1].W);
        // columns per lane in the up phase: 2 when Ddn is even (16-byte loads)
        const int vpl = ((Ddn & 1) == 0 && H->vec_cols != 1) ? 2 : 1;
        const int64_t up_items = ((Ddn + 32 * vpl - 1) / (32 * vpl)) * ((Dup + kUpRows - 1) / kUpRows);
        const int up_grid = grid_cap(sms() * (part != nullptr ? 3 : 4), up_items);
        // standalone up phase: request the epilogue's own element and Y before
        // the gathers (at 3 CTAs/SM for the registers) where that measured
        // faster -- the 128-bit epilogue and rows staged from global memory --
        // unless the schedule fixes it (ctas_cols 1: no, 2: yes)
        const bool pre = H->ctas_cols == 2 || (H->ctas_cols == 0 && (!ep.fast || va == 0));
#define UP64(K, V, F)                                                                                       \
    K<V, F><<<up_grid, 256, 0, s>>>(Xg, Y, (double*)w, (const double*)w_old, Dup, Ddn, up.pn_ptr,             \
        up.pn_npos, up.pn_list, up.states, dn.states, ep, emax, fixed_emax
#define UP64P(V, F, CT)                                                                                     \
    k_up_f64x<V, F, true, CT><<<grid_cap(sms() * CT, up_items), 256, 0, s>>>(Xg, Y, (double*)w,               \
        (const double*)w_old, Dup, Ddn,                                                                    \
        up.pn_ptr, up.pn_npos, up.pn_list, up.states, dn.states, ep, emax, fixed_emax)
#define UP64_R(V, F)                                                                                        \
    if (part != nullptr) { UP64(k_up_step_f64x, V, F), (const double*)v, part, dv); }                      \
    else if (V == 2 && pre) { UP64P(V, F, 3); }                                                            \
    else { UP64(k_up_f64x, V, F)); }
        if (vpl == 2) {
            if (ep.fast) { UP64_R(2, true) } else { UP64_R(2, false) }
        } else {
            if (ep.fast) { UP64_R(1, true) } else { UP64_R(1, false) }
        }
#undef UP64_R
#undef UP64P
#undef UP64
        if (part != nullptr && nparts != nullptr) *nparts = up_grid;
        HUB_CUDA(cudaGetLastError());
        count_launches(1 + extra + (fixed_emax <= 0 ? (w_old ? 2 : 1) : 0));
        return HUB_OK;
    }
    // binary32
    const int va = choose_vec(H->vec_rows, Ddn, 4, 4, 0);
    if (va == 0) return -1;
    Launch LA = shape((size_t)staged_slots(Ddn) * 4 * va, H->ctas_rows);
    LA.blocks = grid_cap(LA.blocks, (Dup + va - 1) / va);
    float* Y = (float*)ybuf;
    // columns per lane in the up phase: the widest aligned vector load, capped by vec_cols
    int vpl = (Ddn & 3) == 0 ? 4 : ((Ddn & 1) == 0 ? 2 : 1);
    if (H->vec_cols > 0 && H->vec_cols < vpl) vpl = H->vec_cols;
#define ROWS32_U(V, E, P, U)                                                                               \
    allow_smem<k_rows_f32<V, E, U>>();                                                                      \
    k_rows_f32<V, E, U><<<LA.blocks, LA.threads, LA.smem, s>>>((float*)const_cast<void*>(v), Y, Dup, Ddn,   \
        dn.blk_off, dn.blk_cnt, P, upd ? (const float*)upd->fo : nullptr, upd ? (float)upd->a : 0.0f,       \
        upd ? (float)upd->inv : 1.0f, upd ? upd->dv : nullptr)
#define ROWS32(V, E, P) if (upd) { ROWS32_U(V, E, P, true); } else { ROWS32_U(V, E, P, false); }
#define BOTH32(M, V, F, P16, P32) if (F) { M(V, uint16_t, P16); } else { M(V, uint32_t, P32); }
    if (va == 4) { BOTH32(ROWS32, 4, dn16, dn.ent16, dn.ent32) }
    else if (va == 2) { BOTH32(ROWS32, 2, dn16, dn.ent16, dn.ent32) }
    else { BOTH32(ROWS32, 1, dn16, dn.ent16, dn.ent32) }
#undef BOTH32
#undef ROWS32
#undef ROWS32_U
    int up_grid = 0;
#define UP32(V)                                                                                            \
    {                                                                                                      \
        up_grid = grid_cap(sms() * (part != nullptr ? up32_ctas<V, true>() : up32_ctas<V, false>()),      \
                           ((Ddn + 32 * V - 1) / (32 * V)) * ((Dup + kUpRows - 1) / kUpRows));             \
        if (part != nullptr)                                                                               \
            k_up_f32<V, true><<<up_grid, 256, 0, s>>>((const float*)v, Y, (float*)w, (const float*)w_old,  \
                Dup, Ddn, up.pn_ptr, up.pn_npos, up.pn_list, up.states, dn.states, (float)-H->t,           \
                (float)H->U, (float)-beta, part, dv);                                                      \
        else                                                                                               \
            k_up_f32<V, false><<<up_grid, 256, 0, s>>>((const float*)v, Y, (float*)w, (const float*)w_old, \
                Dup, Ddn, up.pn_ptr, up.pn_npos, up.pn_list, up.states, dn.states, (float)-H->t,           \
                (float)H->U, (float)-beta, part, nullptr);                                                 \
    }
    if (vpl == 4) { UP32(4) } else if (vpl == 2) { UP32(2) } else { UP32(1) }
#undef UP32
    if (part != nullptr && nparts != nullptr) *nparts = up_grid;
    HUB_CUDA(cudaGetLastError());
    count_launches(2);
    return HUB_OK;
}

}  // namespace hub
