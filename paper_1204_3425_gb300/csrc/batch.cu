// Many sectors solved in one persistent launch (Sec. 2.2, Algorithm 1,
// run entirely on the device for each sector).
//
// The paper measured that sectors below ~10 sites leave a GPU idle (Sec. 5:
// 16 % occupancy at 8 sites).  Here one cooperative launch solves a whole
// batch in two parts:
//  * sectors above a size threshold advance in lock step, one Lanczos step per
//    grid-synchronous sweep whose phases spread the rows of every active
//    sector over all warps (sweep_solve);
//  * the rest are tasks of one CTA each, claimed by the CTAs from a global
//    counter (largest work first); a task that fits keeps the fixed-point copy
//    of its Lanczos vector in shared memory.
// Rows staged in shared memory take their down-hops from the coloured row
// table of the single-sector kernels (row_blocks.cuh), built here for 8-byte
// slots.
// Grid barriers are bounded (a timeout sets an error word; later waits fail
// fast).  Every reduction is summed in a fixed order, so the result of a
// sector does not depend on which other sectors share the launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "row_blocks.cuh"
#include "splitmix.cuh"

namespace hub {
namespace {

constexpr int kBatchThreads = 480;   // 15 warps: two CTAs per SM leave each warp a 945-element row slice
constexpr int kCheckEvery = 4;        // Ritz-value test every few steps

// Per-shape schedule bits (the autotuner's table, one entry per sector shape):
constexpr int kModeFlat = 1;    // a one-CTA task keeps its whole fixed-point vector in shared memory when it fits
constexpr int kModeStage = 2;   // a warp-per-row pass stages the row in shared memory for the down-hops
constexpr int kModeDefault = kModeFlat | kModeStage;

struct SectorDesc {
    int64_t Dup, Ddn, D;
    int64_t voff;          // element offset of the sector's vectors in the pools
    int64_t up_rp, dn_rp;  // offsets of the row pointers in the rowptr pool
    int64_t up_ent, dn_ent;
    int64_t up_st, dn_st;
    int64_t ab;            // offset of its a/b history (2 * max_iters doubles)
    int64_t dn_blk;        // first group of its down-spin row table in the block pools (-1: none)
    double t, U;
    int32_t mode;          // schedule bits of its shape (kModeFlat, kModeStage)
    int32_t pad;
    unsigned long long seed;   // queued tasks: start vector drawn in place from this seed
};

struct BatchParams {
    const SectorDesc* sec;
    const int* tasks;      // one-CTA sector ids, largest work first, claimed through claim[2]
    int ntasks;
    const int32_t* rp;     // pooled row pointers
    const uint32_t* ent;   // pooled packed hop entries (target << 1) | neg
    const uint32_t* st;    // pooled basis words
    const int64_t* bo;     // pooled row tables (coloured for 8-byte slots): first entry of each group
    const int32_t* bc;     //   half-blocks of 4 slots per group
    const uint16_t* be;    //   entries (15-bit staged slot index, bit 15 = sign -1)
    const double* v0;      // caller start vectors (concatenated)
    double* f;             // Lanczos vector pools (workspace)
    double* g;
    int2* xg;              // global fixed-point copies (sectors not staged in shared memory)
    double* ab;            // a/b histories
    lanczos_result* res;   // [sector]
    int* err;              // batch error word
    int max_iters;         // stride of the a/b histories
    int iter_cap;          // steps at most (<= max_iters; shorter in autotuner trials)
    double tol;
    int smem_elems;        // capacity of the shared fixed-point buffer
    int mode_force;        // >= 0: schedule bits for every sector (autotuner trials); -1: per sector
    long long spin_limit;  // bounded waits
    // grid-synchronous sweep (sectors above the schedule's size threshold)
    int nswp;
    int sweep_ctas;        // the first sweep_ctas CTAs run the sweep; the others start on the tasks at once
    const int* swp;        // [nswp] sector ids
    const int64_t* rowoff; // [nswp + 1] prefix sums of their D_up
    const int32_t* rowsec; // [rowoff[nswp]] sweep index k of each row
    double* rowpart;       // [rowoff[nswp]][3] per-row partial sums
    struct SweepState* sst;// [nswp]
    unsigned int* gbar;    // grid barrier counter
    int* nactive;          // sectors of the sweep still iterating
    unsigned long long* claim; // [3] row counters of the sweep's element and update phases, task counter
    // queue mode (hubbard_queue_*; q_posted == nullptr: a batch): tasks are
    // posted while the kernel runs; task n uses descriptor / vector / result
    // slot n % q_cap, its start vector drawn from its seed
    const volatile unsigned int* q_posted;  // host-mapped: tasks posted so far
    const volatile unsigned int* q_stop;    // host-mapped: nonzero -> leave once nothing is left to claim
    unsigned int* q_claim;                  // device: tasks claimed so far
    volatile unsigned int* q_done;          // host-mapped, per slot: task number + 1 once its result is written
    int q_cap;
    long long q_idle;                       // polls of an empty queue before the kernel leaves
};

__device__ __forceinline__ unsigned int ld_acquire_sys(const volatile unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// a queued task's descriptor, read through L2 (the slot was rewritten by the host since the last task in it)
__device__ __forceinline__ SectorDesc load_desc_cg(const SectorDesc* p) {
    static_assert(sizeof(SectorDesc) % 8 == 0, "descriptor of 8-byte words");
    SectorDesc d;
    const long long* src = reinterpret_cast<const long long*>(p);
    long long* dst = reinterpret_cast<long long*>(&d);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(SectorDesc) / 8); ++i) dst[i] = __ldcg(src + i);
    return d;
}

// Lanczos state of a swept sector between the phases of one iteration.
struct SweepState {
    double beta, alpha, ib, amax, prev;
    int fused, active, m, broke;
};

__device__ __forceinline__ int2 fixed47(double x) {
    // |x| <= 1: X = round(x 2^47), split as (lo 24 bits, hi)
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & ((1ull << 52) - 1);
    if (e != 0) mant |= (1ull << 52);
    const int ee = e > 0 ? e : 1;
    const int rs = max(1023 - ee + 5, 1);
    long long X = (rs >= 60) ? 0 : (long long)((mant + (1ull << (rs - 1))) >> rs);
    if (b >> 63) X = -X;
    return make_int2((int)(X & 0xFFFFFF), (int)(X >> 24));
}

__device__ __forceinline__ double block_reduce(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];      // same order in every thread
    return s;
}

// barrier number `gen` (1, 2, ...) among `nctas` CTAs: returns false on timeout
__device__ bool grid_barrier(unsigned int* ctr, int nctas, unsigned gen, long long limit, int* err, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        const unsigned target = (unsigned)nctas * gen;
        long long it = 0;
        int ok = 1;
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (*(volatile int*)err != 0 || ++it > limit) {     // fail fast after any timeout
                ok = 0;
                atomicExch(err, (int)HUB_ETIMEOUT);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// ---- device tridiagonal helpers (thread-serial; m <= max_iters) -------------
// Number of eigenvalues of T_m below x: sign changes of the characteristic
// polynomials p_0 = 1, p_1 = a_0 - x, p_k = (a_{k-1} - x) p_{k-1} - b_{k-2}^2 p_{k-2}
// (Sturm sequence).  No division (the binary64 divide is slow on this part);
// both terms are rescaled by 2^-600 / 2^600 when they leave a safe range.
// A zero p_k takes the sign of p_{k-1}.
__device__ __noinline__ int d_sturm(const double* a, const double* b, int m, double x) {
    double p0 = 1.0, p1 = a[0] - x;
    int c = (p1 < 0.0) ? 1 : 0;
    bool s1 = (p1 != 0.0) ? (p1 < 0.0) : false;       // sign used for counting
    for (int i = 1; i < m; ++i) {
        const double p2 = (a[i] - x) * p1 - (b[i - 1] * b[i - 1]) * p0;
        const bool s2 = (p2 != 0.0) ? (p2 < 0.0) : s1;
        if (s2 != s1) ++c;
        s1 = s2;
        p0 = p1;
        p1 = p2;
        const double mag = fmax(fabs(p0), fabs(p1));
        if (mag > 0x1p600) {
            p0 *= 0x1p-600;
            p1 *= 0x1p-600;
        } else if (mag < 0x1p-600 && mag > 0.0) {
            p0 *= 0x1p600;
            p1 *= 0x1p600;
        }
    }
    return c;
}

// Lowest eigenvalue of T_m by multisection over the whole CTA: every thread
// evaluates the Sturm count at its own point of the bracket, which shrinks by
// blockDim + 1 per round.  prev (or NaN) is an upper bound from an earlier
// step (interlacing).  Returns the same value in every thread.
__device__ double cta_lowest_eig(const double* a, const double* b, int m, double prev, int* flags, double* sh2) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double glo = a[0], ghi = a[0];
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        glo = fmin(glo, a[i] - r);
        ghi = fmax(ghi, a[i] + r);
    }
    double lo = glo, hi = ghi;
    if (prev == prev) {
        // warm bracket [prev - 1e-6, prev + 1e-12] (relative), checked by two threads
        const double wl = prev - 1e-6 * fmax(1.0, fabs(prev)), wh = prev + 1e-12 * fmax(1.0, fabs(prev));
        if (tid == 0) flags[0] = (wl > glo) ? (d_sturm(a, b, m, wl) == 0) : 0;
        if (tid == 1 % nt) flags[1] = (wh < ghi) ? (d_sturm(a, b, m, wh) >= 1) : 0;
        __syncthreads();
        const bool okl = flags[0] != 0, okh = flags[1] != 0;
        __syncthreads();
        if (okh) hi = wh;
        if (okl && okh) lo = wl;
    }
    for (int round = 0; round < 12; ++round) {
        if (!(hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
        const double x = lo + (hi - lo) * (double)(tid + 1) / (double)(nt + 1);
        // the first point with a positive count bounds the eigenvalue; taken as the
        // smallest such thread index (computed counts need not be monotone in x
        // near an eigenvalue, and the choice must not depend on timing)
        int* kmin = reinterpret_cast<int*>(sh2);
        if (tid == 0) *kmin = nt;
        __syncthreads();
        if (d_sturm(a, b, m, x) >= 1) atomicMin(kmin, tid);
        __syncthreads();
        const int k = *kmin;
        const double nlo = k == 0 ? lo : lo + (hi - lo) * (double)k / (double)(nt + 1);
        const double nhi = k == nt ? hi : lo + (hi - lo) * (double)(k + 1) / (double)(nt + 1);
        lo = nlo;
        hi = nhi;
        __syncthreads();
    }
    return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of T_m for eigenvalue th: solve the
// eigen-equations backwards from y_m = 1 (the lowest eigenvector grows in that
// direction), rescaling by powers of two; returns 1 / |y|.
__device__ __noinline__ double d_last_component(const double* a, const double* b, int m, double th) {
    if (m == 1) return 1.0;
    double y1 = 1.0;                                   // y_m
    double y0 = -(a[m - 1] - th) / b[m - 2];           // y_{m-1}
    double n2 = 1.0 + y0 * y0;
    double scale_log = 0.0;                            // n2 and the y's carry 2^scale_log
    for (int i = m - 2; i >= 1; --i) {
        // row i: b_{i-1} y_{i-1} + (a_i - th) y_i + b_i y_{i+1} = 0
        const double ym = -((a[i] - th) * y0 + b[i] * y1) / b[i - 1];
        y1 = y0;
        y0 = ym;
        n2 += ym * ym;
        const double mag = fmax(fabs(y0), fabs(y1));
        if (mag > 0x1p300) {
            y0 *= 0x1p-300;
            y1 *= 0x1p-300;
            n2 *= 0x1p-600;
            scale_log += 600.0;
        }
    }
    // |y|^2 = n2 * 2^scale_log; y_m was 1 in the unscaled frame
    return exp2(-0.5 * scale_log) / sqrt(n2);
}

// One sector as seen by the element pass.
struct SecView {
    const int2* X;         // fixed-point copy of f (global)
    const double* f;
    double* g;
    const int32_t *urp, *drp;
    const uint32_t *uent, *dent, *ust, *dst;
    int64_t Ddn;
    double U, scale;       // scale = -t * 2^-47
    // down-spin row table (nullptr: per-lane CSR lists instead); used when the
    // row is staged with its zero slots
    const int64_t* dbo = nullptr;
    const int32_t* dbc = nullptr;
    const uint16_t* dbe = nullptr;
};

// A row staged for the coloured down-hop table: Ddn rounded up to 32, then the
// zero slots its padding entries read (8-byte slots fall in 16 bank groups, so
// 16 zero slots cover every group).
constexpr int kRowZeroSlots = 16;
__host__ __device__ __forceinline__ int64_t row_slots(int64_t Ddn) { return (Ddn + 31) / 32 * 32 + kRowZeroSlots; }

// Row u of q = H f - beta g (Eqs. split1) by one warp, the fixed-point copy in
// global memory (L2): the row is staged in buf (when given) for the
// down-hops, up-hops read whole neighbour rows with lanes over columns
// (coalesced; the row's hop list is held in the lanes, the column loop is
// warp-uniform).  With V.dbo and a staged row (buf holds row_slots(Ddn)
// elements) the down-hops walk the coloured row table: the same slot count
// for all lanes of a group and no shared-memory bank conflicts; otherwise each
// lane walks its own CSR list.  Adds this lane's <q,f>, <q,q>, <f,f> over the row.
__device__ __forceinline__ void row_pass(const SecView& V, int64_t u, int2* buf, double beta, double& ap,
                                         double& qq, double& ff) {
    const int lane = threadIdx.x & 31;
    const int64_t Ddn = V.Ddn;
    const int2* xr = V.X + u * Ddn;
    const bool blocks = buf != nullptr && V.dbo != nullptr;
    if (buf != nullptr) {
        for (int64_t d = lane; d < Ddn; d += 32) buf[d] = __ldcg(xr + d);
        if (blocks && lane < kRowZeroSlots) buf[(Ddn + 31) / 32 * 32 + lane] = make_int2(0, 0);
        __syncwarp();
        xr = buf;
    }
    const int32_t kb = V.urp[u], ke = V.urp[u + 1];
    const int nh = ke - kb;
    const uint32_t mine = lane < nh ? V.uent[kb + lane] : 0u;
    const uint32_t su_u = V.ust[u];
    for (int64_t d0 = 0; d0 < Ddn; d0 += 32) {
        const int64_t d = d0 + lane;
        const bool act = d < Ddn;
        const int64_t dd = act ? d : Ddn - 1;
        int lo = 0, hi = 0;
        if (nh <= 32) {
#pragma unroll 4
            for (int k = 0; k < nh; ++k) {
                const uint32_t e = __shfl_sync(0xffffffffu, mine, k);
                const int2 x = __ldcg(V.X + (int64_t)(e >> 1) * Ddn + dd);
                if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
            }
        } else {
            for (int32_t k = kb; k < ke; ++k) {
                const uint32_t e = V.uent[k];
                const int2 x = __ldcg(V.X + (int64_t)(e >> 1) * Ddn + dd);
                if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
            }
        }
        if (blocks) {
            // padding slots (and the lanes past Ddn) read a zero slot
            for_each_hop<uint16_t>(V.dbe + V.dbo[d0 >> 5], V.dbc[d0 >> 5], lane, [&](uint32_t e) {
                const int s = RowEnt<uint16_t>::sgn(e);
                const int2 x = buf[RowEnt<uint16_t>::idx(e)];
                lo += s * x.x;
                hi += s * x.y;
            });
        } else {
            for (int32_t k = V.drp[dd]; k < V.drp[dd + 1]; ++k) {
                const uint32_t e = V.dent[k];
                const int2 x = buf != nullptr ? xr[e >> 1] : __ldcg(xr + (e >> 1));
                if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
            }
        }
        if (act) {
            const int64_t j = u * Ddn + d;
            const long long Sx = ((long long)hi << 24) + (long long)lo;
            const double fj = __ldcg(V.f + j);
            const double q = fma(-beta, __ldcg(V.g + j), fma(V.U * (double)__popc(su_u & V.dst[d]), fj, V.scale * (double)Sx));
            V.g[j] = q;
            ap = fma(q, fj, ap);
            qq = fma(q, q, qq);
            ff = fma(fj, fj, ff);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-synchronous sweep over the larger sectors (Algorithm 1 for all of them
// in lock step).  Every phase spreads the rows of all active sectors over all
// warps of the launch, so the load balances whatever the mix of sizes:
//   E  q = H f - beta g for every row (row_pass); per-row partials of
//      <q,f>, <q,q>, <f,f>;
//   R  one CTA per sector: a_j, b_{j+1} from the partials (the explicit
//      |q - a f| pass near breakdown), the Ritz test, the stop decision;
//   U  f_{j+1} = (q - a f) / b_{j+1} and its fixed-point copy.
// Phases are separated by bounded grid barriers; per-row partials are summed
// in row order, so a sector's result does not depend on the rest of the batch.
// Vector data written in one phase and read in another goes through L2
// (__ldcg): the near-breakdown pass of phase R rewrites rows that other SMs
// read next.
__device__ __noinline__ bool sweep_solve(const BatchParams& P, int2* xs, double* red, int* flag, int* sh_flags,
                                         double* sh_k, int* sh_stop, double* sh_out) {
    unsigned ggen = 0;
    const int G = P.sweep_ctas;                        // CTAs of the sweep: blockIdx.x < G
    auto gsync = [&]() -> bool {
        ++ggen;
        return grid_barrier(P.gbar, G, ggen, P.spin_limit, P.err, flag);
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw_all = (int64_t)G * nwarps;
    const int64_t nrows = P.rowoff[P.nswp];
    auto locate = [&](int64_t r) -> int { return __ldg(P.rowsec + r); };   // k: rowoff[k] <= r < rowoff[k + 1]
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.nactive = P.nswp;
    // rows of the element and update phases are claimed one at a time (heaviest
    // sectors first), so warps that drew cheap rows take more of them
    auto claim = [&](int c) -> int64_t {
        unsigned long long r = 0ull;
        if (lane == 0) r = atomicAdd(P.claim + c, 1ull);
        return (int64_t)__shfl_sync(0xffffffffu, r, 0);
    };
    // a claimed row of a sector that has stopped: move the counter past the
    // sector's last row (the counter only grows, so every row it skips is of
    // that sector), and the other warps stop claiming its rows one by one
    auto skip_sector = [&](int c, int k) {
        if (lane == 0) atomicMax(P.claim + c, (unsigned long long)P.rowoff[k + 1]);
    };
    // |v0|^2 by rows, then per sector
    for (int64_t r = gw; r < nrows; r += nw_all) {
        const int k = locate(r);
        const SectorDesc S = P.sec[P.swp[k]];
        const double* v0 = P.v0 + S.voff + (r - P.rowoff[k]) * S.Ddn;
        double nn = 0.0;
        for (int64_t d = lane; d < S.Ddn; d += 32) nn = fma(v0[d], v0[d], nn);
        nn = warp_sum(nn);
        if (lane == 0) P.rowpart[3 * r] = nn;
    }
    if (!gsync()) return false;
    for (int k = blockIdx.x; k < P.nswp; k += G) {
        const SectorDesc S = P.sec[P.swp[k]];
        double nn = 0.0;
        for (int64_t u = threadIdx.x; u < S.Dup; u += blockDim.x) nn += __ldcg(P.rowpart + 3 * (P.rowoff[k] + u));
        nn = block_reduce(nn, red);
        if (threadIdx.x == 0) {
            SweepState st{};
            st.ib = 1.0 / sqrt(nn);
            st.amax = 1.0;
            st.prev = __longlong_as_double(0x7ff8000000000000ll);   // NaN: no previous Ritz value
            st.active = 1;
            P.sst[k] = st;
        }
    }
    if (!gsync()) return false;
    // f_1 = v0 / |v0|, f_0 = 0 and the fixed-point copy of f_1
    for (int64_t r = gw; r < nrows; r += nw_all) {
        const int k = locate(r);
        const SectorDesc S = P.sec[P.swp[k]];
        const double ib = __ldcg(&P.sst[k].ib);
        const int64_t j0 = S.voff + (r - P.rowoff[k]) * S.Ddn;
        for (int64_t d = lane; d < S.Ddn; d += 32) {
            const double x = P.v0[j0 + d] * ib;
            P.f[j0 + d] = x;
            P.g[j0 + d] = 0.0;
            P.xg[j0 + d] = fixed47(x);
        }
    }
    if (!gsync()) return false;
    int nact = P.nswp;
    for (int it = 0; it < P.iter_cap && nact > 0; ++it) {
        double* fp = (it & 1) ? P.g : P.f;          // f_j and f_{j-1} swap pools each step
        double* gp = (it & 1) ? P.f : P.g;
        // E
        for (int64_t r = claim(0); r < nrows; r = claim(0)) {
            const int k = locate(r);
            if (!__ldcg(&P.sst[k].active)) {
                skip_sector(0, k);
                continue;
            }
            const SectorDesc S = P.sec[P.swp[k]];
            // warps of one CTA work on rows of different sectors: each owns a
            // fixed slice of the shared buffer, long rows read from L2 instead
            const int64_t slice = P.smem_elems / nwarps;
            const int mode = P.mode_force >= 0 ? P.mode_force : S.mode;
            int2* buf = (mode & kModeStage) && S.Ddn <= slice ? xs + (int64_t)warp * slice : nullptr;
            const bool blk = S.dn_blk >= 0 && row_slots(S.Ddn) <= slice;
            const SecView V{P.xg + S.voff, fp + S.voff, gp + S.voff, P.rp + S.up_rp, P.rp + S.dn_rp,
                            P.ent + S.up_ent, P.ent + S.dn_ent, P.st + S.up_st, P.st + S.dn_st, S.Ddn, S.U,
                            -S.t * 0x1p-47, blk ? P.bo + S.dn_blk : nullptr, blk ? P.bc + S.dn_blk : nullptr,
                            P.be};
            double ap = 0.0, qq = 0.0, ff = 0.0;
            row_pass(V, r - P.rowoff[k], buf, __ldcg(&P.sst[k].beta), ap, qq, ff);
            ap = warp_sum(ap);
            qq = warp_sum(qq);
            ff = warp_sum(ff);
            if (lane == 0) {
                P.rowpart[3 * r] = ap;
                P.rowpart[3 * r + 1] = qq;
                P.rowpart[3 * r + 2] = ff;
            }
        }
        if (!gsync()) return false;
        // R
        if (blockIdx.x == 0 && threadIdx.x == 0) P.claim[1] = 0ull;   // U of this step starts after a barrier
        for (int k = blockIdx.x; k < P.nswp; k += G) {
            SweepState st = P.sst[k];
            if (!st.active) continue;
            const int sid = P.swp[k];
            const SectorDesc S = P.sec[sid];
            double sv[3] = {0.0, 0.0, 0.0};
            for (int64_t u = threadIdx.x; u < S.Dup; u += blockDim.x)
                for (int q = 0; q < 3; ++q) sv[q] += __ldcg(P.rowpart + 3 * (P.rowoff[k] + u) + q);
            for (int q = 0; q < 3; ++q) sv[q] = block_reduce(sv[q], red);
            const double alpha = sv[0];
            double b2 = sv[1] - 2.0 * alpha * alpha + alpha * alpha * sv[2];
            const bool fused = b2 > 1e-6 * sv[1];
            if (!fused) {                               // near breakdown: form q - a f explicitly
                double bp = 0.0;
                for (int64_t j = S.voff + threadIdx.x; j < S.voff + S.D; j += blockDim.x) {
                    const double x = fma(-alpha, __ldcg(fp + j), __ldcg(gp + j));
                    gp[j] = x;
                    bp = fma(x, x, bp);
                }
                b2 = block_reduce(bp, red);
            }
            const double bn = sqrt(fmax(b2, 0.0));
            double* A = P.ab + S.ab;
            double* B = A + P.max_iters;
            if (threadIdx.x == 0) {
                A[it] = alpha;
                B[it] = bn;
            }
            const int m = it + 1;
            const int mcap = (int)((int64_t)P.iter_cap < S.D ? (int64_t)P.iter_cap : S.D);
            st.amax = fmax(st.amax, fmax(fabs(alpha), bn));
            st.broke = bn <= 1e-13 * st.amax;
            if (st.broke || (m >= 8 && (m % (m >= 32 ? 2 * kCheckEvery : kCheckEvery)) == 0) || m == mcap) {
                __syncthreads();                         // A, B written by thread 0
                const double th = cta_lowest_eig(A, B, m, st.prev, sh_flags, sh_k);
                if (threadIdx.x == 0) {
                    const double rho = bn * d_last_component(A, B, m, th);
                    const int conv = st.broke || (rho < P.tol * fmax(1.0, fabs(th)));
                    *sh_stop = conv || m == mcap;
                    sh_out[0] = th;
                    sh_out[1] = rho;
                    if (*sh_stop) {
                        lanczos_result res;
                        res.energy = th;
                        res.residual = rho;
                        res.err_bound = 0.0;             // set on the host (hubbard_batch_results)
                        res.iters = m;
                        res.breakdown = st.broke;
                        res.status = conv ? HUB_OK : HUB_ENOTCONV;
                        res.reserved = 0;
                        P.res[sid] = res;
                    }
                }
                __syncthreads();
                st.prev = sh_out[0];
                if (*sh_stop) st.active = 0;
            }
            if (threadIdx.x == 0) {
                st.alpha = alpha;
                st.beta = bn;
                st.ib = 1.0 / bn;
                st.fused = fused;
                st.m = m;
                P.sst[k] = st;
                if (!st.active) atomicSub(P.nactive, 1);
            }
            __syncthreads();
        }
        if (!gsync()) return false;
        // U
        if (blockIdx.x == 0 && threadIdx.x == 0) P.claim[0] = 0ull;   // E of the next step starts after a barrier
        for (int64_t r = claim(1); r < nrows; r = claim(1)) {
            const int k = locate(r);
            if (!__ldcg(&P.sst[k].active)) {
                skip_sector(1, k);
                continue;
            }
            const SectorDesc S = P.sec[P.swp[k]];
            const double alpha = __ldcg(&P.sst[k].alpha), ib = __ldcg(&P.sst[k].ib);
            const int fused = __ldcg(&P.sst[k].fused);
            const int64_t j0 = S.voff + (r - P.rowoff[k]) * S.Ddn;
            // four elements per lane in flight: every load of a group before its stores
            for (int64_t d0 = lane; d0 < S.Ddn; d0 += 128) {
                double fv[4], gv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t d = d0 + 32 * i;
                    fv[i] = (fused && d < S.Ddn) ? __ldcg(fp + j0 + d) : 0.0;
                    gv[i] = d < S.Ddn ? __ldcg(gp + j0 + d) : 0.0;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t d = d0 + 32 * i;
                    if (d < S.Ddn) {
                        const double x = (fused ? fma(-alpha, fv[i], gv[i]) : gv[i]) * ib;
                        gp[j0 + d] = x;
                        P.xg[j0 + d] = fixed47(x);
                    }
                }
            }
        }
        if (!gsync()) return false;
        nact = __ldcg(P.nactive);
    }
    return true;
}

__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_lanczos(BatchParams P) {
    extern __shared__ __align__(16) int2 xs[];
    __shared__ double red[kBatchThreads / 32];
    __shared__ int flag, stop;
    __shared__ double sh_theta, sh_rho;
    __shared__ double sh_prev;
    __shared__ int sh_flags[kBatchThreads];
    __shared__ double sh_k[1];
    __shared__ double sh_out[2];
    // the larger sectors first, in lock step over the whole grid; then the
    // smaller ones, one CTA each
    if (P.nswp > 0 && (int)blockIdx.x < P.sweep_ctas && !sweep_solve(P, xs, red, &flag, sh_flags, sh_k, &stop, sh_out))
        return;
    __shared__ int sh_task;
    const bool queued = P.q_posted != nullptr;
    while (true) {
        // the next task (largest work first) goes to the CTA that asks first;
        // queued: a task number is taken only once that task has been posted,
        // so a CTA that leaves an idle queue holds none
        if (threadIdx.x == 0) {
            if (!queued) {
                sh_task = (int)atomicAdd(P.claim + 2, 1ull);
            } else {
                sh_task = -1;
                for (long long it = 0; it < P.q_idle; ++it) {
                    const unsigned c = *(volatile unsigned int*)P.q_claim;
                    const unsigned n = ld_acquire_sys(P.q_posted);
                    if (c < n) {
                        if (atomicCAS(P.q_claim, c, c + 1u) == c) {
                            sh_task = (int)c;
                            break;
                        }
                        continue;
                    }
                    if (*P.q_stop != 0u) break;
                    __nanosleep(it < 256 ? 200 : 2000);
                }
            }
        }
        __syncthreads();
        const int ti = sh_task;
        __syncthreads();
        if (queued ? ti < 0 : ti >= P.ntasks) break;
        const int sid = queued ? ti % P.q_cap : P.tasks[ti];
        const SectorDesc S = queued ? load_desc_cg(P.sec + sid) : P.sec[sid];
        const int64_t D = S.D, Ddn = S.Ddn, Dup = S.Dup;
        const int64_t j0 = 0, j1 = D;
        const int mode = P.mode_force >= 0 ? P.mode_force : S.mode;
        const bool in_smem = (mode & kModeFlat) && D <= P.smem_elems;
        // per-warp row buffer for the global-memory path (rows of the fixed-point copy)
        const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
        // (row_slots(Ddn) per warp for the coloured down-hop table, else Ddn)
        const bool blk = S.dn_blk >= 0 && row_slots(Ddn) * nwarps <= P.smem_elems;
        const int64_t rstride = blk ? row_slots(Ddn) : Ddn;
        const bool rowbuf = (mode & kModeStage) && !in_smem && rstride * nwarps <= P.smem_elems;
        int2* X = in_smem ? xs : (P.xg + S.voff);
        double* f = P.f + S.voff;
        double* g = P.g + S.voff;
        const double* v0 = queued ? nullptr : P.v0 + S.voff;
        auto v0at = [&](int64_t j) -> double { return queued ? splitmix_uniform(S.seed, j) : v0[j]; };
        const int32_t* urp = P.rp + S.up_rp;
        const int32_t* drp = P.rp + S.dn_rp;
        const uint32_t* uent = P.ent + S.up_ent;
        const uint32_t* dent = P.ent + S.dn_ent;
        const uint32_t* ust = P.st + S.up_st;
        const uint32_t* dst = P.st + S.dn_st;
        double* A = P.ab + S.ab;
        double* B = A + P.max_iters;
        // block sums of nv <= 3 values (in place), in a fixed order
        auto cta_sum = [&](int nv, double* v) {
            for (int q = 0; q < nv; ++q) v[q] = block_reduce(v[q], red);
        };
        // f_1 = v0 / |v0|, f_0 = 0, and the fixed-point copy of f_1 (|f| <= 1)
        double nn[1] = {0.0};
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double x = v0at(j);
            nn[0] = fma(x, x, nn[0]);
        }
        cta_sum(1, nn);
        const double inv0 = 1.0 / sqrt(nn[0]);
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double x = v0at(j) * inv0;
            f[j] = x;
            g[j] = 0.0;
            X[j] = fixed47(x);
        }
        __syncthreads();
        const double scale = -S.t * 0x1p-47;           // -t times the fixed-point unit
        const int mcap = (int)((int64_t)P.iter_cap < D ? (int64_t)P.iter_cap : D);
        double beta = 0.0, theta = 0.0, rho = 0.0;
        int m = 0, broke = 0, conv = 0;
        if (threadIdx.x == 0) sh_prev = __longlong_as_double(0x7ff8000000000000ll);   // NaN: no previous value
        double amax = 1.0;
        for (int it = 0; it < mcap; ++it) {
            // q = H f - beta g  (Eqs. split1) with <q, f>, <q, q>, <f, f>
            double ap = 0.0, qq = 0.0, ff = 0.0;
            auto element = [&](int64_t u, int64_t d, int lo, int hi) {
                const int64_t j = u * Ddn + d;
                const long long Sx = ((long long)hi << 24) + (long long)lo;
                const double fj = f[j];
                const double q = fma(-beta, g[j], fma(S.U * (double)__popc(ust[u] & dst[d]), fj, scale * (double)Sx));
                g[j] = q;
                ap = fma(q, fj, ap);
                qq = fma(q, q, qq);
                ff = fma(fj, fj, ff);
            };
            if (in_smem) {
                // whole fixed-point vector in shared memory: flat loop over elements
                // (D <= smem_elems, so 32-bit index arithmetic)
                const int Dd = (int)Ddn;
                for (int jj = (int)j0 + threadIdx.x; jj < (int)j1; jj += blockDim.x) {
                    const int u = jj / Dd, d = jj - u * Dd;
                    int lo = 0, hi = 0;
                    for (int32_t k = urp[u]; k < urp[u + 1]; ++k) {
                        const uint32_t e = uent[k];
                        const int2 x = X[(int)(e >> 1) * Dd + d];
                        if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
                    }
                    const int rowb = u * Dd;
                    for (int32_t k = drp[d]; k < drp[d + 1]; ++k) {
                        const uint32_t e = dent[k];
                        const int2 x = X[rowb + (int)(e >> 1)];
                        if (e & 1u) { lo -= x.x; hi -= x.y; } else { lo += x.x; hi += x.y; }
                    }
                    element(u, d, lo, hi);
                }
            } else {
                // global copy (L2): a warp per row (row_pass)
                const SecView V{X, f, g, urp, drp, uent, dent, ust, dst, Ddn, S.U, scale,
                                blk ? P.bo + S.dn_blk : nullptr, blk ? P.bc + S.dn_blk : nullptr, P.be};
                int2* buf = rowbuf ? xs + (int64_t)warp * rstride : nullptr;
                for (int64_t u = warp; u < Dup; u += nwarps) row_pass(V, u, buf, beta, ap, qq, ff);
            }
            double sv[3] = {ap, qq, ff};
            cta_sum(3, sv);
            const double alpha = sv[0];
            // |q - alpha f|^2 = <q,q> - 2 alpha <q,f> + alpha^2 <f,f>, unless that
            // cancels more than six digits (near breakdown): then form it
            double b2 = sv[1] - 2.0 * alpha * alpha + alpha * alpha * sv[2];
            const bool fused = b2 > 1e-6 * sv[1];
            if (!fused) {
                double bp[1] = {0.0};
                for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
                    const double r = fma(-alpha, f[j], g[j]);
                    g[j] = r;
                    bp[0] = fma(r, r, bp[0]);
                }
                cta_sum(1, bp);
                b2 = bp[0];
            }
            const double bn = sqrt(fmax(b2, 0.0));
            if (threadIdx.x == 0) {
                A[it] = alpha;
                B[it] = bn;
            }
            m = it + 1;
            amax = fmax(amax, fmax(fabs(alpha), bn));
            if (bn <= 1e-13 * amax) broke = 1;
            // Ritz test
            if (broke || (m >= 8 && (m % (m >= 32 ? 2 * kCheckEvery : kCheckEvery)) == 0) || m == mcap) {
                __syncthreads();                             // A, B written by thread 0
                const double th = cta_lowest_eig(A, B, m, sh_prev, sh_flags, sh_k);
                if (threadIdx.x == 0) {
                    const double sl = d_last_component(A, B, m, th);
                    sh_prev = th;
                    sh_theta = th;
                    sh_rho = bn * sl;
                    stop = broke || (sh_rho < P.tol * fmax(1.0, fabs(th)));
                }
                __syncthreads();
                theta = sh_theta;
                rho = sh_rho;
                if (stop) {
                    conv = 1;
                    break;
                }
            }
            // f_{j+1} = (q - alpha f) / beta_next (rounded as axpy then scale) and
            // its fixed-point copy; the old f becomes f_{j-1}
            const double ib = 1.0 / bn;
            for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
                const double x = (fused ? fma(-alpha, f[j], g[j]) : g[j]) * ib;
                g[j] = x;
                X[j] = fixed47(x);
            }
            __syncthreads();
            double* tmp = f;
            f = g;
            g = tmp;
            beta = bn;
        }
        if (threadIdx.x == 0) {
            lanczos_result r;
            r.energy = theta;
            r.residual = rho;
            r.err_bound = 0.0;                           // set on the host (hubbard_batch_results)
            r.iters = m;
            r.breakdown = broke;
            r.status = conv ? HUB_OK : HUB_ENOTCONV;
            r.reserved = 0;
            P.res[sid] = r;
            if (queued) {
                __threadfence_system();                      // result and a/b history before the flag
                P.q_done[sid] = (unsigned)ti + 1u;
            }
        }
        __syncthreads();
    }
}

// A bounded grid barrier that cannot complete (it expects one CTA more than
// launched): every CTA gives up after `limit` polls and sets the error word.
__global__ void k_wait_probe(unsigned int* ctr, long long limit, int* err) {
    __shared__ int flag;
    grid_barrier(ctr, (int)gridDim.x + 1, 1, limit, err, &flag);
}

}  // namespace
}  // namespace hub

// ---------------------------------------------------------------------------
struct hubbard_batch {
    int device = 0;
    int n = 0;
    std::vector<hub::SectorDesc> sec;          // host copy
    std::vector<int64_t> voff;                 // n + 1 vector offsets
    int64_t total = 0;                         // sum of D
    std::vector<double> cost;                  // per-sector work estimate
    std::vector<int> hops1;                    // per-sector W_up + W_dn + 1 (error-bound floor)
    // schedule table: one entry per sector shape (D_up, D_dn, W_up + W_dn)
    struct Shape {
        int64_t Dup, Ddn;
        int W, count, mode;
    };
    std::vector<Shape> shapes;
    std::vector<int> shape_of;                 // per sector
    bool desc_dirty = false;                   // modes changed since the last descriptor upload
    hub::SectorDesc* d_sec = nullptr;
    int32_t* d_rp = nullptr;
    uint32_t* d_ent = nullptr;
    uint32_t* d_st = nullptr;
    int64_t* d_bo = nullptr;                   // row-table pools
    int32_t* d_bc = nullptr;
    uint16_t* d_be = nullptr;
    // schedule
    int64_t elems_per_cta = 1 << 14;
    int task_ctas = 0;                         // CTAs that start on the one-CTA tasks while the rest sweep
    int* d_tasks = nullptr;
    int ntasks = 0;
    size_t tasks_cap = 0;
    int grid = 0;
    int smem_elems = 0;
    int sched_max_iters = -1;
    int64_t sched_elems = -1;
    // grid-synchronous sweep: sectors above the threshold
    int nswp = 0;
    int* d_swp = nullptr;
    int64_t* d_rowoff = nullptr;
    int32_t* d_rowsec = nullptr;
    int64_t rows_all = 0;                      // sum of D_up over all sectors (workspace bound)
    cudaStream_t mem_stream = nullptr;         // stream of its allocations (batch_create_streamed)
};

namespace hub {
namespace {

struct Cached {
    int64_t rp_off, ent_off, st_off, D, W;
    double hops;   // mean hops per state
    int64_t blk;   // first group of the row table in the block pools (-1: none)
};

// row tables are built for spins whose staged row could fit a warp's slice
constexpr int64_t kRowTableMaxD = 4064;

struct RowPools {
    std::vector<int64_t> bo;
    std::vector<int32_t> bc;
    std::vector<uint16_t> be;
};

int batch_upload(hubbard_batch* B, const std::vector<int32_t>& rp, const std::vector<uint32_t>& ent,
                 const std::vector<uint32_t>& st, const RowPools& rows) {
    const cudaStream_t ms = B->mem_stream;
    auto up = [ms](auto** dst, const auto& v) -> int {
        using T = std::remove_reference_t<decltype(v[0])>;
        const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
        cudaError_t e = dev_alloc((void**)dst, bytes, ms);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch tables)");
        if (!v.empty()) {
            e = dev_upload(*dst, v.data(), v.size() * sizeof(T), ms);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch tables)");
        }
        return HUB_OK;
    };
    int rc;
    if ((rc = up(&B->d_rp, rp)) || (rc = up(&B->d_ent, ent)) || (rc = up(&B->d_st, st))) return rc;
    if ((rc = up(&B->d_bo, rows.bo)) || (rc = up(&B->d_bc, rows.bc)) || (rc = up(&B->d_be, rows.be))) return rc;
    return up(&B->d_sec, B->sec);
}

void batch_free(hubbard_batch* B) {
    const cudaStream_t ms = B->mem_stream;
    dev_free(B->d_sec, ms);
    dev_free(B->d_rp, ms);
    dev_free(B->d_ent, ms);
    dev_free(B->d_st, ms);
    dev_free(B->d_bo, ms);
    dev_free(B->d_bc, ms);
    dev_free(B->d_be, ms);
    dev_free(B->d_tasks, ms);
    dev_free(B->d_swp, ms);
    dev_free(B->d_rowoff, ms);
    dev_free(B->d_rowsec, ms);
}

int kernel_shape_impl(int* smem_elems, int* grid);
// dynamic shared memory (bytes; elements to *smem_elems) and grid (two CTAs
// per SM) of the batch kernel; sets the kernel's shared-memory attribute
int kernel_shape(int* smem_elems, int* grid) { return kernel_shape_impl(smem_elems, grid); }

int batch_grid(hubbard_batch* B, int* smem_elems) {
    int grid = 0;
    const int smem = kernel_shape(smem_elems, &grid);
    if (smem > 0) B->grid = grid;
    return smem;
}

int kernel_shape_impl(int* smem_elems, int* grid) {
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0, optin = 0, per_sm_bytes = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_batch_lanczos) != cudaSuccess) return -1;
    // two CTAs per SM, each with half of the SM's shared memory (less the
    // per-CTA reservation and the kernel's static buffers) for fixed-point staging
    int smem = per_sm_bytes / 2 - 1024 - (int)fa.sharedSizeBytes;
    smem = std::min(smem, optin - (int)fa.sharedSizeBytes) / 16 * 16;
    if (smem < 16 * 1024) return -1;
    *smem_elems = smem / (int)sizeof(int2);
    cudaError_t e = cudaFuncSetAttribute(k_batch_lanczos, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return -1;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_lanczos, kBatchThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return -1;
    *grid = sms * std::min(per_sm, 2);
    return smem;
}

// Sectors above elems_per_cta elements go to the sweep, ordered by the cost of
// their rows (heaviest first); the rest are one-CTA tasks ordered by work
// (largest first).  The kernel hands both out dynamically in these orders.
int batch_schedule(hubbard_batch* B) {
    // sectors above the threshold: the grid-synchronous sweep
    std::vector<int> swp;
    std::vector<int64_t> rowoff(1, 0);
    std::vector<int> order;
    for (int s = 0; s < B->n; ++s) {
        if (B->sec[s].D > B->elems_per_cta) swp.push_back(s);
        else order.push_back(s);
    }
    // heaviest rows first (rows are claimed dynamically in this order)
    std::stable_sort(swp.begin(), swp.end(), [&](int a, int b) {
        return B->cost[a] / (double)B->sec[a].Dup > B->cost[b] / (double)B->sec[b].Dup;
    });
    std::vector<int32_t> rowsec;
    for (int s : swp) {
        rowsec.insert(rowsec.end(), (size_t)B->sec[s].Dup, (int32_t)(rowoff.size() - 1));
        rowoff.push_back(rowoff.back() + B->sec[s].Dup);
    }
    // the rest: one CTA per sector, largest work first (claimed dynamically)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->cost[a] > B->cost[b]; });
    const cudaStream_t ms = B->mem_stream;
    dev_free(B->d_swp, ms);
    dev_free(B->d_rowoff, ms);
    dev_free(B->d_rowsec, ms);
    B->d_swp = nullptr;
    B->d_rowoff = nullptr;
    B->d_rowsec = nullptr;
    B->nswp = (int)swp.size();
    {
        cudaError_t e = dev_alloc((void**)&B->d_swp, std::max<size_t>(swp.size(), 1) * sizeof(int), ms);
        if (e == cudaSuccess) e = dev_alloc((void**)&B->d_rowoff, rowoff.size() * sizeof(int64_t), ms);
        if (e == cudaSuccess) e = dev_alloc((void**)&B->d_rowsec, std::max<size_t>(rowsec.size(), 1) * sizeof(int32_t), ms);
        if (e == cudaSuccess && !rowsec.empty())
            e = dev_upload(B->d_rowsec, rowsec.data(), rowsec.size() * sizeof(int32_t), ms);
        if (e == cudaSuccess && !swp.empty())
            e = dev_upload(B->d_swp, swp.data(), swp.size() * sizeof(int), ms);
        if (e == cudaSuccess)
            e = dev_upload(B->d_rowoff, rowoff.data(), rowoff.size() * sizeof(int64_t), ms);
        if (e != cudaSuccess) return cuda_fail(e, "batch sweep list upload");
    }
    dev_free(B->d_tasks, ms);
    B->d_tasks = nullptr;
    B->ntasks = (int)order.size();
    cudaError_t e = dev_alloc((void**)&B->d_tasks, std::max<size_t>(order.size(), 1) * sizeof(int), ms);
    if (e == cudaSuccess && !order.empty())
        e = dev_upload(B->d_tasks, order.data(), order.size() * sizeof(int), ms);
    if (e != cudaSuccess) return cuda_fail(e, "batch schedule upload");
    e = dev_upload(B->d_sec, B->sec.data(), B->sec.size() * sizeof(SectorDesc), ms);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
    B->sched_elems = B->elems_per_cta;
    return HUB_OK;
}

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct WsLayout {
    size_t f, g, xg, ab, res, err, rowpart, sst, gbar, total;
};

WsLayout batch_layout(const hubbard_batch* B, int max_iters) {
    WsLayout L{};
    size_t o = 0;
    const size_t T = (size_t)B->total, n = (size_t)B->n;
    L.f = o; o += al256(T * 8);
    L.g = o; o += al256(T * 8);
    L.xg = o; o += al256(T * 8);
    L.ab = o; o += al256(n * 2 * (size_t)max_iters * 8);
    L.res = o; o += al256(n * sizeof(lanczos_result));
    L.err = o; o += 256;
    L.rowpart = o; o += al256((size_t)B->rows_all * 3 * 8);
    L.sst = o; o += al256(n * sizeof(SweepState));
    L.gbar = o; o += 256;                  // grid barrier counter, active-sector count, row and task counters
    L.total = o;
    return L;
}

// One cooperative launch: the sweep over the schedule's sweep list (when
// `sweep`), then the one-CTA tasks d_tasks[0 .. ntasks).  mode_force >= 0
// gives every sector those schedule bits (autotuner trials).
int batch_launch(hubbard_batch* B, const double* v0_all, int max_iters, double tol, char* ws, const WsLayout& L,
                 cudaStream_t s, const int* d_tasks, int ntasks, bool sweep, int mode_force, int iter_cap) {
    // the barrier counter and the error word start at zero
    HUB_CUDA(cudaMemsetAsync(ws + L.err, 0, 4, s));
    HUB_CUDA(cudaMemsetAsync(ws + L.gbar, 0, 64, s));
    BatchParams P;
    P.sec = B->d_sec;
    P.tasks = d_tasks;
    P.ntasks = ntasks;
    P.rp = B->d_rp;
    P.ent = B->d_ent;
    P.st = B->d_st;
    P.bo = B->d_bo;
    P.bc = B->d_bc;
    P.be = B->d_be;
    P.v0 = v0_all;
    P.f = (double*)(ws + L.f);
    P.g = (double*)(ws + L.g);
    P.xg = (int2*)(ws + L.xg);
    P.ab = (double*)(ws + L.ab);
    P.res = (lanczos_result*)(ws + L.res);
    P.err = (int*)(ws + L.err);
    P.max_iters = max_iters;
    P.iter_cap = std::min(max_iters, iter_cap);
    P.tol = tol > 0.0 ? tol : 1e-10;
    P.smem_elems = B->smem_elems;
    P.mode_force = mode_force;
    P.spin_limit = 20000000;            // ~2.5 s of 128 ns sleeps per barrier
    P.nswp = sweep ? B->nswp : 0;
    {
        const int g = B->nswp == 0 ? 0 : B->grid;
        P.sweep_ctas = std::max(1, g - std::min(B->task_ctas, std::max(0, B->ntasks)));
        if (B->task_ctas >= g) P.sweep_ctas = std::max(1, g / 2);
    }
    P.swp = B->d_swp;
    P.rowoff = B->d_rowoff;
    P.rowsec = B->d_rowsec;
    P.rowpart = (double*)(ws + L.rowpart);
    P.sst = (SweepState*)(ws + L.sst);
    P.gbar = (unsigned int*)(ws + L.gbar);
    P.nactive = (int*)(ws + L.gbar + 4);
    P.claim = (unsigned long long*)(ws + L.gbar + 16);
    P.q_posted = nullptr;
    P.q_stop = nullptr;
    P.q_claim = nullptr;
    P.q_done = nullptr;
    P.q_cap = 1;
    P.q_idle = 0;
    void* args[] = {&P};
    const size_t smem = (size_t)B->smem_elems * sizeof(int2);
    // without sweep sectors every CTA takes one-CTA tasks: a batch of a few
    // sectors then occupies only as many CTAs as it has tasks, and the rest of
    // the GPU stays free for concurrent work on other streams
    const int grid = P.nswp == 0 ? std::max(1, std::min(B->grid, ntasks)) : B->grid;
    HUB_CUDA(cudaLaunchCooperativeKernel((const void*)k_batch_lanczos, dim3(grid), dim3(kBatchThreads), args, smem, s));
    count_launches(1);
    return HUB_OK;
}

}  // namespace
}  // namespace hub

using namespace hub;

extern "C" {

int hubbard_batch_create(const hubbard_sector_desc* sectors, int n_sectors, hubbard_batch_t* out) {
    return batch_create_streamed(sectors, n_sectors, nullptr, out);
}

}  // extern "C"

int hub::batch_create_streamed(const hubbard_sector_desc* sectors, int n_sectors, cudaStream_t ms,
                               hubbard_batch_t* out) {
    clear_error();
    if (out == nullptr || n_sectors < 1 || sectors == nullptr) return fail(HUB_EINVAL, "bad batch arguments");
    *out = nullptr;
    hubbard_batch* B = new (std::nothrow) hubbard_batch();
    if (B == nullptr) return fail(HUB_ENOMEM, "host allocation");
    B->mem_stream = ms;
    cudaGetDevice(&B->device);
    B->n = n_sectors;
    std::vector<int32_t> rp;
    std::vector<uint32_t> ent, st;
    RowPools rows;
    std::map<std::tuple<int, std::vector<std::pair<int, int>>, int>, Cached> cache;
    std::map<std::tuple<int64_t, int64_t, int>, int> shape_ids;
    auto spin = [&](int ns, const std::vector<std::pair<int, int>>& bl, int N) -> Cached {
        auto key = std::make_tuple(ns, bl, N);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
        SpinTables T;
        build_spin_tables(ns, N, bl, T);
        Cached c{(int64_t)rp.size(), (int64_t)ent.size(), (int64_t)st.size(), T.D, T.W,
                 T.D ? (double)T.tgt.size() / (double)T.D : 0.0, -1};
        if (T.D <= kRowTableMaxD) {
            RowBlocks rb;
            build_row_blocks(T, 8, rb);
            if (rb.narrow) {
                const int64_t base = (int64_t)rows.be.size();  // a multiple of 128 entries: 16-byte aligned
                c.blk = (int64_t)rows.bo.size();
                for (size_t g = 0; g < rb.boff.size(); ++g) {
                    rows.bo.push_back(base + rb.boff[g]);
                    rows.bc.push_back(rb.bcnt[g]);
                }
                for (uint32_t e : rb.ent) rows.be.push_back((uint16_t)e);
            }
        }
        rp.insert(rp.end(), T.rowptr.begin(), T.rowptr.end());
        for (size_t k = 0; k < T.tgt.size(); ++k) ent.push_back(((uint32_t)T.tgt[k] << 1) | (T.sign[k] < 0 ? 1u : 0u));
        st.insert(st.end(), T.states.begin(), T.states.end());
        cache.emplace(key, c);
        return c;
    };
    B->voff.assign((size_t)n_sectors + 1, 0);
    try {
        for (int i = 0; i < n_sectors; ++i) {
            const hubbard_sector_desc& d = sectors[i];
            if (d.ns < 1 || d.ns > 32 || d.nup < 0 || d.nup > d.ns || d.ndn < 0 || d.ndn > d.ns ||
                d.n_bonds < 0 || (d.n_bonds > 0 && d.bonds == nullptr) || !std::isfinite(d.t) || !std::isfinite(d.U)) {
                delete B;
                return fail(HUB_EINVAL, "batch: invalid sector " + std::to_string(i));
            }
            std::vector<std::pair<int, int>> bl;
            std::vector<std::pair<int, int>> seen;
            for (int b = 0; b < d.n_bonds; ++b) {
                const int x = d.bonds[2 * b], y = d.bonds[2 * b + 1];
                const std::pair<int, int> key(std::min(x, y), std::max(x, y));
                if (x < 0 || x >= d.ns || y < 0 || y >= d.ns || x == y ||
                    std::find(seen.begin(), seen.end(), key) != seen.end()) {
                    delete B;
                    return fail(HUB_EINVAL, "batch: bad or duplicate bond in sector " + std::to_string(i));
                }
                seen.push_back(key);
                bl.emplace_back(x, y);
            }
            const Cached cu = spin(d.ns, bl, d.nup), cd = spin(d.ns, bl, d.ndn);
            if (cu.W + cd.W > 127) {
                delete B;
                return fail(HUB_EINVAL, "batch: more than 127 hops per state in sector " + std::to_string(i));
            }
            SectorDesc s{};
            s.Dup = cu.D;
            s.Ddn = cd.D;
            s.D = cu.D * cd.D;
            if (s.D > (int64_t)1 << 31) {
                delete B;
                return fail(HUB_EINVAL, "batch: sector dimension above 2^31");
            }
            s.voff = B->total;
            s.up_rp = cu.rp_off;
            s.dn_rp = cd.rp_off;
            s.up_ent = cu.ent_off;
            s.dn_ent = cd.ent_off;
            s.up_st = cu.st_off;
            s.dn_st = cd.st_off;
            s.dn_blk = cd.blk;
            s.t = d.t;
            s.U = d.U;
            {
                const auto key = std::make_tuple(s.Dup, s.Ddn, (int)(cu.W + cd.W));
                auto it = shape_ids.find(key);
                if (it == shape_ids.end()) {
                    it = shape_ids.emplace(key, (int)B->shapes.size()).first;
                    B->shapes.push_back({s.Dup, s.Ddn, (int)(cu.W + cd.W), 0, kModeDefault});
                }
                B->shapes[(size_t)it->second].count++;
                B->shape_of.push_back(it->second);
                s.mode = kModeDefault;
            }
            B->sec.push_back(s);
            B->cost.push_back((double)s.D * (cu.hops + cd.hops + 8.0));
            B->hops1.push_back(cu.W + cd.W + 1);
            B->rows_all += s.Dup;
            B->total += (s.D + 1) / 2 * 2;           // keep every sector 16-byte aligned
            B->voff[(size_t)i + 1] = B->total;
        }
    } catch (const std::bad_alloc&) {
        delete B;
        return fail(HUB_ENOMEM, "host allocation (batch tables)");
    }
    int rc = batch_upload(B, rp, ent, st, rows);
    if (rc == HUB_OK && batch_grid(B, &B->smem_elems) < 0) rc = fail(HUB_ECUDA, "batch kernel occupancy");
    if (rc != HUB_OK) {
        std::string msg = hubbard_last_error();
        batch_free(B);
        delete B;
        return fail(rc, msg);
    }
    *out = B;
    return HUB_OK;
}

extern "C" {

void hubbard_batch_destroy(hubbard_batch_t B) {
    if (B == nullptr) return;
    // a batch tied to a stream frees in that stream's order
    if (B->mem_stream == nullptr) cudaDeviceSynchronize();
    batch_free(B);
    delete B;
}

int hubbard_batch_vector_offsets(hubbard_batch_t B, int64_t* offsets) {
    clear_error();
    if (B == nullptr || offsets == nullptr) return fail(HUB_EINVAL, "null argument");
    std::memcpy(offsets, B->voff.data(), B->voff.size() * sizeof(int64_t));
    return HUB_OK;
}

size_t hubbard_batch_workspace_bytes(hubbard_batch_t B, int max_iters) {
    if (B == nullptr || max_iters < 1) return 0;
    return batch_layout(B, max_iters).total;
}

int hubbard_batch_set_schedule(hubbard_batch_t B, int64_t elems_per_cta) {
    clear_error();
    if (B == nullptr || elems_per_cta < 1) return fail(HUB_EINVAL, "bad schedule");
    B->elems_per_cta = elems_per_cta;
    return HUB_OK;
}

int hubbard_batch_solve_async(hubbard_batch_t B, const double* v0_all, int max_iters, double tol, void* workspace,
                              size_t ws_bytes, void* stream) {
    clear_error();
    if (B == nullptr || v0_all == nullptr || max_iters < 1) return fail(HUB_EINVAL, "bad batch solve arguments");
    if ((reinterpret_cast<uintptr_t>(v0_all) & 15u) || workspace == nullptr ||
        (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return fail(HUB_EINVAL, "v0 must be 16-byte and workspace 256-byte aligned");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != B->device) return fail(HUB_EINVAL, "batch created on another device");
    const WsLayout L = batch_layout(B, max_iters);
    if (ws_bytes < L.total) return fail(HUB_ENOMEM, "batch workspace too small");
    int rc;
    // descriptors: a/b history offsets depend on max_iters
    // (both uploaded synchronously: fix them before capturing this call in a graph)
    bool dirty = false;
    if (B->sched_max_iters != max_iters) {
        for (int i = 0; i < B->n; ++i) B->sec[(size_t)i].ab = (int64_t)i * 2 * max_iters;
        B->sched_max_iters = max_iters;
        dirty = true;
    }
    if (B->sched_elems != B->elems_per_cta) {
        if ((rc = batch_schedule(B))) return rc;      // uploads the descriptors too
        dirty = false;
        B->desc_dirty = false;
    }
    if (dirty || B->desc_dirty) {
        HUB_CUDA(dev_upload(B->d_sec, B->sec.data(), B->sec.size() * sizeof(SectorDesc), B->mem_stream));
        B->desc_dirty = false;
    }
    return batch_launch(B, v0_all, max_iters, tol, (char*)workspace, L, (cudaStream_t)stream, B->d_tasks, B->ntasks,
                        true, -1, max_iters);
}

int hubbard_batch_results(hubbard_batch_t B, const void* workspace, int max_iters, void* stream,
                          lanczos_result* results) {
    clear_error();
    if (B == nullptr || workspace == nullptr || results == nullptr) return fail(HUB_EINVAL, "null argument");
    const WsLayout L = batch_layout(B, max_iters);
    cudaStream_t s = (cudaStream_t)stream;
    int err = 0;
    HUB_CUDA(cudaMemcpyAsync(results, (const char*)workspace + L.res, (size_t)B->n * sizeof(lanczos_result),
                             cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaMemcpyAsync(&err, (const char*)workspace + L.err, 4, cudaMemcpyDeviceToHost, s));
    // a/b histories, for the a-posteriori error bound of every sector
    std::vector<double> ab;
    try {
        ab.resize((size_t)B->n * 2 * (size_t)max_iters);
    } catch (const std::bad_alloc&) {
        return fail(HUB_ENOMEM, "host allocation (batch a/b histories)");
    }
    HUB_CUDA(cudaMemcpyAsync(ab.data(), (const char*)workspace + L.ab, ab.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    HUB_CUDA(cudaStreamSynchronize(s));
    if (err != 0) return fail(err, "batch: a grid barrier timed out");
    for (int i = 0; i < B->n; ++i) {
        lanczos_result& r = results[i];
        const int m = r.iters;
        if (m < 1 || m > max_iters) {
            r.err_bound = INFINITY;
            continue;
        }
        const double* A = ab.data() + (size_t)i * 2 * max_iters;
        const double* Bv = A + max_iters;
        const double gap = tridiag_gap_lower(A, Bv, m, Bv[m - 1], r.energy);
        r.err_bound = energy_error_bound(r.residual, gap) +
                      rounding_floor(B->hops1[(size_t)i], HUB_F64, tridiag_scale(A, Bv, m));
    }
    return HUB_OK;
}

int hubbard_selftest_wait_timeout(void* stream) {
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    char* buf = nullptr;
    HUB_CUDA(cudaMalloc((void**)&buf, 256));
    int err = 0;
    cudaError_t e = cudaMemsetAsync(buf, 0, 256, s);
    if (e == cudaSuccess) {
        k_wait_probe<<<2, 64, 0, s>>>((unsigned int*)buf, 2000, (int*)(buf + 128));
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, buf + 128, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe");
    if (err == HUB_ETIMEOUT) return fail(HUB_ETIMEOUT, "bounded wait gave up as intended");
    return fail(HUB_EDEVICE, "bounded wait did not report its timeout");
}

int hubbard_batch_autotune(hubbard_batch_t B, const double* v0_all, int max_iters, double tol, void* workspace,
                           size_t ws_bytes, void* stream, int64_t* chosen) {
    clear_error();
    if (B == nullptr) return fail(HUB_EINVAL, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    // the first solve checks the arguments and fixes the descriptors for max_iters
    int rc = hubbard_batch_solve_async(B, v0_all, max_iters, tol, workspace, ws_bytes, stream);
    if (rc != HUB_OK) return rc;
    HUB_CUDA(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    HUB_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(HUB_ECUDA, "event");
    }
    // a warm-up run, then the timed one; < 0 on failure (rc set)
    auto timed = [&](auto&& launch) -> float {
        float ms = -1.0f;
        for (int rep = 0; rep < 2 && rc == HUB_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) rc = fail(HUB_ECUDA, "event");
            if (rc == HUB_OK) rc = launch();
            if (rc == HUB_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = fail(HUB_ECUDA, "event");
            if (rc == HUB_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(HUB_ECUDA, "event sync");
        }
        if (rc == HUB_OK) cudaEventElapsedTime(&ms, e0, e1);
        return rc == HUB_OK ? ms : -1.0f;
    };
    // 1. per-shape schedule bits of the one-CTA tasks: for every shape that is
    // a task under the largest threshold tried, up to one grid of its sectors
    // is solved alone as tasks for 16 steps in each candidate mode -- the whole vector in
    // shared memory (when it fits) or warp-per-row passes over the L2 copy,
    // with or without the row staged for the down-hops -- and the fastest mode
    // (the default unless another is 3 % faster) goes into the shape's entry
    const int64_t kMaxTask = (int64_t)1 << 17;
    constexpr int kTrialSteps = 16;                   // steps per trial solve (the cost per step is what differs)
    const WsLayout L = batch_layout(B, max_iters);
    std::vector<std::vector<int>> members(B->shapes.size());
    for (int i = 0; i < B->n; ++i) members[(size_t)B->shape_of[(size_t)i]].push_back(i);
    int* d_trial = nullptr;
    const size_t trial_cap = (size_t)std::max(1, B->grid);
    if (dev_alloc((void**)&d_trial, trial_cap * sizeof(int), B->mem_stream) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(HUB_ENOMEM, "autotune trial list");
    }
    for (size_t k = 0; k < B->shapes.size() && rc == HUB_OK; ++k) {
        auto& sh = B->shapes[k];
        const int64_t D = sh.Dup * sh.Ddn;
        if (D > kMaxTask || members[k].empty()) continue;
        std::vector<int> ids(members[k].begin(), members[k].begin() + std::min(members[k].size(), trial_cap));
        if (cudaMemcpyAsync(d_trial, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = fail(HUB_ECUDA, "autotune trial upload");
            break;
        }
        const int cands_flat[] = {kModeDefault, kModeStage};
        const int cands_rows[] = {kModeStage, 0};
        const int* cands = D <= B->smem_elems ? cands_flat : cands_rows;
        float t[2];
        for (int c = 0; c < 2 && rc == HUB_OK; ++c)
            t[c] = timed([&] {
                return batch_launch(B, v0_all, max_iters, tol, (char*)workspace, L, s, d_trial, (int)ids.size(),
                                    false, cands[c], kTrialSteps);
            });
        if (rc == HUB_OK) sh.mode = (t[1] < 0.97f * t[0]) ? cands[1] : cands[0];
    }
    dev_free(d_trial, B->mem_stream);
    for (int i = 0; i < B->n; ++i) B->sec[(size_t)i].mode = B->shapes[(size_t)B->shape_of[(size_t)i]].mode;
    B->desc_dirty = true;
    // 2. the size threshold between the grid-wide sweep and the tasks: full
    // solves for elems_per_cta in 2^12 .. 2^17 with the shapes' modes
    const int64_t cands[] = {1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16, kMaxTask};
    float best = 1e30f;
    int64_t best_e = B->elems_per_cta;
    for (int64_t c : cands) {
        if (rc != HUB_OK) break;
        B->elems_per_cta = c;
        const float ms =
            timed([&] { return hubbard_batch_solve_async(B, v0_all, max_iters, tol, workspace, ws_bytes, stream); });
        if (rc == HUB_OK && ms < best) {
            best = ms;
            best_e = c;
        }
    }
    B->elems_per_cta = best_e;
    // 3. how many CTAs start on the one-CTA tasks while the rest sweep
    //    (the tasks then overlap the sweep's lightly loaded last steps)
    int best_t = 0;
    if (rc == HUB_OK) {
        float best_t_ms = 1e30f;
        for (int tcand : {0, 16, 32, 48, 64}) {
            B->task_ctas = tcand;
            const float ms =
                timed([&] { return hubbard_batch_solve_async(B, v0_all, max_iters, tol, workspace, ws_bytes, stream); });
            if (rc != HUB_OK) break;
            if (ms < best_t_ms) {
                best_t_ms = ms;
                best_t = tcand;
            }
        }
    }
    B->task_ctas = best_t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen) *chosen = best_e;
    return rc;
}

int hubbard_batch_get_schedule(hubbard_batch_t B, int64_t* elems_per_cta, int* task_ctas) {
    clear_error();
    if (B == nullptr) return fail(HUB_EINVAL, "null batch");
    if (elems_per_cta) *elems_per_cta = B->elems_per_cta;
    if (task_ctas) *task_ctas = B->task_ctas;
    return HUB_OK;
}

int hubbard_batch_set_task_ctas(hubbard_batch_t B, int task_ctas) {
    clear_error();
    if (B == nullptr || task_ctas < 0) return fail(HUB_EINVAL, "bad task CTA count");
    B->task_ctas = task_ctas;
    return HUB_OK;
}

int hubbard_batch_set_shape_mode(hubbard_batch_t B, int shape, int mode) {
    clear_error();
    if (B == nullptr || shape < 0 || shape >= (int)B->shapes.size() || mode < 0 || mode > kModeDefault)
        return fail(HUB_EINVAL, "bad shape or mode");
    B->shapes[(size_t)shape].mode = mode;
    for (int i = 0; i < B->n; ++i)
        if (B->shape_of[(size_t)i] == shape) B->sec[(size_t)i].mode = mode;
    B->desc_dirty = true;
    return HUB_OK;
}

int hubbard_batch_schedule_table(hubbard_batch_t B, int64_t* rows, int cap, int* n_out) {
    clear_error();
    if (B == nullptr || n_out == nullptr || cap < 0 || (cap > 0 && rows == nullptr))
        return fail(HUB_EINVAL, "bad schedule table arguments");
    *n_out = (int)B->shapes.size();
    for (int k = 0; k < std::min(cap, *n_out); ++k) {
        const auto& sh = B->shapes[(size_t)k];
        int64_t* r = rows + 6 * (size_t)k;
        r[0] = sh.Dup;
        r[1] = sh.Ddn;
        r[2] = sh.W;
        r[3] = sh.count;
        r[4] = sh.Dup * sh.Ddn > B->elems_per_cta ? 2 : 1;
        r[5] = sh.mode;
    }
    return HUB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Queued solver (hubbard_queue_*): the batch kernel's one-CTA task path kept
// running while sectors are posted.  A task is one sector solved by one CTA
// (Algorithm 1 on the device, as in a batch).  Slot n % capacity holds task
// n's descriptor, vectors, a/b history and result; the host publishes a task
// by raising the posted count in host-mapped memory after its descriptor has
// been copied, a CTA takes task numbers below that count, and writes the
// result and then the slot's done word (task number + 1) to host-mapped memory.
// The kernel runs as up to 8 workers (launches on the queue's streams), one
// more started while unfinished tasks outnumber the running workers' CTAs; a
// worker leaves ~2 ms after it last claimed a task (the first after ~20 ms)
// or at destroy; a task number is only ever taken once posted, so leaving
// loses none.  Hop tables are cached per (lattice, particle number) in device
// pools that grow (with the workers stopped) as new ones are needed.
struct hubbard_queue {
    int device = 0;
    int cap = 0;
    int64_t max_dim = 0, vstride = 0;
    int max_iters = 0;
    double tol = 0.0;
    int ctas = 0;
    int smem_elems = 0;
    std::mutex mu;
    // workers: launches of the task kernel over this queue, each on its own
    // stream with `ctas` CTAs; another starts while posted tasks outnumber the
    // CTAs of the running ones, so the solver's width follows the backlog
    static constexpr int kWorkers = 8;
    cudaStream_t ks[kWorkers] = {};
    bool wrun[kWorkers] = {};
    int wctas[kWorkers] = {};
    int resident = 0;                          // CTAs of the workers running at the last check
    std::chrono::steady_clock::time_point checked{};
    cudaStream_t cstream = nullptr;            // uploads and reads
    // device
    hub::SectorDesc* d_sec = nullptr;          // [cap]
    double* d_f = nullptr;                     // [cap * vstride] each
    double* d_g = nullptr;
    int2* d_xg = nullptr;
    double* d_ab = nullptr;                    // [cap * 2 * max_iters]
    int* d_err = nullptr;
    unsigned int* d_claim = nullptr;
    // table pools (device, with host-side fill counts and capacities in elements)
    int32_t* d_rp = nullptr;
    uint32_t* d_ent = nullptr;
    uint32_t* d_st = nullptr;
    int64_t* d_bo = nullptr;
    int32_t* d_bc = nullptr;
    uint16_t* d_be = nullptr;
    size_t n_rp = 0, n_ent = 0, n_st = 0, n_bo = 0, n_bc = 0, n_be = 0;
    size_t c_rp = 0, c_ent = 0, c_st = 0, c_bo = 0, c_bc = 0, c_be = 0;
    // host-mapped
    unsigned int* h_ctl = nullptr;             // [0] posted, [1] stop
    unsigned int* h_done = nullptr;            // [cap]
    lanczos_result* h_res = nullptr;           // [cap]
    unsigned int* m_ctl = nullptr;             // device views of the mapped buffers
    unsigned int* m_done = nullptr;
    lanczos_result* m_res = nullptr;
    // host state
    struct Cached {
        int64_t rp, ent, st, D;
        int W;
        int64_t blk;
    };
    std::map<std::tuple<int, std::vector<std::pair<int, int>>, int>, Cached> cache;
    uint64_t posted = 0;
    std::vector<int64_t> slot_ticket;          // task in the slot not yet harvested, -1: free
    std::vector<int> slot_hops1;               // W_up + W_dn + 1 of that task
    std::unordered_map<int64_t, lanczos_result> finished;
};

namespace hub {
namespace {

// appends n elements to a device pool (capacity in elements), growing it
// 2x (copying the old contents) when full; the caller has stopped the kernel
// before a pool may move.  Regions start on 256-byte boundaries, so no cache
// line mixes the tables of two uploads.
template <typename T>
int pool_append(T** pool, size_t* used, size_t* capn, const T* src, size_t n, cudaStream_t s, bool* moved,
                int64_t* at, size_t align = 256 / sizeof(T)) {
    const size_t start = (*used + align - 1) / align * align;
    if (start + n > *capn) {
        size_t nc = std::max<size_t>(*capn * 2, start + n + align);
        T* np = nullptr;
        if (cudaMalloc((void**)&np, nc * sizeof(T)) != cudaSuccess) return fail(HUB_ENOMEM, "queue table pool");
        if (*used > 0) HUB_CUDA(cudaMemcpyAsync(np, *pool, *used * sizeof(T), cudaMemcpyDeviceToDevice, s));
        HUB_CUDA(cudaStreamSynchronize(s));
        cudaFree(*pool);
        *pool = np;
        *capn = nc;
        *moved = true;
    }
    if (n > 0) HUB_CUDA(cudaMemcpyAsync(*pool + start, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    *used = start + n;
    *at = (int64_t)start;
    return HUB_OK;
}

}  // namespace
}  // namespace hub

namespace hub {
namespace {

void queue_set_stop(hubbard_queue* Q, unsigned v) {
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile unsigned int*)(Q->h_ctl + 1) = v;
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

bool queue_any_running(const hubbard_queue* Q) {
    for (int w = 0; w < hubbard_queue::kWorkers; ++w)
        if (Q->wrun[w]) return true;
    return false;
}

// lets the running workers finish every posted task and leave
int queue_stop_kernel(hubbard_queue* Q) {
    if (!queue_any_running(Q)) return HUB_OK;
    queue_set_stop(Q, 1u);
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < hubbard_queue::kWorkers; ++w) {
        if (!Q->wrun[w]) continue;
        const cudaError_t ew = cudaStreamSynchronize(Q->ks[w]);
        if (e == cudaSuccess) e = ew;
        Q->wrun[w] = false;
    }
    Q->resident = 0;
    queue_set_stop(Q, 0u);
    if (e != cudaSuccess) return cuda_fail(e, "queue kernel");
    return HUB_OK;
}

// device tables of one spin species (cached per lattice and particle number).
// Called without the queue's lock: the host tables of a new species are built
// unlocked (milliseconds for the larger ones), then appended under the lock.
int queue_spin(hubbard_queue* Q, int ns, const std::vector<std::pair<int, int>>& bl, int N,
               hubbard_queue::Cached* out) {
    const auto key = std::make_tuple(ns, bl, N);
    {
        std::lock_guard<std::mutex> lk(Q->mu);
        auto it = Q->cache.find(key);
        if (it != Q->cache.end()) {
            *out = it->second;
            return HUB_OK;
        }
    }
    SpinTables T;
    build_spin_tables(ns, N, bl, T);
    std::vector<uint32_t> ent(T.tgt.size());
    for (size_t k = 0; k < T.tgt.size(); ++k) ent[k] = ((uint32_t)T.tgt[k] << 1) | (T.sign[k] < 0 ? 1u : 0u);
    RowBlocks rb;
    bool rows = false;
    std::vector<uint16_t> be;
    if (T.D <= kRowTableMaxD) {
        build_row_blocks(T, 8, rb);
        rows = rb.narrow;
        if (rows) {
            be.resize(rb.ent.size());
            for (size_t i = 0; i < rb.ent.size(); ++i) be[i] = (uint16_t)rb.ent[i];
        }
    }
    std::lock_guard<std::mutex> lk(Q->mu);
    {
        auto it = Q->cache.find(key);                    // built meanwhile by another caller
        if (it != Q->cache.end()) {
            *out = it->second;
            return HUB_OK;
        }
    }
    // a pool that must grow moves: the kernel leaves first
    // (the per-group arrays bo and bc advance in step: the same alignment, 64 groups)
    auto fits = [](size_t used, size_t capn, size_t n, size_t align) {
        return (used + align - 1) / align * align + n <= capn;
    };
    const bool grow = !fits(Q->n_rp, Q->c_rp, T.rowptr.size(), 64) || !fits(Q->n_ent, Q->c_ent, ent.size(), 64) ||
                      !fits(Q->n_st, Q->c_st, T.states.size(), 64) ||
                      (rows && (!fits(Q->n_bo, Q->c_bo, rb.boff.size(), 64) ||
                                !fits(Q->n_bc, Q->c_bc, rb.bcnt.size(), 64) || !fits(Q->n_be, Q->c_be, be.size(), 128)));
    int rc;
    if (grow && (rc = queue_stop_kernel(Q))) return rc;
    bool moved = false;
    hubbard_queue::Cached c{0, 0, 0, T.D, T.W, -1};
    if ((rc = pool_append(&Q->d_rp, &Q->n_rp, &Q->c_rp, T.rowptr.data(), T.rowptr.size(), Q->cstream, &moved, &c.rp)))
        return rc;
    if ((rc = pool_append(&Q->d_ent, &Q->n_ent, &Q->c_ent, ent.data(), ent.size(), Q->cstream, &moved, &c.ent)))
        return rc;
    if ((rc = pool_append(&Q->d_st, &Q->n_st, &Q->c_st, T.states.data(), T.states.size(), Q->cstream, &moved, &c.st)))
        return rc;
    if (rows) {
        int64_t be_at = 0, bc_at = 0;
        if ((rc = pool_append(&Q->d_be, &Q->n_be, &Q->c_be, be.data(), be.size(), Q->cstream, &moved, &be_at)))
            return rc;
        std::vector<int64_t> bo(rb.boff.size());
        for (size_t g = 0; g < bo.size(); ++g) bo[g] = be_at + rb.boff[g];
        if ((rc = pool_append(&Q->d_bo, &Q->n_bo, &Q->c_bo, bo.data(), bo.size(), Q->cstream, &moved, &c.blk, 64)))
            return rc;
        if ((rc = pool_append(&Q->d_bc, &Q->n_bc, &Q->c_bc, rb.bcnt.data(), rb.bcnt.size(), Q->cstream, &moved,
                              &bc_at, 64)))
            return rc;
        if (bc_at != c.blk) {
            // the two per-group arrays are indexed by the same group number
            return fail(HUB_EDEVICE, "queue row-table pools out of step");
        }
    }
    HUB_CUDA(cudaStreamSynchronize(Q->cstream));
    Q->cache.emplace(key, c);
    *out = c;
    return HUB_OK;
}

}  // namespace
}  // namespace hub

namespace hub {
namespace {

// launches the task kernel over the queue on worker w (the caller holds the lock)
int queue_launch(hubbard_queue* Q, int w, int ctas) {
    BatchParams P{};
    P.sec = Q->d_sec;
    P.tasks = nullptr;
    P.ntasks = 0;
    P.rp = Q->d_rp;
    P.ent = Q->d_ent;
    P.st = Q->d_st;
    P.bo = Q->d_bo;
    P.bc = Q->d_bc;
    P.be = Q->d_be;
    P.v0 = nullptr;
    P.f = Q->d_f;
    P.g = Q->d_g;
    P.xg = Q->d_xg;
    P.ab = Q->d_ab;
    P.res = Q->m_res;
    P.err = Q->d_err;
    P.max_iters = Q->max_iters;
    P.iter_cap = Q->max_iters;
    P.tol = Q->tol;
    P.smem_elems = Q->smem_elems;
    P.mode_force = -1;
    P.spin_limit = 20000000;
    P.nswp = 0;
    P.q_posted = Q->m_ctl;
    P.q_stop = Q->m_ctl + 1;
    P.q_claim = Q->d_claim;
    P.q_done = Q->m_done;
    P.q_cap = Q->cap;
    // worker 0 waits ~20 ms (2-us sleeps) for the next task, so a new arrival
    // finds resident CTAs; the others leave after ~2 ms with nothing left to
    // claim, giving their SMs back to the rest of the device
    P.q_idle = w == 0 ? 10000 : 1200;
    k_batch_lanczos<<<ctas, kBatchThreads, (size_t)Q->smem_elems * sizeof(int2), Q->ks[w]>>>(P);
    HUB_CUDA(cudaGetLastError());
    count_launches(1);
    Q->wrun[w] = true;
    Q->wctas[w] = ctas;
    return HUB_OK;
}

// retires finished workers and starts one more while the tasks not yet
// finished outnumber the CTAs of the running workers
int queue_scale(hubbard_queue* Q) {
    int outstanding = 0;
    for (int k = 0; k < Q->cap; ++k) outstanding += Q->slot_ticket[(size_t)k] >= 0 ? 1 : 0;
    // the workers' streams are queried only when more CTAs may be needed or
    // every 2 ms (each query is a driver call the other lanes' launches wait on)
    const auto now = std::chrono::steady_clock::now();
    if (outstanding <= Q->resident && now - Q->checked < std::chrono::milliseconds(2)) return HUB_OK;
    Q->checked = now;
    int resident = 0, free_w = -1;
    for (int w = 0; w < hubbard_queue::kWorkers; ++w) {
        if (Q->wrun[w] && cudaStreamQuery(Q->ks[w]) == cudaSuccess) Q->wrun[w] = false;
        if (Q->wrun[w]) resident += Q->wctas[w];
        else if (free_w < 0) free_w = w;
    }
    Q->resident = resident;
    if (outstanding > resident && free_w >= 0) {
        const int c = std::min(Q->ctas, outstanding - resident);
        Q->resident += c;
        return queue_launch(Q, free_w, c);
    }
    return HUB_OK;
}

// moves finished tasks' results (with their a-posteriori bounds) to the host
// map and frees their slots; relaunches the kernel if it left with tasks posted
int queue_harvest(hubbard_queue* Q) {
    std::vector<int> ready;
    for (int k = 0; k < Q->cap; ++k) {
        const int64_t t = Q->slot_ticket[(size_t)k];
        if (t < 0) continue;
        const unsigned d = *(volatile unsigned int*)(Q->h_done + k);
        if (d == (unsigned)(t + 1)) ready.push_back(k);
    }
    if (!ready.empty()) {
        std::atomic_thread_fence(std::memory_order_acquire);
        const size_t m = (size_t)2 * Q->max_iters;
        std::vector<double> ab(ready.size() * m);
        for (size_t i = 0; i < ready.size(); ++i)
            HUB_CUDA(cudaMemcpyAsync(ab.data() + i * m, Q->d_ab + (size_t)ready[i] * m, m * sizeof(double),
                                     cudaMemcpyDeviceToHost, Q->cstream));
        HUB_CUDA(cudaStreamSynchronize(Q->cstream));
        for (size_t i = 0; i < ready.size(); ++i) {
            const int k = ready[i];
            lanczos_result r;
            std::memcpy(&r, (const void*)(Q->h_res + k), sizeof r);
            const int it = r.iters;
            if (it >= 1 && it <= Q->max_iters) {
                const double* A = ab.data() + i * m;
                const double* Bv = A + Q->max_iters;
                const double gap = tridiag_gap_lower(A, Bv, it, Bv[it - 1], r.energy);
                r.err_bound = energy_error_bound(r.residual, gap) +
                              rounding_floor(Q->slot_hops1[(size_t)k], HUB_F64, tridiag_scale(A, Bv, it));
            } else {
                r.err_bound = INFINITY;
            }
            Q->finished[Q->slot_ticket[(size_t)k]] = r;
            Q->slot_ticket[(size_t)k] = -1;
        }
    }
    return queue_scale(Q);
}

void queue_free(hubbard_queue* Q) {
    if (Q->h_ctl != nullptr && queue_any_running(Q)) {
        queue_set_stop(Q, 1u);
        for (int w = 0; w < hubbard_queue::kWorkers; ++w)
            if (Q->wrun[w]) cudaStreamSynchronize(Q->ks[w]);
    }
    if (Q->cstream) cudaStreamSynchronize(Q->cstream);
    cudaFree(Q->d_sec);
    cudaFree(Q->d_f);
    cudaFree(Q->d_g);
    cudaFree(Q->d_xg);
    cudaFree(Q->d_ab);
    cudaFree(Q->d_err);
    cudaFree(Q->d_claim);
    cudaFree(Q->d_rp);
    cudaFree(Q->d_ent);
    cudaFree(Q->d_st);
    cudaFree(Q->d_bo);
    cudaFree(Q->d_bc);
    cudaFree(Q->d_be);
    if (Q->h_ctl) cudaFreeHost(Q->h_ctl);
    if (Q->h_done) cudaFreeHost(Q->h_done);
    if (Q->h_res) cudaFreeHost(Q->h_res);
    for (int w = 0; w < hubbard_queue::kWorkers; ++w)
        if (Q->ks[w]) cudaStreamDestroy(Q->ks[w]);
    if (Q->cstream) cudaStreamDestroy(Q->cstream);
    delete Q;
}

}  // namespace
}  // namespace hub

extern "C" {

int hubbard_queue_create(int capacity, int64_t max_dim, int max_iters, double tol, int ctas, hubbard_queue_t* out) {
    using namespace hub;
    clear_error();
    if (out == nullptr || capacity < 1 || capacity > (1 << 20) || max_dim < 1 || max_dim > ((int64_t)1 << 31) ||
        max_iters < 1 || ctas < 0 || !(tol >= 0.0))
        return fail(HUB_EINVAL, "bad queue arguments");
    *out = nullptr;
    hubbard_queue* Q = new (std::nothrow) hubbard_queue();
    if (Q == nullptr) return fail(HUB_ENOMEM, "host allocation");
    cudaGetDevice(&Q->device);
    Q->cap = capacity;
    Q->max_dim = max_dim;
    Q->vstride = (max_dim + 1) / 2 * 2;           // every slot's vectors 16-byte aligned
    Q->max_iters = max_iters;
    Q->tol = tol > 0.0 ? tol : 1e-10;
    int grid = 0;
    if (kernel_shape(&Q->smem_elems, &grid) < 0) {
        queue_free(Q);
        return fail(HUB_ECUDA, "queue kernel occupancy");
    }
    Q->ctas = ctas > 0 ? std::min(ctas, grid) : grid;
    Q->slot_ticket.assign((size_t)capacity, -1);
    Q->slot_hops1.assign((size_t)capacity, 1);
    const size_t nv = (size_t)capacity * (size_t)Q->vstride;
    cudaError_t e = cudaStreamCreateWithFlags(&Q->cstream, cudaStreamNonBlocking);
    for (int w = 0; w < hubbard_queue::kWorkers && e == cudaSuccess; ++w)
        e = cudaStreamCreateWithFlags(&Q->ks[w], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_sec, (size_t)capacity * sizeof(SectorDesc));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_f, nv * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_g, nv * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_xg, nv * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_ab, (size_t)capacity * 2 * max_iters * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_err, 256);
    if (e == cudaSuccess) e = cudaMalloc((void**)&Q->d_claim, 256);
    if (e == cudaSuccess) e = cudaMemset(Q->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaMemset(Q->d_claim, 0, 256);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&Q->h_ctl, 256, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&Q->h_done, (size_t)capacity * sizeof(unsigned int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&Q->h_res, (size_t)capacity * sizeof(lanczos_result), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&Q->m_ctl, Q->h_ctl, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&Q->m_done, Q->h_done, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&Q->m_res, Q->h_res, 0);
    if (e != cudaSuccess) {
        queue_free(Q);
        return cuda_fail(e, "queue allocation");
    }
    // table pools sized for a few hundred small sectors' tables, so that
    // growing one (which waits for the running tasks) stays rare
    {
        Q->c_rp = (size_t)1 << 20;
        Q->c_ent = (size_t)8 << 20;
        Q->c_st = (size_t)1 << 20;
        Q->c_bo = (size_t)1 << 18;
        Q->c_bc = (size_t)1 << 18;
        Q->c_be = (size_t)4 << 20;
        cudaError_t e2 = cudaMalloc((void**)&Q->d_rp, Q->c_rp * sizeof(int32_t));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&Q->d_ent, Q->c_ent * sizeof(uint32_t));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&Q->d_st, Q->c_st * sizeof(uint32_t));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&Q->d_bo, Q->c_bo * sizeof(int64_t));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&Q->d_bc, Q->c_bc * sizeof(int32_t));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&Q->d_be, Q->c_be * sizeof(uint16_t));
        if (e2 != cudaSuccess) {
            queue_free(Q);
            return cuda_fail(e2, "queue table pools");
        }
    }
    std::memset(Q->h_ctl, 0, 256);
    std::memset(Q->h_done, 0, (size_t)capacity * sizeof(unsigned int));
    std::memset((void*)Q->h_res, 0, (size_t)capacity * sizeof(lanczos_result));
    *out = Q;
    return HUB_OK;
}

int hubbard_queue_post(hubbard_queue_t Q, const hubbard_sector_desc* d, uint64_t seed, int64_t* ticket) {
    using namespace hub;
    clear_error();
    if (Q == nullptr || d == nullptr || ticket == nullptr) return fail(HUB_EINVAL, "null argument");
    if (d->ns < 1 || d->ns > 32 || d->nup < 0 || d->nup > d->ns || d->ndn < 0 || d->ndn > d->ns || d->n_bonds < 0 ||
        (d->n_bonds > 0 && d->bonds == nullptr) || !std::isfinite(d->t) || !std::isfinite(d->U))
        return fail(HUB_EINVAL, "queue: invalid sector");
    std::vector<std::pair<int, int>> bl;
    for (int b = 0; b < d->n_bonds; ++b) {
        const int x = d->bonds[2 * b], y = d->bonds[2 * b + 1];
        const std::pair<int, int> key(std::min(x, y), std::max(x, y));
        if (x < 0 || x >= d->ns || y < 0 || y >= d->ns || x == y)
            return fail(HUB_EINVAL, "queue: bad bond");
        for (const auto& q : bl)
            if (std::min(q.first, q.second) == key.first && std::max(q.first, q.second) == key.second)
                return fail(HUB_EINVAL, "queue: duplicate bond");
        bl.emplace_back(x, y);
    }
    int rc;
    hubbard_queue::Cached cu{}, cd{};
    if ((rc = queue_spin(Q, d->ns, bl, d->nup, &cu)) || (rc = queue_spin(Q, d->ns, bl, d->ndn, &cd))) return rc;
    std::lock_guard<std::mutex> lk(Q->mu);
    if (Q->posted >= 0x7FFFFFFFull) return fail(HUB_ENOMEM, "queue: 2^31 - 1 posts made");   // task numbers are 31-bit
    if ((rc = queue_harvest(Q))) return rc;
    const int k = (int)(Q->posted % (uint64_t)Q->cap);
    if (Q->slot_ticket[(size_t)k] >= 0) return HUB_EPENDING;     // full: the oldest task's slot is still in use
    if (cu.W + cd.W > 127) return fail(HUB_EINVAL, "queue: more than 127 hops per state");
    if (cu.D * cd.D > Q->max_dim) return fail(HUB_EINVAL, "queue: sector above the queue's max_dim");
    SectorDesc s{};
    s.Dup = cu.D;
    s.Ddn = cd.D;
    s.D = cu.D * cd.D;
    s.voff = (int64_t)k * Q->vstride;
    s.up_rp = cu.rp;
    s.dn_rp = cd.rp;
    s.up_ent = cu.ent;
    s.dn_ent = cd.ent;
    s.up_st = cu.st;
    s.dn_st = cd.st;
    s.ab = (int64_t)k * 2 * Q->max_iters;
    s.dn_blk = cd.blk;
    s.t = d->t;
    s.U = d->U;
    s.mode = kModeDefault;
    s.seed = (unsigned long long)seed;
    HUB_CUDA(cudaMemcpyAsync(Q->d_sec + k, &s, sizeof s, cudaMemcpyHostToDevice, Q->cstream));
    HUB_CUDA(cudaStreamSynchronize(Q->cstream));
    Q->slot_ticket[(size_t)k] = (int64_t)Q->posted;
    Q->slot_hops1[(size_t)k] = cu.W + cd.W + 1;
    *(volatile unsigned int*)(Q->h_done + k) = 0u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile unsigned int*)Q->h_ctl = (unsigned int)(Q->posted + 1);       // publish
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *ticket = (int64_t)Q->posted;
    ++Q->posted;
    return queue_scale(Q);
}

int hubbard_queue_prepare(hubbard_queue_t Q, const hubbard_sector_desc* d) {
    using namespace hub;
    clear_error();
    if (Q == nullptr || d == nullptr) return fail(HUB_EINVAL, "null argument");
    if (d->ns < 1 || d->ns > 32 || d->nup < 0 || d->nup > d->ns || d->ndn < 0 || d->ndn > d->ns || d->n_bonds < 0 ||
        (d->n_bonds > 0 && d->bonds == nullptr))
        return fail(HUB_EINVAL, "queue: invalid sector");
    std::vector<std::pair<int, int>> bl;
    for (int b = 0; b < d->n_bonds; ++b) {
        const int x = d->bonds[2 * b], y = d->bonds[2 * b + 1];
        if (x < 0 || x >= d->ns || y < 0 || y >= d->ns || x == y) return fail(HUB_EINVAL, "queue: bad bond");
        bl.emplace_back(x, y);
    }
    hubbard_queue::Cached cu{}, cd{};
    int rc;
    if ((rc = queue_spin(Q, d->ns, bl, d->nup, &cu)) || (rc = queue_spin(Q, d->ns, bl, d->ndn, &cd))) return rc;
    return HUB_OK;
}

int hubbard_queue_poll(hubbard_queue_t Q, int64_t ticket, lanczos_result* out) {
    using namespace hub;
    clear_error();
    if (Q == nullptr || out == nullptr) return fail(HUB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(Q->mu);
    if (ticket < 0 || (uint64_t)ticket >= Q->posted) return fail(HUB_EINVAL, "unknown ticket");
    int rc;
    if ((rc = queue_harvest(Q))) return rc;
    auto it = Q->finished.find(ticket);
    if (it == Q->finished.end()) {
        if (Q->slot_ticket[(size_t)(ticket % Q->cap)] != ticket) return fail(HUB_EINVAL, "ticket already collected");
        int err = 0;
        if (!queue_any_running(Q) &&
            cudaMemcpyAsync(&err, Q->d_err, sizeof err, cudaMemcpyDeviceToHost, Q->cstream) == cudaSuccess &&
            cudaStreamSynchronize(Q->cstream) == cudaSuccess && err != 0)
            return fail(err, "queue kernel reported an error");
        return HUB_EPENDING;
    }
    *out = it->second;
    Q->finished.erase(it);
    return HUB_OK;
}

int hubbard_queue_collect(hubbard_queue_t Q, int64_t* tickets, lanczos_result* out, int cap, int* n_out) {
    using namespace hub;
    clear_error();
    if (Q == nullptr || n_out == nullptr || cap < 0 || (cap > 0 && (tickets == nullptr || out == nullptr)))
        return fail(HUB_EINVAL, "bad collect arguments");
    std::lock_guard<std::mutex> lk(Q->mu);
    *n_out = 0;
    int rc;
    if ((rc = queue_harvest(Q))) return rc;
    int n = 0;
    for (auto it = Q->finished.begin(); it != Q->finished.end() && n < cap;) {
        tickets[n] = it->first;
        out[n] = it->second;
        ++n;
        it = Q->finished.erase(it);
    }
    *n_out = n;
    return HUB_OK;
}

void hubbard_queue_destroy(hubbard_queue_t Q) {
    if (Q == nullptr) return;
    hub::queue_free(Q);
}

}  // extern "C"
