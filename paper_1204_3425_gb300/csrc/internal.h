// Internal declarations shared by the library's translation units.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <memory>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/hubbard.h"

namespace hub {

// thread-local last-error message (hubbard_last_error)
void set_error(const std::string& msg);
void clear_error();
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Device memory of an object tied to one stream (ms != nullptr): allocated,
// uploaded and freed in that stream's order, so releasing it does not wait for
// the whole device (cudaFree would).  ms == nullptr: cudaMalloc / cudaMemcpy /
// cudaFree.
inline cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t ms) {
    return ms ? cudaMallocAsync(p, bytes, ms) : cudaMalloc(p, bytes);
}
inline void dev_free(void* p, cudaStream_t ms) {
    if (p == nullptr) return;
    if (ms) cudaFreeAsync(p, ms);
    else cudaFree(p);
}
// host -> device; pageable sources are staged before the call returns
inline cudaError_t dev_upload(void* dst, const void* src, size_t bytes, cudaStream_t ms) {
    return ms ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ms)
              : cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}

#define HUB_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return ::hub::cuda_fail(e_, #call); \
    } while (0)

// Per-spin host tables (Sec. 2.1 basis; Eq. H-Kroneckersum factors).
struct SpinTables {
    int ns = 0, n = 0;
    int64_t D = 0;
    int W = 0;                       // max hops per state
    std::vector<uint32_t> states;    // ascending basis words
    std::vector<int32_t> rowptr;     // CSR by source row r (= output row, H symmetric)
    std::vector<int32_t> tgt;        // target rank r'
    std::vector<int8_t> sign;        // +1 / -1: <r'|H|r> = -t * sign
};

// Builds the basis and hopping table of one spin species.
void build_spin_tables(int ns, int n, const std::vector<std::pair<int, int>>& bonds, SpinTables& out);

// Row-phase hop table of one spin (the SELL-32/8 layout of DevSpin::blk_off /
// blk_cnt / ent16 / ent32), its slots coloured for staged elements of eb bytes
// (4, 8 or 16).  narrow: entries fit 16 bits (15-bit index, sign in bit 15).
struct RowBlocks {
    std::vector<int64_t> boff;       // [groups] first entry of each group
    std::vector<int32_t> bcnt;       // [groups] half-blocks of 4 slots
    std::vector<uint32_t> ent;       // every group a multiple of 128 entries
    bool narrow = false;
};
void build_row_blocks(const SpinTables& T, int eb, RowBlocks& out);

// Device copy of one spin's tables.
struct DevSpin {
    uint32_t* states = nullptr;      // [D]
    int32_t* rowptr = nullptr;       // [D+1]
    uint32_t* ent = nullptr;         // [nnz] packed (target << 1) | (sign < 0)
    // the row-phase table in blocks of 8 slots per lane ("SELL-32/8"): group g
    // starts at blk_off[g] (in entries) and has blk_cnt[g] half-blocks of 4
    // slots: blk_cnt[g] / 2 blocks of 8 (block b of lane l holds slots
    // 8b .. 8b+7 at blk_off[g] + (b*32 + l)*8), then, when blk_cnt[g] is odd,
    // one block of 4 (lane l's at blk_off[g] + nfull*256 + l*4).  Entry = staged
    // slot index with the top bit set for sign -1; 16-bit (ent16) when the index
    // fits 15 bits, else 32-bit (ent32).  Indices >= D point at zero slots.
    int64_t* blk_off = nullptr;      // [groups]
    int32_t* blk_cnt = nullptr;      // [groups]
    uint16_t* ent16 = nullptr;
    uint32_t* ent32 = nullptr;
    // per-state hop list with the +1 targets first, then the -1 targets:
    // targets of state r at pn_list[pn_ptr[r] .. pn_ptr[r+1]), the first
    // pn_npos[r] of them with sign +1 (used where the list is warp-uniform)
    int32_t* pn_ptr = nullptr;       // [D+1]
    int32_t* pn_npos = nullptr;      // [D]
    uint32_t* pn_list = nullptr;     // [nnz]
};

}  // namespace hub

namespace hub {
// Host and device tables of one spin species, shared by every handle with the
// same device, lattice and particle number (read-only once uploaded; the
// device arrays are freed with the last owner).
struct SpinEntry;
// Device staging and streams of hubbard_apply_host (allocated on first use).
struct HostPipe;
}

struct hubbard_sector {
    int device = 0;
    int ns = 0, nup = 0, ndn = 0;
    double t = 0.0, U = 0.0;
    std::vector<std::pair<int, int>> bonds;
    hub::SpinTables host[2];                   // copies of the shared host tables
    hub::DevSpin dev[2];                       // device pointers owned by spin_owner
    std::shared_ptr<hub::SpinEntry> spin_owner[2];
    int64_t Dup = 0, Ddn = 0, D = 0;
    // fixed-point scratch for the F64 fast path, allocated on first use
    void* fx_scratch = nullptr;
    size_t fx_bytes = 0;
    // two-phase H*v schedule (0 = automatic; hubbard_set_schedule): rows per
    // row-phase block, up-phase columns per lane, row-phase CTAs per SM
    // (ctas_cols is accepted and reserved)
    int vec_rows = 0, vec_cols = 0, ctas_rows = 0, ctas_cols = 0;
    int fixed_emax_host = 1023;      // host copy for the device word used by the fixed-scale fallback
    // small device scratch for reductions: partial sums, status words
    double* red = nullptr;           // [kRedSlots]
    int* status = nullptr;           // [4]
    // device-resident Lanczos control (LzDev) and a/b history for lz_cap steps
    void* lz = nullptr;
    int lz_cap = 0;
    // stream of the handle's own allocations (nullptr: cudaMalloc / cudaFree;
    // set by sector_create_streamed for handles that live on one stream)
    cudaStream_t mem_stream = nullptr;
    // hubbard_apply_host: two slots of device staging, three streams
    hub::HostPipe* host_pipe = nullptr;
};

namespace hub {
constexpr int kRedSlots = 4096;      // partial-sum slots for block reductions
constexpr int kRedBlocks = 1024;     // grid size of reduction kernels (<= kRedSlots/2)
constexpr int kPartStride = 1024;    // stride of the partial arrays of a fused three-value reduction

// process-wide count of kernel launches (hubbard_kernel_launches)
void count_launches(int n);

// Handles and batches whose allocations live on one stream (server lanes):
// created like hubbard_sector_create / hubbard_batch_create, released without
// a device-wide synchronisation (the caller's later work on that stream is
// ordered after the frees; work on other streams is not waited for).
int sector_create_streamed(int Ns, const int32_t* bonds, int n_bonds, int Nup, int Ndn, double t, double U,
                           cudaStream_t ms, hubbard_t* out);
int batch_create_streamed(const hubbard_sector_desc* sectors, int n_sectors, cudaStream_t ms, hubbard_batch_t* out);

// Device-resident control of a Lanczos run (Algorithm 1 steps enqueued without
// a host round trip): the scalars the next step's kernels read, written by the
// one-CTA kernels that close each step (k_lz_finish, k_lz_finish2).
struct LzDev {
    double beta;      // b_j: coefficient of w_old (= f_{j-1}) in the next H*v
    double ua, uinv;  // the next row phase's deferred update f <- (f + ua fo) * uinv
    double a;         // a_j of the step in progress
    int j;            // steps closed so far (index of the step in progress)
    int fused;        // the step in progress took beta^2 from the fused sums
    int pad[2];
};

// A Lanczos vector update deferred into the next H*v (Algorithm 1, the
// normalisation of the new vector): before v is used, every element becomes
// v <- (v + a fo) * inv, rounded as launch_axpy_scale (one fused multiply-add,
// then one multiplication), and is written back to v.  The row phase applies
// it while staging rows, which saves the separate pass over three vectors.
// dv != nullptr: a and inv are read on the device from dv->ua, dv->uinv.
struct RowUpdate {
    const void* fo;
    double a, inv;
    const LzDev* dv = nullptr;
};

// kernels.cu launchers -------------------------------------------------------
int launch_hv_reference(const hubbard_sector* H, const void* v, void* w, int dtype, cudaStream_t s);
// part != nullptr: also reduce <w, v>, <w, w> and <v, v> into
// part[kRedSlots-1], part[kRedSlots-2], part[kRedSlots-3] (fused Lanczos
// reductions); *fused tells whether that happened (the kernel path in use may
// not support it).
// upd != nullptr: v is first updated in place as RowUpdate describes.
// dv != nullptr (device-resident step): beta is read on the device from
// dv->beta, and the fused sums are closed by k_lz_finish into dv and the
// history arrays ha, hb (requires part).
int launch_hv_fast(hubbard_sector* H, const void* v, void* w, int dtype, double beta,
                   const void* w_old, int fixed_emax, cudaStream_t s, double* part = nullptr,
                   bool* fused = nullptr, const RowUpdate* upd = nullptr, LzDev* dv = nullptr,
                   double* ha = nullptr, double* hb = nullptr);
// hv_phases.cu: two-phase shared-memory H*v; -1 when the staging buffers do not fit.
// fixed_emax > 0 fixes the fixed-point exponent bound (vectors of norm <= 1:
// 1023); otherwise it is computed from v and w_old.
// part != nullptr: the up phase writes per-CTA partials of <w, v>, <w, w> and
// <v, v> at part[b], part[kPartStride + b], part[2 kPartStride + b];
// *nparts = their count (<= kPartStride).
// upd != nullptr: v is first updated in place (fused into the row phase where
// it stages rows in shared memory); -1 is returned before anything is launched.
int launch_hv_phases(hubbard_sector* H, const void* v, void* w, int dtype, double beta, const void* w_old,
                     void* ybuf, int fixed_emax, cudaStream_t s, double* part = nullptr, int* nparts = nullptr,
                     const RowUpdate* upd = nullptr, const LzDev* dv = nullptr);
// whether launch_hv_phases fuses the Lanczos reductions for this sector and dtype
bool hv_phases_fuse(const hubbard_sector* H, int dtype);
// whether a fused launch_hv_phases call with a fixed exponent bound enqueues
// only kernels (no host-memory copies), so a CUDA graph can capture it
bool hv_phases_capturable(const hubbard_sector* H, int dtype);
// max biased binary64 exponent of |v| folded into *emax (atomicMax; caller zeroes it)
void launch_max_exponent(const double* v, int64_t n, int* emax, cudaStream_t s);
// binary64 -> (lo, hi) fixed point with the exponent bound *emax (read on the device)
void launch_to_fixed(const double* v, int64_t n, void* X, const int* emax, cudaStream_t s);
int launch_dot(const hubbard_sector* H, const void* x, const void* y, int64_t n, int dtype,
               double* partials, cudaStream_t s);
int reduce_partials_host(double* partials, cudaStream_t s, double* out);
// the three sums of a fused reduction: out[k] = part[kRedSlots-1-k]
int reduce_partials3_host(double* partials, cudaStream_t s, double out[3]);
// y <- (y + a x) * inv, rounded as launch_axpy_nrm2 followed by launch_scale
// (dv != nullptr: a and inv read on the device from dv->ua, dv->uinv)
int launch_axpy_scale(double a, double inv, const void* x, void* y, int64_t n, int dtype, cudaStream_t s,
                      const LzDev* dv = nullptr);
// the explicit branch of a device-resident step: when dv->fused is 0,
// y <- y - dv->a x with partial sums of y^2 in partials, then k_lz_finish2
// sums them and closes the step (no-ops when the step was closed fused)
int launch_lz_explicit(LzDev* dv, const void* x, void* y, int64_t n, int dtype, double* partials, double* hb,
                       cudaStream_t s);
// k_lz_finish: the fused sums of an up phase (np per-CTA partials) closed into dv, ha, hb
int launch_lz_finish(double* part, int np, LzDev* dv, double* ha, double* hb, cudaStream_t s);
int launch_axpy(double a, const void* x, void* y, int64_t n, int dtype, cudaStream_t s);
int launch_axpy_nrm2(double a, const void* x, void* y, int64_t n, int dtype, double* partials,
                     cudaStream_t s);
int launch_scale(double a, void* y, int64_t n, int dtype, cudaStream_t s);
int launch_copy_normalise(const void* x, void* y, int64_t n, int dtype, double inv_norm, cudaStream_t s);
int launch_f64_to_f32_scaled(const double* x, float* y, int64_t n, double a, cudaStream_t s);
int launch_fill_splitmix(void* v, int64_t n, unsigned long long seed, int64_t start, int dtype, cudaStream_t s);
int launch_psi_accumulate(const float* f, double* psi, int64_t n, double sj, bool init, cudaStream_t s);
int launch_psi_accumulate_f64(const double* f, double* psi, int64_t n, double sj, bool init, cudaStream_t s);
// psi = sum_{j<m} s_j f_j, f_j = base + j * stride (binary32), s on the device;
// bit-identical to m successive launch_psi_accumulate calls
int launch_psi_multi(const float* base, int64_t stride, int m, const double* s_dev, double* psi, int64_t n,
                     cudaStream_t s);

// A <- A + ca f, B <- B + cb f (binary64)
int launch_acc2_f64(const double* f, double* A, double* B, int64_t n, double ca, double cb, cudaStream_t s);
// A <- A + sum_{j<m} c_j f_j, B <- B + sum_{j<m} c_{m+j} f_j, f_j = base + j * stride
// (binary64), c on the device; bit-identical to m successive launch_acc2_f64 calls
int launch_combine2_f64(const double* base, int64_t stride, int m, const double* c_dev, double* A, double* B,
                        int64_t n, cudaStream_t s);

// krylov.cpp ------------------------------------------------------------------
// Eigenvalues lam[0..m) of the symmetric tridiagonal T (diag a, off-diag
// b[0..m-2]) by implicit-shift QR, and rows rows[0..zrows) of its eigenvector
// matrix: Z[r * m + k] = component rows[r] of the eigenvector of lam[k].
// false if the iteration does not converge.
bool tridiag_eigen(const double* a, const double* b, int m, double* lam, double* Z, int zrows, const int* rows);
// eigenvalues and the first and last rows of the eigenvector matrix of T_m,
// from which |e_m^T exp(-i T_m tau) e_1| is evaluated at any tau in O(m)
struct KrylovEnds {
    int m = 0;
    std::vector<double> lam, z0, zl;
};
bool krylov_exp_ends(const double* a, const double* b, int m, KrylovEnds& out);
double krylov_last_coeff(const KrylovEnds& K, double tau);
// y = exp(-i T_m tau) e_1 (real and imaginary parts, m each)
bool krylov_exp_coeffs(const double* a, const double* b, int m, double tau, double* yre, double* yim);

// tridiag.cpp -----------------------------------------------------------------
// Lowest eigenvalue of the symmetric tridiagonal T (diag a[0..m-1], off-diag
// b[0..m-2]) and the last component of its normalised eigenvector.
void tridiag_lowest(const double* a, const double* b, int m, double* theta, double* s_last);
// the whole normalised lowest eigenvector s[0..m)
void tridiag_lowest_vector(const double* a, const double* b, int m, double* theta, double* s);
// k-th smallest eigenvalue (k = 0 is the lowest)
double tridiag_kth(const double* a, const double* b, int m, int k);
// Lower estimate of the gap lambda_2 - theta from the Lanczos tridiagonal
// T_m (b_next = b_{m+1}): (theta_2 - rho_2) - theta, with theta_2 the lowest
// Ritz value above theta that is not a copy of it and rho_2 = b_{m+1} |s_m|
// its residual estimate.  Valid when no eigenvalue of H other than the one
// near theta lies below theta_2 - rho_2.  <= 0 when T_m resolves no gap.
double tridiag_gap_lower(const double* a, const double* b, int m, double b_next, double theta);
// a-posteriori bound on |theta - E0| from a residual norm rho and a gap lower
// estimate: min(rho, rho^2 / (gap / kGapSafety)) when gap > 0 (Temple-type),
// else rho.  The gap comes from Lanczos Ritz pairs, which can place the
// eigenvalue they resolve above lambda_2 when lambda_2 itself is not yet
// resolved (a 2.2x overestimate was seen in a serving trace), so only a tenth
// of it is trusted.
constexpr double kGapSafety = 10.0;
inline double energy_error_bound(double rho, double gap) {
    if (gap > 0.0) return std::min(rho, rho * rho * kGapSafety / gap);
    return rho;
}
// floor of the computed energy's rounding error: hops of one H*v element
// (hops_plus_one = W_up + W_dn + 1, or any upper bound of it) times the unit
// of the H*v arithmetic (2^-47: the binary64 path rounds unit vectors to that
// fixed-point grid; 2^-24: binary32) times scale = max(1, max|a_j|, max b_j)
// (a bound on |H| restricted to the Krylov space)
inline double rounding_floor(int hops_plus_one, int dtype, double scale) {
    return (double)hops_plus_one * (dtype == HUB_F64 ? 0x1p-47 : 0x1p-24) * scale;
}
inline double tridiag_scale(const double* a, const double* b, int m) {
    double s = 1.0;
    for (int i = 0; i < m; ++i) s = std::max(s, std::max(std::fabs(a[i]), std::fabs(b[i])));
    return s;
}

}  // namespace hub
