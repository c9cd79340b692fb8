/* hubbard.h - C ABI of the GB300 Hubbard exact-diagonalization hot path.
 *
 * Method: T. Siro and A. Harju, "Exact diagonalization of the Hubbard model
 * on graphics processing units" (arXiv:1204.3425).  The library computes,
 * in one fixed (N_up, N_dn) sector of
 *
 *     H = -t sum_<ij> sum_sigma (c+_{i sigma} c_{j sigma} + h.c.)
 *         + U sum_i n_{i up} n_{i dn}                              (Eq. 1)
 *
 * the product w = H v and the Lanczos ground state (Sec. 2.2, Algorithm 1).
 *
 * Conventions (Sec. 2.1):
 *   - a spin configuration is an Ns-bit word, bit i set <=> site i occupied;
 *   - i_sigma is the position of that word in the ascending list of Ns-bit
 *     words with N_sigma bits set; the vector index is
 *         J = i_up * D_dn + i_dn,   D_sigma = C(Ns, N_sigma)  (Eq. J-formula)
 *     so a vector is a row-major D_up x D_dn matrix (the "subvectors" of
 *     Fig. 2 are its rows);
 *   - basis states put all up creators left of all down creators, sites in
 *     ascending order; a hop of a spin-sigma electron picks up (-1) per
 *     same-spin electron on sites strictly between origin and destination.
 *
 * General rules for every call:
 *   - Return value: HUB_OK (0) or a positive hub_status code; a message is
 *     then available from hubbard_last_error() (thread-local).  No call
 *     aborts the process or throws across the ABI.
 *   - Device pointers are plain CUDA device addresses on the current device,
 *     owned by the caller unless stated.  They must be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return only device results are asynchronous on
 *     that stream; calls that return host results synchronise the stream.
 *   - dtype: HUB_F64 (IEEE binary64 vectors) or HUB_F32 (binary32 vectors).
 *     The F64 path keeps binary64 storage but accumulates hop sums in exact
 *     integer fixed point (see hubbard_apply).
 */
#ifndef HUBBARD_H
#define HUBBARD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hubbard_sector* hubbard_t;

typedef enum {
    HUB_OK = 0,
    HUB_EINVAL = 1,    /* invalid argument (sizes, pointers, alignment, ranges)   */
    HUB_ENOMEM = 2,    /* device or host allocation failed, or workspace too small */
    HUB_ECUDA = 3,     /* a CUDA runtime call failed                               */
    HUB_ENOTCONV = 4,  /* Lanczos hit max_iters before the residual test passed    */
    HUB_ETIMEOUT = 5,  /* a bounded device wait gave up                            */
    HUB_EDEVICE = 6,   /* a kernel reported an error through its status word       */
    HUB_EPENDING = 7   /* hubbard_server_poll: the request has not finished yet    */
} hub_status;

typedef enum { HUB_F64 = 0, HUB_F32 = 1 } hub_dtype;

/* ---------------------------------------------------------------------------
 * Sector handle (Sec. 2.1 basis and ranking; Sec. 4.2 Kronecker split).
 *
 * hubbard_sector_create builds, on the host, the ascending basis of each spin
 * (Eq. J-formula) and the per-spin hopping tables of H_up and H_dn
 * (Eq. H-Kroneckersum): for every rank r and every bond with exactly one end
 * occupied, the target rank r' and the Jordan-Wigner sign of Sec. 2.1.  It
 * copies them to the current device and returns an opaque handle.  The
 * tables of one spin depend only on (device, Ns, bonds, N): handles with the
 * same ones share a single read-only device copy (also between the two spins
 * when Nup = Ndn), and the library keeps the 256 most recently built table
 * sets after their last handle is gone, so re-creating a sector skips the
 * build.  Each handle has its own t, U, schedule and scratch.
 *   Ns      number of sites, 1..32
 *   bonds   host array of 2*n_bonds int32: (i0, j0, i1, j1, ...), 0 <= i,j < Ns,
 *           i != j, no unordered pair repeated.  n_bonds may be 0.
 *   Nup,Ndn 0..Ns electrons of each spin
 *   t, U    finite hopping amplitude and on-site interaction of Eq. (1)
 *   out     receives the handle (NULL on failure)
 * Errors: HUB_EINVAL for any violated rule above or D_sigma > 2^30 (never
 * binding: with Ns <= 32, D_sigma <= C(32, 16) = 601080390 < 2^30);
 *         HUB_ENOMEM / HUB_ECUDA on allocation or copy failure.
 * The handle is tied to the device that was current at creation; every later
 * call must run with that device current.  Not thread-safe per handle.
 * ------------------------------------------------------------------------- */
int hubbard_sector_create(int Ns, const int32_t* bonds, int n_bonds, int Nup, int Ndn,
                          double t, double U, hubbard_t* out);

/* Releases the handle (synchronising the device first): its scratch is freed,
 * and its tables when no other handle or the recent-table cache holds them.
 * NULL is a no-op. */
void hubbard_sector_destroy(hubbard_t H);

/* Dimensions D_up, D_dn and maximum hops per state W_up, W_dn (any may be NULL). */
int hubbard_sector_info(hubbard_t H, int64_t* D_up, int64_t* D_dn, int32_t* W_up, int32_t* W_dn);

/* Number of stored (target, sign) entries of H_sigma (spin 0 = up, 1 = down). */
int64_t hubbard_table_nnz(hubbard_t H, int spin);

/* Canonical host copy of one spin's basis and hopping table, for bit-exact
 * comparison (Sec. 2.1 matrix elements).  Host buffers, caller-owned:
 *   states[D_sigma]      ascending basis words
 *   rowptr[D_sigma + 1]  CSR row pointers
 *   tgt[nnz], sign[nnz]  for row r, every r' with <r'|H_sigma|r> = -t*sign != 0,
 *                        sorted by r'
 * Any pointer may be NULL to skip that array. */
int hubbard_export_tables(hubbard_t H, int spin, uint32_t* states, int32_t* rowptr,
                          int32_t* tgt, int8_t* sign);

/* Host-only variant of the per-spin table build (no device needed), for
 * testing the basis and sign tables on machines without a GPU.  Call once
 * with states/rowptr/tgt/sign all NULL to get *D and *nnz, then again with
 * host buffers of those sizes.  Same argument rules as hubbard_sector_create
 * for Ns, bonds and N. */
int hubbard_host_spin_tables(int Ns, const int32_t* bonds, int n_bonds, int N, int64_t* D, int64_t* nnz,
                             uint32_t* states, int32_t* rowptr, int32_t* tgt, int8_t* sign);

/* Host-only copy of the row-phase hop table of one spin (the layout the
 * down-hop gathers of hubbard_apply and of the batched solver walk; Sec. 4.3
 * restated for shared-memory staging), for testing its invariants without a
 * GPU.  States are taken in groups of 32 (group g = states 32g .. 32g+31, one
 * per lane).  Group g holds bcnt[g] half-blocks of 4 slots per lane starting at
 * entry boff[g]: bcnt[g] / 2 blocks of 8 slots (slot s < 8 * (bcnt[g] / 2) of
 * lane l at boff[g] + ((s / 8) * 32 + l) * 8 + s % 8), then, when bcnt[g] is
 * odd, one block of 4 (slot s of lane l at boff[g] + (bcnt[g] / 2) * 256 +
 * l * 4 + s - 8 * (bcnt[g] / 2)).  Entry = staged slot index in the low 15 bits
 * (narrow) or 31 bits, sign -1 in the bit above; the hops of a state are its
 * entries with index < D, the others point at zero slots (index >= D rounded
 * up to 32).  Slots are coloured for staged elements of elem_bytes (4, 8 or 16)
 * bytes: within every wavefront phase (min(32, 128 / elem_bytes) lanes) the
 * entries of one slot have distinct index mod 128 / elem_bytes (bank group).
 * Call once with boff/bcnt/ent NULL to get *groups and *entries, then with
 * host buffers of those sizes.  Same argument rules as hubbard_host_spin_tables. */
int hubbard_host_row_table(int Ns, const int32_t* bonds, int n_bonds, int N, int elem_bytes, int64_t* groups,
                           int64_t* entries, int* narrow, int64_t* boff, int32_t* bcnt, uint32_t* ent);

/* ---------------------------------------------------------------------------
 * w = H v  (Sec. 4.3: the fused up-hop, down-hop and interaction kernel,
 * Algorithms 2-4, restated for sm_103a).
 *   v, w   device vectors of D = D_up*D_dn elements of `dtype`, row-major
 *          D_up x D_dn (Fig. 2), 16-byte aligned, w must not overlap v.
 * HUB_F64: the hop sums are exact integer sums of the elements of v rounded
 * to a common fixed-point grid of 2^-48 * 2^ceil(log2 max|v|); the result is
 * within 1e-12 * |t| * max|v| of the exact product (max-abs).  This path uses
 * a device workspace owned by the handle, allocated on first use (the first
 * call may therefore allocate; later calls do not).
 * HUB_F32: binary32 arithmetic throughout.
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int hubbard_apply(hubbard_t H, const void* v, void* w, int dtype, void* stream);

/* w_host = H v_host with both vectors in host memory (same product and
 * accuracy as hubbard_apply).  The call copies v_host to device staging owned
 * by the handle, applies H, and copies the result back into w_host, on three
 * streams of the handle, with two staging slots: consecutive calls overlap
 * (the upload of call i+1 and the download of call i-1 run during the H*v of
 * call i) when the host buffers are page-locked; with pageable buffers the
 * copies are synchronous.  Returns once the work is enqueued; `stream` waits
 * for the download, so w_host holds the result once `stream` has reached this
 * call.  The upload is not ordered after earlier work on `stream`: v_host must
 * hold the input when the call is made and stay unchanged, and w_host must not
 * be read or written, until `stream` has reached the call.  The first call,
 * and a call with another dtype, allocates 4 * D elements of staging (freed
 * with the handle).  Calls on one handle, of this and the other functions,
 * must not run concurrently (they share the handle's scratch).  HUB_EINVAL:
 * null or overlapping vectors, a device pointer, a bad dtype, a handle from
 * hubbard_server's lanes; HUB_ECUDA on a CUDA error. */
int hubbard_apply_host(hubbard_t H, const void* v_host, void* w_host, int dtype, void* stream);

/* Same as hubbard_apply, reference kernel: one thread per element and native
 * arithmetic of `dtype` (binary64 DADD/DFMA for HUB_F64), the paper's own
 * kernel organisation (Sec. 4.3, Algorithms 2-4: each thread gathers its
 * element's up- and down-hops and adds the interaction), no workspace.
 * Kept as the parity anchor for the fast path. */
int hubbard_apply_reference(hubbard_t H, const void* v, void* w, int dtype, void* stream);

/* Launch schedule of the two-phase H*v for this handle (the hook an
 * autotuner drives; Sec. 4.3 reports the paper's own tuning knob, several
 * elements per thread).  vec_rows: rows of V staged per row-phase block;
 * vec_cols: columns per lane in the up phase (each 0 = automatic, else 1, 2
 * or 4; binary64 uses at most 2, and a width the row length does not divide
 * is narrowed); ctas_rows: row-phase CTAs per SM (0 = automatic, 1 or 2);
 * ctas_cols: binary64 up phase of a standalone H*v (0 = automatic; 1 = 4 CTAs
 * per SM, epilogue operands loaded after the hop sum; 2 = 3 CTAs per SM, the
 * own element and row-phase sum requested before it).  A choice whose buffers
 * do not fit in shared memory falls back to the largest one that does.
 * Results do not depend on the schedule: every output sums its hops in one
 * fixed order (binary32) or exactly (binary64 fixed point). */
int hubbard_set_schedule(hubbard_t H, int vec_rows, int vec_cols, int ctas_rows, int ctas_cols);

/* Autotuner for the schedule above (the paper tunes elements per thread by
 * hand, Sec. 4.3): times three hubbard_apply calls (after a
 * warm one) for every vec_rows x vec_cols in {1, 2 (, 4 for binary32)},
 * ctas_rows in {1, 2} and (binary64) ctas_cols in {1, 2} on the caller's v, w
 * (device, dtype, as hubbard_apply;
 * w is overwritten), keeps the fastest on the handle and writes it to
 * chosen[4] = {vec_rows, vec_cols, ctas_rows, ctas_cols} (nullable).
 * Synchronises `stream`.  On error the previous schedule is kept. */
int hubbard_autotune_schedule(hubbard_t H, const void* v, void* w, int dtype, void* stream, int* chosen);

/* ---------------------------------------------------------------------------
 * Binary64 w = H v that allocates no device memory.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc at the point where they need H*v: code that runs
 * while another framework owns the device allocator, code under a hard
 * memory budget, or hot loops that must never reach the allocator.  Such a
 * caller creates the handle beforehand (hubbard_sector_create allocates the
 * tables) and then calls this function with its own v and w.
 *
 * It runs the binary64 fixed-point kernels of hubbard_apply, but its scratch
 * (the fixed-point copy of v and one exponent word) lives in a file-scope
 * device array of HUBBARD_NOALLOC_MAX_ELEMS * 8 bytes (16 MiB) that every
 * GPU loading the library holds until process exit.
 *   - D_up * D_dn above HUBBARD_NOALLOC_MAX_ELEMS: HUB_EINVAL, nothing runs.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address with cudaGetSymbolAddress; make that first call
 *     before any stream capture.
 *   - Every call, from any thread or stream, shares the one array and leaves
 *     its contents behind; calls whose GPU work overlaps (concurrent streams
 *     or threads) race on it and must be serialised by the caller.
 *   - Sectors with more than 127 hops per state (W_up + W_dn > 127) take the
 *     native binary64 kernel of hubbard_apply_reference, which needs no
 *     scratch; every other sector takes the fixed-point kernels.
 * Same accuracy and argument rules as hubbard_apply with HUB_F64.
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
#define HUBBARD_NOALLOC_MAX_ELEMS (1 << 21)
int hubbard_apply_noalloc(hubbard_t H, const void* v, void* w, void* stream);

/* ---------------------------------------------------------------------------
 * Lanczos vector operations (the dot product, norm and update of
 * Algorithm 1), n elements of dtype, results accumulated in binary64 in a
 * fixed reduction order (deterministic for a given n and dtype).  Device
 * vectors; host scalar results; dot and nrm2 synchronise `stream`.
 * ------------------------------------------------------------------------- */
int hubbard_vec_dot(const void* x, const void* y, int64_t n, int dtype, void* stream, double* out);
int hubbard_vec_nrm2(const void* x, int64_t n, int dtype, void* stream, double* out);
/* y <- y + a*x  (asynchronous) */
int hubbard_vec_axpy(double a, const void* x, void* y, int64_t n, int dtype, void* stream);

/* Seeded start vector on the device (the paper asks for a random start
 * vector, Algorithm 1): v[i] = 2 x - 1 with x the top 53 bits of SplitMix64
 * (Steele, Lea, Flood 2014) at counter seed * 2^40 + start + i, divided by
 * 2^53; binary32 rounds the binary64 value.  Asynchronous. */
int hubbard_fill_start_vector(void* v, int64_t n, uint64_t seed, int64_t start, int dtype, void* stream);

/* ---------------------------------------------------------------------------
 * One step of Algorithm 1 in the two-vector form of Eqs. (split1):
 *   g <- H f - beta_j g;  alpha_j = g.f;  g <- g - alpha_j f;
 *   beta_{j+1} = |g|;  g <- g / beta_{j+1}  (skipped when beta_{j+1} == 0)
 * f must have norm 1.  f, g device vectors of D elements.  Writes alpha_j
 * and beta_{j+1} to *alpha, *beta_next (host).  Synchronises `stream`.
 * The H*v kernels also reduce g.f, g.g and f.f, so beta_{j+1}^2 =
 * g.g - 2 alpha_j^2 + alpha_j^2 f.f without another pass; when that
 * difference cancels more than six digits of g.g, |g - alpha_j f| is formed
 * explicitly.  The update rounds as an axpy followed by a scale.
 * ------------------------------------------------------------------------- */
int hubbard_lanczos_step(hubbard_t H, const void* f, void* g, double beta_j, int dtype,
                         void* stream, double* alpha, double* beta_next);

/* ---------------------------------------------------------------------------
 * Lanczos ground state (Sec. 2.2, Algorithm 1, two-vector form).
 *   v0         device start vector of D elements (dtype); normalised inside,
 *              not modified
 *   max_iters  >= 1; the iteration count is also capped at D
 *   tol        stop when rho = beta_{m+1} * |s_m| < tol (s = lowest
 *              eigenvector of the tridiagonal T_m); tol <= 0 runs exactly
 *              max_iters steps (or to breakdown)
 *   workspace  device buffer of at least lanczos_workspace_bytes(H, dtype)
 *              bytes, caller-owned, 256-byte aligned
 *   psi_out    optional binary64 device vector of D elements (16-byte
 *              aligned, not overlapping the workspace) receiving the
 *              normalised Ritz vector psi = sum_j s_j f_j of the lowest Ritz
 *              value.  The Lanczos vectors are not stored: a second pass
 *              replays the same recurrence with the recorded a_j, b_j (the
 *              kernels are deterministic, so the replayed f_j are the ones of
 *              the first pass) and accumulates psi in binary64, which doubles
 *              the H*v count.  NULL skips it.
 *   alpha_out, beta_out  optional host arrays of max_iters doubles receiving
 *              a_1..a_m and b_2..b_{m+1}
 *   out        host result: energy (lowest Ritz value), residual rho,
 *              err_bound, iters, status, breakdown flag
 * err_bound is the a-posteriori bound min(rho, 10 rho^2 / gap) on
 * |energy - E0|, gap = (theta_2 - rho_2) - energy from the second distinct
 * Ritz pair of T_m (theta_2, residual estimate rho_2); when T_m resolves no
 * positive gap it is rho.  The quadratic form assumes that no eigenvalue of H
 * other than E0 (counted once if degenerate) lies below a tenth of that gap
 * above E0: the estimate is not rigorous (a Ritz pair can resolve an
 * eigenvalue above an unresolved lambda_2), hence the factor 10.  A rounding floor
 * (W_up + W_dn + 1) u max(1, max|a_j|, max b_j) is added, u = 2^-47 for
 * HUB_F64 (the fixed-point grid of unit vectors) and 2^-24 for HUB_F32.
 * Breakdown (beta_{m+1} <= 1e-13 * max(1, max|a|, max b)) counts as
 * converged.  Returns HUB_ENOTCONV (with the best energy in *out) when
 * max_iters is reached with tol > 0 and rho >= tol.  Synchronises `stream`.
 * Each new vector f_{j+1} = (g - a_j f_j) / b_{j+1} is completed by the next
 * step's H*v while it stages its rows (same roundings as the separate update
 * of hubbard_lanczos_step), so the workspace holds no finished vector on return.
 * ------------------------------------------------------------------------- */
typedef struct {
    double energy;
    double residual;
    double err_bound;
    int32_t iters;
    int32_t status;
    int32_t breakdown;
    int32_t reserved;
} lanczos_result;

size_t lanczos_workspace_bytes(hubbard_t H, int dtype);

int lanczos_ground_state(hubbard_t H, const void* v0, int max_iters, double tol, int dtype,
                         void* workspace, size_t ws_bytes, void* psi_out, void* stream,
                         double* alpha_out, double* beta_out, lanczos_result* out);

/* Number of kernels this library has launched in this process (all threads,
 * all devices) - instrumentation for benchmarks and tests. */
uint64_t hubbard_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Ground state in binary32 with binary64 refinement (Sec. 2.2, Algorithm 1,
 * run in binary32; the paper benchmarks both precisions, Sec. 5).
 *   1. binary32 Lanczos (H*v and vectors binary32; a_j, b_j reductions
 *      accumulated in float-float, ~48 bits) until rho < 2e-6 max(1,|theta|);
 *   2. Ritz vector psi = sum_j s_j f_j accumulated in binary64: from the f_j
 *      stored in the workspace's spare room, and past the last stored one
 *      by replaying the same binary32 recurrence with the stored a_j, b_j
 *      (bit-identical f_j, so psi is the same however many were stored);
 *   3. binary64 Rayleigh quotient theta = <psi|H|psi> and residual
 *      |H psi - theta psi| with the binary64 H*v;
 *   4. if the error bound below exceeds tol max(1,|theta|): a short binary64
 *      Lanczos run started from psi (at most 150 steps).
 *   v0          binary64 device start vector (normalised inside)
 *   workspace   >= lanczos_refined_workspace_bytes(H) bytes (40 D), 256-aligned;
 *               every further 4 D bytes (rounded up to 256) stores one more
 *               binary32 Lanczos vector, i.e. saves one replayed step
 *   psi_out     optional binary64 device vector receiving the normalised psi
 *               of step 2
 *   out         energy (binary64 Rayleigh quotient or polished Ritz value),
 *               residual (|H psi - theta psi| in binary64, or the polish's
 *               Ritz residual estimate), error_bound, binary32 energy, gap,
 *               iteration counts, status
 * gap is a lower estimate of lambda_2 - E0 from the binary32 run:
 * (theta_2 - rho_2) - theta with theta_2 its second distinct Ritz value and
 * rho_2 that Ritz pair's residual estimate (a Ritz value alone only bounds
 * lambda_2 from above).  error_bound = min(residual, 10 residual^2 / gap), or
 * the residual when gap <= 0, plus the binary64 rounding floor of
 * lanczos_ground_state; the quadratic form assumes no eigenvalue other than
 * E0 lies within a tenth of gap above it.  The polish runs until
 * error_bound <= tol * max(1, |energy|) / 2 (at most 150 binary64 steps);
 * status is HUB_OK exactly when error_bound <= tol * max(1, |energy|).
 * Returns HUB_ENOTCONV otherwise.  Synchronises stream.
 * ------------------------------------------------------------------------- */
typedef struct {
    double energy;
    double residual;
    double error_bound;
    double energy_f32;
    double gap;
    int32_t iters_f32;
    int32_t iters_f64;
    int32_t status;
    int32_t replayed;          /* Lanczos steps replayed for psi (0: all vectors were stored) */
} lanczos_refined_result;

size_t lanczos_refined_workspace_bytes(hubbard_t H);

int lanczos_ground_state_refined(hubbard_t H, const void* v0, int max_iters, double tol, void* workspace,
                                 size_t ws_bytes, void* psi_out, void* stream, lanczos_refined_result* out);

/* ---------------------------------------------------------------------------
 * Time propagation psi(t) = exp(-i H t) v (the other use of the H*v kernel
 * the paper names, Sec. 6; the paper gives no scheme).  Short iterative
 * Lanczos: from a real start p the Lanczos vectors f_j of Algorithm 1 (the
 * binary64 H*v and step kernels of lanczos_ground_state) give
 *   exp(-i H tau) p ~ |p| sum_{j<m} y_j f_j,   y = exp(-i T_m tau) e_1,
 * with T_m the Lanczos tridiagonal (Eq. Tmatrix; its eigendecomposition by
 * implicit-shift QR on the host) and the a-posteriori error estimate
 *   est(tau) = |p| b_{m+1} |y_{m-1}|.
 * A complex v = v_re + i v_im is propagated as its two real parts (H is real).
 * Steps: the Lanczos run of each real part stops once est(remaining time) is
 * within its share of tol * |v| * remaining / |t| (checked every 4 steps), or
 * at krylov_max steps; then the step tau is the longest that meets that
 * budget for both parts (bisection), the state becomes exp(-i H tau) v, and
 * the loop repeats until |t| is used up.  The summed estimates are therefore
 * about tol * |v|; the estimate is not a proven bound.
 *   v_re, v_im  binary64 device vectors of D elements (v_im may be NULL: a
 *               real v), 16-byte aligned, not inside the workspace
 *   t           propagation time (any sign; 0 copies v)
 *   krylov_max  1 .. 1024: Lanczos steps per propagation step at most
 *   tol         > 0: relative accuracy target, see above
 *   workspace   >= hubbard_evolve_workspace_bytes(H, krylov_max, 0) bytes
 *               (6 vectors: two Lanczos vectors, the H*v scratch, the current
 *               state), 256-aligned.  With hubbard_evolve_workspace_bytes(H,
 *               krylov_max, 1) bytes the Lanczos vectors of both real parts
 *               are stored and combined in one pass; with less, each part's
 *               recurrence is replayed to combine them (twice the H*v count,
 *               bit-identical result)
 *   out_re, out_im  binary64 device vectors receiving psi(t), 16-byte
 *               aligned, disjoint from each other and the workspace; they may
 *               alias v_re / v_im (v is copied into the workspace first)
 *   info        steps taken, H*v count, largest Krylov dimension, summed
 *               error estimates, |psi(t)|, status
 * Errors: HUB_EINVAL (arguments, non-finite t or tol, more than 127 hops per
 * state), HUB_ENOMEM (workspace too small), HUB_ENOTCONV (the tridiagonal QR
 * did not converge, or a step would have to be shorter than 1e-12 |t|:
 * tol too strict for krylov_max), HUB_ECUDA.  Synchronises stream.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t steps;             /* propagation steps (Krylov restarts + 1) */
    int32_t hv;                /* H*v applications, replays included */
    int32_t krylov_dim;        /* largest Lanczos run of any step */
    int32_t status;
    double err_estimate;       /* sum over steps and parts of est(tau) */
    double norm;               /* |psi(t)|_2 */
} hubbard_evolve_info;

size_t hubbard_evolve_workspace_bytes(hubbard_t H, int krylov_max, int store_basis);

int hubbard_time_evolve(hubbard_t H, const void* v_re, const void* v_im, double t, int krylov_max, double tol,
                        void* workspace, size_t ws_bytes, void* out_re, void* out_im, void* stream,
                        hubbard_evolve_info* info);

/* Host-only helper of hubbard_time_evolve, for testing without a GPU:
 * y = exp(-i T tau) e_1 for the m x m symmetric tridiagonal T with diagonal
 * a[0..m) and off-diagonal b[0..m-1) (y_re, y_im: m each).  m in 1..4096.
 * HUB_EINVAL for bad arguments or non-finite inputs, HUB_ENOTCONV if the QR
 * iteration does not converge. */
int hubbard_host_krylov_exp(const double* a, const double* b, int m, double tau, double* y_re, double* y_im);

/* ---------------------------------------------------------------------------
 * Many sectors solved in one persistent launch (Algorithm 1 for every
 * sector, entirely on the device; the paper notes that small sectors leave
 * the GPU idle, Sec. 5).  A batch owns the hopping tables of all its sectors
 * (tables are shared between sectors with the same lattice and filling).
 * One cooperative kernel solves the batch: sectors above elems_per_cta
 * elements (the schedule knob hubbard_batch_autotune chooses) advance in lock
 * step, every Lanczos step spread over the whole grid; the others are solved
 * by one CTA each, in shared memory when the vector fits (~14000 elements).
 * Results do not depend on which other sectors share the batch (fixed-order
 * reductions).
 * ------------------------------------------------------------------------- */
typedef struct hubbard_batch* hubbard_batch_t;

typedef struct {
    int32_t ns, nup, ndn, n_bonds;
    const int32_t* bonds;      /* host, 2 * n_bonds, same rules as hubbard_sector_create */
    double t, U;
} hubbard_sector_desc;

/* Builds and uploads the tables of n_sectors sectors (host descriptors). */
int hubbard_batch_create(const hubbard_sector_desc* sectors, int n_sectors, hubbard_batch_t* out);
void hubbard_batch_destroy(hubbard_batch_t B);

/* offsets[n_sectors + 1]: sector i's start vector occupies elements
 * offsets[i] .. offsets[i] + D_i of the concatenated binary64 v0 buffer
 * (offsets are even, so every sector is 16-byte aligned). */
int hubbard_batch_vector_offsets(hubbard_batch_t B, int64_t* offsets);

/* Device workspace bytes for hubbard_batch_solve_async with this max_iters. */
size_t hubbard_batch_workspace_bytes(hubbard_batch_t B, int max_iters);

/* Size threshold (>= 1): sectors of more than elems_per_cta elements are
 * solved by the whole grid in lock step, the others by one CTA each. */
int hubbard_batch_set_schedule(hubbard_batch_t B, int64_t elems_per_cta);

/* One launch solving every sector to rho < tol * max(1, |theta|) (or
 * breakdown, or max_iters capped at D).  v0_all: device, 16-byte aligned.
 * Asynchronous on `stream`; results stay in the workspace until
 * hubbard_batch_results.  The first call for a given max_iters / schedule
 * uploads descriptors synchronously; later calls only enqueue two memsets and
 * one cooperative launch, so they can be captured in a CUDA graph. */
int hubbard_batch_solve_async(hubbard_batch_t B, const double* v0_all, int max_iters, double tol, void* workspace,
                              size_t ws_bytes, void* stream);

/* Copies the per-sector results (host array of n_sectors); synchronises
 * `stream`.  err_bound is computed here on the host from each sector's a/b
 * history, as lanczos_ground_state defines it.  HUB_ETIMEOUT if a grid
 * barrier gave up. */
int hubbard_batch_results(hubbard_batch_t B, const void* workspace, int max_iters, void* stream,
                          lanczos_result* results);

/* Failure-path self-test (the paper has no counterpart): launches two CTAs
 * on the batch kernel's bounded grid barrier set to expect three, so the wait
 * cannot complete; each CTA gives up after 2000 polls (well under a
 * millisecond) and sets the error word.  Returns HUB_ETIMEOUT when the bound
 * and the error path work (the expected result), HUB_EDEVICE if the timeout
 * was not reported, HUB_ECUDA on a CUDA error.  Allocates 256 bytes of device
 * memory for the call; synchronises `stream`. */
int hubbard_selftest_wait_timeout(void* stream);

/* Autotuner of the batch's schedule (the paper tunes its kernels' shape by
 * measurement, Sec. 4.3).  First, per sector shape (D_up, D_dn, W = W_up +
 * W_dn) small enough to be a one-CTA task: up to one grid of that shape's
 * sectors is solved alone for 16 steps in each candidate mode --
 * the whole vector in shared memory when it fits, or warp-per-row passes over
 * the L2 copy with or without the row staged in shared memory for the
 * down-hops -- and the fastest (the default unless another is 3 % faster) is
 * kept in the batch's schedule table.  Then full solves for elems_per_cta in
 * {2^12 .. 2^17} pick the sweep/task threshold (written to *chosen), and
 * then the number of CTAs that start on the tasks while the rest sweep
 * (hubbard_batch_set_task_ctas; 0, 16, 32, 48 or 64).  The
 * table persists in the batch and is used by every later solve (including a
 * graph-captured one).  Each sector's arithmetic depends only on its own
 * shape's entry and on whether it is swept, so results stay independent of
 * the other sectors under a given table.  v0_all, workspace and ws_bytes as
 * for hubbard_batch_solve_async; the workspace's results are overwritten.
 * Synchronises `stream`. */
int hubbard_batch_autotune(hubbard_batch_t B, const double* v0_all, int max_iters, double tol, void* workspace,
                           size_t ws_bytes, void* stream, int64_t* chosen);

/* The schedule table, one row of six int64 per distinct sector shape, in
 * order of first appearance: {D_up, D_dn, W_up + W_dn, number of sectors of
 * that shape, path (1: one-CTA task, 2: grid-wide sweep, by the current
 * threshold), mode bits (1: a task keeps its whole vector in shared memory
 * when it fits; 2: warp-per-row passes stage the row in shared memory for the
 * down-hops; 3 is the default)}.  rows: host, 6 * cap int64 (may be NULL when
 * cap = 0); writes min(cap, shapes) rows and sets *n_shapes to the number of
 * shapes.  HUB_EINVAL on a null batch or n_shapes, or rows NULL with cap > 0. */
int hubbard_batch_schedule_table(hubbard_batch_t B, int64_t* rows, int cap, int* n_shapes);

/* Sets the mode bits (0 .. 3, as in the schedule table) of shape number
 * `shape` (its row in hubbard_batch_schedule_table), e.g. to pin a table
 * measured earlier; the next solve uploads the descriptors synchronously.
 * HUB_EINVAL on a null batch or an out-of-range shape or mode. */
int hubbard_batch_set_shape_mode(hubbard_batch_t B, int shape, int mode);

/* CTAs (0 by default) that start on the one-CTA tasks at once while the rest
 * of the grid runs the sweep (the sweep CTAs join the tasks when it ends);
 * capped at the number of tasks, and at half the grid.  A sector's arithmetic
 * does not depend on it.  HUB_EINVAL on a null batch or a negative count. */
int hubbard_batch_set_task_ctas(hubbard_batch_t B, int task_ctas);

/* The batch's current sweep/task threshold and task-CTA count (either
 * pointer may be NULL).  HUB_EINVAL on a null batch. */
int hubbard_batch_get_schedule(hubbard_batch_t B, int64_t* elems_per_cta, int* task_ctas);

/* ---------------------------------------------------------------------------
 * Queued solver: the batch kernel's one-CTA task path kept running while
 * sectors are posted (Algorithm 1 on the device for each sector, as in a
 * batch; the paper notes that small sectors leave the GPU idle, Sec. 5).  A
 * posted sector is taken by the next CTA of the running kernel that frees up,
 * so work joins the device while other sectors are being solved.  Capacity
 * slots each hold one task's descriptor, vectors (max_dim elements), a/b
 * history and result.  The kernel runs as up to 8 workers (launches on
 * streams of the queue) of at most `ctas` CTAs each (0: two per SM): another
 * starts while the unfinished tasks outnumber the running workers' CTAs, and
 * a worker leaves ~2 ms after it last found a task to claim (the first one
 * after ~20 ms), so the solver's width follows the backlog; posts and polls
 * start them.
 * Each task draws its start vector from its seed exactly as
 * hubbard_fill_start_vector does, stops on rho < tol * max(1, |theta|) (tol 0:
 * 1e-10), breakdown or max_iters (capped at D), and gets err_bound as
 * lanczos_ground_state defines it.  A task's arithmetic depends only on its
 * sector, so its result is the same whatever else is queued.  Hop tables are
 * cached per (lattice, particle number); the kernel leaves before a table pool
 * has to grow.  Calls on one queue are serialised internally; destroy must not
 * race other calls.
 * ------------------------------------------------------------------------- */
typedef struct hubbard_queue* hubbard_queue_t;

/* Allocates capacity * (24 * max_dim + 16 * max_iters) bytes of device
 * memory, 52 MB of table pools (grown when needed) and a few host-mapped
 * words.  HUB_EINVAL on
 * capacity outside [1, 2^20], max_dim outside [1, 2^31], max_iters < 1,
 * ctas < 0 or tol < 0; HUB_ENOMEM / HUB_ECUDA on allocation failure. */
int hubbard_queue_create(int capacity, int64_t max_dim, int max_iters, double tol, int ctas, hubbard_queue_t* out);

/* Posts one sector (host descriptor; same rules as hubbard_batch_create) with
 * the seed of its start vector; *ticket numbers the posts from 0.  Returns
 * HUB_EPENDING without posting when the oldest unfinished task still holds
 * the slot this post needs (the queue is full: poll, then post again);
 * HUB_EINVAL for a bad sector, more than 127 hops per state or D > max_dim;
 * HUB_ENOMEM after 2^31 - 1 posts to one queue. */
int hubbard_queue_post(hubbard_queue_t Q, const hubbard_sector_desc* sector, uint64_t seed, int64_t* ticket);

/* Builds and uploads the hop tables of a sector's two spin species, if not
 * cached yet, without posting it (a caller can warm the cache from another
 * thread; the host tables are built without holding the queue's lock).
 * HUB_EINVAL for a bad sector. */
int hubbard_queue_prepare(hubbard_queue_t Q, const hubbard_sector_desc* sector);

/* HUB_OK with the result once the task has finished (each result is returned
 * once), HUB_EPENDING before that; HUB_EINVAL for an unknown or already
 * collected ticket.  Does not block. */
int hubbard_queue_poll(hubbard_queue_t Q, int64_t ticket, lanczos_result* out);

/* Up to cap finished results not yet returned, in any order, with their
 * tickets (host arrays of cap); *n_found = how many.  Does not block. */
int hubbard_queue_collect(hubbard_queue_t Q, int64_t* tickets, lanczos_result* out, int cap, int* n_found);

/* Lets the kernel finish what was posted, then frees everything. */
void hubbard_queue_destroy(hubbard_queue_t Q);

/* ---------------------------------------------------------------------------
 * Continuous-batching ground-state server (the paper notes that a small
 * sector alone leaves the GPU idle, Sec. 5; this serves many requests at once).
 * Requests are queued by hubbard_server_submit and taken by worker lanes (host
 * threads, each with its own non-blocking stream) as soon as a lane is free and
 * the request's device-memory footprint fits what remains of the budget, first
 * come first served within each queue:
 *   D <= small_max_dim                : the small queue.  With a GPU, one
 *       small lane posts each small request to a queued solver
 *       (hubbard_queue_*) as soon as it arrives: the request joins the
 *       persistent kernel that is already solving the earlier ones, on its
 *       next free CTA (small_ctas CTAs, 0: 16; the rest of the GPU stays
 *       with the big lanes); the queue's memory (up to 1024 slots of
 *       small_max_dim elements, within a quarter of the budget) is taken
 *       from the budget when the server starts.  With host_solver (or small_ctas < 0), small lanes take every
 *       small request waiting (up to batch_max, within the budget) into one
 *       micro-batch instead.  tol is relative, rho < tol max(1, |theta|);
 *   small_max_dim < D <= mid_max_dim  : a big lane, binary64 Lanczos
 *       (lanczos_ground_state, absolute rho < tol);
 *   D > mid_max_dim                   : a big lane, binary32 Lanczos with
 *       binary64 refinement (lanczos_ground_state_refined, tol relative on the
 *       error bound), keeping up to store_vectors binary32 Lanczos vectors
 *       within a quarter of the spare budget and 16 GB; a request the
 *       refinement cannot certify is solved again by the binary64 Lanczos
 *       (its result then reports path 1).
 * Requests that arrive while others run are admitted as lanes and memory free
 * up, and their work overlaps on the device.  Handles, batches and buffers of
 * a lane are allocated on its stream, so finishing a request never waits for
 * the whole device.  A request whose solve fails carries that status; the
 * others are unaffected.  Start vectors: hubbard_fill_start_vector(seed).
 *
 * host_solver (testing without a GPU): when non-NULL, lanes call it instead
 * of any CUDA work, with the request, its path (0 batch, 1 binary64,
 * 2 refined) and a result to fill; its return value is the request's status.
 * It is called from the lane threads, concurrently.
 * ------------------------------------------------------------------------- */
typedef struct hubbard_server* hubbard_server_t;

typedef struct {
    int32_t ns, nup, ndn, n_bonds;
    const int32_t* bonds;      /* host, 2 * n_bonds; copied by submit */
    double t, U;
    uint64_t seed;             /* start vector (hubbard_fill_start_vector) */
} hubbard_request;

typedef int (*hubbard_host_solver)(void* ctx, uint64_t ticket, const hubbard_request* req, int path,
                                   lanczos_result* out);

typedef struct {
    double hbm_budget;         /* bytes of device memory for requests (<= 0: 80 % of the free memory) */
    int32_t small_lanes;       /* lanes of the small queue (micro-batch mode: concurrent micro-batches) */
    int32_t big_lanes;         /* concurrent single-sector solves */
    int64_t small_max_dim;
    int64_t mid_max_dim;
    int32_t max_iters;         /* <= 0: 1000 */
    int32_t batch_max;         /* requests per micro-batch (<= 0: 1024) */
    int32_t store_vectors;     /* binary32 Lanczos vectors kept per refined request (>= 0) */
    int32_t small_ctas;        /* CTAs of the queued small-sector solver (0: 16; < 0: micro-batches) */
    double tol;                /* <= 0: 1e-10 */
    hubbard_host_solver host_solver;
    void* host_ctx;
} hubbard_server_opts;

typedef struct {
    lanczos_result result;     /* energy, residual, err_bound, iters, status, breakdown */
    int32_t path;              /* 0 batch, 1 binary64, 2 refined */
    int32_t reserved;
    double t_submit, t_admit, t_done;   /* seconds since the server was created */
} hubbard_served;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t verified;          /* completed with status HUB_OK and err_bound <= 1e-9 max(1, |energy|) */
    int64_t running, queued, max_backlog;
    int64_t batches, batched_requests, binary64_solves, refined_solves;
    double budget_bytes, peak_bytes, free_bytes;
} hubbard_server_stats;

/* Starts the lanes.  HUB_EINVAL for no lane, negative thresholds or, with a
 * host solver, no budget; HUB_ECUDA without a device. */
int hubbard_server_create(const hubbard_server_opts* opts, hubbard_server_t* out);
/* Queues one request (non-blocking); *ticket identifies it.  HUB_ENOMEM when
 * its footprint exceeds the whole budget, HUB_EINVAL for a bad sector. */
int hubbard_server_submit(hubbard_server_t S, const hubbard_request* req, uint64_t* ticket);
/* HUB_OK with *out filled once the request has finished (its own status in
 * out->result.status), HUB_EPENDING before (out holds its times so far). */
int hubbard_server_poll(hubbard_server_t S, uint64_t ticket, hubbard_served* out);
/* Blocks until the request finishes or timeout_s passes (HUB_ETIMEOUT). */
int hubbard_server_wait(hubbard_server_t S, uint64_t ticket, double timeout_s, hubbard_served* out);
int hubbard_server_stats_get(hubbard_server_t S, hubbard_server_stats* out);
/* Stops taking work, lets running requests finish, joins the lanes; queued
 * requests are dropped. */
void hubbard_server_destroy(hubbard_server_t S);

/* Message for the last failing call on this thread ("" if none). */
const char* hubbard_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HUBBARD_H */
