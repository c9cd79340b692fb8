// C ABI entry points (include/hubbard.h): argument checks, device tables,
// dispatch to the kernels, and the Lanczos driver (Sec. 2.2, Algorithm 1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "internal.h"

namespace hub {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return HUB_ECUDA;
}

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t elem_size(int dtype) { return dtype == HUB_F64 ? 8 : 4; }

int check_handle(hubbard_t H) {
    if (H == nullptr) return fail(HUB_EINVAL, "null handle");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != H->device)
        return fail(HUB_EINVAL, "handle was created on another device");
    return HUB_OK;
}

int check_dtype(int dtype) {
    if (dtype != HUB_F64 && dtype != HUB_F32) return fail(HUB_EINVAL, "dtype must be HUB_F64 or HUB_F32");
    return HUB_OK;
}

template <typename T>
int upload(T** dst, const T* src, size_t n) {
    *dst = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tables)");
    if (n > 0) HUB_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return HUB_OK;
}

void free_spin_dev(DevSpin& d) {
    cudaFree(d.states);
    cudaFree(d.rowptr);
    cudaFree(d.ent);
    cudaFree(d.blk_off);
    cudaFree(d.blk_cnt);
    cudaFree(d.ent16);
    cudaFree(d.ent32);
    cudaFree(d.pn_ptr);
    cudaFree(d.pn_npos);
    cudaFree(d.pn_list);
    d = DevSpin{};
}

}  // namespace

// Staging of hubbard_apply_host: call i uses slot i % 2 -- its input copied
// to v[slot] on `up`, H applied on `comp`, the result copied back from
// w[slot] on `down` -- so consecutive calls overlap (upload i+1 | H*v i |
// download i-1).  Events order the reuse of a slot after the call two back.
struct HostPipe {
    int dtype = -1;
    size_t bytes = 0;
    void* v[2] = {nullptr, nullptr};
    void* w[2] = {nullptr, nullptr};
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t uploaded[2] = {}, computed[2] = {}, downloaded[2] = {};
    bool used[2] = {false, false};
    unsigned long long calls = 0;
};

void host_pipe_free(hubbard_sector* H) {
    HostPipe* P = H->host_pipe;
    if (P == nullptr) return;
    for (cudaStream_t st : {P->up, P->comp, P->down})
        if (st) cudaStreamSynchronize(st);
    for (int b = 0; b < 2; ++b) {
        cudaFree(P->v[b]);
        cudaFree(P->w[b]);
        for (cudaEvent_t e : {P->uploaded[b], P->computed[b], P->downloaded[b]})
            if (e) cudaEventDestroy(e);
    }
    for (cudaStream_t st : {P->up, P->comp, P->down})
        if (st) cudaStreamDestroy(st);
    delete P;
    H->host_pipe = nullptr;
}

namespace {

void free_dev(hubbard_sector* H) {
    host_pipe_free(H);
    for (int s = 0; s < 2; ++s) {
        H->dev[s] = DevSpin{};                 // owned by the shared entry
        H->spin_owner[s].reset();
    }
    dev_free(H->fx_scratch, H->mem_stream);
    H->fx_scratch = nullptr;
    H->fx_bytes = 0;
    dev_free(H->red, H->mem_stream);
    dev_free(H->status, H->mem_stream);
    dev_free(H->lz, H->mem_stream);
    H->red = nullptr;
    H->status = nullptr;
    H->lz = nullptr;
    H->lz_cap = 0;
}

// Slot assignment for the row-phase gathers of one group of 32 states.
// Lanes are split into phases of `pl` lanes (one shared-memory wavefront each
// for an element of `eb` bytes: 128/eb bank groups).  Within a phase, a hop
// of lane l to target t is an edge (l, t mod groups) of a bipartite multigraph;
// a proper edge colouring with Delta = max degree colours (Koenig) gives slots
// in which no two lanes of a phase hit the same bank group.  Colouring by
// alternating paths.  Returns, per lane, the slot of each of its hops.
struct SlotColouring {
    int slots = 0;
    std::vector<std::vector<int>> slot_of;   // [lane][hop index] -> slot
};

static SlotColouring colour_group(const std::vector<std::vector<int32_t>>& lane_tgts, int eb) {
    const int ngroups = std::max(1, 128 / eb);
    const int pl = std::max(1, std::min(32, 128 / eb));   // lanes per wavefront phase
    SlotColouring R;
    R.slot_of.resize(lane_tgts.size());
    for (size_t l = 0; l < lane_tgts.size(); ++l) R.slot_of[l].assign(lane_tgts[l].size(), -1);
    for (size_t p0 = 0; p0 < lane_tgts.size(); p0 += pl) {
        const size_t p1 = std::min(lane_tgts.size(), p0 + pl);
        struct E { int l, g; size_t lane, k; };
        std::vector<E> edges;
        std::vector<int> degl(pl, 0), degg(ngroups, 0);
        for (size_t l = p0; l < p1; ++l)
            for (size_t k = 0; k < lane_tgts[l].size(); ++k) {
                const int g = (int)(lane_tgts[l][k] % ngroups);
                edges.push_back({(int)(l - p0), g, l, k});
                degl[l - p0]++;
                degg[g]++;
            }
        int D = 0;
        for (int x : degl) D = std::max(D, x);
        for (int x : degg) D = std::max(D, x);
        std::vector<std::vector<int>> atl(pl, std::vector<int>(D, -1)), atg(ngroups, std::vector<int>(D, -1));
        std::vector<int> col(edges.size(), -1);
        for (size_t ei = 0; ei < edges.size(); ++ei) {
            const int l = edges[ei].l, g = edges[ei].g;
            int a = 0, b = 0;
            while (atl[l][a] >= 0) ++a;
            while (atg[g][b] >= 0) ++b;
            if (atg[g][a] >= 0) {
                // flip the a/b alternating path that starts at g along colour a
                std::vector<int> path;
                bool at_g = true;
                int node = g, cur = a;
                while (true) {
                    const int e = at_g ? atg[node][cur] : atl[node][cur];
                    if (e < 0) break;
                    path.push_back(e);
                    node = at_g ? edges[e].l : edges[e].g;
                    at_g = !at_g;
                    cur = (cur == a) ? b : a;
                }
                for (int e : path) {
                    atl[edges[e].l][col[e]] = -1;
                    atg[edges[e].g][col[e]] = -1;
                }
                for (int e : path) {
                    col[e] = (col[e] == a) ? b : a;
                    atl[edges[e].l][col[e]] = e;
                    atg[edges[e].g][col[e]] = e;
                }
            }
            col[ei] = a;
            atl[l][a] = (int)ei;
            atg[g][a] = (int)ei;
        }
        for (size_t ei = 0; ei < edges.size(); ++ei) R.slot_of[edges[ei].lane][edges[ei].k] = col[ei];
        R.slots = std::max(R.slots, D);
    }
    // validate: every hop has a slot in [0, slots) and no lane uses a slot twice;
    // otherwise fall back to consecutive slots (correct, only slower)
    bool ok = true;
    for (size_t l = 0; l < R.slot_of.size() && ok; ++l) {
        std::vector<char> used((size_t)std::max(R.slots, 1), 0);
        for (int s : R.slot_of[l]) {
            if (s < 0 || s >= R.slots || used[(size_t)s]) { ok = false; break; }
            used[(size_t)s] = 1;
        }
    }
    if (!ok) {
        R.slots = 0;
        for (size_t l = 0; l < R.slot_of.size(); ++l) {
            for (size_t k = 0; k < R.slot_of[l].size(); ++k) R.slot_of[l][k] = (int)k;
            R.slots = std::max(R.slots, (int)R.slot_of[l].size());
        }
    }
    return R;
}

// sign-split list: per row the +1 targets first, then the -1 targets, each
// ascending; npos[r] = number of +1 targets of row r
void sign_split_list(const SpinTables& T, std::vector<int32_t>& npos, std::vector<uint32_t>& pnl) {
    npos.assign((size_t)T.D, 0);
    pnl.assign(T.tgt.size(), 0u);
    for (int64_t r = 0; r < T.D; ++r) {
        int32_t o = T.rowptr[(size_t)r], np = 0;
        for (int32_t k = T.rowptr[(size_t)r]; k < T.rowptr[(size_t)r + 1]; ++k)
            if (T.sign[(size_t)k] > 0) { pnl[(size_t)o++] = (uint32_t)T.tgt[(size_t)k]; ++np; }
        for (int32_t k = T.rowptr[(size_t)r]; k < T.rowptr[(size_t)r + 1]; ++k)
            if (T.sign[(size_t)k] < 0) pnl[(size_t)o++] = (uint32_t)T.tgt[(size_t)k];
        npos[(size_t)r] = np;
    }
}

int upload_spin(const SpinTables& T, DevSpin& d) {
    std::vector<uint32_t> ent(T.tgt.size());
    for (size_t k = 0; k < T.tgt.size(); ++k)
        ent[k] = ((uint32_t)T.tgt[k] << 1) | (T.sign[k] < 0 ? 1u : 0u);
    // SELL-32/8 for the row phase, coloured for the element size the row phase
    // will stage (16 bytes when a 16-byte-per-state row fits in shared memory,
    // else 8, else 4)
    const int64_t smem_budget = 220 * 1024;
    const int eb = ((T.D + 64) * 16 <= smem_budget) ? 16 : (((T.D + 64) * 8 <= smem_budget) ? 8 : 4);
    RowBlocks rb;
    build_row_blocks(T, eb, rb);
    const std::vector<int64_t>& boff = rb.boff;
    const std::vector<int32_t>& bcnt = rb.bcnt;
    const bool narrow = rb.narrow;
    std::vector<uint32_t>& bent = rb.ent;
    if (bent.empty()) bent.push_back(0u);
    std::vector<int32_t> npos;
    std::vector<uint32_t> pnl;
    sign_split_list(T, npos, pnl);
    int rc;
    if ((rc = upload(&d.pn_ptr, T.rowptr.data(), T.rowptr.size()))) return rc;
    if ((rc = upload(&d.pn_npos, npos.data(), npos.size()))) return rc;
    if ((rc = upload(&d.pn_list, pnl.data(), pnl.size()))) return rc;
    if ((rc = upload(&d.blk_off, boff.data(), boff.size()))) return rc;
    if ((rc = upload(&d.blk_cnt, bcnt.data(), bcnt.size()))) return rc;
    if (narrow) {
        std::vector<uint16_t> e16(bent.size());
        for (size_t i = 0; i < bent.size(); ++i) e16[i] = (uint16_t)bent[i];
        if ((rc = upload(&d.ent16, e16.data(), e16.size()))) return rc;
    } else {
        if ((rc = upload(&d.ent32, bent.data(), bent.size()))) return rc;
    }
    if ((rc = upload(&d.states, T.states.data(), T.states.size()))) return rc;
    if ((rc = upload(&d.rowptr, T.rowptr.data(), T.rowptr.size()))) return rc;
    if ((rc = upload(&d.ent, ent.data(), ent.size()))) return rc;
    return HUB_OK;
}

// binary64: row-phase sums Y (int64) + fixed-point copy X (int2); binary32 uses the first half
int ensure_fx_scratch(hubbard_sector* H) {
    const size_t need = (size_t)H->D * 16;
    if (H->fx_bytes >= need) return HUB_OK;
    dev_free(H->fx_scratch, H->mem_stream);
    H->fx_scratch = nullptr;
    H->fx_bytes = 0;
    cudaError_t e = dev_alloc(&H->fx_scratch, std::max<size_t>(need, 256), H->mem_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fixed-point scratch)");
    H->fx_bytes = need;
    return HUB_OK;
}

// hop sums of up to 127 terms fit the two int32 fixed-point accumulators
bool fixed_point_ok(const hubbard_sector* H) { return H->host[0].W + H->host[1].W <= 127; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct SpinEntry {
    SpinTables host;
    DevSpin dev;
    int device = 0;
    ~SpinEntry() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != device) cudaSetDevice(device);
        free_spin_dev(dev);
        if (cur >= 0 && cur != device) cudaSetDevice(cur);
    }
};

namespace {
// Process-wide table cache: (device, Ns, bonds, N) -> entry.  Handles share
// entries; the most recently used kSpinCacheKeep entries stay alive after
// their last handle is gone, so creating the same sector again (a solve
// loop, a server) skips the table build, colouring and upload.
using SpinKey = std::tuple<int, int, std::vector<std::pair<int, int>>, int>;
constexpr size_t kSpinCacheKeep = 256;
std::mutex g_spin_mu;
std::map<SpinKey, std::weak_ptr<SpinEntry>> g_spin_index;
std::list<std::shared_ptr<SpinEntry>> g_spin_recent;

std::shared_ptr<SpinEntry> spin_lookup(const SpinKey& key) {
    std::lock_guard<std::mutex> lk(g_spin_mu);
    auto it = g_spin_index.find(key);
    if (it == g_spin_index.end()) return nullptr;
    std::shared_ptr<SpinEntry> e = it->second.lock();
    if (e == nullptr) g_spin_index.erase(it);
    return e;
}

// registers e (or returns the entry another thread registered meanwhile)
std::shared_ptr<SpinEntry> spin_insert(const SpinKey& key, std::shared_ptr<SpinEntry> e) {
    std::shared_ptr<SpinEntry> dropped;
    std::lock_guard<std::mutex> lk(g_spin_mu);
    auto it = g_spin_index.find(key);
    if (it != g_spin_index.end()) {
        std::shared_ptr<SpinEntry> other = it->second.lock();
        if (other != nullptr) return other;
    }
    g_spin_index[key] = e;
    g_spin_recent.push_front(e);
    if (g_spin_recent.size() > kSpinCacheKeep) {
        dropped = std::move(g_spin_recent.back());     // freed after the lock is released
        g_spin_recent.pop_back();
    }
    return e;
}

int spin_tables(int device, int ns, const std::vector<std::pair<int, int>>& bl, int n,
                std::shared_ptr<SpinEntry>& out) {
    const SpinKey key(device, ns, bl, n);
    out = spin_lookup(key);
    if (out != nullptr) return HUB_OK;
    auto e = std::make_shared<SpinEntry>();
    e->device = device;
    try {
        build_spin_tables(ns, n, bl, e->host);
    } catch (const std::bad_alloc&) {
        return fail(HUB_ENOMEM, "host allocation (tables)");
    }
    const int rc = upload_spin(e->host, e->dev);
    if (rc != HUB_OK) return rc;
    out = spin_insert(key, e);
    return HUB_OK;
}
}  // namespace

// Row-phase table of one spin (SELL-32/8): per group of 32 states, slots
// assigned by bank-conflict-free colouring for staged elements of eb bytes, in
// blocks of 8 slots per lane, contiguous per lane.  Entry = staged slot index,
// top bit set for sign -1.  The staged row is followed by 32 zero slots
// starting at Dr = D rounded up to 32; a slot a lane does not use points at the
// zero slot of a bank group no other lane of its wavefront phase uses (so
// padding adds zero without a branch and without a conflict).  Every group
// holds a multiple of 128 entries, so each starts 16-byte aligned.
void build_row_blocks(const SpinTables& T, int eb, RowBlocks& out) {
    const int ngroups = 128 / eb;
    const int planes = std::min(32, ngroups);
    const int64_t Dr = (T.D + 31) / 32 * 32;
    const bool narrow = Dr + 32 <= 32767;            // 15-bit index + sign
    out.narrow = narrow;
    const uint32_t negbit = narrow ? 0x8000u : 0x80000000u;
    const int64_t groups = (T.D + 31) / 32;
    std::vector<int64_t>& boff = out.boff;
    std::vector<int32_t>& bcnt = out.bcnt;
    boff.assign((size_t)groups, 0);
    bcnt.assign((size_t)groups, 0);
    int64_t btotal = 0;
    std::vector<SlotColouring> colours((size_t)groups);
    for (int64_t g = 0; g < groups; ++g) {
        std::vector<std::vector<int32_t>> lt;
        for (int64_t r = 32 * g; r < std::min<int64_t>(T.D, 32 * g + 32); ++r)
            lt.emplace_back(T.tgt.begin() + T.rowptr[(size_t)r], T.tgt.begin() + T.rowptr[(size_t)r + 1]);
        colours[(size_t)g] = colour_group(lt, eb);
        boff[(size_t)g] = btotal;
        bcnt[(size_t)g] = (colours[(size_t)g].slots + 3) / 4;      // half-blocks of 4 slots
        btotal += (int64_t)bcnt[(size_t)g] * 32 * 4;
    }
    std::vector<uint32_t>& bent = out.ent;
    bent.assign((size_t)btotal, (uint32_t)Dr);
    for (int64_t g = 0; g < groups; ++g) {
        const SlotColouring& C = colours[(size_t)g];
        const int nslot = bcnt[(size_t)g] * 4;
        const int nfull = bcnt[(size_t)g] / 2;                        // blocks of 8 slots, then maybe one of 4
        auto pos = [&](int l, int s) -> int64_t {
            if (s < nfull * 8) return boff[(size_t)g] + ((int64_t)(s / 8) * 32 + l) * 8 + s % 8;
            return boff[(size_t)g] + (int64_t)nfull * 32 * 8 + (int64_t)l * 4 + (s - nfull * 8);
        };
        // entry[lane][slot], -1 = padding
        std::vector<std::vector<int64_t>> grid(32, std::vector<int64_t>((size_t)nslot, -1));
        for (int64_t r = 32 * g; r < std::min<int64_t>(T.D, 32 * g + 32); ++r) {
            const int lane = (int)(r % 32);
            for (int32_t k = T.rowptr[(size_t)r], c = 0; k < T.rowptr[(size_t)r + 1]; ++k, ++c)
                grid[(size_t)lane][(size_t)C.slot_of[(size_t)lane][(size_t)c]] = k;
        }
        for (int s = 0; s < nslot; ++s) {
            for (int p0 = 0; p0 < 32; p0 += planes) {
                std::vector<char> used((size_t)ngroups, 0);
                for (int l = p0; l < p0 + planes; ++l) {
                    const int64_t k = grid[(size_t)l][(size_t)s];
                    if (k >= 0) used[(size_t)(T.tgt[(size_t)k] % ngroups)] = 1;
                }
                int freeg = 0;
                while (freeg < ngroups && used[(size_t)freeg]) ++freeg;
                if (freeg == ngroups) freeg = 0;          // cannot happen: a padded lane leaves a group free
                for (int l = p0; l < p0 + planes; ++l) {
                    const int64_t k = grid[(size_t)l][(size_t)s];
                    const uint32_t e = k >= 0 ? ((uint32_t)T.tgt[(size_t)k] | (T.sign[(size_t)k] < 0 ? negbit : 0u))
                                              : (uint32_t)(Dr + freeg);
                    bent[(size_t)pos(l, s)] = e;
                }
            }
        }
    }
}

}  // namespace hub

using namespace hub;

extern "C" {

const char* hubbard_last_error(void) { return g_last_error.c_str(); }

uint64_t hubbard_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

static long double comb_ld(int n, int k) {
    long double c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

// Validates Ns, the bond list and one filling; fills `bl`.
static int check_lattice(int Ns, const int32_t* bonds, int n_bonds, int N, std::vector<std::pair<int, int>>& bl) {
    if (Ns < 1 || Ns > 32) return fail(HUB_EINVAL, "Ns must be in 1..32");
    if (N < 0 || N > Ns) return fail(HUB_EINVAL, "N_up, N_dn must be in 0..Ns");
    if (n_bonds < 0 || (n_bonds > 0 && bonds == nullptr)) return fail(HUB_EINVAL, "bad bond list");
    bl.clear();
    std::set<std::pair<int, int>> seen;
    for (int b = 0; b < n_bonds; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || i >= Ns || j < 0 || j >= Ns) return fail(HUB_EINVAL, "bond endpoint out of range");
        if (i == j) return fail(HUB_EINVAL, "self bond");
        auto key = std::make_pair(std::min(i, j), std::max(i, j));
        if (!seen.insert(key).second) return fail(HUB_EINVAL, "duplicate bond");
        bl.emplace_back(i, j);
    }
    // D_sigma = C(Ns, N_sigma) must stay below 2^30 (packed table entries)
    if (comb_ld(Ns, N) > (long double)(1 << 30)) return fail(HUB_EINVAL, "D_sigma exceeds 2^30");
    return HUB_OK;
}

int hubbard_host_spin_tables(int Ns, const int32_t* bonds, int n_bonds, int N, int64_t* D, int64_t* nnz,
                             uint32_t* states, int32_t* rowptr, int32_t* tgt, int8_t* sign) {
    clear_error();
    std::vector<std::pair<int, int>> bl;
    int rc = check_lattice(Ns, bonds, n_bonds, N, bl);
    if (rc) return rc;
    SpinTables T;
    try {
        build_spin_tables(Ns, N, bl, T);
    } catch (const std::bad_alloc&) {
        return fail(HUB_ENOMEM, "host allocation (tables)");
    }
    if (D) *D = T.D;
    if (nnz) *nnz = (int64_t)T.tgt.size();
    if (states) std::memcpy(states, T.states.data(), T.states.size() * sizeof(uint32_t));
    if (rowptr) std::memcpy(rowptr, T.rowptr.data(), T.rowptr.size() * sizeof(int32_t));
    if (tgt) std::memcpy(tgt, T.tgt.data(), T.tgt.size() * sizeof(int32_t));
    if (sign) std::memcpy(sign, T.sign.data(), T.sign.size() * sizeof(int8_t));
    return HUB_OK;
}

int hubbard_host_row_table(int Ns, const int32_t* bonds, int n_bonds, int N, int elem_bytes, int64_t* groups,
                           int64_t* entries, int* narrow, int64_t* boff, int32_t* bcnt, uint32_t* ent) {
    clear_error();
    if (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) return fail(HUB_EINVAL, "elem_bytes must be 4, 8 or 16");
    std::vector<std::pair<int, int>> bl;
    int rc = check_lattice(Ns, bonds, n_bonds, N, bl);
    if (rc) return rc;
    SpinTables T;
    RowBlocks rb;
    try {
        build_spin_tables(Ns, N, bl, T);
        build_row_blocks(T, elem_bytes, rb);
    } catch (const std::bad_alloc&) {
        return fail(HUB_ENOMEM, "host allocation (tables)");
    }
    if (groups) *groups = (int64_t)rb.boff.size();
    if (entries) *entries = (int64_t)rb.ent.size();
    if (narrow) *narrow = rb.narrow ? 1 : 0;
    if (boff) std::memcpy(boff, rb.boff.data(), rb.boff.size() * sizeof(int64_t));
    if (bcnt) std::memcpy(bcnt, rb.bcnt.data(), rb.bcnt.size() * sizeof(int32_t));
    if (ent) std::memcpy(ent, rb.ent.data(), rb.ent.size() * sizeof(uint32_t));
    return HUB_OK;
}

int hubbard_sector_create(int Ns, const int32_t* bonds, int n_bonds, int Nup, int Ndn, double t, double U,
                          hubbard_t* out) {
    return sector_create_streamed(Ns, bonds, n_bonds, Nup, Ndn, t, U, nullptr, out);
}

}  // extern "C"

int hub::sector_create_streamed(int Ns, const int32_t* bonds, int n_bonds, int Nup, int Ndn, double t, double U,
                                cudaStream_t ms, hubbard_t* out) {
    clear_error();
    if (out == nullptr) return fail(HUB_EINVAL, "out is null");
    *out = nullptr;
    std::vector<std::pair<int, int>> bl;
    int rc0 = check_lattice(Ns, bonds, n_bonds, Nup, bl);
    if (rc0 == HUB_OK) rc0 = check_lattice(Ns, bonds, n_bonds, Ndn, bl);
    if (rc0) return rc0;
    if (!std::isfinite(t) || !std::isfinite(U)) return fail(HUB_EINVAL, "t and U must be finite");
    hubbard_sector* H = new (std::nothrow) hubbard_sector();
    if (H == nullptr) return fail(HUB_ENOMEM, "host allocation");
    if (cudaGetDevice(&H->device) != cudaSuccess) {
        delete H;
        return fail(HUB_ECUDA, "no CUDA device");
    }
    H->mem_stream = ms;
    H->ns = Ns;
    H->nup = Nup;
    H->ndn = Ndn;
    H->t = t;
    H->U = U;
    H->bonds = bl;
    int rc = spin_tables(H->device, Ns, bl, Nup, H->spin_owner[0]);
    if (rc == HUB_OK) rc = spin_tables(H->device, Ns, bl, Ndn, H->spin_owner[1]);
    if (rc == HUB_OK) {
        try {
            for (int s = 0; s < 2; ++s) {
                H->host[s] = H->spin_owner[s]->host;
                H->dev[s] = H->spin_owner[s]->dev;
            }
        } catch (const std::bad_alloc&) {
            rc = fail(HUB_ENOMEM, "host allocation (tables)");
        }
    }
    H->Dup = H->host[0].D;
    H->Ddn = H->host[1].D;
    H->D = H->Dup * H->Ddn;
    if (rc == HUB_OK) {
        cudaError_t e = dev_alloc((void**)&H->red, kRedSlots * sizeof(double), ms);
        if (e == cudaSuccess) e = dev_alloc((void**)&H->status, 4 * sizeof(int), ms);
        if (e == cudaSuccess)
            e = ms ? cudaMemsetAsync(H->status, 0, 4 * sizeof(int), ms) : cudaMemset(H->status, 0, 4 * sizeof(int));
        if (e == cudaSuccess)
            e = ms ? cudaMemsetAsync(H->red, 0, kRedSlots * sizeof(double), ms)
                   : cudaMemset(H->red, 0, kRedSlots * sizeof(double));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(reduction scratch)");
    }
    if (rc != HUB_OK) {
        std::string msg = g_last_error;
        free_dev(H);
        delete H;
        return fail(rc, msg);
    }
    *out = H;
    return HUB_OK;
}

extern "C" {

void hubbard_sector_destroy(hubbard_t H) {
    if (H == nullptr) return;
    // a handle tied to a stream frees in that stream's order; any other waits
    // for the device, since its scratch may be in use on any stream
    if (H->mem_stream == nullptr) cudaDeviceSynchronize();
    free_dev(H);
    delete H;
}

int hubbard_sector_info(hubbard_t H, int64_t* D_up, int64_t* D_dn, int32_t* W_up, int32_t* W_dn) {
    clear_error();
    if (H == nullptr) return fail(HUB_EINVAL, "null handle");
    if (D_up) *D_up = H->Dup;
    if (D_dn) *D_dn = H->Ddn;
    if (W_up) *W_up = H->host[0].W;
    if (W_dn) *W_dn = H->host[1].W;
    return HUB_OK;
}

int64_t hubbard_table_nnz(hubbard_t H, int spin) {
    if (H == nullptr || (spin != 0 && spin != 1)) return -1;
    return (int64_t)H->host[spin].tgt.size();
}

int hubbard_export_tables(hubbard_t H, int spin, uint32_t* states, int32_t* rowptr, int32_t* tgt, int8_t* sign) {
    clear_error();
    if (H == nullptr) return fail(HUB_EINVAL, "null handle");
    if (spin != 0 && spin != 1) return fail(HUB_EINVAL, "spin must be 0 (up) or 1 (down)");
    const SpinTables& T = H->host[spin];
    if (states) std::memcpy(states, T.states.data(), T.states.size() * sizeof(uint32_t));
    if (rowptr) std::memcpy(rowptr, T.rowptr.data(), T.rowptr.size() * sizeof(int32_t));
    if (tgt) std::memcpy(tgt, T.tgt.data(), T.tgt.size() * sizeof(int32_t));
    if (sign) std::memcpy(sign, T.sign.data(), T.sign.size() * sizeof(int8_t));
    return HUB_OK;
}

static int check_apply(hubbard_t H, const void* v, void* w, int dtype) {
    int rc;
    if ((rc = check_handle(H))) return rc;
    if ((rc = check_dtype(dtype))) return rc;
    if (v == nullptr || w == nullptr) return fail(HUB_EINVAL, "null vector");
    if (!aligned16(v) || !aligned16(w)) return fail(HUB_EINVAL, "vectors must be 16-byte aligned");
    const size_t bytes = (size_t)H->D * elem_size(dtype);
    const char* a = (const char*)v;
    const char* b = (const char*)w;
    if (a < b + bytes && b < a + bytes) return fail(HUB_EINVAL, "v and w overlap");
    return HUB_OK;
}

int hubbard_apply(hubbard_t H, const void* v, void* w, int dtype, void* stream) {
    clear_error();
    int rc = check_apply(H, v, w, dtype);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == HUB_F64 && !fixed_point_ok(H)) return launch_hv_reference(H, v, w, dtype, s);
    if ((rc = ensure_fx_scratch(H))) return rc;
    return launch_hv_fast(H, v, w, dtype, 0.0, nullptr, 0, s);
}

int hubbard_apply_host(hubbard_t H, const void* v_host, void* w_host, int dtype, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_handle(H))) return rc;
    if ((rc = check_dtype(dtype))) return rc;
    if (v_host == nullptr || w_host == nullptr) return fail(HUB_EINVAL, "null vector");
    if (H->mem_stream != nullptr) return fail(HUB_EINVAL, "host apply on a stream-owned handle");
    const size_t bytes = (size_t)H->D * elem_size(dtype);
    const char* a = (const char*)v_host;
    const char* b = (const char*)w_host;
    if (a < b + bytes && b < a + bytes) return fail(HUB_EINVAL, "v and w overlap");
    cudaPointerAttributes pa{};
    for (const void* p : {v_host, (const void*)w_host})
        if (cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeDevice)
            return fail(HUB_EINVAL, "hubbard_apply_host takes host buffers");
    cudaGetLastError();                                  // a plain host pointer may leave an error behind
    HostPipe* P = H->host_pipe;
    if (P != nullptr && (P->dtype != dtype || P->bytes != bytes)) {
        host_pipe_free(H);
        P = nullptr;
    }
    if (P == nullptr) {
        P = new (std::nothrow) HostPipe;
        if (P == nullptr) return fail(HUB_ENOMEM, "host allocation (host apply staging)");
        H->host_pipe = P;
        P->dtype = dtype;
        P->bytes = bytes;
        cudaError_t e = cudaSuccess;
        for (cudaStream_t* st : {&P->up, &P->comp, &P->down})
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            for (cudaEvent_t* ev : {&P->uploaded[k], &P->computed[k], &P->downloaded[k]})
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMalloc(&P->v[k], std::max<size_t>(bytes, 256));
            if (e == cudaSuccess) e = cudaMalloc(&P->w[k], std::max<size_t>(bytes, 256));
        }
        if (e != cudaSuccess) {
            host_pipe_free(H);
            return cuda_fail(e, "host apply staging");
        }
    }
    const int k = (int)(P->calls & 1ull);
    // upload: v[k] is free once the call two back has been computed
    if (P->used[k]) HUB_CUDA(cudaStreamWaitEvent(P->up, P->computed[k], 0));
    HUB_CUDA(cudaMemcpyAsync(P->v[k], v_host, bytes, cudaMemcpyHostToDevice, P->up));
    HUB_CUDA(cudaEventRecord(P->uploaded[k], P->up));
    // compute: after the upload, and once w[k] has been downloaded by the call two back
    HUB_CUDA(cudaStreamWaitEvent(P->comp, P->uploaded[k], 0));
    if (P->used[k]) HUB_CUDA(cudaStreamWaitEvent(P->comp, P->downloaded[k], 0));
    if (dtype == HUB_F64 && !fixed_point_ok(H)) {
        rc = launch_hv_reference(H, P->v[k], P->w[k], dtype, P->comp);
    } else {
        rc = ensure_fx_scratch(H);
        if (rc == HUB_OK) rc = launch_hv_fast(H, P->v[k], P->w[k], dtype, 0.0, nullptr, 0, P->comp);
    }
    if (rc != HUB_OK) return rc;
    HUB_CUDA(cudaEventRecord(P->computed[k], P->comp));
    // download, then `stream` waits for it
    HUB_CUDA(cudaStreamWaitEvent(P->down, P->computed[k], 0));
    HUB_CUDA(cudaMemcpyAsync(w_host, P->w[k], bytes, cudaMemcpyDeviceToHost, P->down));
    HUB_CUDA(cudaEventRecord(P->downloaded[k], P->down));
    HUB_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, P->downloaded[k], 0));
    P->used[k] = true;
    ++P->calls;
    return HUB_OK;
}

int hubbard_set_schedule(hubbard_t H, int vec_rows, int vec_cols, int ctas_rows, int ctas_cols) {
    clear_error();
    if (H == nullptr) return fail(HUB_EINVAL, "null handle");
    auto ok_vec = [](int v) { return v == 0 || v == 1 || v == 2 || v == 4; };
    auto ok_cta = [](int c) { return c >= 0 && c <= 2; };
    if (!ok_vec(vec_rows) || !ok_vec(vec_cols) || !ok_cta(ctas_rows) || !ok_cta(ctas_cols))
        return fail(HUB_EINVAL, "schedule: vec in {0,1,2,4}, ctas in {0,1,2}");
    H->vec_rows = vec_rows;
    H->vec_cols = vec_cols;
    H->ctas_rows = ctas_rows;
    H->ctas_cols = ctas_cols;
    return HUB_OK;
}

int hubbard_autotune_schedule(hubbard_t H, const void* v, void* w, int dtype, void* stream, int* chosen) {
    clear_error();
    int rc = check_apply(H, v, w, dtype);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int vmax = dtype == HUB_F64 ? 2 : 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(HUB_ECUDA, "autotune events");
    }
    const int saved[4] = {H->vec_rows, H->vec_cols, H->ctas_rows, H->ctas_cols};
    float best = -1.0f;
    int pick[4] = {0, 0, 0, 0};
    for (int vr = 1; vr <= vmax && rc == HUB_OK; vr *= 2)
        for (int vc = 1; vc <= vmax && rc == HUB_OK; vc *= 2)
            for (int cr = 1; cr <= 2 && rc == HUB_OK; ++cr)
            for (int cc = 1; cc <= (dtype == HUB_F64 ? 2 : 1) && rc == HUB_OK; ++cc) {
                H->vec_rows = vr;
                H->vec_cols = vc;
                H->ctas_rows = cr;
                H->ctas_cols = dtype == HUB_F64 ? cc : 0;
                if ((rc = hubbard_apply(H, v, w, dtype, stream))) break;    // warm (allocates scratch)
                cudaEventRecord(e0, s);
                for (int k = 0; k < 3 && rc == HUB_OK; ++k) rc = hubbard_apply(H, v, w, dtype, stream);
                cudaEventRecord(e1, s);
                if (rc) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = fail(HUB_ECUDA, "autotune timing");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (best < 0.0f || ms < best) {
                    best = ms;
                    pick[0] = vr;
                    pick[1] = vc;
                    pick[2] = cr;
                    pick[3] = H->ctas_cols;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        H->vec_rows = saved[0];
        H->vec_cols = saved[1];
        H->ctas_rows = saved[2];
        H->ctas_cols = saved[3];
        return rc;
    }
    H->vec_rows = pick[0];
    H->vec_cols = pick[1];
    H->ctas_rows = pick[2];
    H->ctas_cols = pick[3];
    if (chosen != nullptr) std::memcpy(chosen, pick, sizeof(pick));
    return HUB_OK;
}

int hubbard_apply_reference(hubbard_t H, const void* v, void* w, int dtype, void* stream) {
    clear_error();
    int rc = check_apply(H, v, w, dtype);
    if (rc) return rc;
    return launch_hv_reference(H, v, w, dtype, (cudaStream_t)stream);
}

static int check_vec(const void* x, int64_t n, int dtype) {
    int rc;
    if ((rc = check_dtype(dtype))) return rc;
    if (n < 0) return fail(HUB_EINVAL, "negative length");
    if (n > 0 && x == nullptr) return fail(HUB_EINVAL, "null vector");
    if (!aligned16(x)) return fail(HUB_EINVAL, "vectors must be 16-byte aligned");
    return HUB_OK;
}

// Reductions use a small per-thread scratch allocated once per device thread.
static double* reduction_scratch() {
    static thread_local double* p = nullptr;
    static thread_local int dev = -1;
    int cur = 0;
    cudaGetDevice(&cur);
    if (p == nullptr || dev != cur) {
        p = nullptr;
        if (cudaMalloc((void**)&p, kRedSlots * sizeof(double)) != cudaSuccess) p = nullptr;
        dev = cur;
    }
    return p;
}

int hubbard_fill_start_vector(void* v, int64_t n, uint64_t seed, int64_t start, int dtype, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_vec(v, n, dtype))) return rc;
    if (start < 0) return fail(HUB_EINVAL, "negative start");
    return launch_fill_splitmix(v, n, (unsigned long long)seed, start, dtype, (cudaStream_t)stream);
}

int hubbard_vec_dot(const void* x, const void* y, int64_t n, int dtype, void* stream, double* out) {
    clear_error();
    int rc;
    if ((rc = check_vec(x, n, dtype)) || (rc = check_vec(y, n, dtype))) return rc;
    if (out == nullptr) return fail(HUB_EINVAL, "out is null");
    double* red = reduction_scratch();
    if (red == nullptr) return fail(HUB_ENOMEM, "reduction scratch");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = launch_dot(nullptr, x, y, n, dtype, red, s))) return rc;
    return reduce_partials_host(red, s, out);
}

int hubbard_vec_nrm2(const void* x, int64_t n, int dtype, void* stream, double* out) {
    double s2 = 0.0;
    int rc = hubbard_vec_dot(x, x, n, dtype, stream, &s2);
    if (rc) return rc;
    *out = std::sqrt(s2);
    return HUB_OK;
}

int hubbard_vec_axpy(double a, const void* x, void* y, int64_t n, int dtype, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_vec(x, n, dtype)) || (rc = check_vec(y, n, dtype))) return rc;
    return launch_axpy(a, x, y, n, dtype, (cudaStream_t)stream);
}

// One Lanczos step (Eqs. split1, Algorithm 1) on caller vectors.
// fixed_emax: 1023 when f and g are known to have norm <= 1 (inside the
// solver), 0 to derive the fixed-point scale from the data.
// One step of Algorithm 1 in the two-vector form: g <- H f - beta_j g,
// a_j = <g, f>, beta_{j+1} = |g - a_j f|.  The H*v kernels also reduce <g, f>,
// <g, g> and <f, f> (fused, deterministic), so that
//   beta_{j+1}^2 = <g, g> - 2 a_j^2 + a_j^2 <f, f>
// without another pass; when that difference cancels more than six digits of
// <g, g> (near breakdown), or the kernel path cannot fuse, g - a_j f is formed
// and its norm taken explicitly.  *pending (may be null when normalise) tells
// how g is left:
//   true : g = H f - beta_j g; finish with launch_axpy_scale(-a_j, 1/beta_{j+1}),
//          or pass that update as `upd` to the next step, whose row phase applies it
//   false: g = H f - beta_j g - a_j f; finish with launch_scale(1/beta_{j+1})
// Every finish rounds as axpy then scale, so each leaves the same f_{j+1}.
// upd (may be null): the previous step's pending update, applied to f first.
static int lanczos_step_impl(hubbard_t H, const void* f, void* g, double beta_j, int dtype, cudaStream_t s,
                             double* alpha, double* beta_next, bool normalise, int fixed_emax,
                             bool* pending = nullptr, const RowUpdate* upd = nullptr,
                             const void* w_old = nullptr) {
    int rc;
    if (dtype == HUB_F64 && !fixed_point_ok(H))
        return fail(HUB_EINVAL, "lanczos step: more than 127 hops per state is not supported");
    bool fused = false;
    // g <- H f - beta_j g  (Eqs. split1), fused into the H*v kernels with the
    // reductions; upd: f itself is first completed by the previous step's update.
    // w_old != nullptr: g <- H f - beta_j w_old (the same operations per element)
    if ((rc = launch_hv_fast(H, f, g, dtype, beta_j, w_old != nullptr ? w_old : g, fixed_emax, s, H->red, &fused,
                             upd)))
        return rc;
    double a = 0.0, b2 = 0.0;
    bool pend = false;
    if (fused) {
        double r[3];
        if ((rc = reduce_partials3_host(H->red, s, r))) return rc;
        a = r[0];
        b2 = r[1] - 2.0 * a * a + a * a * r[2];
        pend = b2 > 1e-6 * r[1];
    } else {
        if ((rc = launch_dot(H, g, f, H->D, dtype, H->red, s))) return rc;
        if ((rc = reduce_partials_host(H->red, s, &a))) return rc;
    }
    if (!pend) {
        if ((rc = launch_axpy_nrm2(-a, f, g, H->D, dtype, H->red, s))) return rc;
        if ((rc = reduce_partials_host(H->red, s, &b2))) return rc;
    }
    const double b = std::sqrt(std::max(b2, 0.0));
    if (normalise && b > 0.0) {
        if (pend) rc = launch_axpy_scale(-a, 1.0 / b, f, g, H->D, dtype, s);
        else rc = launch_scale(1.0 / b, g, H->D, dtype, s);
        if (rc) return rc;
        pend = false;
    } else if (normalise && pend) {
        if ((rc = launch_axpy_nrm2(-a, f, g, H->D, dtype, H->red, s))) return rc;
        pend = false;
    }
    if (pending != nullptr) *pending = pend;
    *alpha = a;
    *beta_next = b;
    return HUB_OK;
}

int hubbard_lanczos_step(hubbard_t H, const void* f, void* g, double beta_j, int dtype, void* stream,
                         double* alpha, double* beta_next) {
    clear_error();
    int rc = check_apply(H, f, g, dtype);
    if (rc) return rc;
    if (alpha == nullptr || beta_next == nullptr) return fail(HUB_EINVAL, "null output");
    if ((rc = ensure_fx_scratch(H))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = lanczos_step_impl(H, f, g, beta_j, dtype, s, alpha, beta_next, true, 0);
    if (rc == HUB_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "lanczos step");
    }
    return rc;
}

size_t lanczos_workspace_bytes(hubbard_t H, int dtype) {
    if (H == nullptr || (dtype != HUB_F64 && dtype != HUB_F32)) return 0;
    const size_t vec = align_up((size_t)H->D * elem_size(dtype), 256);
    // two Lanczos vectors + the H*v scratch (binary64: int64 row sums + fixed-point copy)
    return 2 * vec + align_up((size_t)H->D * 16, 256);
}

// Algorithm 1 in the two-vector form on caller buffers f, g (D elements of
// dtype each; the handle's H*v scratch must already point at 16 D bytes).
// f receives v0 / |v0| (v0 of dtype v0_dtype; binary64 -> binary32 allowed).
// Returns the a_j, b_{j+1} sequences and the lowest Ritz value.
struct LanczosRun {
    std::vector<double> a, b;
    double theta = 0.0, rho = 0.0;
    bool broke = false, converged = false;
};

// A caller's own stop test, run after each recorded step (in place of the
// residual tests, which then need tol = rel_tol = 0); true ends the run.
using LanczosStop = std::function<bool(const LanczosRun&)>;

// store (optional): f_j is also copied to store + j * store_stride bytes for
// j < store_cap (the Ritz vector is then one pass over the stored vectors).
static int lanczos_core_host(hubbard_t H, const void* v0, int v0_dtype, int max_iters, double tol, int dtype,
                             void* f, void* g, cudaStream_t s, LanczosRun& R, double rel_tol, char* store,
                             size_t store_stride, int store_cap, const LanczosStop* stop);

// The handle's device-resident Lanczos control block and a/b history for
// cap steps (grown on demand; freed with the handle).
static int ensure_lz(hubbard_sector* H, int cap) {
    if (H->lz != nullptr && H->lz_cap >= cap) return HUB_OK;
    dev_free(H->lz, H->mem_stream);
    H->lz = nullptr;
    H->lz_cap = 0;
    const size_t bytes = 256 + 2 * (size_t)cap * sizeof(double);
    cudaError_t e = dev_alloc(&H->lz, bytes, H->mem_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(Lanczos control)");
    H->lz_cap = cap;
    return HUB_OK;
}

// Records step m-1 (a_m, b_{m+1} appended to R) and applies the run's stop
// tests in the order of Algorithm 1's loop; returns true when the run ends.
static bool lanczos_record_step(LanczosRun& R, double aj, double bn, double tol, double rel_tol,
                                const LanczosStop* stop = nullptr) {
    R.a.push_back(aj);
    double s_last = 1.0;
    tridiag_lowest(R.a.data(), R.b.data(), (int)R.a.size(), &R.theta, &s_last);
    R.rho = bn * std::fabs(s_last);
    double scale = 1.0;
    for (double x : R.a) scale = std::max(scale, std::fabs(x));
    for (double x : R.b) scale = std::max(scale, x);
    R.b.push_back(bn);
    if (bn <= 1e-13 * scale) {
        R.broke = true;
        R.converged = true;
        return true;
    }
    if ((tol > 0.0 && R.rho < tol) || (rel_tol > 0.0 && R.rho < rel_tol * std::max(1.0, std::fabs(R.theta)))) {
        R.converged = true;
        return true;
    }
    if (stop != nullptr && (*stop)(R)) {
        R.converged = true;
        return true;
    }
    return false;
}

// Algorithm 1 in the two-vector form on caller buffers f, g (D elements of
// dtype each; the handle's H*v scratch must already point at 16 D bytes).
// f receives v0 / |v0| (v0 of dtype v0_dtype; binary64 -> binary32 allowed).
// store (optional): f_j is also copied to store + j * store_stride bytes for
// j < store_cap (the Ritz vector is then one pass over the stored vectors).
//
// Device-resident: every step's scalars (beta_j for the H*v, the deferred
// update's coefficients, a_j and b_{j+1}) are formed and consumed on the
// device (k_lz_finish, k_lz_finish2), so steps are enqueued in chunks with no
// host round trip inside a chunk; after each chunk the recorded a_j, b_{j+1}
// come back and the host runs the tridiagonal stop test on every step of it,
// in order.  A chunk can run a few steps past the one that stops the run:
// those steps only overwrite f, g (and stored vectors past it), never the
// recorded values of the steps before.  The kernels and roundings are those of
// the host-driven step, so the a_j, b_{j+1} are the same bit for bit.
// Chunks are longer for small sectors (where a round trip costs more than a
// step); sectors of more than 2.7e6 elements (one step per chunk) and those
// whose H*v kernels do not fuse the reductions take the host-driven loop.
// steps per chunk of the device-resident loop: about 4e6 / D (a round trip is
// worth a few steps of a small sector)
static int lanczos_chunk(hubbard_t H) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)(4e6 / (double)H->D)));
}

// whether lanczos_core takes the host-driven loop: one step per round trip
// gains nothing over it (its explicit branch costs no launches when unused;
// same results either way), and it needs fused reductions and the scratch
static bool lanczos_host_driven(hubbard_t H, int dtype) {
    return lanczos_chunk(H) == 1 || !hv_phases_fuse(H, dtype) || H->fx_bytes < (size_t)H->D * 16;
}

static int lanczos_core(hubbard_t H, const void* v0, int v0_dtype, int max_iters, double tol, int dtype, void* f,
                        void* g, cudaStream_t s, LanczosRun& R, double rel_tol = 0.0, char* store = nullptr,
                        size_t store_stride = 0, int store_cap = 0, const LanczosStop* stop = nullptr) {
    const int chunk = lanczos_chunk(H);
    if (lanczos_host_driven(H, dtype))
        return lanczos_core_host(H, v0, v0_dtype, max_iters, tol, dtype, f, g, s, R, rel_tol, store, store_stride,
                                 store_cap, stop);
    int rc;
    const int m_cap = (int)std::min<int64_t>(max_iters, H->D);
    if ((rc = ensure_lz(H, m_cap))) return rc;
    LzDev* dv = reinterpret_cast<LzDev*>(H->lz);
    double* ha = reinterpret_cast<double*>((char*)H->lz + 256);
    double* hb = ha + H->lz_cap;
    double n0 = 0.0;
    if ((rc = launch_dot(H, v0, v0, H->D, v0_dtype, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0))) return rc;
    n0 = std::sqrt(n0);
    if (!(n0 > 0.0) || !std::isfinite(n0)) return fail(HUB_EINVAL, "start vector has zero or non-finite norm");
    if (v0_dtype == dtype) rc = launch_copy_normalise(v0, f, H->D, dtype, 1.0 / n0, s);
    else rc = launch_f64_to_f32_scaled((const double*)v0, (float*)f, H->D, 1.0 / n0, s);
    if (rc) return rc;
    const size_t vbytes = (size_t)H->D * elem_size(dtype);
    if (store_cap > 0 && cudaMemcpyAsync(store, f, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(HUB_ECUDA, "store f_0");
    if (cudaMemsetAsync(g, 0, vbytes, s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
    const LzDev init{0.0, 0.0, 1.0, 0.0, 0, 1, {0, 0}};
    if (cudaMemcpyAsync(dv, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(HUB_ECUDA, "Lanczos control upload");
    std::vector<double> ab(2 * (size_t)chunk);
    // one Lanczos step: g <- H f_j - b_j g with f_j completed from the previous
    // step inside the row phase, then the explicit branch (a no-op when fused)
    auto step = [&](void* fj, void* gj, bool first, uint64_t& launches, cudaStream_t st) -> int {
        const uint64_t c0 = hubbard_kernel_launches();
        RowUpdate upd{gj, 0.0, 1.0, dv};
        bool fused = false;
        int r = launch_hv_fast(H, fj, gj, dtype, 0.0, gj, 1023, st, H->red, &fused, first ? nullptr : &upd, dv, ha, hb);
        if (r == HUB_OK && !fused) r = fail(HUB_ECUDA, "device-resident Lanczos: fused reductions unavailable");
        if (r == HUB_OK) r = launch_lz_explicit(dv, fj, gj, H->D, dtype, H->red, hb, st);
        launches = hubbard_kernel_launches() - c0;
        return r;
    };
    // Small sectors are bound by kernel launches: with no vectors to store, the
    // steps of either parity (f, g or g, f) are the same launches every time, so
    // each is captured once as a CUDA graph (after one step run directly, which
    // also settles every kernel attribute) and replayed on the caller's stream.
    // Capture runs on a private stream (the legacy default stream cannot be
    // captured); nothing executes during capture.
    bool graphs = chunk > 1 && store_cap == 0 && m_cap > 4 && hv_phases_capturable(H, dtype);
    cudaGraphExec_t gx[2] = {nullptr, nullptr};
    uint64_t glaunch[2] = {0, 0};
    cudaStream_t cap = nullptr;
    if (graphs && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        graphs = false;
    }
    struct GraphGuard {
        cudaGraphExec_t* g;
        cudaStream_t cap;
        ~GraphGuard() {
            for (int i = 0; i < 2; ++i)
                if (g[i]) cudaGraphExecDestroy(g[i]);
            if (cap) cudaStreamDestroy(cap);
        }
    } gguard{gx, cap};
    int j = 0;
    bool done = false;
    while (!done && j < m_cap) {
        const int j0 = j;
        const int j1 = std::min(m_cap, j0 + chunk);
        for (; j < j1; ++j) {
            const int par = j & 1;
            if (graphs && j >= 1 && gx[par] == nullptr) {
                cudaGraph_t gr = nullptr;
                const cudaError_t e0 = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e0 != cudaSuccess) return cuda_fail(e0, "Lanczos step capture");
                uint64_t n = 0;
                const int r = step(f, g, false, n, cap);
                const cudaError_t e = cudaStreamEndCapture(cap, &gr);
                if (r != HUB_OK) {
                    if (gr) cudaGraphDestroy(gr);
                    return r;
                }
                if (e != cudaSuccess) return cuda_fail(e, "Lanczos step capture");
                const cudaError_t e2 = cudaGraphInstantiate(&gx[par], gr, 0);
                cudaGraphDestroy(gr);
                if (e2 != cudaSuccess) return cuda_fail(e2, "Lanczos step graph");
                glaunch[par] = n;
                count_launches(-(int)n);              // captured, not run: counted at each replay
            }
            if (graphs && j >= 1) {
                if (cudaGraphLaunch(gx[par], s) != cudaSuccess) return fail(HUB_ECUDA, "Lanczos step graph launch");
                count_launches((int)glaunch[par]);
            } else {
                uint64_t n = 0;
                if ((rc = step(f, g, j == 0, n, s))) return rc;
            }
            // f holds the final f_j from here on
            if (j >= 1 && j < store_cap &&
                cudaMemcpyAsync(store + (size_t)j * store_stride, f, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return fail(HUB_ECUDA, "store f_j");
            std::swap(f, g);
        }
        // the recorded a_j, b_{j+1} of the chunk, then the stop tests step by step
        if (cudaMemcpyAsync(ab.data(), ha + j0, (size_t)(j1 - j0) * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(ab.data() + chunk, hb + j0, (size_t)(j1 - j0) * sizeof(double), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return fail(HUB_ECUDA, "Lanczos history download");
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "lanczos synchronise");
        for (int q = 0; q < j1 - j0 && !done; ++q)
            done = lanczos_record_step(R, ab[(size_t)q], ab[(size_t)chunk + q], tol, rel_tol, stop);
    }
    if (tol <= 0.0 && rel_tol <= 0.0) R.converged = true;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "lanczos synchronise");
    return HUB_OK;
}

static int lanczos_core_host(hubbard_t H, const void* v0, int v0_dtype, int max_iters, double tol, int dtype,
                             void* f, void* g, cudaStream_t s, LanczosRun& R, double rel_tol, char* store,
                             size_t store_stride, int store_cap, const LanczosStop* stop) {
    int rc;
    double n0 = 0.0;
    if ((rc = launch_dot(H, v0, v0, H->D, v0_dtype, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0))) return rc;
    n0 = std::sqrt(n0);
    if (!(n0 > 0.0) || !std::isfinite(n0)) return fail(HUB_EINVAL, "start vector has zero or non-finite norm");
    if (v0_dtype == dtype) rc = launch_copy_normalise(v0, f, H->D, dtype, 1.0 / n0, s);
    else rc = launch_f64_to_f32_scaled((const double*)v0, (float*)f, H->D, 1.0 / n0, s);
    if (rc) return rc;
    const size_t vbytes = (size_t)H->D * elem_size(dtype);
    if (store_cap > 0 && cudaMemcpyAsync(store, f, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(HUB_ECUDA, "store f_0");
    if (cudaMemsetAsync(g, 0, (size_t)H->D * elem_size(dtype), s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
    const int m_cap = (int)std::min<int64_t>(max_iters, H->D);
    double bj = 0.0;
    // f_{j+1} = (g - a_j f_j) / b_{j+1} is left to the next step's row phase,
    // which completes it while staging its rows
    RowUpdate upd{};
    bool have_upd = false;
    for (int j = 0; j < m_cap; ++j) {
        double aj = 0.0, bn = 0.0;
        bool pending = false;
        if ((rc = lanczos_step_impl(H, f, g, bj, dtype, s, &aj, &bn, false, 1023, &pending,
                                    have_upd ? &upd : nullptr)))
            return rc;
        have_upd = false;
        // f holds the final f_j from here on
        if (j >= 1 && j < store_cap &&
            cudaMemcpyAsync(store + (size_t)j * store_stride, f, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(HUB_ECUDA, "store f_j");
        if (lanczos_record_step(R, aj, bn, tol, rel_tol, stop)) break;
        if (pending) {
            upd = RowUpdate{f, -aj, 1.0 / bn};
            have_upd = true;
        } else if ((rc = launch_scale(1.0 / bn, g, H->D, dtype, s))) {
            return rc;
        }
        std::swap(f, g);
        bj = bn;
    }
    if (tol <= 0.0 && rel_tol <= 0.0) R.converged = true;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "lanczos synchronise");
    return HUB_OK;
}

// points the handle's H*v scratch at a caller region for the duration of a call
struct ScratchGuard {
    hubbard_sector* H;
    void* p;
    size_t n;
    ScratchGuard(hubbard_sector* h, void* region, size_t bytes) : H(h), p(h->fx_scratch), n(h->fx_bytes) {
        H->fx_scratch = region;
        H->fx_bytes = bytes;
    }
    ~ScratchGuard() {
        H->fx_scratch = p;
        H->fx_bytes = n;
    }
};

// psi <- (init ? 0 : psi) + s f for a Lanczos vector f of dtype
static int psi_accumulate(const void* f, int dtype, double* psi, int64_t n, double sj, bool init, cudaStream_t s) {
    if (dtype == HUB_F64) return launch_psi_accumulate_f64((const double*)f, psi, n, sj, init, s);
    return launch_psi_accumulate((const float*)f, psi, n, sj, init, s);
}

// Ritz vector psi = sum_j s_j f_j (binary64, accumulated in j order) of a
// finished lanczos_core run, by replaying its recurrence: f_0 = v0 / |v0| as
// in the run, then g <- H f_j - b_j g with the recorded b_j, and f_{j+1} =
// (g - a_j f_j) / b_{j+1} completed inside the next H*v (the run's own
// kernels with the same operands, hence the same f_j bit for bit).  f, g:
// two vectors of dtype; psi is normalised on return.
static int replay_ritz_vector(hubbard_t H, const void* v0, int v0_dtype, int dtype, const LanczosRun& R,
                              const std::vector<double>& sv, void* f, void* g, double* psi, cudaStream_t s) {
    int rc;
    const int m = (int)R.a.size();
    double n0 = 0.0;
    if ((rc = launch_dot(H, v0, v0, H->D, v0_dtype, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0)))
        return rc;
    if (v0_dtype == dtype) rc = launch_copy_normalise(v0, f, H->D, dtype, 1.0 / std::sqrt(n0), s);
    else rc = launch_f64_to_f32_scaled((const double*)v0, (float*)f, H->D, 1.0 / std::sqrt(n0), s);
    if (rc) return rc;
    if (cudaMemsetAsync(g, 0, (size_t)H->D * elem_size(dtype), s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
    if ((rc = psi_accumulate(f, dtype, psi, H->D, sv[0], true, s))) return rc;
    RowUpdate ru{};
    bool have = false;
    for (int j = 0; j + 1 < m; ++j) {
        const double bj = j == 0 ? 0.0 : R.b[(size_t)j - 1];
        if ((rc = launch_hv_fast(H, f, g, dtype, bj, g, 1023, s, nullptr, nullptr, have ? &ru : nullptr))) return rc;
        if (have && (rc = psi_accumulate(f, dtype, psi, H->D, sv[(size_t)j], false, s))) return rc;
        ru = RowUpdate{f, -R.a[(size_t)j], 1.0 / R.b[(size_t)j]};
        have = true;
        std::swap(f, g);
    }
    if (have) {
        if ((rc = launch_axpy_scale(ru.a, ru.inv, ru.fo, f, H->D, dtype, s))) return rc;
        if ((rc = psi_accumulate(f, dtype, psi, H->D, sv[(size_t)m - 1], false, s))) return rc;
    }
    double pn = 0.0;
    if ((rc = launch_dot(H, psi, psi, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &pn))) return rc;
    return launch_scale(1.0 / std::sqrt(pn), psi, H->D, HUB_F64, s);
}

int lanczos_ground_state(hubbard_t H, const void* v0, int max_iters, double tol, int dtype, void* workspace,
                         size_t ws_bytes, void* psi_out, void* stream, double* alpha_out, double* beta_out,
                         lanczos_result* out) {
    clear_error();
    int rc;
    if ((rc = check_handle(H))) return rc;
    if ((rc = check_dtype(dtype))) return rc;
    if (out == nullptr) return fail(HUB_EINVAL, "out is null");
    std::memset(out, 0, sizeof(*out));
    if (v0 == nullptr || !aligned16(v0)) return fail(HUB_EINVAL, "v0 null or not 16-byte aligned");
    if (max_iters < 1) return fail(HUB_EINVAL, "max_iters must be >= 1");
    if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return fail(HUB_EINVAL, "workspace null or not 256-byte aligned");
    if (ws_bytes < lanczos_workspace_bytes(H, dtype)) return fail(HUB_ENOMEM, "workspace too small");
    if (dtype == HUB_F64 && !fixed_point_ok(H))
        return fail(HUB_EINVAL, "lanczos: more than 127 hops per state is not supported");
    if (psi_out != nullptr) {
        if (!aligned16(psi_out)) return fail(HUB_EINVAL, "psi_out not 16-byte aligned");
        const char* p = (const char*)psi_out;
        const char* w0 = (const char*)workspace;
        if (p < w0 + ws_bytes && w0 < p + (size_t)H->D * 8) return fail(HUB_EINVAL, "psi_out overlaps the workspace");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vec = align_up((size_t)H->D * elem_size(dtype), 256);
    char* ws = (char*)workspace;
    ScratchGuard guard(H, ws + 2 * vec, (size_t)H->D * 16);
    LanczosRun R;
    if ((rc = lanczos_core(H, v0, dtype, max_iters, tol, dtype, ws, ws + vec, s, R))) return rc;
    const int m = (int)R.a.size();
    if (alpha_out) std::memcpy(alpha_out, R.a.data(), m * sizeof(double));
    if (beta_out) std::memcpy(beta_out, R.b.data(), m * sizeof(double));
    const double gap = tridiag_gap_lower(R.a.data(), R.b.data(), m, R.b.back(), R.theta);
    if (psi_out != nullptr) {
        std::vector<double> sv((size_t)m);
        double th = 0.0;
        tridiag_lowest_vector(R.a.data(), R.b.data(), m, &th, sv.data());
        if ((rc = replay_ritz_vector(H, v0, dtype, dtype, R, sv, ws, ws + vec, (double*)psi_out, s))) return rc;
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "lanczos synchronise");
    }
    out->energy = R.theta;
    out->residual = R.rho;
    out->err_bound = energy_error_bound(R.rho, gap) +
                     rounding_floor(H->host[0].W + H->host[1].W + 1, dtype, tridiag_scale(R.a.data(), R.b.data(), m));
    out->iters = m;
    out->breakdown = R.broke ? 1 : 0;
    out->status = R.converged ? HUB_OK : HUB_ENOTCONV;
    if (!R.converged) return fail(HUB_ENOTCONV, "max_iters reached before the residual test passed");
    return HUB_OK;
}

// binary64 Lanczos steps of the refined solver's polish (at most)
constexpr int kPolishSteps = 150;

size_t lanczos_refined_workspace_bytes(hubbard_t H) {
    if (H == nullptr) return 0;
    const size_t D = (size_t)H->D;
    // psi (8D) | H*v scratch (16D) | w (8D) | f, g binary32 (4D + 4D)
    return align_up(D * 8, 256) + align_up(D * 16, 256) + align_up(D * 8, 256) + 2 * align_up(D * 4, 256);
}

int lanczos_ground_state_refined(hubbard_t H, const void* v0, int max_iters, double tol, void* workspace,
                                 size_t ws_bytes, void* psi_out, void* stream, lanczos_refined_result* out) {
    clear_error();
    int rc;
    if ((rc = check_handle(H))) return rc;
    if (out == nullptr) return fail(HUB_EINVAL, "out is null");
    std::memset(out, 0, sizeof(*out));
    if (v0 == nullptr || !aligned16(v0)) return fail(HUB_EINVAL, "v0 null or not 16-byte aligned");
    if (psi_out != nullptr && !aligned16(psi_out)) return fail(HUB_EINVAL, "psi_out not 16-byte aligned");
    if (max_iters < 1) return fail(HUB_EINVAL, "max_iters must be >= 1");
    if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return fail(HUB_EINVAL, "workspace null or not 256-byte aligned");
    if (ws_bytes < lanczos_refined_workspace_bytes(H)) return fail(HUB_ENOMEM, "workspace too small");
    if (!fixed_point_ok(H)) return fail(HUB_EINVAL, "refined lanczos: more than 127 hops per state");
    if (!(tol > 0.0)) tol = 1e-10;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t D = (size_t)H->D;
    char* ws = (char*)workspace;
    double* psi = (double*)ws;
    char* scr = ws + align_up(D * 8, 256);
    double* w = (double*)(scr + align_up(D * 16, 256));
    float* f = (float*)((char*)w + align_up(D * 8, 256));
    float* g = (float*)((char*)f + align_up(D * 4, 256));
    ScratchGuard guard(H, scr, D * 16);
    // workspace beyond the minimum stores the binary32 Lanczos vectors
    const size_t base_bytes = lanczos_refined_workspace_bytes(H);
    const size_t slot = align_up(D * 4, 256);
    const int store_cap = (int)std::min<size_t>((ws_bytes - base_bytes) / slot, (size_t)kRedSlots);
    char* store = ws + base_bytes;

    // 1. binary32 Lanczos: stop when the Ritz estimate reaches binary32 level
    LanczosRun R;
    if ((rc = lanczos_core(H, v0, HUB_F64, max_iters, 0.0, HUB_F32, f, g, s, R, 2e-6, store, slot, store_cap)))
        return rc;
    const int m = (int)R.a.size();
    std::vector<double> sv((size_t)m);
    double theta32 = 0.0;
    tridiag_lowest_vector(R.a.data(), R.b.data(), m, &theta32, sv.data());
    // lower estimate of lambda_2 - E0: the second distinct Ritz value minus its
    // Ritz residual (a Ritz value alone bounds lambda_2 only from above)
    const double gap = tridiag_gap_lower(R.a.data(), R.b.data(), m, R.b.back(), theta32);
    out->energy_f32 = theta32;
    out->iters_f32 = m;
    out->gap = gap;

    // 2. Ritz vector psi = sum_j s_j f_j in binary64, accumulated in j order:
    //    one pass over the k = min(m, store_cap) stored f_j, then (k < m) a
    //    replay of the same binary32 recurrence with the stored a, b from the
    //    last two stored vectors (every kernel is deterministic, so the f_j
    //    and psi are bit-identical whatever k is)
    const int k = std::min(m, store_cap);
    if (k >= 1) {
        if (cudaMemcpyAsync(H->red, sv.data(), (size_t)k * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(HUB_ECUDA, "upload s");
        if ((rc = launch_psi_multi((const float*)store, (int64_t)(slot / 4), k, H->red, psi, H->D, s))) return rc;
    }
    out->replayed = m - std::max(k, 1);
    if (k < m) {
        float* ff = f;
        float* gg = g;
        int j0 = 0;
        if (k >= 2) {
            // resume from the stored f_{k-2}, f_{k-1}
            if (cudaMemcpyAsync(ff, store + (size_t)(k - 1) * slot, D * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(gg, store + (size_t)(k - 2) * slot, D * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return fail(HUB_ECUDA, "resume from stored vectors");
            j0 = k - 1;
        } else {
            double n0 = 0.0;
            if ((rc = launch_dot(H, v0, v0, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0)))
                return rc;
            if ((rc = launch_f64_to_f32_scaled((const double*)v0, ff, H->D, 1.0 / std::sqrt(n0), s))) return rc;
            if (cudaMemsetAsync(gg, 0, D * 4, s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
            if (k == 0 && (rc = launch_psi_accumulate(ff, psi, H->D, sv[0], true, s))) return rc;
        }
        // each update f_{j+1} = (g - a_j f_j) / b_{j+1} is completed by the next
        // step's row phase (same roundings as launch_axpy_scale), the last one
        // by a pass of its own
        RowUpdate ru{};
        bool have = false;
        for (int j = j0; j + 1 < m; ++j) {
            const double bj = j == 0 ? 0.0 : R.b[(size_t)j - 1];
            if ((rc = launch_hv_fast(H, ff, gg, HUB_F32, bj, gg, 1023, s, nullptr, nullptr, have ? &ru : nullptr)))
                return rc;
            if (have && (rc = launch_psi_accumulate(ff, psi, H->D, sv[(size_t)j], false, s))) return rc;
            ru = RowUpdate{ff, -R.a[(size_t)j], 1.0 / R.b[(size_t)j]};
            have = true;
            std::swap(ff, gg);
        }
        if (have) {
            if ((rc = launch_axpy_scale(ru.a, ru.inv, ru.fo, ff, H->D, HUB_F32, s))) return rc;
            if ((rc = launch_psi_accumulate(ff, psi, H->D, sv[(size_t)m - 1], false, s))) return rc;
        }
    }
    double pn = 0.0;
    if ((rc = launch_dot(H, psi, psi, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &pn))) return rc;
    if ((rc = launch_scale(1.0 / std::sqrt(pn), psi, H->D, HUB_F64, s))) return rc;
    if (psi_out != nullptr)
        if (cudaMemcpyAsync(psi_out, psi, D * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(HUB_ECUDA, "copy psi");

    // 3. binary64 Rayleigh quotient and residual of psi (|psi| = 1)
    if ((rc = launch_hv_fast(H, psi, w, HUB_F64, 0.0, nullptr, 0, s))) return rc;
    double th = 0.0, r2 = 0.0;
    if ((rc = launch_dot(H, psi, w, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &th))) return rc;
    if ((rc = launch_axpy_nrm2(-th, psi, w, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &r2)))
        return rc;
    out->energy = th;
    out->residual = std::sqrt(std::max(r2, 0.0));
    const double floor64 = rounding_floor(H->host[0].W + H->host[1].W + 1, HUB_F64,
                                          std::max(1.0, std::fabs(th) + out->residual));
    out->error_bound = energy_error_bound(out->residual, gap) + floor64;
    out->iters_f64 = 0;

    // 4. short binary64 Lanczos polish from psi when the bound misses tol * |theta|
    if (!(out->error_bound <= tol * std::max(1.0, std::fabs(th)))) {
        // polish workspace: f, g (binary64) over [scratch .. end], scratch after them
        char* base = scr;
        double* pf = (double*)base;
        double* pg = (double*)(base + align_up(D * 8, 256));
        char* pscr = base + 2 * align_up(D * 8, 256);
        if (2 * align_up(D * 8, 256) + D * 16 > (size_t)((char*)workspace + ws_bytes - base))
            return fail(HUB_ENOMEM, "workspace too small for the binary64 polish");
        ScratchGuard g2(H, pscr, D * 16);
        LanczosRun P;
        // stop as soon as the bound meets tol: rho^2 / gap when a gap is
        // resolved, else rho itself
        // target: the bound (quadratic part plus the rounding floor) at half of
        // tol; the gap stays the binary32 run's (a polish started from psi
        // resolves little of lambda_2: its second Ritz pair overestimated the
        // gap threefold in a test)
        const double want = tol * std::max(1.0, std::fabs(th));
        const double rho_target = gap > 0.0 ? std::sqrt(0.5 * want * gap / kGapSafety) : 0.5 * want;
        if ((rc = lanczos_core(H, psi, HUB_F64, kPolishSteps, rho_target, HUB_F64, pf, pg, s, P))) return rc;
        const int mp = (int)P.a.size();
        out->energy = P.theta;
        out->residual = P.rho;
        out->error_bound = energy_error_bound(P.rho, gap) +
                           rounding_floor(H->host[0].W + H->host[1].W + 1, HUB_F64,
                                          tridiag_scale(P.a.data(), P.b.data(), mp));
        out->iters_f64 = mp;
    }
    out->status = (out->error_bound <= tol * std::max(1.0, std::fabs(out->energy))) ? HUB_OK : HUB_ENOTCONV;
    if (out->status != HUB_OK) return fail(HUB_ENOTCONV, "refined energy bound above tol");
    return HUB_OK;
}

}  // extern "C"

// ---- time propagation (Sec. 6: the other use of H*v; short iterative Lanczos) ----

// Algorithm 1 (binary64, host-driven) with the Lanczos vectors kept in the
// stored basis itself: f_j is slot j (store + j * stride bytes) from the
// start, step j writes H f_j - b_j f_{j-1} into slot j+1 (into spare past the
// last slot) and reads f_{j-1} from slot j-1, and the next step's row phase
// completes that slot into f_{j+1} in place, so no vector is copied.  The
// kernels and their operands are those of lanczos_core_host (per element the
// same operations whether or not w_old is the output vector), hence the same
// a_j, b_{j+1} and f_j bit for bit.  At most `slots` steps.
static int lanczos_core_in_store(hubbard_t H, const void* v0, int slots, char* store, size_t stride, void* spare,
                                 cudaStream_t s, LanczosRun& R, const LanczosStop* stop) {
    int rc;
    double n0 = 0.0;
    if ((rc = launch_dot(H, v0, v0, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0))) return rc;
    n0 = std::sqrt(n0);
    if (!(n0 > 0.0) || !std::isfinite(n0)) return fail(HUB_EINVAL, "start vector has zero or non-finite norm");
    auto slot = [&](int j) -> void* { return j < slots ? (void*)(store + (size_t)j * stride) : spare; };
    if ((rc = launch_copy_normalise(v0, slot(0), H->D, HUB_F64, 1.0 / n0, s))) return rc;
    if (cudaMemsetAsync(slot(1), 0, (size_t)H->D * 8, s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
    const int m_cap = (int)std::min<int64_t>(slots, H->D);
    double bj = 0.0;
    RowUpdate upd{};
    bool have_upd = false;
    for (int j = 0; j < m_cap; ++j) {
        void* f = slot(j);
        void* w = slot(j + 1);
        const void* w_old = j == 0 ? w : slot(j - 1);
        double aj = 0.0, bn = 0.0;
        bool pending = false;
        if ((rc = lanczos_step_impl(H, f, w, bj, HUB_F64, s, &aj, &bn, false, 1023, &pending,
                                    have_upd ? &upd : nullptr, w_old)))
            return rc;
        have_upd = false;
        if (lanczos_record_step(R, aj, bn, 0.0, 0.0, stop)) break;
        if (pending) {
            upd = RowUpdate{f, -aj, 1.0 / bn};
            have_upd = true;
        } else if ((rc = launch_scale(1.0 / bn, w, H->D, HUB_F64, s))) {
            return rc;
        }
        bj = bn;
    }
    R.converged = true;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "lanczos synchronise");
    return HUB_OK;
}

// A <- A + sum_j ca_j f_j, B <- B + sum_j cb_j f_j over the Lanczos vectors of a
// finished lanczos_core run from p, by replaying its recurrence as
// replay_ritz_vector does (same kernels and operands, hence the same f_j bit
// for bit); the accumulation is the one launch_combine2_f64 does over stored
// vectors, so both routes give the same A, B.
static int replay_combine2(hubbard_t H, const void* p, const LanczosRun& R, const std::vector<double>& ca,
                           const std::vector<double>& cb, double* A, double* B, void* f, void* g, cudaStream_t s) {
    int rc;
    const int m = (int)R.a.size();
    double n0 = 0.0;
    if ((rc = launch_dot(H, p, p, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &n0))) return rc;
    if ((rc = launch_copy_normalise(p, f, H->D, HUB_F64, 1.0 / std::sqrt(n0), s))) return rc;
    if (cudaMemsetAsync(g, 0, (size_t)H->D * 8, s) != cudaSuccess) return fail(HUB_ECUDA, "memset");
    if ((rc = launch_acc2_f64((const double*)f, A, B, H->D, ca[0], cb[0], s))) return rc;
    RowUpdate ru{};
    bool have = false;
    for (int j = 0; j + 1 < m; ++j) {
        const double bj = j == 0 ? 0.0 : R.b[(size_t)j - 1];
        if ((rc = launch_hv_fast(H, f, g, HUB_F64, bj, g, 1023, s, nullptr, nullptr, have ? &ru : nullptr))) return rc;
        if (have && (rc = launch_acc2_f64((const double*)f, A, B, H->D, ca[(size_t)j], cb[(size_t)j], s))) return rc;
        ru = RowUpdate{f, -R.a[(size_t)j], 1.0 / R.b[(size_t)j]};
        have = true;
        std::swap(f, g);
    }
    if (have) {
        if ((rc = launch_axpy_scale(ru.a, ru.inv, ru.fo, f, H->D, HUB_F64, s))) return rc;
        if ((rc = launch_acc2_f64((const double*)f, A, B, H->D, ca[(size_t)m - 1], cb[(size_t)m - 1], s))) return rc;
    }
    return HUB_OK;
}

static size_t evolve_vec_bytes(hubbard_t H) { return align_up((size_t)H->D * 8, 256); }

extern "C" {

size_t hubbard_evolve_workspace_bytes(hubbard_t H, int krylov_max, int store_basis) {
    if (H == nullptr || krylov_max < 1 || krylov_max > 1024) return 0;
    const size_t vec = evolve_vec_bytes(H);
    const int k = (int)std::min<int64_t>(krylov_max, H->D);
    return 6 * vec + (store_basis ? 2 * (size_t)k * vec : 0);
}

int hubbard_time_evolve(hubbard_t H, const void* v_re, const void* v_im, double t, int krylov_max, double tol,
                        void* workspace, size_t ws_bytes, void* out_re, void* out_im, void* stream,
                        hubbard_evolve_info* info) {
    clear_error();
    int rc;
    if (info == nullptr) return fail(HUB_EINVAL, "info is null");
    std::memset(info, 0, sizeof(*info));
    info->status = HUB_EINVAL;
    if ((rc = check_handle(H))) return rc;
    if (v_re == nullptr || !aligned16(v_re) || (v_im != nullptr && !aligned16(v_im)))
        return fail(HUB_EINVAL, "v_re null, or v_re / v_im not 16-byte aligned");
    if (out_re == nullptr || out_im == nullptr || !aligned16(out_re) || !aligned16(out_im))
        return fail(HUB_EINVAL, "out_re / out_im null or not 16-byte aligned");
    if (!std::isfinite(t)) return fail(HUB_EINVAL, "t must be finite");
    if (krylov_max < 1 || krylov_max > 1024) return fail(HUB_EINVAL, "krylov_max must be in 1..1024");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(HUB_EINVAL, "tol must be positive and finite");
    if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return fail(HUB_EINVAL, "workspace null or not 256-byte aligned");
    if (!fixed_point_ok(H)) return fail(HUB_EINVAL, "time evolution: more than 127 hops per state is not supported");
    const size_t vbytes = (size_t)H->D * 8;
    auto overlap = [&](const void* x, size_t nx, const void* y, size_t ny) {
        const char* a = (const char*)x;
        const char* b = (const char*)y;
        return a < b + ny && b < a + nx;
    };
    if (overlap(out_re, vbytes, out_im, vbytes)) return fail(HUB_EINVAL, "out_re and out_im overlap");
    for (const void* q : {v_re, v_im, (const void*)out_re, (const void*)out_im})
        if (q != nullptr && overlap(q, vbytes, workspace, ws_bytes)) return fail(HUB_EINVAL, "a vector overlaps the workspace");
    info->status = HUB_ENOMEM;
    if (ws_bytes < hubbard_evolve_workspace_bytes(H, krylov_max, 0)) return fail(HUB_ENOMEM, "workspace too small");
    info->status = HUB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int kmax = (int)std::min<int64_t>(krylov_max, H->D);
    const size_t vec = evolve_vec_bytes(H);
    char* ws = (char*)workspace;
    void* f = ws;
    void* g = ws + vec;
    ScratchGuard guard(H, ws + 2 * vec, (size_t)H->D * 16);
    double* part[2] = {(double*)(ws + 4 * vec), (double*)(ws + 5 * vec)};   // state: real, imaginary part
    char* store = ws + 6 * vec;
    const bool stored = ws_bytes >= hubbard_evolve_workspace_bytes(H, krylov_max, 1);
    // large sectors (host-driven steps): the recurrence runs in the stored basis, no copies
    const bool in_store = stored && lanczos_host_driven(H, HUB_F64);
    double* A = (double*)out_re;
    double* B = (double*)out_im;

    if (cudaMemcpyAsync(part[0], v_re, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(HUB_ECUDA, "copy v_re");
    bool has_im = v_im != nullptr;
    if (has_im && cudaMemcpyAsync(part[1], v_im, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(HUB_ECUDA, "copy v_im");
    double nn[2] = {0.0, 0.0};
    for (int q = 0; q < (has_im ? 2 : 1); ++q)
        if ((rc = launch_dot(H, part[q], part[q], H->D, HUB_F64, H->red, s)) ||
            (rc = reduce_partials_host(H->red, s, &nn[q])))
            return rc;
    const double nv = std::sqrt(nn[0] + nn[1]);
    if (!std::isfinite(nv)) return fail(HUB_EINVAL, "v has non-finite elements");
    if (t == 0.0 || nv == 0.0) {
        if (cudaMemcpyAsync(A, part[0], vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            (has_im ? cudaMemcpyAsync(B, part[1], vbytes, cudaMemcpyDeviceToDevice, s)
                    : cudaMemsetAsync(B, 0, vbytes, s)) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(HUB_ECUDA, "copy v");
        info->norm = nv;
        return HUB_OK;
    }
    const double tabs = std::fabs(t), sgn = t > 0.0 ? 1.0 : -1.0;
    double rem = tabs;
    constexpr int kMaxSteps = 100000;
    struct Run {
        int q = 0;
        double nu = 0.0;
        LanczosRun R;
        KrylovEnds E;
    };
    while (rem > 0.0) {
        if (info->steps >= kMaxSteps) return fail(HUB_ENOTCONV, "time evolution: too many steps");
        // norms of the parts of the current state; each part's share of the budget
        for (int q = 0; q < 2; ++q) {
            nn[q] = 0.0;
            if (q == 1 && !has_im) continue;
            if ((rc = launch_dot(H, part[q], part[q], H->D, HUB_F64, H->red, s)) ||
                (rc = reduce_partials_host(H->red, s, &nn[q])))
                return rc;
            nn[q] = std::sqrt(nn[q]);
        }
        const double nsum = nn[0] + nn[1];
        std::vector<Run> runs;
        for (int q = 0; q < 2; ++q) {
            if (!(nn[q] > 0.0)) continue;
            Run run;
            run.q = q;
            run.nu = nn[q];
            // budget of this part for a step tau: tol |v| (tau / |t|) (nu / sum of the parts' nu)
            const double share = tol * nv * (nn[q] / nsum) / tabs;
            const double target = rem;
            const LanczosStop stop = [&, share, target](const LanczosRun& Rr) {
                const int m = (int)Rr.a.size();
                if (m % 4 != 0 && m < kmax) return false;
                KrylovEnds E;
                if (!krylov_exp_ends(Rr.a.data(), Rr.b.data(), m, E)) return false;
                return run.nu * Rr.b.back() * krylov_last_coeff(E, sgn * target) <= share * target;
            };
            char* st = stored ? store + (size_t)q * kmax * vec : nullptr;
            if (in_store) rc = lanczos_core_in_store(H, part[q], kmax, st, vec, g, s, run.R, &stop);
            else rc = lanczos_core(H, part[q], HUB_F64, kmax, 0.0, HUB_F64, f, g, s, run.R, 0.0, st, vec,
                                   stored ? kmax : 0, &stop);
            if (rc) return rc;
            const int m = (int)run.R.a.size();
            if (!krylov_exp_ends(run.R.a.data(), run.R.b.data(), m, run.E))
                return fail(HUB_ENOTCONV, "time evolution: tridiagonal QR did not converge");
            info->hv += m;
            info->krylov_dim = std::max(info->krylov_dim, m);
            runs.push_back(std::move(run));
        }
        // the longest step every part's estimate allows
        double tau = rem;
        for (const Run& r : runs) {
            const double share = tol * nv * (r.nu / nsum) / tabs;
            auto est = [&](double x) { return r.nu * r.R.b.back() * krylov_last_coeff(r.E, sgn * x); };
            if (est(tau) <= share * tau) continue;
            double lo = 0.0, hi = tau;
            for (int it = 0; it < 80; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (est(mid) <= share * mid) lo = mid;
                else hi = mid;
            }
            tau = lo;
        }
        // a step shorter than 1e-12 |t| (unless it ends the propagation) means tol cannot be met
        if (!(tau >= std::min(rem, 1e-12 * tabs)) || !(tau > 0.0))
            return fail(HUB_ENOTCONV, "time evolution: tol too strict for krylov_max");
        if (tau > rem) tau = rem;
        // psi(tau) = sum over parts of i^q nu_q sum_j y_j f_j into (A, B)
        if (cudaMemsetAsync(A, 0, vbytes, s) != cudaSuccess || cudaMemsetAsync(B, 0, vbytes, s) != cudaSuccess)
            return fail(HUB_ECUDA, "memset");
        for (const Run& r : runs) {
            const int m = (int)r.R.a.size();
            std::vector<double> yre((size_t)m), yim((size_t)m), ca((size_t)m), cb((size_t)m);
            if (!krylov_exp_coeffs(r.R.a.data(), r.R.b.data(), m, sgn * tau, yre.data(), yim.data()))
                return fail(HUB_ENOTCONV, "time evolution: tridiagonal QR did not converge");
            info->err_estimate += r.nu * r.R.b.back() * std::hypot(yre[(size_t)m - 1], yim[(size_t)m - 1]);
            for (int j = 0; j < m; ++j) {
                // real part: (re, im) += nu (Re y, Im y) f_j; imaginary part: i nu y f_j = nu (-Im y, Re y) f_j
                ca[(size_t)j] = r.nu * (r.q == 0 ? yre[(size_t)j] : -yim[(size_t)j]);
                cb[(size_t)j] = r.nu * (r.q == 0 ? yim[(size_t)j] : yre[(size_t)j]);
            }
            if (stored) {
                std::vector<double> c(2 * (size_t)m);
                std::copy(ca.begin(), ca.end(), c.begin());
                std::copy(cb.begin(), cb.end(), c.begin() + m);
                if (cudaMemcpyAsync(H->red, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess)
                    return fail(HUB_ECUDA, "upload coefficients");
                const double* base = (const double*)(store + (size_t)r.q * kmax * vec);
                if ((rc = launch_combine2_f64(base, (int64_t)(vec / 8), m, H->red, A, B, H->D, s))) return rc;
            } else {
                if ((rc = replay_combine2(H, part[r.q], r.R, ca, cb, A, B, f, g, s))) return rc;
                info->hv += m - 1;
            }
        }
        ++info->steps;
        rem -= tau;
        if (rem <= 1e-15 * tabs) rem = 0.0;
        if (rem > 0.0) {
            if (cudaMemcpyAsync(part[0], A, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(part[1], B, vbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return fail(HUB_ECUDA, "copy state");
            has_im = true;
        }
    }
    double pr = 0.0, pi = 0.0;
    if ((rc = launch_dot(H, A, A, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &pr)) ||
        (rc = launch_dot(H, B, B, H->D, HUB_F64, H->red, s)) || (rc = reduce_partials_host(H->red, s, &pi)))
        return rc;
    info->norm = std::sqrt(pr + pi);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HUB_ECUDA, "time evolution synchronise");
    return HUB_OK;
}

}  // extern "C"
