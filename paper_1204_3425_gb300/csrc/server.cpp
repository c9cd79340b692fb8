// Continuous-batching ground-state server (include/hubbard.h, hubbard_server_*).
//
// Requests (one sector each) are queued by hubbard_server_submit and picked up
// by worker lanes as soon as a lane is free and the request's device-memory
// footprint fits what remains of the budget; results are collected with
// hubbard_server_poll / hubbard_server_wait.  The paper motivates the design
// (Sec. 5): a small sector alone leaves most of the GPU idle, so work from
// many requests has to share the device.
//   * small requests: with a GPU, a prep lane makes their hop tables and one
//     lane posts them, as they arrive, to a queued persistent solver
//     (hubbard_queue_*) whose CTAs take each new sector while they run, and
//     answers what it finishes; without one (host solver) or with
//     small_ctas < 0, every small request waiting when a small lane frees up
//     joins one task-only launch of the batched solver (hubbard_batch_*);
//   * big lanes: one request each, on the lane's own stream -- mid-sized
//     sectors by the binary64 Lanczos (device-resident steps), larger ones by
//     the binary32 Lanczos with binary64 refinement, keeping binary32 Lanczos
//     vectors in spare budget for the Ritz vector.
// Lanes run concurrently on non-blocking streams; every handle, batch and
// buffer a lane creates lives on its stream (stream-ordered allocation), so
// finishing a request never waits for the whole device.
// A request whose solve fails is answered with that status; the others go on.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { kPathBatch = 0, kPathBinary64 = 1, kPathRefined = 2 };

struct Req {
    uint64_t ticket = 0;
    std::vector<int32_t> bonds;
    hubbard_request desc{};
    int64_t D = 0;
    int path = 0;
    size_t footprint = 0;      // bytes held while it runs (stored vectors added at admission)
    int state = 0;             // 0 queued, 1 running, 2 done
    hubbard_served out{};
};

double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

}  // namespace

struct hubbard_server {
    hubbard_server_opts opts{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> small_q, big_q;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    size_t budget = 0, free_bytes = 0, peak = 0;
    hubbard_server_stats st{};
    bool stop = false;
    bool queued_small = false;                 // small requests go to a queued persistent solver
    int queue_cap = 0;                         // its slots
    bool queue_ready = false;                  // its lane has warmed the solver up
    hubbard_queue_t queue = nullptr;
    std::deque<Req*> prep_q;                   // small requests whose hop tables are being made
    std::vector<std::thread> threads;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// bytes a request holds while it runs, without optional stored vectors
size_t base_footprint(const hubbard_server* S, int path, int64_t D) {
    const size_t d = (size_t)D;
    if (path == kPathBatch)                        // v0 + f, g, fixed-point copy, row partials + a/b history
        return 56 * d + 16 * (size_t)S->opts.max_iters + 4096;
    if (path == kPathBinary64)                     // v0 + two vectors + H*v scratch
        return 40 * d + (1u << 20);
    return 48 * d + (1u << 20);                    // v0 + refined workspace (psi, scratch, w, f, g)
}

void take(hubbard_server* S, size_t bytes) {
    S->free_bytes -= bytes;
    S->peak = std::max(S->peak, S->budget - S->free_bytes);
}

void finish(hubbard_server* S, Req* r, const lanczos_result& res, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->out.result = res;
    r->out.result.status = status;
    r->out.t_done = S->now();
    r->state = 2;
    S->free_bytes += r->footprint;
    S->st.running -= 1;
    S->st.completed += 1;
    if (status != HUB_OK) S->st.failed += 1;
    else if (res.err_bound <= 1e-9 * std::max(1.0, std::fabs(res.energy))) S->st.verified += 1;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

// ---- GPU work of the lanes --------------------------------------------------
// stream-ordered allocation aligned to 256 bytes (the solvers' workspace rule)
struct DevBuf {
    void* raw = nullptr;
    char* p = nullptr;
    cudaStream_t st = nullptr;
    bool alloc(size_t bytes, cudaStream_t s) {
        st = s;
        if (cudaMallocAsync(&raw, bytes + 256, s) != cudaSuccess) {
            raw = nullptr;
            return false;
        }
        p = (char*)(((uintptr_t)raw + 255) & ~(uintptr_t)255);
        return true;
    }
    ~DevBuf() {
        if (raw) cudaFreeAsync(raw, st);
    }
};

int solve_batch_gpu(hubbard_server* S, const std::vector<Req*>& batch, cudaStream_t st,
                    std::vector<lanczos_result>& res) {
    std::vector<hubbard_sector_desc> descs(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
        const hubbard_request& q = batch[i]->desc;
        descs[i] = hubbard_sector_desc{q.ns, q.nup, q.ndn, q.n_bonds, q.bonds, q.t, q.U};
    }
    hubbard_batch_t B = nullptr;
    int rc = hub::batch_create_streamed(descs.data(), (int)descs.size(), st, &B);
    if (rc) return rc;
    std::vector<int64_t> off(batch.size() + 1);
    DevBuf vb, wb;
    const size_t wsb = hubbard_batch_workspace_bytes(B, S->opts.max_iters);
    rc = hubbard_batch_vector_offsets(B, off.data());
    if (rc == HUB_OK && !vb.alloc((size_t)std::max<int64_t>(off.back(), 2) * 8, st))
        rc = hub::fail(HUB_ENOMEM, "server: batch start vectors");
    if (rc == HUB_OK && !wb.alloc(wsb, st)) rc = hub::fail(HUB_ENOMEM, "server: batch workspace");
    double* v0 = (double*)vb.p;
    void* ws = wb.p;
    for (size_t i = 0; rc == HUB_OK && i < batch.size(); ++i)
        rc = hubbard_fill_start_vector(v0 + off[i], batch[i]->D, batch[i]->desc.seed, 0, HUB_F64, st);
    // every sector is a one-CTA task: small micro-batches never start a grid-wide sweep
    if (rc == HUB_OK) rc = hubbard_batch_set_schedule(B, INT64_MAX / 4);
    if (rc == HUB_OK) rc = hubbard_batch_solve_async(B, v0, S->opts.max_iters, S->opts.tol, ws, wsb, st);
    if (rc == HUB_OK) {
        res.assign(batch.size(), lanczos_result{});
        rc = hubbard_batch_results(B, ws, S->opts.max_iters, st, res.data());
    }
    hubbard_batch_destroy(B);
    return rc;
}

int solve_big_gpu(hubbard_server* S, Req* r, size_t store_bytes, cudaStream_t st, lanczos_result& res) {
    const hubbard_request& q = r->desc;
    hubbard_t H = nullptr;
    int rc = hub::sector_create_streamed(q.ns, q.bonds, q.n_bonds, q.nup, q.ndn, q.t, q.U, st, &H);
    if (rc) return rc;
    DevBuf vb, wb;
    if (!vb.alloc((size_t)r->D * 8, st)) rc = hub::fail(HUB_ENOMEM, "server: v0");
    double* v0 = (double*)vb.p;
    if (rc == HUB_OK) rc = hubbard_fill_start_vector(v0, r->D, q.seed, 0, HUB_F64, st);
    if (rc == HUB_OK && r->path == kPathBinary64) {
        const size_t wsb = lanczos_workspace_bytes(H, HUB_F64);
        if (!wb.alloc(wsb, st)) rc = hub::fail(HUB_ENOMEM, "server: workspace");
        void* ws = wb.p;
        // the binary64 solver's absolute test rho < tol (at least as strict as
        // the relative test of the other paths whenever |E0| >= 1)
        if (rc == HUB_OK)
            rc = lanczos_ground_state(H, v0, S->opts.max_iters, S->opts.tol, HUB_F64, ws, wsb, nullptr, st, nullptr,
                                      nullptr, &res);
    } else if (rc == HUB_OK) {
        const size_t wsb = lanczos_refined_workspace_bytes(H) + store_bytes;
        if (!wb.alloc(wsb, st)) rc = hub::fail(HUB_ENOMEM, "server: workspace");
        void* ws = wb.p;
        lanczos_refined_result rr{};
        if (rc == HUB_OK) rc = lanczos_ground_state_refined(H, v0, S->opts.max_iters, S->opts.tol, ws, wsb, nullptr, st, &rr);
        res.energy = rr.energy;
        res.residual = rr.residual;
        res.err_bound = rr.error_bound;
        res.iters = rr.iters_f32 + rr.iters_f64;
        res.status = rr.status;
        res.breakdown = 0;
        if (rc == HUB_ENOTCONV) {
            // the refinement could not certify tol (a gap too small to resolve in
            // its polish): the binary64 Lanczos, in the same workspace, certifies
            // through its own Ritz estimates
            r->out.path = kPathBinary64;
            const int it0 = res.iters;
            rc = lanczos_ground_state(H, v0, S->opts.max_iters, S->opts.tol, HUB_F64, ws, wsb, nullptr, st, nullptr,
                                      nullptr, &res);
            res.iters += it0;
        }
    }
    hubbard_sector_destroy(H);
    return rc;
}

// ---- lanes ------------------------------------------------------------------
void small_lane(hubbard_server* S) {
    cudaStream_t st = nullptr;
    if (!S->opts.host_solver) {
        cudaSetDevice(S->device);
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    }
    while (true) {
        std::vector<Req*> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || (!S->small_q.empty() && S->small_q.front()->footprint <= S->free_bytes);
            });
            if (S->stop) break;
            // every small request that waits, in arrival order, while it fits
            size_t bytes = 0;
            while (!S->small_q.empty() && (int)batch.size() < S->opts.batch_max &&
                   bytes + S->small_q.front()->footprint <= S->free_bytes) {
                Req* r = S->small_q.front();
                S->small_q.pop_front();
                bytes += r->footprint;
                r->state = 1;
                r->out.t_admit = S->now();
                batch.push_back(r);
            }
            take(S, bytes);
            S->st.running += (int64_t)batch.size();
            S->st.batches += 1;
            S->st.batched_requests += (int64_t)batch.size();
        }
        std::vector<lanczos_result> res;
        int rc = HUB_OK;
        if (S->opts.host_solver) {
            res.assign(batch.size(), lanczos_result{});
            for (size_t i = 0; i < batch.size(); ++i) {
                const int ri = S->opts.host_solver(S->opts.host_ctx, batch[i]->ticket, &batch[i]->desc, kPathBatch, &res[i]);
                if (ri != HUB_OK) res[i].status = ri;
            }
        } else {
            rc = solve_batch_gpu(S, batch, st, res);
            cudaStreamSynchronize(st);
        }
        for (size_t i = 0; i < batch.size(); ++i) {
            const lanczos_result ri = rc == HUB_OK ? res[i] : lanczos_result{};
            finish(S, batch[i], ri, rc != HUB_OK ? rc : ri.status);
        }
    }
    if (st) cudaStreamDestroy(st);
}

// The small queue with a GPU: every small request is posted to one queued
// solver as soon as it is taken (its CTAs solve posted sectors while others
// are being posted); finished results are collected and answered.
void queue_lane(hubbard_server* S) {
    cudaSetDevice(S->device);
    hubbard_queue_t Q = S->queue;
    const int qrc = Q != nullptr ? HUB_OK : HUB_ECUDA;
    std::deque<Req*> local;                                   // taken, not yet posted (queue full)
    std::unordered_map<int64_t, Req*> inflight;
    const int kCollect = 256;
    std::vector<int64_t> tks(kCollect);
    std::vector<lanczos_result> rs(kCollect);
    // warm-up: one two-site sector through the solver, so the first requests
    // do not pay for the first launch (create waits for this)
    if (qrc == HUB_OK) {
        const int32_t dimer[2] = {0, 1};
        const hubbard_sector_desc d{2, 1, 1, 1, dimer, 1.0, 0.0};
        int64_t tk = -1;
        if (hubbard_queue_post(Q, &d, 1, &tk) == HUB_OK) {
            const auto end = Clock::now() + std::chrono::seconds(10);
            int n = 0;
            while (Clock::now() < end && hubbard_queue_collect(Q, tks.data(), rs.data(), kCollect, &n) == HUB_OK &&
                   n == 0)
                std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->queue_ready = true;
    }
    S->cv_done.notify_all();
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (inflight.empty() && local.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->small_q.empty(); });
            if (S->stop && inflight.empty()) break;          // posted requests finish first
            int taken = 0;
            while (!S->stop && !S->small_q.empty()) {
                Req* r = S->small_q.front();
                S->small_q.pop_front();
                r->state = 1;
                r->out.t_admit = S->now();
                S->st.running += 1;
                S->st.batched_requests += 1;
                local.push_back(r);
                ++taken;
            }
            if (taken) S->st.batches += 1;
        }
        bool progress = false;
        // answers whatever has finished (after every post too: a post that builds a
        // new lattice's tables takes milliseconds, and results should not wait on it)
        auto collect = [&] {
            if (Q == nullptr || inflight.empty()) return;
            int n = 0;
            const int rc = hubbard_queue_collect(Q, tks.data(), rs.data(), kCollect, &n);
            if (rc != HUB_OK) {
                for (auto& kv : inflight) finish(S, kv.second, lanczos_result{}, rc);
                inflight.clear();
            }
            for (int i = 0; i < n; ++i) {
                auto it = inflight.find(tks[(size_t)i]);
                if (it == inflight.end()) continue;
                finish(S, it->second, rs[(size_t)i], rs[(size_t)i].status);
                inflight.erase(it);
                progress = true;
            }
        };
        while (!local.empty()) {
            Req* r = local.front();
            if (qrc != HUB_OK) {
                local.pop_front();
                finish(S, r, lanczos_result{}, qrc);
                continue;
            }
            const hubbard_request& q = r->desc;
            const hubbard_sector_desc d{q.ns, q.nup, q.ndn, q.n_bonds, q.bonds, q.t, q.U};
            int64_t tk = -1;
            const int rc = hubbard_queue_post(Q, &d, q.seed, &tk);
            if (rc == HUB_EPENDING) break;                       // every slot busy: collect first
            local.pop_front();
            if (rc != HUB_OK) finish(S, r, lanczos_result{}, rc);
            else inflight.emplace(tk, r);
            collect();
        }
        collect();
        if (!progress && (!inflight.empty() || !local.empty())) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::microseconds(500));
        }
    }
    for (Req* r : local) finish(S, r, lanczos_result{}, HUB_EINVAL);   // taken at stop, never posted
}

// Small requests on their way to the queued solver: their lattice's hop
// tables are made here (milliseconds for a new lattice and filling, nothing
// once cached), so the lane that posts and answers never waits on them.
void prep_lane(hubbard_server* S) {
    cudaSetDevice(S->device);
    while (true) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->prep_q.empty(); });
            if (S->stop) break;
            r = S->prep_q.front();
            S->prep_q.pop_front();
        }
        const hubbard_request& q = r->desc;
        const hubbard_sector_desc d{q.ns, q.nup, q.ndn, q.n_bonds, q.bonds, q.t, q.U};
        hubbard_queue_prepare(S->queue, &d);          // a failure shows again when the request is posted
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->small_q.push_back(r);
        }
        S->cv_work.notify_all();
    }
}

void big_lane(hubbard_server* S) {
    cudaStream_t st = nullptr;
    if (!S->opts.host_solver) {
        cudaSetDevice(S->device);
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    }
    while (true) {
        Req* r = nullptr;
        size_t store_bytes = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // first come, first served: the oldest request runs once its footprint fits
            S->cv_work.wait(lk, [&] {
                return S->stop || (!S->big_q.empty() && S->big_q.front()->footprint <= S->free_bytes);
            });
            if (S->stop) break;
            r = S->big_q.front();
            S->big_q.pop_front();
            if (r->path == kPathRefined) {
                // binary32 Lanczos vectors kept for the Ritz vector (each saves a
                // replayed step): up to store_vectors, within a quarter of the
                // spare budget and 16 GB, so one request does not hold back the
                // admission of the next ones
                const size_t slot = ((size_t)r->D * 4 + 255) / 256 * 256;
                const size_t spare = S->free_bytes - r->footprint;
                const size_t room = std::min<size_t>(spare / 4, (size_t)16 << 30);
                const size_t k = std::min<size_t>((size_t)std::max(0, S->opts.store_vectors), room / slot);
                store_bytes = k * slot;
                r->footprint += store_bytes;
            }
            take(S, r->footprint);
            r->state = 1;
            r->out.t_admit = S->now();
            S->st.running += 1;
            if (r->path == kPathBinary64) S->st.binary64_solves += 1;
            else S->st.refined_solves += 1;
        }
        lanczos_result res{};
        int rc;
        if (S->opts.host_solver) rc = S->opts.host_solver(S->opts.host_ctx, r->ticket, &r->desc, r->path, &res);
        else rc = solve_big_gpu(S, r, store_bytes, st, res);
        finish(S, r, res, rc != HUB_OK ? rc : res.status);
    }
    if (st) cudaStreamDestroy(st);
}

int check_request(const hubbard_request* q) {
    if (q == nullptr) return hub::fail(HUB_EINVAL, "null request");
    if (q->ns < 1 || q->ns > 32 || q->nup < 0 || q->nup > q->ns || q->ndn < 0 || q->ndn > q->ns)
        return hub::fail(HUB_EINVAL, "request: Ns in 1..32 and 0 <= N <= Ns");
    if (q->n_bonds < 0 || (q->n_bonds > 0 && q->bonds == nullptr)) return hub::fail(HUB_EINVAL, "request: bond list");
    for (int b = 0; b < q->n_bonds; ++b) {
        const int i = q->bonds[2 * b], j = q->bonds[2 * b + 1];
        if (i < 0 || i >= q->ns || j < 0 || j >= q->ns || i == j) return hub::fail(HUB_EINVAL, "request: bond endpoint");
    }
    if (!std::isfinite(q->t) || !std::isfinite(q->U)) return hub::fail(HUB_EINVAL, "request: t, U not finite");
    return HUB_OK;
}

}  // namespace

extern "C" {

int hubbard_server_create(const hubbard_server_opts* opts, hubbard_server_t* out) {
    using namespace hub;
    clear_error();
    if (out == nullptr) return fail(HUB_EINVAL, "out is null");
    *out = nullptr;
    hubbard_server_opts o{};
    if (opts) o = *opts;
    if (o.small_lanes < 0 || o.big_lanes < 0 || o.small_lanes + o.big_lanes < 1)
        return fail(HUB_EINVAL, "server: at least one lane");
    if (o.max_iters <= 0) o.max_iters = 1000;
    if (!(o.tol > 0.0)) o.tol = 1e-10;
    if (o.batch_max <= 0) o.batch_max = 1024;
    if (o.small_max_dim < 0 || o.mid_max_dim < 0) return fail(HUB_EINVAL, "server: size thresholds");
    if (o.store_vectors < 0) return fail(HUB_EINVAL, "server: store_vectors");
    hubbard_server* S = new (std::nothrow) hubbard_server();
    if (S == nullptr) return fail(HUB_ENOMEM, "host allocation");
    S->opts = o;
    if (!o.host_solver) {
        if (cudaGetDevice(&S->device) != cudaSuccess) {
            delete S;
            return fail(HUB_ECUDA, "no CUDA device");
        }
        // freed lane memory stays in the device pool for the next request
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    double budget = o.hbm_budget;
    if (!(budget > 0.0)) {
        size_t fr = 0, tot = 0;
        if (o.host_solver || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return fail(HUB_EINVAL, "server: a budget is required");
        }
        budget = 0.8 * (double)fr;
    }
    S->budget = S->free_bytes = (size_t)budget;
    S->st.budget_bytes = (double)S->budget;
    // small requests: a queued persistent solver (GPU) or micro-batches; the
    // queue's slots (vectors of small_max_dim elements and a/b histories) and
    // its table pools come out of the budget now
    S->queued_small = !o.host_solver && o.small_ctas >= 0 && o.small_lanes > 0 && o.small_max_dim > 0;
    if (S->queued_small) {
        const size_t per = 24 * (size_t)((o.small_max_dim + 1) / 2 * 2) + 16 * (size_t)o.max_iters;
        const size_t pools = (size_t)64 << 20;
        const size_t room = S->budget / 4 > pools ? S->budget / 4 - pools : 0;
        S->queue_cap = (int)std::min<size_t>(1024, room / per);
        if (S->queue_cap < 1 ||
            hubbard_queue_create(S->queue_cap, o.small_max_dim, o.max_iters, o.tol, o.small_ctas > 0 ? o.small_ctas : 16,
                                 &S->queue) != HUB_OK) {
            S->queued_small = false;                  // micro-batches instead
            S->queue = nullptr;
        } else {
            S->free_bytes -= (size_t)S->queue_cap * per + pools;
            S->peak = S->budget - S->free_bytes;
        }
    }
    S->t0 = Clock::now();
    try {
        if (S->queued_small) {
            S->threads.emplace_back(queue_lane, S);
            S->threads.emplace_back(prep_lane, S);
        }
        else
            for (int i = 0; i < o.small_lanes; ++i) S->threads.emplace_back(small_lane, S);
        for (int i = 0; i < o.big_lanes; ++i) S->threads.emplace_back(big_lane, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        for (auto& th : S->threads) th.join();
        hubbard_queue_destroy(S->queue);
        delete S;
        return fail(HUB_ENOMEM, "server: threads");
    }
    if (S->queued_small) {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait_for(lk, std::chrono::seconds(30), [&] { return S->queue_ready; });
    }
    *out = S;
    return HUB_OK;
}

int hubbard_server_submit(hubbard_server_t S, const hubbard_request* req, uint64_t* ticket) {
    using namespace hub;
    clear_error();
    if (S == nullptr || ticket == nullptr) return fail(HUB_EINVAL, "null argument");
    int rc = check_request(req);
    if (rc) return rc;
    auto r = std::unique_ptr<Req>(new (std::nothrow) Req());
    if (!r) return fail(HUB_ENOMEM, "host allocation");
    r->bonds.assign(req->bonds, req->bonds + 2 * (size_t)req->n_bonds);
    r->desc = *req;
    r->desc.bonds = r->bonds.empty() ? nullptr : r->bonds.data();
    const double D = binom(req->ns, req->nup) * binom(req->ns, req->ndn);
    if (D > 4e18) return fail(HUB_EINVAL, "request: dimension");
    r->D = (int64_t)D;
    r->path = r->D <= S->opts.small_max_dim ? kPathBatch
                                            : (r->D <= S->opts.mid_max_dim ? kPathBinary64 : kPathRefined);
    r->footprint = (r->path == kPathBatch && S->queued_small) ? 0 : base_footprint(S, r->path, r->D);
    r->out.path = r->path;
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->footprint > S->budget) return fail(HUB_ENOMEM, "request footprint above the server budget");
    if (S->stop) return fail(HUB_EINVAL, "server stopping");
    if ((r->path == kPathBatch && S->opts.small_lanes == 0) || (r->path != kPathBatch && S->opts.big_lanes == 0))
        return fail(HUB_EINVAL, "no lane serves this request size");
    r->ticket = S->next_ticket++;
    r->out.t_submit = S->now();
    (r->path == kPathBatch ? (S->queued_small ? S->prep_q : S->small_q) : S->big_q).push_back(r.get());
    *ticket = r->ticket;
    S->reqs.emplace(r->ticket, std::move(r));
    S->st.submitted += 1;
    S->st.max_backlog =
        std::max<int64_t>(S->st.max_backlog, (int64_t)(S->prep_q.size() + S->small_q.size() + S->big_q.size()));
    S->cv_work.notify_all();
    return HUB_OK;
}

int hubbard_server_poll(hubbard_server_t S, uint64_t ticket, hubbard_served* out) {
    using namespace hub;
    clear_error();
    if (S == nullptr || out == nullptr) return fail(HUB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(HUB_EINVAL, "unknown ticket");
    *out = it->second->out;
    return it->second->state == 2 ? HUB_OK : HUB_EPENDING;
}

int hubbard_server_wait(hubbard_server_t S, uint64_t ticket, double timeout_s, hubbard_served* out) {
    using namespace hub;
    clear_error();
    if (S == nullptr || out == nullptr) return fail(HUB_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(HUB_EINVAL, "unknown ticket");
    Req* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    if (!S->cv_done.wait_until(lk, deadline, [&] { return r->state == 2; })) {
        *out = r->out;
        return fail(HUB_ETIMEOUT, "request not finished within the timeout");
    }
    *out = r->out;
    return HUB_OK;
}

int hubbard_server_stats_get(hubbard_server_t S, hubbard_server_stats* out) {
    using namespace hub;
    clear_error();
    if (S == nullptr || out == nullptr) return fail(HUB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->queued = (int64_t)(S->prep_q.size() + S->small_q.size() + S->big_q.size());
    out->peak_bytes = (double)S->peak;
    out->free_bytes = (double)S->free_bytes;
    return HUB_OK;
}

void hubbard_server_destroy(hubbard_server_t S) {
    if (S == nullptr) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& th : S->threads) th.join();      // running requests finish first
    hubbard_queue_destroy(S->queue);
    delete S;
}

}  // extern "C"
