"""Continuous-batching ground-state server over the C ABI.

Requests (one sector each: lattice, fillings, t, U, seed) arrive over time;
each is answered with its ground-state energy to 1e-9 relative.  Work from
requests that arrive while others run overlaps on the GPU:

* small sectors (D <= small_max_dim) join the next micro-batch of the
  persistent batched solver (hubbard_batch_*): a new micro-batch is launched
  as soon as the previous one finishes and takes every small request that
  arrived meanwhile (binary64, fixed-point hop sums, tol on rho);
* larger sectors are admitted to one of `n_slots` worker slots, each with
  its own CUDA stream, and solved with the binary32 + binary64-refined path
  (lanczos_ground_state_refined); slots run concurrently on the device.

Admission is by device-memory footprint: a request is admitted only when its
buffers fit in what remains of `hbm_budget` bytes; all device buffers of a
request live until it completes, then the footprint is returned.

The scheduler is Python threads; every numerical step runs in the CUDA
library (the ctypes calls release the GIL).  `solver` can be replaced (tests
use a host-only fake to check admission and batching without a GPU).
"""
import math
import threading
import time
from collections import deque


class Request:
    __slots__ = ("id", "arrival_s", "lattice", "ns", "bonds", "nup", "ndn", "t", "U", "seed", "D", "path",
                 "footprint", "t_submit", "t_admit", "t_done", "result")

    def __init__(self, rid, spec, arrival_s=0.0):
        from workload import lattice_by_name
        self.id = rid
        self.arrival_s = float(arrival_s)
        self.lattice = spec["lattice"]
        self.ns, self.bonds = lattice_by_name(spec["lattice"])
        self.nup, self.ndn = int(spec["nup"]), int(spec["ndn"])
        self.t, self.U = float(spec["t"]), float(spec["U"])
        self.seed = int(spec["seed"])
        self.D = math.comb(self.ns, self.nup) * math.comb(self.ns, self.ndn)
        self.path = None
        self.footprint = 0
        self.t_submit = self.t_admit = self.t_done = None
        self.result = None

    def spec(self):
        return (self.ns, self.bonds, self.nup, self.ndn, self.t, self.U)


class GPUSolver:
    """The default solver: the library's batched and refined paths."""

    def __init__(self, max_iters=1000, tol=1e-10, device="cuda:0"):
        import torch

        import paper_1204_3425_gb300 as hub
        self.hub, self.torch = hub, torch
        self.max_iters, self.tol = max_iters, tol
        self.device = torch.device(device)
        hub.load_library()

    # binary32 Lanczos vectors kept for the Ritz vector (each one saves a replayed
    # step): up to 128, within 32 GB per request
    @staticmethod
    def store_vectors(D):
        return int(min(128, 32e9 // (4 * D + 256)))

    # bytes of device memory a request holds while it runs
    @classmethod
    def large_footprint(cls, D):
        return 48 * D + cls.store_vectors(D) * (4 * D + 256) + (1 << 20)

    @staticmethod
    def small_footprint(D):
        return 32 * D + (1 << 12)

    def solve_large(self, req, stream):
        hub, torch = self.hub, self.torch
        with torch.cuda.stream(stream):
            H = hub.hubbard_sector_create(*req.spec())
            try:
                v0 = torch.empty(req.D, dtype=torch.float64, device=self.device)
                hub.hubbard_fill_start_vector(v0, req.seed, stream=stream)
                ws = torch.empty(hub.lanczos_refined_workspace_bytes(H, self.store_vectors(req.D)), dtype=torch.uint8,
                                 device=self.device)
                r = hub.lanczos_ground_state_refined(H, v0, self.max_iters, self.tol, workspace=ws, stream=stream)
                del v0, ws
            finally:
                H.close()
        return dict(energy=r["energy"], residual=r["residual"], error_bound=r["error_bound"],
                    iters=r["iters_f32"] + r["iters_f64"], status=r["status"])

    def solve_batch(self, reqs, stream):
        hub, torch = self.hub, self.torch
        with torch.cuda.stream(stream):
            B = hub.Batch([r.spec() for r in reqs])
            try:
                v0 = torch.zeros(int(B.offsets[-1]), dtype=torch.float64, device=self.device)
                for k, r in enumerate(reqs):
                    hub.hubbard_fill_start_vector(v0[int(B.offsets[k]):int(B.offsets[k]) + r.D], r.seed,
                                                  stream=stream)
                ws = torch.empty(B.workspace_bytes(self.max_iters), dtype=torch.uint8, device=self.device)
                B.solve_async(v0, self.max_iters, self.tol, ws, stream=stream)
                res = B.results(ws, self.max_iters, stream=stream)
                del v0, ws
            finally:
                B.close()
        return [dict(energy=x["energy"], residual=x["residual"], error_bound=None, iters=x["iters"],
                     status=x["status"]) for x in res]

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)


class SolveServer:
    # Defaults measured on the 500 req/s trace: a cooperative micro-batch needs
    # the whole GPU, so batching only sectors that stay in one CTA's shared
    # memory (<= 20000 elements) interferes least with the refined slots.
    def __init__(self, hbm_budget, n_slots=12, small_max_dim=20_000, batch_max=1024, solver=None):
        self.solver = solver if solver is not None else GPUSolver()
        self.budget = int(hbm_budget)
        self.free = int(hbm_budget)
        self.n_slots = n_slots
        self.small_max_dim = small_max_dim
        self.batch_max = batch_max
        self.cv = threading.Condition()
        self.pending_large = deque()
        self.pending_small = deque()
        self.done = []
        self.peak_in_use = 0
        self.max_backlog = 0
        self.batches = []           # sizes of the micro-batches launched
        self.errors = []
        self._stop = False
        self._threads = []
        self.t0 = None

    # ---- public ---------------------------------------------------------------
    def start(self):
        self.t0 = time.perf_counter()
        for i in range(self.n_slots):
            th = threading.Thread(target=self._slot_worker, args=(i,), daemon=True)
            th.start()
            self._threads.append(th)
        th = threading.Thread(target=self._batcher, daemon=True)
        th.start()
        self._threads.append(th)
        return self

    def submit(self, req):
        req.t_submit = time.perf_counter()
        if req.D <= self.small_max_dim:
            req.path = "batch"
            req.footprint = self.solver.small_footprint(req.D)
        else:
            req.path = "refined"
            req.footprint = self.solver.large_footprint(req.D)
        if req.footprint > self.budget:
            raise ValueError(f"request {req.id} needs {req.footprint} bytes, above the budget {self.budget}")
        with self.cv:
            (self.pending_small if req.path == "batch" else self.pending_large).append(req)
            self.max_backlog = max(self.max_backlog, len(self.pending_small) + len(self.pending_large))
            self.cv.notify_all()

    def stop(self):
        with self.cv:
            self._stop = True
            self.cv.notify_all()
        for th in self._threads:
            th.join(timeout=60)

    def wait(self, n, timeout=None):
        end = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while len(self.done) + len(self.errors) < n:
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError(f"{len(self.done)} of {n} requests done")
                self.cv.wait(timeout=left if left is not None else 1.0)
        if self.errors:
            raise RuntimeError(f"{len(self.errors)} requests failed: {self.errors[0]}")

    def run_trace(self, requests, time_scale=1.0, timeout=None):
        """Submits each request at its arrival time (scaled), waits for all, returns stats."""
        if self.t0 is None:
            self.start()
        base = time.perf_counter()
        for req in sorted(requests, key=lambda r: r.arrival_s):
            delay = base + req.arrival_s * time_scale - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            self.submit(req)
        self.wait(len(requests), timeout=timeout)
        return self.stats(requests)

    def stats(self, requests):
        lat = sorted(r.t_done - r.t_submit for r in requests)
        first = min(r.t_submit for r in requests)
        last = max(r.t_done for r in requests)
        q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
        return dict(requests=len(requests), wall_s=last - first, solves_per_s=len(requests) / (last - first),
                    p50_ms=1e3 * q(0.50), p99_ms=1e3 * q(0.99), max_ms=1e3 * lat[-1],
                    max_backlog=self.max_backlog, peak_bytes=self.peak_in_use, budget_bytes=self.budget,
                    n_batches=len(self.batches), mean_batch=(sum(self.batches) / len(self.batches)) if self.batches else 0,
                    large=sum(1 for r in requests if r.path == "refined"), slots=self.n_slots,
                    small_max_dim=self.small_max_dim)

    # ---- internals --------------------------------------------------------------
    def _take(self, nbytes):
        self.free -= nbytes
        self.peak_in_use = max(self.peak_in_use, self.budget - self.free)

    def _finish(self, reqs, results=None, error=None):
        now = time.perf_counter()
        with self.cv:
            for k, r in enumerate(reqs):
                r.t_done = now
                if error is None:
                    r.result = results[k]
                    self.done.append(r)
                else:
                    self.errors.append((r.id, repr(error)))
                self.free += r.footprint
            self.cv.notify_all()

    def _slot_worker(self, slot):
        stream = self.solver.new_stream()
        while True:
            with self.cv:
                # FIFO admission: the oldest large request runs when its footprint fits
                while not self._stop and not (self.pending_large and self.pending_large[0].footprint <= self.free):
                    self.cv.wait(timeout=0.5)
                if self._stop:
                    return
                req = self.pending_large.popleft()
                self._take(req.footprint)
                req.t_admit = time.perf_counter()
            try:
                res = self.solver.solve_large(req, stream)
                self._finish([req], [res])
            except Exception as exc:  # noqa: BLE001  (reported per request)
                self._finish([req], error=exc)

    def _batcher(self):
        stream = self.solver.new_stream()
        while True:
            with self.cv:
                while not self._stop and not (self.pending_small and self.pending_small[0].footprint <= self.free):
                    self.cv.wait(timeout=0.5)
                if self._stop:
                    return
                # every small request that arrived meanwhile, while it fits the budget
                batch, nbytes = [], 0
                while self.pending_small and len(batch) < self.batch_max:
                    fp = self.pending_small[0].footprint
                    if nbytes + fp > self.free:
                        break
                    r = self.pending_small.popleft()
                    batch.append(r)
                    nbytes += fp
                self._take(nbytes)
                now = time.perf_counter()
                for r in batch:
                    r.t_admit = now
                self.batches.append(len(batch))
            try:
                res = self.solver.solve_batch(batch, stream)
                self._finish(batch, res)
            except Exception as exc:  # noqa: BLE001
                self._finish(batch, error=exc)
