"""Trace-driven front end of the native continuous-batching server.

The scheduling and every numerical step run in the library
(hubbard_server_*, csrc/server.cpp): requests are queued with
hubbard_server_submit and taken by lanes (host threads with their own
streams) as lanes and device memory free up; small sectors are posted, as
they arrive, to a queued persistent solver whose CTAs take each new sector as
they free up, mid-sized ones solved in binary64, large ones in binary32 with
binary64 refinement.  This module only submits the
requests of a trace at their arrival times, waits for the answers and
summarises latencies (arrival to answer, on the server's clock) and
throughput.
"""
import math
import time

import numpy as np


class Request:
    __slots__ = ("id", "arrival_s", "lattice", "ns", "bonds", "nup", "ndn", "t", "U", "seed", "D", "ticket",
                 "path", "t_submit", "t_admit", "t_done", "result")

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
        self.ticket = None
        self.path = None
        self.t_submit = self.t_admit = self.t_done = None
        self.result = None

    def spec(self):
        return (self.ns, self.bonds, self.nup, self.ndn, self.t, self.U)


class SolveServer:
    """hbm_budget: bytes of device memory for requests (0: 80 % of the free
    memory); n_slots: big lanes (binary64 / refined solves in flight);
    small_lanes: lanes of the small queue (with a GPU one lane posts to the
    queued solver of small_ctas CTAs, 0: 16; small_ctas < 0 or a host solver:
    concurrent micro-batches); solver (tests without a GPU): a
    callable (ticket, request_dict, path) -> result dict run by the lanes
    instead of the CUDA solvers."""

    def __init__(self, hbm_budget=0.0, n_slots=8, small_lanes=2, small_max_dim=20_000, mid_max_dim=200_000,
                 batch_max=1024, store_vectors=128, max_iters=1000, tol=1e-10, solver=None, small_ctas=0):
        from paper_1204_3425_gb300 import Server
        self.srv = Server(hbm_budget, small_lanes, n_slots, small_max_dim, mid_max_dim, max_iters, batch_max,
                          store_vectors, tol, host_solver=solver, small_ctas=small_ctas)
        self.small_max_dim, self.mid_max_dim, self.n_slots, self.small_lanes = (small_max_dim, mid_max_dim, n_slots,
                                                                               small_lanes)

    def submit(self, req):
        req.ticket = self.srv.submit(*req.spec(), req.seed)

    def collect(self, req, timeout=3600.0):
        r = self.srv.wait(req.ticket, timeout)
        req.result = r
        req.path = r["path"]
        req.t_submit, req.t_admit, req.t_done = r["t_submit"], r["t_admit"], r["t_done"]
        return r

    def run_trace(self, requests, time_scale=1.0, timeout=3600.0):
        """Submits each request at its arrival time (scaled), waits for all, returns stats."""
        base = time.perf_counter()
        for req in sorted(requests, key=lambda r: r.arrival_s):
            delay = base + req.arrival_s * time_scale - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            self.submit(req)
        end = time.perf_counter() + timeout
        for req in requests:
            self.collect(req, max(0.0, end - time.perf_counter()))
        return self.stats(requests)

    def stats(self, requests):
        lat = np.array([r.t_done - r.t_submit for r in requests])
        first = min(r.t_submit for r in requests)
        last = max(r.t_done for r in requests)
        wall = max(last - first, 1e-9)
        ok = [r for r in requests if r.result["status"] == 0]
        failures = {}
        for r in requests:
            if r.result["status"] != 0:
                key = f'{r.path}:{r.result["status"]}'
                failures[key] = failures.get(key, 0) + 1
        verified = [r for r in ok if r.result["err_bound"] <= 1e-9 * max(1.0, abs(r.result["energy"]))]
        by_path = {}
        for pth in sorted({r.path for r in requests}):
            lp = np.array([r.t_done - r.t_submit for r in requests if r.path == pth])
            by_path[pth] = dict(requests=int(lp.size), p50_ms=1e3 * float(np.percentile(lp, 50)),
                                p99_ms=1e3 * float(np.percentile(lp, 99)))
        nat = self.srv.stats()
        return dict(requests=len(requests), wall_s=wall, solves_per_s=len(ok) / wall,
                    verified_solves_per_s=len(verified) / wall, verified=len(verified), failed=len(requests) - len(ok),
                    failures=failures,
                    p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                    max_ms=1e3 * float(lat.max()), latency_by_path=by_path, max_backlog=nat["max_backlog"],
                    peak_bytes=nat["peak_bytes"],
                    budget_bytes=nat["budget_bytes"], n_batches=nat["batches"],
                    mean_batch=(nat["batched_requests"] / nat["batches"]) if nat["batches"] else 0.0,
                    binary64=nat["binary64_solves"], refined=nat["refined_solves"], big_lanes=self.n_slots,
                    small_lanes=self.small_lanes, small_max_dim=self.small_max_dim, mid_max_dim=self.mid_max_dim)

    def stop(self):
        self.srv.close()
