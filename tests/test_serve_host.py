"""Host-side tests of the serving scheduler (no GPU): a fake solver that only
sleeps stands in for the CUDA paths."""
import threading
import time

import pytest

from paper_1204_3425_gb300.serve import Request, SolveServer
from workload import serve_requests


class FakeSolver:
    def __init__(self, scale=2e-9):
        self.scale = scale
        self.lock = threading.Lock()
        self.concurrent_large = 0
        self.max_concurrent_large = 0

    large_footprint = staticmethod(lambda D: 48 * D)
    small_footprint = staticmethod(lambda D: 32 * D)

    def new_stream(self):
        return None

    def solve_large(self, req, stream):
        with self.lock:
            self.concurrent_large += 1
            self.max_concurrent_large = max(self.max_concurrent_large, self.concurrent_large)
        time.sleep(min(0.05, self.scale * req.D))
        with self.lock:
            self.concurrent_large -= 1
        return dict(energy=-float(req.id), residual=0.0, error_bound=0.0, iters=1, status=0)

    def solve_batch(self, reqs, stream):
        time.sleep(0.01)
        return [dict(energy=-float(r.id), residual=0.0, error_bound=None, iters=1, status=0) for r in reqs]


def _reqs(n, rate, seed=3):
    return [Request(k, s, s["arrival_s"]) for k, s in enumerate(serve_requests(n, rate=rate, seed=seed))]


def test_server_completes_and_respects_budget():
    reqs = _reqs(200, rate=2000.0)
    budget = 3 * 48 * max(r.D for r in reqs)          # room for about three of the largest at once
    fake = FakeSolver()
    srv = SolveServer(budget, n_slots=4, small_max_dim=100_000, solver=fake).start()
    st = srv.run_trace(reqs, timeout=120)
    srv.stop()
    assert st["requests"] == 200 and len(srv.done) == 200 and not srv.errors
    assert srv.peak_in_use <= budget
    assert srv.free == budget                            # every footprint returned
    assert all(r.result["energy"] == -float(r.id) for r in reqs)
    assert st["n_batches"] < sum(1 for r in reqs if r.path == "batch")   # small requests were grouped
    assert 1 <= fake.max_concurrent_large <= 4
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_server_rejects_request_above_budget():
    srv = SolveServer(1000, n_slots=1, solver=FakeSolver())
    big = _reqs(50, 100.0)
    r = max(big, key=lambda q: q.D)
    with pytest.raises(ValueError):
        srv.submit(r)


def test_large_requests_admitted_in_arrival_order():
    reqs = [r for r in _reqs(300, 5000.0) if r.D > 100_000][:12]
    fake = FakeSolver(scale=0.0)
    budget = 48 * max(r.D for r in reqs)                # one at a time
    srv = SolveServer(budget, n_slots=3, small_max_dim=100_000, solver=fake).start()
    srv.run_trace(reqs, timeout=60)
    srv.stop()
    admits = [r.t_admit for r in sorted(reqs, key=lambda q: q.arrival_s)]
    assert admits == sorted(admits)
    assert srv.peak_in_use <= budget
    assert fake.max_concurrent_large <= budget // (48 * min(r.D for r in reqs))
