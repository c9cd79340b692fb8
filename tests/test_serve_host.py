"""Host-side tests of the native server's scheduling (no GPU): a Python fake
solver, called by the lanes through the host_solver hook, stands in for the
CUDA paths, so admission by budget, first-come order, micro-batching,
concurrency and failure isolation are checked on CPU."""
import math
import threading
import time

import pytest

import paper_1204_3425_gb300 as hub
from paper_1204_3425_gb300.serve import Request, SolveServer
from workload import serve_requests


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()


class FakeSolver:
    """Sleeps (in proportion to D for big solves); energy = -ticket; counts concurrent big solves."""

    def __init__(self, scale=2e-9, fail_seeds=()):
        self.scale = scale
        self.fail_seeds = set(fail_seeds)
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.calls = []

    def __call__(self, ticket, req, path):
        D = math.comb(req["ns"], req["nup"]) * math.comb(req["ns"], req["ndn"])
        with self.lock:
            self.calls.append((ticket, path))
            if path != 0:
                self.running += 1
                self.max_running = max(self.max_running, self.running)
        try:
            if req["seed"] in self.fail_seeds:
                raise RuntimeError("injected failure")
            # a micro-batch takes a few ms whatever its size, so requests that
            # arrive meanwhile queue up for the next one
            time.sleep(0.004 if path == 0 else min(0.02, self.scale * D))
            return dict(energy=-float(ticket), residual=0.0, err_bound=0.0, iters=1, status=0)
        finally:
            if path != 0:
                with self.lock:
                    self.running -= 1


def _reqs(n, rate, seed=3):
    return [Request(k, s, s["arrival_s"]) for k, s in enumerate(serve_requests(n, rate=rate, seed=seed))]


def _footprint(D, path, max_iters=1000):
    return 56 * D + 16 * max_iters + 4096 if path == "batch" else (40 * D + (1 << 20) if path == "binary64"
                                                                   else 48 * D + (1 << 20))


def test_server_completes_within_budget_and_groups_small_requests():
    reqs = _reqs(200, rate=4000.0)
    big = max(r.D for r in reqs)
    budget = 3 * (48 * big + (1 << 20))                  # room for about three of the largest at once
    fake = FakeSolver()
    srv = SolveServer(budget, n_slots=4, small_lanes=2, small_max_dim=20_000, mid_max_dim=200_000,
                      store_vectors=0, solver=fake)
    st = srv.run_trace(reqs, timeout=120)
    nat = srv.srv.stats()
    srv.stop()
    assert st["requests"] == 200 and st["failed"] == 0 and nat["completed"] == 200
    assert nat["peak_bytes"] <= budget and nat["free_bytes"] == nat["budget_bytes"]   # every footprint returned
    assert all(r.result["energy"] == -float(r.ticket) for r in reqs)
    small = [r for r in reqs if r.path == "batch"]
    assert small and all(r.D <= 20_000 for r in small)
    assert all(r.path == ("binary64" if r.D <= 200_000 else "refined") for r in reqs if r.D > 20_000)
    assert st["n_batches"] < len(small)                   # small requests were grouped
    assert 1 <= fake.max_running <= 4
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_server_rejects_request_above_budget():
    srv = SolveServer(1000.0, n_slots=1, solver=FakeSolver())
    r = max(_reqs(50, 100.0), key=lambda q: q.D)
    with pytest.raises(hub.HubError) as ei:
        srv.submit(r)
    assert ei.value.code == hub.HUB_ENOMEM
    srv.stop()


def test_big_requests_admitted_in_arrival_order():
    reqs = [r for r in _reqs(300, 5000.0) if r.D > 20_000][:12]
    fake = FakeSolver(scale=0.0)
    budget = max(_footprint(r.D, "refined") for r in reqs)          # the largest runs alone
    srv = SolveServer(budget, n_slots=3, small_max_dim=20_000, mid_max_dim=0, store_vectors=0, solver=fake)
    srv.run_trace(reqs, timeout=60)
    nat = srv.srv.stats()
    srv.stop()
    admits = [r.t_admit for r in sorted(reqs, key=lambda q: q.arrival_s)]
    assert admits == sorted(admits)
    assert nat["peak_bytes"] <= budget
    assert 1 <= fake.max_running <= budget // min(_footprint(r.D, "refined") for r in reqs)


def test_failing_request_fails_alone():
    reqs = _reqs(60, rate=3000.0, seed=5)
    bad = {reqs[7].seed, reqs[31].seed}
    fake = FakeSolver(fail_seeds=bad)
    srv = SolveServer(1e12, n_slots=3, small_lanes=1, small_max_dim=20_000, solver=fake)
    st = srv.run_trace(reqs, timeout=60)
    srv.stop()
    assert st["failed"] == 2
    for r in reqs:
        if r.seed in bad:
            assert r.result["status"] == hub.HUB_EDEVICE
        else:
            assert r.result["status"] == 0 and r.result["energy"] == -float(r.ticket)


def test_poll_before_and_after_completion():
    gate = threading.Event()

    def slow(ticket, req, path):
        gate.wait(10)
        return dict(energy=1.5, status=0)

    srv = hub.Server(1e12, small_lanes=0, big_lanes=1, small_max_dim=0, mid_max_dim=1 << 40, host_solver=slow)
    from workload import ring
    tk = srv.submit(8, ring(8), 4, 4, 1.0, 4.0, 1234)
    assert srv.poll(tk) is None                          # HUB_EPENDING
    gate.set()
    r = srv.wait(tk, 10.0)
    assert r["energy"] == 1.5 and r["path"] == "binary64" and r["t_submit"] <= r["t_admit"] <= r["t_done"]
    assert srv.poll(tk)["energy"] == 1.5
    with pytest.raises(hub.HubError):
        srv.poll(tk + 100)                              # unknown ticket
    srv.close()
