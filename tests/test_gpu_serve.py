"""GPU test of the continuous-batching server: a mixed trace of small and
large sectors, every served energy against the CPU oracle (dense, sparse or
matrix-free diagonalisation of Eq. 1, whichever fits), and each answer the
same alone and in the mix."""
import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from paper_1204_3425_gb300.serve import Request, SolveServer
from oracle.energies import ground_energy
from workload import serve_requests

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    return torch.device("cuda:0")


LATS = ["ring8", "ring10", "ring12", "ring14", "sq3x3", "sq4x3"]


def _trace(n, seed):
    return [Request(k, s, s["arrival_s"]) for k, s in
            enumerate(serve_requests(n, rate=500.0, seed=seed, lattices=LATS))]


def _server(**kw):
    args = dict(hbm_budget=60e9, n_slots=4, small_lanes=2, small_max_dim=20_000, mid_max_dim=400_000)
    args.update(kw)
    return SolveServer(**args)


def test_serve_mixed_trace(dev):
    """60 requests of every path (small sectors through the queued persistent
    solver, binary64 and refined lanes), all answered, each energy within 1e-9 of the oracle and
    within its own error bound."""
    reqs = _trace(60, 21)
    srv = _server()
    st = srv.run_trace(reqs, timeout=600)
    srv.stop()
    assert st["requests"] == 60 and st["failed"] == 0
    assert {r.path for r in reqs} == {"batch", "binary64", "refined"}
    assert st["verified"] == 60
    for r in reqs:
        e_ref, route = ground_energy(*r.spec(), seed=r.seed)
        err = abs(r.result["energy"] - e_ref)
        assert err <= 1e-9 * max(1.0, abs(e_ref)), (r.path, r.D, route)
        assert err <= r.result["err_bound"] + 1e-12 * max(1.0, abs(e_ref)), (r.path, r.D, r.result)


def test_serve_alone_equals_in_mix(dev):
    """A request's answer in the mix equals its answer served alone (fixed-order
    reductions on every path), and both match the oracle."""
    reqs = _trace(40, 22)
    srv = _server()
    srv.run_trace(reqs, timeout=600)
    srv.stop()
    picks = ([r for r in reqs if r.path == "batch"][:3] + [r for r in reqs if r.path == "binary64"][:2] +
             [r for r in reqs if r.path == "refined"][:2])
    assert {r.path for r in picks} == {"batch", "binary64", "refined"}
    for r in picks:
        solo = Request(1000 + r.id, dict(lattice=r.lattice, nup=r.nup, ndn=r.ndn, t=r.t, U=r.U, seed=r.seed), 0.0)
        s2 = _server(n_slots=1, small_lanes=1)
        s2.run_trace([solo], timeout=600)
        s2.stop()
        assert solo.path == r.path
        assert solo.result["energy"] == r.result["energy"], (r.path, solo.result, r.result)
        e_ref, _ = ground_energy(*r.spec(), seed=r.seed)
        assert abs(r.result["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))


def test_serve_c_abi_submit_poll(dev):
    """The C ABI directly: submit, poll until done, wait; a bad request is refused."""
    from workload import ring
    srv = hub.Server(8e9, small_lanes=1, big_lanes=2, small_max_dim=20_000, mid_max_dim=400_000)
    free0 = srv.stats()["free_bytes"]                    # the queued solver's memory is reserved at start
    assert free0 < srv.stats()["budget_bytes"]
    tks = [srv.submit(8, ring(8), 4, 4, 1.0, 4.0, 1234), srv.submit(10, ring(10), 5, 5, 1.0, 6.0, 7),
           srv.submit(12, ring(12), 5, 6, 1.0, 4.5, 11)]
    import time
    deadline = time.time() + 120
    res = {}
    while len(res) < len(tks) and time.time() < deadline:
        for tk in tks:
            if tk not in res:
                r = srv.poll(tk)
                if r is not None:
                    res[tk] = r
        time.sleep(0.01)
    assert len(res) == 3
    assert [res[tk]["path"] for tk in tks] == ["batch", "binary64", "refined"]
    for tk, (ns, bonds, nup, ndn, U, seed) in zip(tks, [(8, ring(8), 4, 4, 4.0, 1234), (10, ring(10), 5, 5, 6.0, 7),
                                                      (12, ring(12), 5, 6, 4.5, 11)]):
        e_ref, _ = ground_energy(ns, bonds, nup, ndn, 1.0, U, seed=seed)
        assert res[tk]["status"] == 0 and abs(res[tk]["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))
        assert srv.wait(tk, 1.0)["energy"] == res[tk]["energy"]
    with pytest.raises(hub.HubError):
        srv.submit(4, [(0, 4)], 1, 1, 1.0, 1.0, 1)          # bond endpoint out of range
    st = srv.stats()
    assert st["completed"] == 3 and st["verified"] == 3 and st["free_bytes"] == free0
    srv.close()


def test_serve_small_request_joins_running_work(dev):
    """Continuous batching of small sectors: a request submitted while 24 others
    are being solved by the queued solver (4 CTAs) is taken by its next free CTA
    and answered before the earlier requests are all done -- a micro-batch would
    have made it wait for all of them."""
    import time
    from workload import lattice_by_name, ring
    srv = hub.Server(8e9, small_lanes=1, big_lanes=1, small_max_dim=20_000, mid_max_dim=400_000, small_ctas=4)
    ns, bonds = lattice_by_name("sq3x3")
    early = [srv.submit(ns, bonds, 4, 4, 1.0, 2.0 + 0.25 * k, 100 + k) for k in range(24)]
    time.sleep(0.05)
    late = srv.submit(4, ring(4), 2, 2, 1.0, 4.0, 5)
    r_late = srv.wait(late, 120.0)
    r_early = [srv.wait(tk, 120.0) for tk in early]
    srv.close()
    assert r_late["status"] == 0 and all(r["status"] == 0 for r in r_early)
    assert r_late["t_admit"] < max(r["t_done"] for r in r_early)       # admitted while the others ran
    assert r_late["t_done"] < max(r["t_done"] for r in r_early)        # and answered before they all were
    e_ref, _ = ground_energy(4, ring(4), 2, 2, 1.0, 4.0, seed=5)
    assert abs(r_late["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))
    for k, r in enumerate(r_early[:4]):
        e_ref, _ = ground_energy(ns, bonds, 4, 4, 1.0, 2.0 + 0.25 * k, seed=100 + k)
        assert abs(r["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))


def test_fill_start_vector_matches_host_recipe(dev):
    from workload import start_vector
    for n, seed, start in [(1, 3, 0), (1000, 1234, 0), (4097, 77, 123456789)]:
        v = torch.empty(n, dtype=torch.float64, device=dev)
        hub.hubbard_fill_start_vector(v, seed, start)
        assert np.array_equal(v.cpu().numpy(), start_vector(n, seed=seed, start=start))
        v32 = torch.empty(n, dtype=torch.float32, device=dev)
        hub.hubbard_fill_start_vector(v32, seed, start)
        assert np.array_equal(v32.cpu().numpy(), start_vector(n, seed=seed, start=start).astype(np.float32))
