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


def test_serve_mixed_trace(dev):
    reqs = _trace(60, 21)
    assert any(r.D > 200_000 for r in reqs) and any(r.D <= 200_000 for r in reqs)
    srv = SolveServer(60e9, n_slots=4, small_max_dim=200_000)
    st = srv.run_trace(reqs, timeout=600)
    srv.stop()
    assert st["requests"] == 60 and not srv.errors
    assert all(r.result["status"] == hub.HUB_OK for r in reqs)
    for r in reqs:
        e_ref, route = ground_energy(*r.spec(), seed=r.seed)
        assert abs(r.result["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref)), (r.path, r.D, route)


def test_serve_alone_equals_in_mix(dev):
    reqs = _trace(40, 22)
    srv = SolveServer(60e9, n_slots=4, small_max_dim=200_000)
    srv.run_trace(reqs, timeout=600)
    srv.stop()
    picks = [r for r in reqs if r.path == "batch"][:3] + [r for r in reqs if r.path == "refined"][:2]
    for r in picks:
        solo = Request(1000 + r.id, dict(lattice=r.lattice, nup=r.nup, ndn=r.ndn, t=r.t, U=r.U, seed=r.seed), 0.0)
        s2 = SolveServer(60e9, n_slots=1, small_max_dim=200_000)
        s2.run_trace([solo], timeout=600)
        s2.stop()
        assert solo.path == r.path
        assert abs(solo.result["energy"] - r.result["energy"]) <= 1e-12 * max(1.0, abs(r.result["energy"]))
        e_ref, _ = ground_energy(*r.spec(), seed=r.seed)
        assert abs(r.result["energy"] - e_ref) <= 1e-9 * max(1.0, abs(e_ref))


def test_fill_start_vector_matches_host_recipe(dev):
    from workload import start_vector
    for n, seed, start in [(1, 3, 0), (1000, 1234, 0), (4097, 77, 123456789)]:
        v = torch.empty(n, dtype=torch.float64, device=dev)
        hub.hubbard_fill_start_vector(v, seed, start)
        assert np.array_equal(v.cpu().numpy(), start_vector(n, seed=seed, start=start))
        v32 = torch.empty(n, dtype=torch.float32, device=dev)
        hub.hubbard_fill_start_vector(v32, seed, start)
        assert np.array_equal(v32.cpu().numpy(), start_vector(n, seed=seed, start=start).astype(np.float32))
