"""GPU tests of the queued solver (sectors posted to a persistent kernel while it runs)."""
import math
import time

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
from workload import batch_sectors, lattice_by_name, start_vector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MAXIT = 1000
TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    return torch.device("cuda:0")


def _reqs(n, seed, dmax):
    out = []
    for r in batch_sectors(4 * n, seed=seed):
        ns, _ = lattice_by_name(r["lattice"])
        if math.comb(ns, r["nup"]) * math.comb(ns, r["ndn"]) <= dmax:
            out.append(r)
        if len(out) == n:
            break
    return out


def _spec(r):
    ns, bonds = lattice_by_name(r["lattice"])
    return ns, bonds, r["nup"], r["ndn"], r["t"], r["U"]


def _oracle(spec):
    ns, bonds, nup, ndn, t, U = spec
    S = Sector(ns, bonds, nup, ndn, t, U)
    if S.D <= 1500:
        return float(np.linalg.eigvalsh(S.dense())[0])
    from scipy.sparse.linalg import eigsh
    return float(eigsh(S.explicit(), k=1, which="SA", tol=1e-14, v0=start_vector(S.D, seed=9))[0][0])


def _post_all(Q, reqs):
    """Posts every request (waiting for free slots when full); returns tickets."""
    tickets = []
    for r in reqs:
        while True:
            tk = Q.post(*_spec(r), r["seed"])
            if tk is not None:
                tickets.append(tk)
                break
            time.sleep(0.001)
    return tickets


def test_queue_matches_oracle(dev):
    reqs = _reqs(40, 21, 20000)
    Q = hub.Queue(capacity=64, max_dim=20000, max_iters=MAXIT, tol=TOL)
    tickets = _post_all(Q, reqs)
    res = [Q.wait(tk, 120.0) for tk in tickets]
    Q.close()
    for r, got in zip(reqs, res):
        assert got["status"] == hub.HUB_OK, (r, got)
        e = _oracle(_spec(r))
        assert abs(got["energy"] - e) <= 1e-9 * max(1.0, abs(e)), (r, got, e)
        assert abs(got["energy"] - e) <= got["err_bound"] + 1e-12 * max(1.0, abs(e)), (r, got, e)


def test_queue_alone_equals_in_mix_and_batch_task(dev):
    """A sector's result is bit-identical posted alone, posted among others, and
    solved as a one-CTA task of a batch whose start vectors come from the same seeds."""
    reqs = _reqs(24, 23, 20000)
    Q = hub.Queue(capacity=32, max_dim=20000, max_iters=MAXIT, tol=TOL)
    mix = [Q.wait(tk, 120.0) for tk in _post_all(Q, reqs)]
    Q.close()
    specs = [_spec(r) for r in reqs]
    B = hub.Batch(specs)
    B.set_schedule(1 << 30)                              # every sector a one-CTA task
    v0 = torch.zeros(int(B.offsets[-1]), dtype=torch.float64, device=dev)
    for k, r in enumerate(reqs):
        ns, _, nup, ndn, _, _ = specs[k]
        D = math.comb(ns, nup) * math.comb(ns, ndn)
        hub.hubbard_fill_start_vector(v0[int(B.offsets[k]):int(B.offsets[k]) + D], r["seed"])
    ws = torch.empty(B.workspace_bytes(MAXIT), dtype=torch.uint8, device=dev)
    B.solve_async(v0, MAXIT, TOL, ws)
    bres = B.results(ws, MAXIT)
    B.close()
    for i in range(len(reqs)):
        assert mix[i]["energy"] == bres[i]["energy"] and mix[i]["iters"] == bres[i]["iters"], i
    for i in (0, 11, 23):
        Q1 = hub.Queue(capacity=4, max_dim=20000, max_iters=MAXIT, tol=TOL)
        alone = Q1.wait(Q1.post(*specs[i], reqs[i]["seed"]), 60.0)
        Q1.close()
        assert alone["energy"] == mix[i]["energy"] and alone["iters"] == mix[i]["iters"], i


def test_queue_full_slot_reuse_and_relaunch_after_idle(dev):
    """Eight slots for 30 posts (posts wait for free slots while the kernel runs),
    then an idle pause long enough for the kernel to leave, then more posts."""
    reqs = _reqs(36, 29, 6000)
    Q = hub.Queue(capacity=8, max_dim=6000, max_iters=MAXIT, tol=TOL, ctas=4)
    first = []
    pending = []
    for r in reqs[:30]:
        while True:
            tk = Q.post(*_spec(r), r["seed"])
            if tk is not None:
                pending.append((r, tk))
                break
            # full: collect whatever has finished, then try again
            for item in list(pending):
                got = Q.poll(item[1])
                if got is not None:
                    first.append((item[0], got))
                    pending.remove(item)
            time.sleep(0.0005)
    first += [(r, Q.wait(tk, 120.0)) for r, tk in pending]
    time.sleep(0.5)                                       # the kernel leaves an idle queue
    second = [(r, Q.wait(Q.post(*_spec(r), r["seed"]), 120.0)) for r in reqs[30:]]
    Q.close()
    assert len(first) == 30 and len(second) == 6
    for r, got in first + second:
        assert got["status"] == hub.HUB_OK, (r, got)
        e = _oracle(_spec(r))
        assert abs(got["energy"] - e) <= 1e-9 * max(1.0, abs(e)), (r, got, e)


def test_queue_argument_errors(dev):
    Q = hub.Queue(capacity=4, max_dim=100, max_iters=200, tol=TOL)
    ns, bonds = lattice_by_name("ring8")
    with pytest.raises(hub.HubError) as ei:
        Q.post(ns, bonds, 4, 4, 1.0, 4.0, 1)             # D = 4900 > max_dim
    assert ei.value.code == hub.HUB_EINVAL
    with pytest.raises(hub.HubError):
        Q.post(ns, [(0, 1), (1, 0)], 1, 1, 1.0, 4.0, 1)    # duplicate bond
    with pytest.raises(hub.HubError):
        Q.poll(5)                                         # nothing posted
    tk = Q.post(4, lattice_by_name("ring4")[1], 2, 2, 1.0, 4.0, 7)
    got = Q.wait(tk, 30.0)
    assert got["status"] == hub.HUB_OK
    with pytest.raises(hub.HubError):
        Q.poll(tk)                                        # already collected
    Q.close()
