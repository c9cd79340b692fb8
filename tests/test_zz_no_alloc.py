"""GPU test of hubbard_apply_noalloc, the binary64 H*v entry point that
allocates no device memory (for callers that cannot call cudaMalloc when
they need H*v).  Its output must match hubbard_apply's within the binary64
H*v tolerance, on two calls in a row, and it must refuse sectors larger than
its fixed scratch array.  Collected last on purpose (file name)."""
import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from workload import lattice_by_name, start_vector

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


def _tol(v, t):
    return 1e-12 * float(np.linalg.norm(v)) * max(1.0, abs(t))


@pytest.mark.parametrize("name,nup,ndn,t,U", [("sq3x3", 4, 4, 1.0, 6.0), ("ring12", 6, 6, 1.3, 4.0)])
def test_noalloc_matches_apply_twice(dev, name, nup, ndn, t, U):
    ns, bonds = lattice_by_name(name)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    assert H.D <= hub.HUBBARD_NOALLOC_MAX_ELEMS
    v1 = start_vector(H.D, seed=21)
    # second call: a vector 1e6 times smaller, so a stale exponent word or
    # stale fixed-point data from the first call would show up as a large error
    v2 = 1e-6 * start_vector(H.D, seed=22)
    for v in (v1, v2):
        vd = torch.from_numpy(v).to(dev)
        w_ref = torch.empty_like(vd)
        w_na = torch.full_like(vd, float("nan"))
        hub.hubbard_apply(H, vd, w_ref)
        hub.hubbard_apply_noalloc(H, vd, w_na)
        torch.cuda.synchronize()
        err = (w_na - w_ref).abs().max().item()
        assert err <= _tol(v, t), err
    H.close()


def test_noalloc_rejects_large_sector(dev):
    ns, bonds = lattice_by_name("sq4x4")
    H = hub.hubbard_sector_create(ns, bonds, 5, 5, 1.0, 2.0)        # D = 4368^2 > 2^21
    assert H.D > hub.HUBBARD_NOALLOC_MAX_ELEMS
    v = torch.zeros(H.D, dtype=torch.float64, device=dev)
    w = torch.zeros_like(v)
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_apply_noalloc(H, v, w)
    assert ei.value.code == hub.HUB_EINVAL and "HUBBARD_NOALLOC_MAX_ELEMS" in str(ei.value)
    H.close()
