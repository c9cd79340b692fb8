"""GPU tests of hubbard_apply_noalloc, the binary64 H*v entry point that
allocates no device memory.

It serves callers that cannot call cudaMalloc at the moment they need H*v:
code running while another framework owns the device allocator, code held
to a fixed memory budget, or a hot loop that must never reach the allocator.
Its scratch is a fixed file-scope device array, so it takes sectors of at
most HUBBARD_NOALLOC_MAX_ELEMS elements.

The checks: on a freshly created handle (no H*v scratch allocated yet) the
first call already works; every output agrees with the oracle's explicit
sparse H (Eq. 1) within the binary64 H*v bar and with hubbard_apply's output,
on two calls in a row; the device's free memory does not change across a
call; inputs at the edges of the binary64 range (2^+-900, subnormal, zero)
keep the bar; oversized sectors are refused.  Collected last on purpose
(file name), and independent of the other test files' state.
"""
import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
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


def _tol(nrm, t):
    return 1e-12 * nrm * max(1.0, abs(t))


@pytest.mark.parametrize("name,nup,ndn,t,U", [("sq3x3", 4, 4, 1.0, 6.0), ("ring12", 6, 6, 1.3, 4.0)])
def test_noalloc_matches_oracle_and_apply_twice(dev, name, nup, ndn, t, U):
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    Hx = S.explicit()
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)       # fresh handle: no scratch allocated
    assert H.D <= hub.HUBBARD_NOALLOC_MAX_ELEMS
    v1 = start_vector(H.D, seed=21)
    # second call: a vector 1e6 times smaller, so a stale exponent word or
    # stale fixed-point data from the first call would show up as a large error
    v2 = 1e-6 * start_vector(H.D, seed=22)
    outs = []
    for v in (v1, v2):                                              # noalloc first, before any hubbard_apply
        vd = torch.from_numpy(v).to(dev)
        w_na = torch.full_like(vd, float("nan"))
        hub.hubbard_apply_noalloc(H, vd, w_na)
        torch.cuda.synchronize()
        got = w_na.cpu().numpy()
        assert np.abs(got - Hx @ v).max() <= _tol(np.linalg.norm(v), t)
        outs.append((vd, w_na))
    for v, (vd, w_na) in zip((v1, v2), outs):
        w_ref = torch.empty_like(vd)
        hub.hubbard_apply(H, vd, w_ref)
        torch.cuda.synchronize()
        assert (w_na - w_ref).abs().max().item() <= _tol(np.linalg.norm(v), t)
    H.close()


def test_noalloc_leaves_free_memory_unchanged(dev):
    ns, bonds = lattice_by_name("ring10")
    H = hub.hubbard_sector_create(ns, bonds, 5, 4, 1.0, 3.0)
    v = torch.from_numpy(start_vector(H.D, seed=5)).to(dev)
    w = torch.empty_like(v)
    hub.hubbard_apply_noalloc(H, v, w)              # warm-up: resolves the scratch address on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        hub.hubbard_apply_noalloc(H, v, w)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    H.close()


@pytest.mark.parametrize("scale", [2.0 ** 900, 2.0 ** -900, 1e-310, 3.7e12, 0.0])
@pytest.mark.parametrize("case", [("sq3x3", 4, 5, 1.0, 6.0), ("ring6", 3, 3, 0.75, 2.5), ("ring8", 4, 3, 1.3, 7.0)])
def test_noalloc_extreme_scales(dev, case, scale):
    """The fixed-point grid follows max|v| across the binary64 range; a
    non-dyadic t is applied before the power-of-two scaling, so results at
    subnormal scales keep their precision; the zero vector gives zero."""
    name, nup, ndn, t, U = case
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    u = start_vector(S.D, seed=79)
    v = u * scale
    ref = (S.explicit() @ u) * scale                   # no overflow in the reference
    vd = torch.from_numpy(v).to(dev)
    w = torch.full_like(vd, float("nan"))
    hub.hubbard_apply_noalloc(H, vd, w)
    got = w.cpu().numpy()
    assert np.all(np.isfinite(got))
    if scale == 0.0:
        assert not np.any(got)
    else:
        # subnormal inputs: the grid cannot go below the smallest subnormal
        floor = 4.95e-324 * (S.D ** 0.5) * 64 * max(1.0, abs(t))
        assert np.abs(got - ref).max() <= _tol(np.linalg.norm(u) * scale, t) + floor
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
