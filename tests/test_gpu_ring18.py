"""Config 3 at full size: the 18-site ring, N = (9, 9), D = 48620^2 = 2.36e9.

* binary32 and binary64 H*v on sampled outputs against the oracle's rows of
  H*v (start-vector entries generated on demand from the seeded recipe);
* the binary32 + binary64-refined ground state against the binary64 Lanczos
  on the same GPU and seed (1e-9 relative), and against the oracle's stored
  energy when tests/golden/ring18_n9_9_U4.json exists;
* at U = 8, the refined ground state against the oracle (ring18_n9_9_U8.json);
* at U = 2, the refined ground state against the exact solution of the ring
  (Lieb-Wu Bethe ansatz, ring18_n9_9_U2.json).
"""
import json
import os

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
from workload import lattice_by_name, start_vector_at, start_vector_into

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ring18():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    free, _ = torch.cuda.mem_get_info()
    if free < 140e9:
        pytest.skip("needs ~140 GB of device memory")
    ns, bonds = lattice_by_name("ring18")
    H = hub.hubbard_sector_create(ns, bonds, 9, 9, 1.0, 4.0)
    S = Sector(ns, bonds, 9, 9, 1.0, 4.0)
    v = np.empty(H.D)
    start_vector_into(v, 1234)
    vd = torch.from_numpy(v).to("cuda")
    del v
    yield H, S, vd
    del vd
    H.close()
    torch.cuda.empty_cache()


def test_ring18_hv_sampled_rows(ring18):
    H, S, vd = ring18
    rng = np.random.default_rng(18)
    J = np.concatenate([rng.integers(0, H.D, 3000), np.arange(40), H.D - 1 - np.arange(40)])
    ref = S.rows_of_hv(J, lambda idx: start_vector_at(idx, seed=1234))
    Jt = torch.from_numpy(J).to("cuda")
    w = torch.empty_like(vd)
    hub.hubbard_apply(H, vd, w)                               # binary64 (fixed-point hop sums)
    got = w[Jt].cpu().numpy()
    nrm = float(vd.norm())
    assert np.abs(got - ref).max() <= 1e-12 * nrm
    del w
    v32 = vd.float()
    w32 = torch.empty_like(v32)
    hub.hubbard_apply(H, v32, w32)                            # binary32
    got32 = w32[Jt].double().cpu().numpy()
    tol32 = 4e-7 * (H.Wup + H.Wdn + 1) * max(1.0, 4.0 * 18) * float(vd.abs().max())
    assert np.abs(got32 - ref).max() <= tol32
    del v32, w32
    torch.cuda.empty_cache()


def test_ring18_refined_vs_f64(ring18):
    H, S, vd = ring18
    r32 = hub.lanczos_ground_state_refined(H, vd, 1000, 1e-10)
    assert r32["status"] == hub.HUB_OK, r32
    torch.cuda.empty_cache()
    r64 = hub.lanczos_ground_state(H, vd, 600, 1e-10)
    assert r64["status"] == hub.HUB_OK
    assert abs(r32["energy"] - r64["energy"]) <= 1e-9 * abs(r64["energy"])
    path = os.path.join(GOLD, "ring18_n9_9_U4.json")
    if os.path.exists(path):
        e = json.load(open(path))["e0"]
        assert abs(r32["energy"] - e) <= 1e-9 * abs(e)
        assert abs(r64["energy"] - e) <= 1e-9 * abs(e)


@pytest.mark.parametrize("U", [8.0, 2.0])
def test_ring18_refined_vs_stored_energy(ring18, U):
    """U = 8 (stronger coupling, 258 oracle iterations; the oracle's matrix-free
    Lanczos energy) and U = 2 (the Bethe-ansatz energy): binary32 Lanczos +
    binary64 refinement."""
    _, _, vd = ring18
    path = os.path.join(GOLD, f"ring18_n9_9_U{U:g}.json")
    if not os.path.exists(path):
        pytest.skip(f"no U={U:g} stored value")
    e = json.load(open(path))["e0"]
    ns, bonds = lattice_by_name("ring18")
    H8 = hub.hubbard_sector_create(ns, bonds, 9, 9, 1.0, U)
    try:
        r = hub.lanczos_ground_state_refined(H8, vd, 1000, 1e-10)
        assert r["status"] == hub.HUB_OK, r
        assert abs(r["energy"] - e) <= 1e-9 * abs(e), (r, e)
    finally:
        H8.close()
        torch.cuda.empty_cache()
