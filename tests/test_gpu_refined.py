"""GPU tests of the binary32 Lanczos and the binary32 + binary64-refined ground
state against the CPU oracle (energies within 1e-9 relative)."""
import json
import os

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
from workload import lattice_by_name, start_vector

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    return torch.device("cuda:0")


def _ref_energy(S):
    from scipy.sparse.linalg import eigsh
    if S.D <= 2000:
        return float(np.linalg.eigvalsh(S.dense())[0])
    return float(eigsh(S.explicit(), k=1, which="SA", tol=1e-14, v0=start_vector(S.D, seed=9))[0][0])


CASES = [("ring8", 4, 4, 1.0, 4.0), ("sq3x3", 4, 4, 1.0, 6.0), ("ring10", 5, 5, 1.0, 3.0),
         ("sq4x3", 2, 3, 1.0, 9.0), ("ring12", 3, 4, 1.0, 2.5), ("sq4x2", 3, 5, 1.0, 0.7)]


@pytest.mark.parametrize("case", CASES)
def test_f32_lanczos_energy(dev, case):
    name, nup, ndn, t, U = case
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    e = _ref_energy(S)
    v0 = torch.from_numpy(start_vector(S.D, seed=1234)).to(dev, torch.float32)
    r = hub.lanczos_ground_state(H, v0, 400, 1e-5)
    assert abs(r["energy"] - e) <= 2e-5 * max(1.0, abs(e))


@pytest.mark.parametrize("case", CASES)
def test_refined_energy_small(dev, case):
    name, nup, ndn, t, U = case
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    e = _ref_energy(S)
    v0 = torch.from_numpy(start_vector(S.D, seed=1234)).to(dev)
    psi = torch.empty_like(v0)
    r = hub.lanczos_ground_state_refined(H, v0, 1000, 1e-10, psi_out=psi)
    assert r["status"] == hub.HUB_OK, r
    assert abs(r["energy"] - e) <= 1e-9 * max(1.0, abs(e)), (r, e)
    # the stated bound covers the actual error (up to rounding)
    assert abs(r["energy"] - e) <= max(r["error_bound"], 1e-12 * max(1.0, abs(e)))
    # psi is the binary32 Ritz vector: unit norm, residual small
    p = psi.cpu().numpy()
    assert abs(np.linalg.norm(p) - 1.0) < 1e-12
    Hp = S.explicit() @ p
    th = p @ Hp
    assert np.linalg.norm(Hp - th * p) < 1e-3


def test_refined_sq4x4(dev):
    """4x4, (8,8), U=8: binary32 path refined in binary64 against the stored oracle energy."""
    ns, bonds = lattice_by_name("sq4x4")
    H = hub.hubbard_sector_create(ns, bonds, 8, 8, 1.0, 8.0)
    g = json.load(open(os.path.join(GOLD, "sq4x4_n8_8_U8.json")))
    v0 = torch.from_numpy(start_vector(H.D, seed=1234)).to(dev)
    r = hub.lanczos_ground_state_refined(H, v0, 1000, 1e-10)
    assert r["status"] == hub.HUB_OK, r
    assert abs(r["energy"] - g["e0"]) <= 1e-9 * abs(g["e0"]), r


def test_refined_stored_vectors_equal_replay(dev):
    """With room for the binary32 Lanczos vectors the Ritz vector is summed from
    the stored vectors instead of a replay: same operations in the same order,
    so psi and every reported number are bit-identical; with room for only some
    of them the replay resumes from the last two stored vectors."""
    ns, bonds = lattice_by_name("sq3x3")
    H = hub.hubbard_sector_create(ns, bonds, 4, 5, 1.0, 6.0)
    v0 = torch.from_numpy(start_vector(H.D, seed=21)).to(dev)
    outs = []
    for k in (0, 400, 4):
        psi = torch.empty(H.D, dtype=torch.float64, device=dev)
        r = hub.lanczos_ground_state_refined(H, v0, 1000, 1e-10, psi_out=psi, store_vectors=k)
        outs.append((r, psi))
    (r0, p0), (r1, p1), (r2, p2) = outs
    m = r0["iters_f32"]
    assert m > 4
    assert r0["replayed"] == m - 1 and r1["replayed"] == 0 and r2["replayed"] == m - 4
    for r, p in ((r1, p1), (r2, p2)):
        assert torch.equal(p, p0)
        assert {k: v for k, v in r.items() if k != "replayed"} == {k: v for k, v in r0.items() if k != "replayed"}


def _two_lowest(S):
    """E0 and the next distinct eigenvalue above it (dense, or ARPACK on the
    explicit H; a degenerate ground level counts once, as it does in the
    Temple-type bound)."""
    if S.D <= 2000:
        w = np.linalg.eigvalsh(S.dense())
    else:
        from scipy.sparse.linalg import eigsh
        w = np.sort(eigsh(S.explicit(), k=6, which="SA", tol=1e-14, v0=start_vector(S.D, seed=9))[0])
    above = w[w > w[0] + 1e-8 * max(1.0, abs(w[0]))]
    return float(w[0]), float(above[0])


@pytest.mark.parametrize("case", CASES[:4])
@pytest.mark.parametrize("iters_f32", [12, 1000])
def test_refined_gap_is_lower_estimate_and_bound_covers_error(dev, case, iters_f32):
    """The gap the refined solver reports is a lower estimate of lambda_2 - E0
    (the binary32 run's second Ritz value minus its residual), also when that
    run is cut short after 12 steps and lambda_2 is far from converged; the
    error bound then covers the actual error of the binary64 energy."""
    name, nup, ndn, t, U = case
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    e0, e1 = _two_lowest(S)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    v0 = torch.from_numpy(start_vector(S.D, seed=1234)).to(dev)
    r = hub.lanczos_ground_state_refined(H, v0, iters_f32, 1e-10)
    assert r["gap"] <= (e1 - e0) + 1e-9 * max(1.0, abs(e0)), (r, e1 - e0)
    err = abs(r["energy"] - e0)
    assert err <= r["error_bound"] + 1e-12 * max(1.0, abs(e0)), (r, e0)
    if r["status"] == hub.HUB_OK:
        assert err <= 1e-9 * max(1.0, abs(e0))


@pytest.mark.parametrize("case", CASES[:3] + [("ring6", 3, 3, 1.0, 0.0)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_plain_solver_psi_out_and_err_bound(dev, case, dt):
    """lanczos_ground_state with psi_out: the replayed Ritz vector is a unit
    vector whose binary64 Rayleigh quotient (the oracle's explicit H) is the
    returned energy and whose residual is small; err_bound covers the error."""
    name, nup, ndn, t, U = case
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, t, U)
    e0, _ = _two_lowest(S)
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U)
    tdt = torch.float64 if dt == "f64" else torch.float32
    v0 = torch.from_numpy(start_vector(S.D, seed=1234)).to(dev, tdt)
    psi = torch.full((S.D,), float("nan"), dtype=torch.float64, device=dev)
    tol = 1e-10 if dt == "f64" else 1e-5
    r = hub.lanczos_ground_state(H, v0, 1000, tol, psi_out=psi)
    assert r["status"] == hub.HUB_OK
    p = psi.cpu().numpy()
    assert abs(np.linalg.norm(p) - 1.0) < 1e-12
    Hp = S.explicit() @ p
    th = float(p @ Hp)
    res = float(np.linalg.norm(Hp - th * p))
    if dt == "f64":
        assert abs(r["energy"] - e0) <= 1e-9 * max(1.0, abs(e0))
        assert abs(th - e0) <= 1e-9 * max(1.0, abs(e0))
        assert res <= 1e-6
    else:
        assert abs(th - e0) <= 1e-6 * max(1.0, abs(e0))
        assert res <= 1e-2
    assert abs(r["energy"] - e0) <= r["err_bound"] + 1e-12 * max(1.0, abs(e0))


@pytest.mark.parametrize("iters", [20, 40])
def test_plain_solver_err_bound_when_stopped_early(dev, iters):
    """A run stopped before convergence reports a bound that still covers its
    (large) error: the second Ritz pair then resolves little of the gap."""
    ns, bonds = lattice_by_name("ring10")
    S = Sector(ns, bonds, 5, 5, 1.0, 3.0)
    e0, e1 = _two_lowest(S)
    H = hub.hubbard_sector_create(ns, bonds, 5, 5, 1.0, 3.0)
    v0 = torch.from_numpy(start_vector(S.D, seed=1234)).to(dev)
    r = hub.lanczos_ground_state(H, v0, iters, 0.0)
    err = abs(r["energy"] - e0)
    assert err > 1e-9 * abs(e0)                        # genuinely unconverged
    assert err <= r["err_bound"]
