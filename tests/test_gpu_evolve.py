"""GPU parity of the time propagator psi(t) = exp(-iHt) v (hubbard_time_evolve,
through the C ABI) against the CPU oracle (oracle/propagate.py).

Tolerance: the propagator sizes its steps so that its a-posteriori error
estimates sum to about tol * |v| (an estimate, not a proven bound, of the
truncation of the Krylov expansion), and the binary64 fixed-point H*v adds
rounding of about 1e-15 |v| per step.  The tests ask for
max-abs error <= 10 * tol * |v|_2 + 1e-12 * |v|_2.
"""
import math

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle import propagate as pr
from oracle.basis import Sector
from workload import lattice_by_name, start_vector

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    return torch.device("cuda:0")


def _sector(name, nup, ndn, t, U):
    ns, bonds = lattice_by_name(name)
    return hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U), Sector(ns, bonds, nup, ndn, t, U)


def _start(D, seed, dev, imag=True):
    vr = torch.from_numpy(start_vector(D, seed=seed)).to(dev)
    vi = torch.from_numpy(start_vector(D, seed=seed + 1000)).to(dev) if imag else None
    return vr, vi


def _host(vr, vi):
    v = vr.cpu().numpy().astype(np.complex128)
    if vi is not None:
        v = v + 1j * vi.cpu().numpy()
    return v


def _err_ok(got, want, v, tol=TOL):
    nv = np.linalg.norm(v)
    err = np.abs(got - want).max()
    return err <= 10 * tol * nv + 1e-12 * nv, err


@pytest.mark.parametrize("case,t,K,imag", [
    (("dimer", 1, 1, 1.0, 4.0), 0.9, 40, True),
    (("ring6", 3, 2, 1.0, 4.0), -1.7, 40, True),
    (("sq3x2", 2, 2, 1.0, 7.0), 2.9, 12, True),
    (("ring8", 4, 4, 1.0, 4.0), 0.3, 40, False),
    (("ring8", 4, 4, 1.0, 4.0), 3.1, 16, True),
    (("sq3x3", 2, 3, 0.8, 5.0), -0.6, 24, True),
    (("ring7", 3, 3, 1.3, 0.0), 1.2, 30, False),
])
def test_evolve_matches_oracle(dev, case, t, K, imag):
    """Both routes (stored Lanczos vectors, replayed recurrence) against the
    oracle's eigendecomposition; the two routes agree bit for bit."""
    H, S = _sector(*case)
    vr, vi = _start(S.D, 11, dev, imag)
    want = pr.evolve_dense(S, _host(vr, vi), t)
    outs = []
    for store in (True, False):
        ore, oim, info = hub.hubbard_time_evolve(H, vr, vi, t, krylov_max=K, tol=TOL, store_basis=store)
        got = ore.cpu().numpy() + 1j * oim.cpu().numpy()
        ok, err = _err_ok(got, want, _host(vr, vi))
        assert ok, (case, t, K, store, err, info)
        assert info["status"] == hub.HUB_OK and info["steps"] >= 1 and info["krylov_dim"] <= min(K, S.D)
        assert abs(info["norm"] - np.linalg.norm(want)) <= 1e-9 * np.linalg.norm(want)
        outs.append((ore.clone(), oim.clone(), info))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert outs[1][2]["hv"] > outs[0][2]["hv"]                 # the replay applies H again
    H.close()


def test_short_krylov_forces_steps_and_stays_accurate(dev):
    """krylov_max = 6 over a long time: many propagation steps, same accuracy."""
    H, S = _sector("ring6", 3, 3, 1.0, 3.0)
    vr, vi = _start(S.D, 5, dev)
    ore, oim, info = hub.hubbard_time_evolve(H, vr, vi, 4.0, krylov_max=6, tol=1e-9)
    assert info["steps"] > 10 and info["krylov_dim"] == 6
    ok, err = _err_ok(ore.cpu().numpy() + 1j * oim.cpu().numpy(), pr.evolve_dense(S, _host(vr, vi), 4.0),
                      _host(vr, vi), tol=1e-9)
    assert ok, err
    H.close()


@pytest.mark.parametrize("case,t", [(("ring12", 5, 5, 1.0, 4.0), 0.25), (("sq3x4", 5, 5, 1.0, 6.0), -0.2)])
def test_evolve_large_sectors_vs_expm_multiply(dev, case, t):
    """Sectors of 6.3e5 elements (ragged rows, 2D signs) against the oracle's
    expm_multiply route on the explicit sparse H."""
    H, S = _sector(*case)
    vr, vi = _start(S.D, 21, dev)
    ore, oim, info = hub.hubbard_time_evolve(H, vr, vi, t, krylov_max=40, tol=TOL)
    want = pr.evolve_sparse(S, _host(vr, vi), t)
    ok, err = _err_ok(ore.cpu().numpy() + 1j * oim.cpu().numpy(), want, _host(vr, vi))
    assert ok, (case, err, info)
    H.close()


def test_full_size_sq4x4_invariants(dev):
    """4x4 (8,8) U = 8 (1.66e8 elements): the norm is conserved, the energy
    <psi|H|psi> (the oracle's Kronecker-sum H*v) is conserved, and evolving
    back by -t returns v."""
    from oracle.kron import KronHamiltonian
    ns, bonds = lattice_by_name("sq4x4")
    H = hub.hubbard_sector_create(ns, bonds, 8, 8, 1.0, 8.0)
    v = torch.from_numpy(start_vector(H.D, seed=1234)).to(dev)
    v /= torch.linalg.vector_norm(v)
    ws = torch.empty(hub.hubbard_evolve_workspace_bytes(H, 30, store_basis=False), dtype=torch.uint8, device=dev)
    ore, oim, info = hub.hubbard_time_evolve(H, v, None, 0.05, krylov_max=30, tol=TOL, workspace=ws,
                                             store_basis=False)
    assert abs(info["norm"] - 1.0) <= 1e-9, info
    K = KronHamiltonian(ns, bonds, 8, 8, 1.0, 8.0)
    vh = v.cpu().numpy()
    e0 = float(np.dot(vh, K.hv(vh)))
    pr_, pi_ = ore.cpu().numpy(), oim.cpu().numpy()
    e1 = float(np.dot(pr_, K.hv(pr_)) + np.dot(pi_, K.hv(pi_)))
    assert abs(e1 - e0) <= 5e-8 * max(1.0, abs(e0)), (e0, e1, info)
    del pr_, pi_
    bre, bim, info2 = hub.hubbard_time_evolve(H, ore, oim, -0.05, krylov_max=30, tol=TOL, workspace=ws,
                                              store_basis=False)
    back = torch.sqrt(torch.sum((bre - v) ** 2) + torch.sum(bim ** 2)).item()
    assert back <= 5e-10, (back, info2)
    H.close()


def test_u0_slater_state_full_size_sq4x4(dev):
    """U = 0 on the 4x4 (8,8) sector (1.66e8 elements): a product of Slater
    determinants of orthonormal orbitals propagates as the determinants of its
    orbitals under the one-body exp(-iht) (the oracle's closed form); every
    element is compared."""
    ns, bonds = lattice_by_name("sq4x4")
    rng = np.random.default_rng(3)
    pu = np.linalg.qr(rng.normal(size=(ns, 8)))[0]
    pd = np.linalg.qr(rng.normal(size=(ns, 8)))[0]
    v = pr.slater_state(ns, 8, 8, pu, pd).real.copy()
    H = hub.hubbard_sector_create(ns, bonds, 8, 8, 1.0, 0.0)
    vd = torch.from_numpy(v).to(dev)
    del v
    ws = torch.empty(hub.hubbard_evolve_workspace_bytes(H, 30, store_basis=False), dtype=torch.uint8, device=dev)
    ore, oim, info = hub.hubbard_time_evolve(H, vd, None, 0.05, krylov_max=30, tol=TOL, workspace=ws,
                                             store_basis=False)
    want = pr.slater_evolution(ns, bonds, 1.0, 8, 8, pu, pd, 0.05)
    err = max(np.abs(ore.cpu().numpy() - want.real).max(), np.abs(oim.cpu().numpy() - want.imag).max())
    assert err <= 10 * TOL + 1e-12, (err, info)
    H.close()


def test_large_sector_stored_basis_equals_replay(dev):
    """Ring 14 (6,7), 1.0e7 elements: large enough for the host-driven steps,
    where the recurrence runs inside the stored basis (no copies); it equals
    the replayed route bit for bit, conserves the norm and the energy (oracle
    Kronecker-sum H*v), and a second, complex step goes through both parts."""
    from oracle.kron import KronHamiltonian
    ns, bonds = lattice_by_name("ring14")
    H = hub.hubbard_sector_create(ns, bonds, 6, 7, 1.0, 5.0)
    assert H.D > 4_000_000
    v = torch.from_numpy(start_vector(H.D, seed=8)).to(dev)
    v /= torch.linalg.vector_norm(v)
    outs = []
    for store in (True, False):
        ore, oim, info = hub.hubbard_time_evolve(H, v, None, 0.3, krylov_max=24, tol=TOL, store_basis=store)
        outs.append((ore.clone(), oim.clone(), info))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    ore, oim, info = outs[0]
    assert info["steps"] >= 2 and abs(info["norm"] - 1.0) <= 1e-9, info
    K = KronHamiltonian(ns, bonds, 6, 7, 1.0, 5.0)
    vh = v.cpu().numpy()
    e0 = float(np.dot(vh, K.hv(vh)))
    a, b = ore.cpu().numpy(), oim.cpu().numpy()
    e1 = float(np.dot(a, K.hv(a)) + np.dot(b, K.hv(b)))
    assert abs(e1 - e0) <= 1e-8 * max(1.0, abs(e0)), (e0, e1, info)
    H.close()


def test_ground_state_only_gains_its_phase(dev):
    """The Ritz vector of lanczos_ground_state on ring 12 (5,6) evolves as
    exp(-i E0 t) psi0 up to its residual times t."""
    ns, bonds = lattice_by_name("ring12")
    H = hub.hubbard_sector_create(ns, bonds, 5, 6, 1.0, 4.0)
    v0 = torch.from_numpy(start_vector(H.D, seed=3)).to(dev)
    psi = torch.empty_like(v0)
    r = hub.lanczos_ground_state(H, v0, max_iters=600, tol=1e-11, psi_out=psi)
    t = 0.7
    ore, oim, info = hub.hubbard_time_evolve(H, psi, None, t, krylov_max=40, tol=TOL)
    ph = complex(math.cos(r["energy"] * t), -math.sin(r["energy"] * t))
    err = max((ore - ph.real * psi).abs().max().item(), (oim - ph.imag * psi).abs().max().item())
    assert err <= 10 * TOL + 2 * r["residual"] * t + 1e-12, (err, r["residual"], info)
    H.close()


def test_dimer_closed_form_and_time_symmetry(dev):
    """The dimer against its closed form; for a real v, psi(-t) = conj(psi(t))."""
    H, S = _sector("dimer", 1, 1, 1.0, 4.0)
    v = torch.tensor([0.3, -0.8, 0.1, 0.5], dtype=torch.float64, device=dev)
    for t in (0.37, 2.5):
        ore, oim, _ = hub.hubbard_time_evolve(H, v, None, t, krylov_max=4, tol=1e-12)
        got = ore.cpu().numpy() + 1j * oim.cpu().numpy()
        assert np.abs(got - pr.dimer_evolution(1.0, 4.0, v.cpu().numpy(), t)).max() <= 1e-11
        bre, bim, _ = hub.hubbard_time_evolve(H, v, None, -t, krylov_max=4, tol=1e-12)
        assert (bre - ore).abs().max().item() <= 1e-14 and (bim + oim).abs().max().item() <= 1e-14
    H.close()


def test_edge_cases(dev):
    """t = 0 copies v; a zero v gives zero; outputs may alias the inputs; a
    sector of dimension 1; a one-vector Krylov space cannot meet a strict
    tol (HUB_ENOTCONV); argument errors."""
    H, S = _sector("ring6", 3, 2, 1.0, 4.0)
    vr, vi = _start(S.D, 2, dev)
    ore, oim, info = hub.hubbard_time_evolve(H, vr, vi, 0.0)
    assert torch.equal(ore, vr) and torch.equal(oim, vi) and info["steps"] == 0
    z = torch.zeros_like(vr)
    ore, oim, info = hub.hubbard_time_evolve(H, z, None, 1.0)
    assert float(ore.abs().max()) == 0.0 and float(oim.abs().max()) == 0.0
    want = pr.evolve_dense(S, _host(vr, vi), 0.8)
    a, b = vr.clone(), vi.clone()
    hub.hubbard_time_evolve(H, a, b, 0.8, out_re=a, out_im=b)
    assert _err_ok(a.cpu().numpy() + 1j * b.cpu().numpy(), want, _host(vr, vi))[0]
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_time_evolve(H, vr, None, 1.0, krylov_max=1, tol=1e-14)
    assert ei.value.code == hub.HUB_ENOTCONV
    for kw in (dict(krylov_max=0), dict(krylov_max=1025), dict(tol=0.0), dict(tol=float("nan"))):
        with pytest.raises(hub.HubError) as ei:
            hub.hubbard_time_evolve(H, vr, None, 1.0, **kw)
        assert ei.value.code == hub.HUB_EINVAL, kw
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_time_evolve(H, vr, None, float("inf"))
    assert ei.value.code == hub.HUB_EINVAL
    small = torch.empty(16, dtype=torch.uint8, device=dev)
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_time_evolve(H, vr, None, 1.0, workspace=small)
    assert ei.value.code == hub.HUB_ENOMEM
    both = torch.empty(S.D + 2, dtype=torch.float64, device=dev)
    with pytest.raises(hub.HubError) as ei:                  # out_re and out_im overlap
        hub.hubbard_time_evolve(H, vr, None, 1.0, out_re=both[:S.D], out_im=both[2:])
    assert ei.value.code == hub.HUB_EINVAL
    H.close()
    H1, S1 = _sector("ring4", 4, 4, 1.0, 2.0)                 # D = 1: every site doubly occupied, E = 4 U
    one = torch.ones(1, dtype=torch.float64, device=dev)
    ore, oim, info = hub.hubbard_time_evolve(H1, one, None, 0.9)
    e = float(S1.dense()[0, 0])
    assert abs(ore.item() - math.cos(e * 0.9)) <= 1e-14 and abs(oim.item() + math.sin(e * 0.9)) <= 1e-14
    H1.close()
