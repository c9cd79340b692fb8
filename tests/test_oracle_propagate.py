"""Pins of the time-propagation oracle (oracle/propagate.py): closed forms,
brute force and the invariants of exp(-iHt), plus planted mistakes they catch."""
import numpy as np
import pytest

from oracle import propagate as pr
from oracle.basis import Sector
from workload import lattice_by_name, ring, start_vector


def _cvec(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)


@pytest.mark.parametrize("t_hop,U,time", [(1.0, 4.0, 0.37), (0.7, 0.0, -1.9), (1.3, 9.5, 2.6), (1.0, -2.0, 0.05)])
def test_dense_matches_dimer_closed_form(t_hop, U, time):
    v = _cvec(4, 1)
    got = pr.evolve_dense(pr.dimer_sector(t_hop, U), v, time)
    assert np.abs(got - pr.dimer_evolution(t_hop, U, v, time)).max() <= 1e-13 * np.linalg.norm(v)


@pytest.mark.parametrize("ns,time", [(3, 0.8), (5, -1.4), (8, 2.3), (11, 0.61)])
def test_dense_matches_ring_one_pair_closed_form(ns, time):
    """U = 0, one electron of each spin: the Kronecker product of the
    plane-wave one-body propagator."""
    S = Sector(ns, ring(ns), 1, 1, 1.0, 0.0)
    v = _cvec(S.D, ns)
    got = pr.evolve_dense(S, v, time)
    assert np.abs(got - pr.ring_one_pair_evolution(ns, 1.0, v, time)).max() <= 1e-12 * np.linalg.norm(v)


@pytest.mark.parametrize("name,nup,ndn,U,time", [
    ("ring6", 3, 2, 4.0, 0.37), ("sq2x3", 2, 2, 7.0, -1.3), ("ring5", 2, 2, 1.5, 2.2), ("sq3x3", 2, 1, 3.0, 0.9),
])
def test_dense_matches_taylor_series(name, nup, ndn, U, time):
    """Sectors with Jordan-Wigner signs (several electrons per spin, 2D)."""
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, 1.0, U)
    v = _cvec(S.D, 3)
    got = pr.evolve_dense(S, v, time)
    assert np.abs(got - pr.evolve_taylor(S, v, time)).max() <= 1e-11 * np.linalg.norm(v)


@pytest.mark.parametrize("name,nup,ndn,U,time", [("ring8", 4, 4, 4.0, 0.7), ("sq2x4", 3, 2, 6.0, -0.45)])
def test_sparse_route_matches_dense(name, nup, ndn, U, time):
    ns, bonds = lattice_by_name(name)
    S = Sector(ns, bonds, nup, ndn, 1.0, U)
    v = _cvec(S.D, 5)
    got = pr.evolve_sparse(S, v, time)
    assert np.abs(got - pr.evolve_dense(S, v, time)).max() <= 1e-11 * np.linalg.norm(v)


@pytest.mark.parametrize("name,nup,ndn,time", [("ring6", 3, 2, 0.9), ("sq2x3", 2, 3, -1.4), ("ring7", 3, 3, 2.1),
                                              ("sq3x3", 2, 2, 0.6)])
def test_dense_matches_slater_determinants_at_u0(name, nup, ndn, time):
    """U = 0 with several electrons of a spin: the Jordan-Wigner signs of the
    many-body propagation against determinants of propagated orbitals."""
    ns, bonds = lattice_by_name(name)
    rng = np.random.default_rng(7)
    phi_up = rng.normal(size=(ns, nup)) + 1j * rng.normal(size=(ns, nup))
    phi_dn = rng.normal(size=(ns, ndn)) + 1j * rng.normal(size=(ns, ndn))
    S = Sector(ns, bonds, nup, ndn, 1.0, 0.0)
    v = pr.slater_state(ns, nup, ndn, phi_up, phi_dn)
    want = pr.slater_evolution(ns, bonds, 1.0, nup, ndn, phi_up, phi_dn, time)
    got = pr.evolve_dense(S, v, time)
    assert np.abs(got - want).max() <= 1e-11 * np.linalg.norm(v)


def test_invariants_of_the_propagator():
    """Unitarity, energy conservation, the group property, time reversal and
    (real H, real v) psi(-t) = conj(psi(t)); an eigenvector only gains its phase."""
    ns, bonds = lattice_by_name("ring7")
    S = Sector(ns, bonds, 3, 2, 1.0, 5.0)
    H = S.explicit()
    v = _cvec(S.D, 11)
    p1 = pr.evolve_dense(S, v, 0.8)
    assert abs(np.linalg.norm(p1) - np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(v)
    e0 = np.vdot(v, H @ v).real
    assert abs(np.vdot(p1, H @ p1).real - e0) <= 1e-11 * np.linalg.norm(v) ** 2 * max(1.0, abs(e0))
    p2 = pr.evolve_dense(S, p1, 1.1)
    assert np.abs(p2 - pr.evolve_dense(S, v, 1.9)).max() <= 1e-12 * np.linalg.norm(v)
    assert np.abs(pr.evolve_dense(S, p1, -0.8) - v).max() <= 1e-12 * np.linalg.norm(v)
    vr = start_vector(S.D, seed=4)
    assert np.abs(pr.evolve_dense(S, vr, -0.6) - np.conj(pr.evolve_dense(S, vr, 0.6))).max() <= 1e-12
    w, phi = np.linalg.eigh(S.dense())
    k = 3
    assert np.abs(pr.evolve_dense(S, phi[:, k], 1.7) - np.exp(-1.7j * w[k]) * phi[:, k]).max() <= 1e-12


def test_dimer_ground_state_gains_its_phase():
    """The dimer ground state, from its closed form, picks up exp(-i E0 t):
    fixes the sign of the time in exp(-iHt)."""
    t_hop, U, time = 1.0, 4.0, 0.9
    W = np.sqrt(U * U / 4 + 4 * t_hop * t_hop)
    E0 = U / 2 - W
    # eigenvector of [[U, -2t], [-2t, 0]] at E0 in (a, s), mapped to J = 0..3
    alpha, sigma = 2 * t_hop, U - E0
    n = np.hypot(alpha, sigma)
    alpha, sigma = alpha / n, sigma / n
    r2 = np.sqrt(0.5)
    phi = np.array([r2 * alpha, r2 * sigma, r2 * sigma, r2 * alpha])
    S = pr.dimer_sector(t_hop, U)
    assert np.abs(S.dense() @ phi - E0 * phi).max() <= 1e-14
    for f in (lambda v, tt: pr.evolve_dense(S, v, tt), lambda v, tt: pr.dimer_evolution(t_hop, U, v, tt)):
        assert np.abs(f(phi, time) - np.exp(-1j * E0 * time) * phi).max() <= 1e-14


# ---- planted mistakes: the pins above must catch them -----------------------
def test_planted_time_sign_is_caught(monkeypatch):
    orig = pr.evolve_dense
    monkeypatch.setattr(pr, "evolve_dense", lambda S, v, t: orig(S, v, -t))
    v = _cvec(4, 1)
    got = pr.evolve_dense(pr.dimer_sector(1.0, 4.0), v, 0.37)
    assert np.abs(got - pr.dimer_evolution(1.0, 4.0, v, 0.37)).max() > 1e-3


def test_planted_dropped_interaction_is_caught(monkeypatch):
    monkeypatch.setattr(Sector, "diagonal", lambda self: np.zeros(self.D))
    v = _cvec(4, 2)
    got = pr.evolve_dense(pr.dimer_sector(1.0, 4.0), v, 0.5)
    assert np.abs(got - pr.dimer_evolution(1.0, 4.0, v, 0.5)).max() > 1e-3


def test_planted_bosonic_sign_is_caught(monkeypatch):
    """A sign-free hop changes the dynamics of a sector with two electrons of
    one spin on a ring (the Taylor route uses the same H, so the comparison
    is with the correct H's dense propagation)."""
    ns, bonds = lattice_by_name("ring5")
    S = Sector(ns, bonds, 2, 1, 1.0, 3.0)
    v = _cvec(S.D, 6)
    want = pr.evolve_dense(S, v, 0.9)
    orig = Sector._hop

    def bosonic(self, occ, a, b):
        valid, new, sign = orig(self, occ, a, b)
        return valid, new, np.ones_like(sign)

    monkeypatch.setattr(Sector, "_hop", bosonic)
    got = pr.evolve_dense(Sector(ns, bonds, 2, 1, 1.0, 3.0), v, 0.9)
    assert np.abs(got - want).max() > 1e-3
    # and the determinant pin fails for it at U = 0
    rng = np.random.default_rng(7)
    phi_up, phi_dn = rng.normal(size=(ns, 2)), rng.normal(size=(ns, 1))
    vs = pr.slater_state(ns, 2, 1, phi_up, phi_dn)
    bos = pr.evolve_dense(Sector(ns, bonds, 2, 1, 1.0, 0.0), vs, 0.9)
    assert np.abs(bos - pr.slater_evolution(ns, bonds, 1.0, 2, 1, phi_up, phi_dn, 0.9)).max() > 1e-3
