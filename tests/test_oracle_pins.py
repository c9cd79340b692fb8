"""Pins for the CPU oracle: values the paper prints, closed forms, symmetries
and brute force, each independent of the oracle's own code paths."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import closed_forms as cf
from oracle.basis import Sector, sector_dim, spin_states
from oracle.bethe import lieb_wu_ground_energy
from oracle.kron import KronHamiltonian
from oracle.lanczos import ground_energy_dense, lanczos_full, lanczos_plain
from workload import dimer, ring, square, start_vector, splitmix64

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RING4 = ring(4)


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def e0(ns, bonds, nup, ndn, t, U):
    """Lowest eigenvalue: dense eigvalsh for small sectors, scipy's sparse
    eigensolver (a library routine) for larger ones."""
    S = Sector(ns, bonds, nup, ndn, t, U)
    if S.D <= 2500:
        return ground_energy_dense(S.dense())
    from scipy.sparse.linalg import eigsh
    return float(eigsh(S.explicit(), k=1, which="SA", tol=1e-14, v0=start_vector(S.D, seed=9))[0][0])


# ---- Sec. 2.1: labelling -------------------------------------------------
def test_table1_labelling():
    S = Sector(4, RING4, 2, 3)
    assert S.D == 24
    for up, dn, iu, idn, J in _rows("table1.txt"):
        u, d = S.unrank(int(J))
        assert (int(u), int(d)) == (int(up, 2), int(dn, 2))
        assert int(J) == int(iu) * math.comb(4, 3) + int(idn)
        assert int(S.rank(np.array([int(up, 2)]), np.array([int(dn, 2)]))[0]) == int(J)


def test_worked_J_example():
    # 0101 x 1101 -> i_up = 1, i_dn = 2, J = 1*4 + 2 = 6
    assert list(spin_states(4, 2)).index(0b0101) == 1
    assert list(spin_states(4, 3)).index(0b1101) == 2
    assert int(Sector(4, RING4, 2, 3).rank(np.array([0b0101]), np.array([0b1101]))[0]) == 6


def test_dimensions_quoted_in_paper():
    assert sector_dim(12, 6, 6) == 853776
    assert round(sector_dim(14, 7, 7) / 1e6, 1) == 11.8
    assert round(sector_dim(16, 8, 8) / 1e6) == 166
    for ns, n in [(4, 2), (8, 3), (10, 5)]:
        assert len(spin_states(ns, n)) == math.comb(ns, n)
        assert np.all(np.diff(spin_states(ns, n)) > 0)


# ---- Sec. 2.1: matrix elements and signs ----------------------------------
@pytest.mark.parametrize("t", [1.0, 1.7])
def test_paper_sign_examples(t):
    H = Sector(4, RING4, 2, 3, t, 0.0).dense()
    for bra, ket, val in _rows("sign_examples.txt"):
        assert H[int(bra), int(ket)] == pytest.approx(int(val) * t, abs=0)


def _paper_rule_table(ns, bonds, n):
    """The paper's stated rule, literally: -1 per same-spin electron on sites
    whose labels lie strictly between origin and destination."""
    st = [s for s in range(1 << ns) if bin(s).count("1") == n]
    idx = {s: k for k, s in enumerate(st)}
    out = {}
    for k, s in enumerate(st):
        for i, j in bonds:
            for a, b in ((i, j), (j, i)):          # electron b -> a
                if (s >> b) & 1 and not (s >> a) & 1:
                    lo, hi = min(a, b), max(a, b)
                    between = sum((s >> m) & 1 for m in range(lo + 1, hi))
                    out[(idx[s ^ (1 << a) ^ (1 << b)], k)] = (-1) ** between
    return out


@pytest.mark.parametrize("ns,bonds,n", [(4, RING4, 2), (6, ring(6), 3), (6, square(3, 2), 2),
                                        (9, square(3, 3), 4), (8, square(4, 2), 5)])
def test_generic_jw_equals_paper_rule(ns, bonds, n):
    S = Sector(ns, bonds, n, n)
    states, rowptr, tgt, sign = S.spin_table(0)
    got = {}
    for r in range(len(states)):
        for k in range(rowptr[r], rowptr[r + 1]):
            got[(int(tgt[k]), r)] = int(sign[k])
    assert got == _paper_rule_table(ns, bonds, n)


@pytest.mark.parametrize("ns,bonds", [(8, ring(8)), (16, square(4, 4)), (12, square(4, 3)),
                                      (6, square(3, 2)), (8, square(4, 2))])
def test_hop_count_formula(ns, bonds):
    # each bond connects the states with exactly one end occupied: 2*C(Ns-2, N-1)
    for n in range(0, ns + 1):
        if math.comb(ns, n) > 20000:
            continue
        S = Sector(ns, bonds, n, 0)
        _, rowptr, _, _ = S.spin_table(0)
        assert rowptr[-1] == len(bonds) * 2 * (math.comb(ns - 2, n - 1) if n >= 1 else 0)


@pytest.mark.parametrize("ns,bonds,nup,ndn,U", [(8, ring(8), 4, 4, 4.0), (6, square(3, 2), 2, 5, 2.5),
                                                (9, square(3, 3), 3, 4, 7.0)])
def test_trace_and_hermiticity(ns, bonds, nup, ndn, U):
    H = Sector(ns, bonds, nup, ndn, 1.3, U).explicit()
    assert H.diagonal().sum() == pytest.approx(U * ns * math.comb(ns - 1, nup - 1) * math.comb(ns - 1, ndn - 1))
    assert abs(H - H.T).max() == 0.0
    # spin tables: r -> r' with sign s  <=>  r' -> r with sign s
    S = Sector(ns, bonds, nup, ndn, 1.3, U)
    for spin in (0, 1):
        _, rowptr, tgt, sign = S.spin_table(spin)
        pairs = {(r, int(tgt[k])): int(sign[k]) for r in range(len(rowptr) - 1)
                 for k in range(rowptr[r], rowptr[r + 1])}
        assert all(pairs[(b, a)] == s for (a, b), s in pairs.items())


def test_kronecker_sum_equals_explicit():
    # Eq. H-Kroneckersum: H_hop = H_up (x) I_dn + I_up (x) H_dn
    S = Sector(6, square(3, 2), 3, 2, 0.9, 2.0)
    Hu, Hd = S.spin_matrix(0), S.spin_matrix(1)
    K = sp.kron(Hu, sp.identity(S.Ddn)) + sp.kron(sp.identity(S.Dup), Hd) + sp.diags(S.diagonal())
    assert abs(K - S.explicit()).max() < 1e-15


# ---- closed forms -------------------------------------------------------
@pytest.mark.parametrize("t,U", [(1.0, 4.0), (1.0, 0.0), (0.7, 3.3), (2.0, 12.0)])
def test_dimer(t, U):
    assert e0(2, dimer(), 1, 1, t, U) == pytest.approx(cf.dimer_energy(t, U), abs=1e-13)
    if (t, U) == (1.0, 4.0):
        assert cf.dimer_energy(t, U) == pytest.approx(-0.82842712474619, abs=1e-13)


@pytest.mark.parametrize("ns,bonds,nup,ndn", [(6, ring(6), 4, 5), (6, ring(6), 2, 3), (6, square(3, 2), 5, 5),
                                              (8, ring(8), 6, 3)])
def test_atomic_limit(ns, bonds, nup, ndn):
    assert e0(ns, bonds, nup, ndn, 0.0, 2.5) == pytest.approx(cf.atomic_energy(ns, nup, ndn, 2.5), abs=1e-13)


@pytest.mark.parametrize("ns,bonds,nup,ndn", [(8, ring(8), 4, 4), (7, ring(7), 3, 2), (6, ring(6), 3, 3),
                                              (6, square(3, 2), 2, 3), (9, square(3, 3), 4, 4),
                                              (8, square(4, 2), 3, 5)])
def test_free_fermions(ns, bonds, nup, ndn):
    assert e0(ns, bonds, nup, ndn, 1.0, 0.0) == pytest.approx(cf.free_energy(ns, bonds, nup, ndn, 1.0), abs=1e-12)


def test_free_fermion_values():
    # one-body values, brute force on the Ns x Ns hopping matrix
    assert cf.free_energy(8, ring(8), 4, 4, 1.0) == pytest.approx(-4 - 4 * math.sqrt(2), abs=1e-12)
    assert cf.free_energy(16, square(4, 4), 8, 8, 1.0) == pytest.approx(-24.0, abs=1e-12)


@pytest.mark.parametrize("ns,bonds", [(6, ring(6)), (8, square(4, 2))])
def test_particle_hole(ns, bonds):
    U = 3.0
    for nup, ndn in [(1, 2), (2, 2), (1, 4), (3, 2)]:
        a = e0(ns, bonds, nup, ndn, 1.0, U)
        b = e0(ns, bonds, ns - nup, ns - ndn, 1.0, U)
        assert b == pytest.approx(a + U * (ns - nup - ndn), abs=1e-12)


def test_spin_flip_and_relabelling():
    ns, bonds = 9, square(3, 3)
    assert e0(ns, bonds, 2, 5, 1.0, 4.0) == pytest.approx(e0(ns, bonds, 5, 2, 1.0, 4.0), abs=1e-11)
    rng = np.random.default_rng(7)
    perm = rng.permutation(ns)
    pb = [(int(perm[i]), int(perm[j])) for i, j in bonds]
    for nup, ndn in [(2, 3), (1, 1), (2, 7)]:
        A = np.linalg.eigvalsh(Sector(ns, bonds, nup, ndn, 1.0, 4.0).dense())
        B = np.linalg.eigvalsh(Sector(ns, pb, nup, ndn, 1.0, 4.0).dense())
        assert np.abs(A - B).max() < 1e-11


# ---- Lanczos (Sec. 2.2) ---------------------------------------------------
def test_lanczos_matches_dense_ring8():
    S = Sector(8, ring(8), 4, 4, 1.0, 4.0)
    H = S.explicit()
    ed = ground_energy_dense(H.toarray())
    v0 = start_vector(S.D, seed=1234)
    r1 = lanczos_plain(lambda x: H @ x, v0, 100)
    r2 = lanczos_full(lambda x: H @ x, v0, 200, tol=1e-10)
    assert r1["energy"] == pytest.approx(ed, rel=1e-12)
    assert r2["energy"] == pytest.approx(ed, rel=1e-12)
    assert r2["residual"] < 1e-10


def test_lanczos_variational_and_a1():
    S = Sector(6, square(3, 2), 3, 3, 1.0, 5.0)
    H = S.explicit()
    ed = ground_energy_dense(H.toarray())
    v0 = start_vector(S.D, seed=3)
    f = v0 / np.linalg.norm(v0)
    thetas = [lanczos_full(lambda x: H @ x, v0, m)["energy"] for m in range(1, 25)]
    assert all(b <= a + 1e-12 for a, b in zip(thetas, thetas[1:]))
    assert all(th >= ed - 1e-12 for th in thetas)
    # a_1 is the Rayleigh quotient of the normalised start vector
    assert lanczos_plain(lambda x: H @ x, v0, 1)["a"][0] == pytest.approx(f @ (H @ f), rel=1e-14)


def test_lanczos_breakdown_on_tiny_sector():
    S = Sector(4, RING4, 1, 1, 1.0, 2.0)     # D = 16
    H = S.explicit()
    r = lanczos_full(lambda x: H @ x, start_vector(S.D, seed=5), 50)
    assert r["breakdown"] and r["iters"] <= S.D
    assert r["energy"] == pytest.approx(ground_energy_dense(H.toarray()), abs=1e-12)


# ---- sampled rows and the matrix-free C path ------------------------------
@pytest.mark.parametrize("ns,bonds,nup,ndn", [(8, ring(8), 4, 4), (9, square(3, 3), 4, 5), (6, square(3, 2), 1, 5)])
def test_rows_and_kron_match_explicit(ns, bonds, nup, ndn):
    S = Sector(ns, bonds, nup, ndn, 1.1, 6.0)
    v = start_vector(S.D, seed=11)
    ref = S.explicit() @ v
    J = np.random.default_rng(0).integers(0, S.D, 300)
    assert np.abs(S.rows_of_hv(J, v) - ref[J]).max() < 1e-13
    K = KronHamiltonian(ns, bonds, nup, ndn, 1.1, 6.0)
    assert np.abs(K.hv(v) - ref).max() < 1e-13


def test_golden_ring8_consistent():
    import json
    g = json.load(open(os.path.join(GOLD, "ring8_n4_4_U4.json")))
    assert g["e0_dense"] == pytest.approx(-4.603526299989137, abs=1e-12)
    assert g["lanczos_energy"] == pytest.approx(g["e0_dense"], rel=1e-12)


# ---- Sec. 1: the exact solution of the ring (Lieb-Wu Bethe ansatz) ----------
BETHE_SMALL = [(4, 1, 1, 1.0, 4.0), (4, 2, 2, 1.0, 4.0), (6, 3, 3, 1.0, 4.0), (6, 3, 2, 1.0, 5.0),
               (7, 3, 3, 1.0, 2.0), (8, 3, 3, 1.0, 6.0), (6, 1, 1, 1.0, 1.0), (8, 4, 4, 1.0, 4.0),
               (8, 4, 4, 0.7, 3.0), (10, 3, 3, 1.0, 4.0), (10, 5, 5, 1.0, 8.0), (9, 4, 3, 1.0, 2.5)]


@pytest.mark.parametrize("L,nup,ndn,t,U", BETHE_SMALL)
def test_bethe_ansatz_matches_diagonalisation(L, nup, ndn, t, U):
    """The Lieb-Wu equations against diagonalisation of the explicit H."""
    assert lieb_wu_ground_energy(L, nup, ndn, t, U) == pytest.approx(e0(L, ring(L), nup, ndn, t, U),
                                                                      rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("L,n", [(8, 3), (8, 4), (9, 4), (12, 5), (18, 9), (18, 8)])
def test_bethe_ansatz_polarised_is_free_fermions(L, n):
    """One spin species only (M = 0): the equations decouple to k = 2 pi I / L and
    the energy is that of free fermions on the ring, for any U."""
    ef = cf.free_energy(L, ring(L), n, 0, 1.0)
    for U in (0.5, 7.0):
        assert lieb_wu_ground_energy(L, n, 0, 1.0, U) == pytest.approx(ef, rel=1e-13, abs=1e-13)


def test_planted_bethe_parity_error_is_caught(monkeypatch):
    """A plausible mistake in the Bethe-ansatz oracle (the spin quantum numbers'
    parity rule inverted) fails the dense-diagonalisation pin."""
    import oracle.bethe as ob
    real = ob._consecutive

    def flipped(n, half):
        # ring 8, N = 8, M = 4: the sets of size M are the spin quantum numbers J
        return real(n, (not half) if n == 4 else half)

    monkeypatch.setattr(ob, "_consecutive", flipped)
    try:
        e_wrong = ob.lieb_wu_ground_energy(8, 4, 4, 1.0, 4.0)
    except ValueError:
        return                                           # no root at all: caught as well
    assert abs(e_wrong - e0(8, ring(8), 4, 4, 1.0, 4.0)) > 1e-3


def test_bethe_ansatz_open_shell_is_outside_its_class():
    # two electrons of each spin on 6 sites: the consecutive-quantum-number
    # states miss the ground state (so the pins above are not vacuous)
    assert lieb_wu_ground_energy(6, 2, 2, 1.0, 3.0) > e0(6, ring(6), 2, 2, 1.0, 3.0) + 0.1


@pytest.mark.parametrize("U", [4.0, 8.0])
def test_ring18_stored_energies_match_bethe_ansatz(U):
    """The stored 18-site energies (the oracle's matrix-free Lanczos on D = 2.4e9)
    against the exact solution."""
    import json
    g = json.load(open(os.path.join(GOLD, f"ring18_n9_9_U{U:g}.json")))
    assert g["e0"] == pytest.approx(lieb_wu_ground_energy(18, 9, 9, 1.0, U), rel=1e-12)


# ---- seeded inputs ----------------------------------------------------------
def test_splitmix64_reference_outputs():
    # first outputs of the published SplitMix64 reference for states 0 and 1234567
    assert int(splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF
    assert int(splitmix64(np.array([1234567], dtype=np.uint64))[0]) == 6457827717110365317
    v = start_vector(1000, seed=1234)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert np.array_equal(start_vector(10, seed=1234, start=500), v[500:510])


# ---- planted mistakes: the pins above must catch them -----------------------
def test_planted_sign_error_is_caught(monkeypatch):
    orig = Sector._hop

    def bosonic(self, occ, a, b):
        valid, new, sign = orig(self, occ, a, b)
        return valid, new, np.ones_like(sign)

    monkeypatch.setattr(Sector, "_hop", bosonic)
    assert abs(e0(8, ring(8), 4, 4, 1.0, 0.0) - cf.free_energy(8, ring(8), 4, 4, 1.0)) > 0.5


def test_planted_transposed_rank_is_caught(monkeypatch):
    def swapped(self, J):
        J = np.asarray(J, dtype=np.int64)
        return self.up[J % self.Dup], self.dn[J // self.Dup]

    monkeypatch.setattr(Sector, "unrank", swapped)
    S = Sector(4, RING4, 2, 3)
    up, dn, *_ = _rows("table1.txt")[1]
    u, d = S.unrank(1)
    assert (int(u), int(d)) != (int(up, 2), int(dn, 2))


def test_planted_dropped_interaction_is_caught(monkeypatch):
    monkeypatch.setattr(Sector, "diagonal", lambda self: np.zeros(self.D))
    assert abs(e0(2, dimer(), 1, 1, 1.0, 4.0) - cf.dimer_energy(1.0, 4.0)) > 0.1


@pytest.mark.parametrize("name,nup,ndn,U", [("ring6", 3, 3, 4.0), ("sq3x3", 2, 3, 6.5), ("ring7", 3, 2, 2.0)])
def test_energy_routes_agree(name, nup, ndn, U):
    """The three routes of oracle.energies (dense, eigsh on the explicit H,
    matrix-free Kronecker-sum Lanczos) give the same E0 where all apply."""
    from oracle.energies import ground_energy
    from workload import lattice_by_name
    ns, bonds = lattice_by_name(name)
    es = {r: ground_energy(ns, bonds, nup, ndn, 1.0, U, route=r)[0] for r in ("dense", "eigsh", "lanczos")}
    ref = es["dense"]
    for r, e in es.items():
        assert abs(e - ref) <= 1e-11 * max(1.0, abs(ref)), (r, e, ref)
