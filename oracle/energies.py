"""Ground-state energy of one sector by the cheapest exact oracle route.

Test infrastructure only (imported by tests/ and by the benchmark's
CPU-baseline leg, never by the library).  E0 is the smallest eigenvalue of
Eq. (1) in the (N_up, N_dn) sector (Sec. 2.1); the route depends on size:

  * D <= 3000: dense diagonalisation of the explicit H (numpy eigvalsh);
  * D <= 300000: scipy's eigsh (implicitly restarted Lanczos, ARPACK) on the
    explicit sparse H, tolerance 1e-14;
  * larger: the plain-C Kronecker-sum H*v (the paper's CPU scheme, Sec. 5)
    driven by Algorithm 1 in its two-vector form to rho < 1e-11 (the lowest
    Ritz value is unaffected by the loss of orthogonality; Sec. 2.2).

Each route is one of the oracle's pinned routines; tests/test_oracle_pins.py
checks that adjacent routes agree where both apply.
"""
from .basis import Sector
from .lanczos import ground_energy_dense

DENSE_MAX = 3000
EIGSH_MAX = 300_000


def ground_energy(ns, bonds, nup, ndn, t, U, seed=1234, route=None):
    """Returns (E0, route name).  `seed` fixes the start vector of the iterative routes."""
    from workload import start_vector
    S = Sector(ns, bonds, nup, ndn, t, U)
    if route is None:
        route = "dense" if S.D <= DENSE_MAX else ("eigsh" if S.D <= EIGSH_MAX else "lanczos")
    if S.D == 1 or route == "dense":
        return ground_energy_dense(S.dense()), "dense"
    if route == "eigsh":
        from scipy.sparse.linalg import eigsh
        w = eigsh(S.explicit(), k=1, which="SA", tol=1e-14, v0=start_vector(S.D, seed=seed))[0]
        return float(w[0]), "eigsh"
    from .kron import KronHamiltonian, lanczos_matrix_free
    K = KronHamiltonian(ns, bonds, nup, ndn, t, U)
    r = lanczos_matrix_free(K, start_vector(S.D, seed=seed), min(S.D, 3000), tol=1e-11, inplace=True)
    return float(r["energy"]), "lanczos"
