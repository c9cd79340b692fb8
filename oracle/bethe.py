"""Ground-state energy of the periodic Hubbard ring from the Bethe ansatz.

Test infrastructure only: imported by tests/ and tests/golden/ scripts, never by
the library.

The paper (Sec. 1) notes that the one-dimensional model has an exact solution
(Lieb and Wu).  That solution gives an independent check of the ring energies the
oracle's Lanczos produces, at sizes where no explicit matrix fits.  This module
restates the published Lieb-Wu equations (E. H. Lieb and F. Y. Wu, Phys. Rev.
Lett. 20, 1445 (1968)) for H = -t sum (c+ c + h.c.) + U sum n_up n_dn on L sites
with periodic boundary conditions for the fermions (which is what the
Jordan-Wigner signs of Sec. 2.1 give on a ring), N electrons of which M carry
the minority spin.  With u = U / (4t) and theta(x) = 2 arctan(x), the real
charge momenta k_j (j = 1..N) and spin rapidities L_a (a = 1..M) of the ground
state solve, in logarithmic form,

    L k_j                                  = 2 pi I_j - sum_b theta((sin k_j - L_b) / u)
    sum_j theta((L_a - sin k_j) / u)       = 2 pi J_a + sum_b theta((L_a - L_b) / (2u))

and E = -2t sum_j cos k_j.  Taking the logarithm of the product form fixes the
parities: I_j is an integer when M is even and a half-odd integer when M is odd;
J_a is an integer when N - M + 1 is even and a half-odd integer when it is odd.
The ground state takes consecutive quantum numbers, as symmetric about zero as
their parity allows.  When the parity forbids a symmetric set there are two
candidates; all candidates are solved and the lowest energy is returned.  That
class holds the ground state for the fillings the tests use (checked against
dense diagonalisation there); fillings whose non-interacting ground state is an
open shell (e.g. two electrons of each spin on 5 or 6 sites) can have their
ground state outside it, which the tests show and avoid.
"""
import numpy as np
from scipy.optimize import root


def _theta(x):
    return 2.0 * np.arctan(x)


def _consecutive(n, half):
    """n consecutive numbers on Z (half=False) or Z + 1/2 (half=True), as
    symmetric about 0 as the grid allows (one or two candidate sets)."""
    off = 0.5 if half else 0.0
    centre = -(n - 1) / 2.0
    sets = []
    for start in (centre, centre - 0.5, centre + 0.5):
        if abs((start - off) - round(start - off)) < 1e-9:
            sets.append(start + np.arange(n, dtype=np.float64))
    return sets


def _solve(L, N, M, u, I, J):
    """Roots (k, L) of the logarithmic equations for one choice of I, J;
    returns (energy / t, max residual)."""
    two_pi_I = 2.0 * np.pi * I
    two_pi_J = 2.0 * np.pi * J

    def residual(x):
        k, lam = x[:N], x[N:]
        sk = np.sin(k)
        f = L * k + _theta((sk[:, None] - lam[None, :]) / u).sum(axis=1) - two_pi_I
        g = (_theta((lam[:, None] - sk[None, :]) / u).sum(axis=1)
             - _theta((lam[:, None] - lam[None, :]) / (2.0 * u)).sum(axis=1) - two_pi_J)
        return np.concatenate([f, g])

    # start: free momenta, and spin rapidities of the strong-coupling limit
    k0 = two_pi_I / L
    lam0 = u * np.tan(np.pi * J / N)
    x0 = np.concatenate([k0, lam0])
    best_x, best_r = x0, np.inf
    for method in ("hybr", "lm"):
        sol = root(residual, x0, method=method, tol=1e-15)
        r = float(np.abs(residual(sol.x)).max())
        if r < best_r:
            best_x, best_r = sol.x, r
        if best_r < 1e-12:
            break
    return -2.0 * float(np.cos(best_x[:N]).sum()), best_r


def lieb_wu_ground_energy(L, n_up, n_dn, t=1.0, U=0.0, max_residual=1e-11):
    """Lowest energy over the consecutive-quantum-number states of the ring with
    L sites, n_up + n_dn <= L electrons; U > 0.  Raises ValueError when no
    candidate solves the equations to max_residual."""
    if not U > 0.0 or not t > 0.0:
        raise ValueError("the logarithmic equations need U > 0 and t > 0")
    N, M = n_up + n_dn, min(n_up, n_dn)
    if N > L:
        raise ValueError("more electrons than sites: use particle-hole symmetry first")
    if N == 0:
        return 0.0
    u = U / (4.0 * t)
    energies = []
    for I in _consecutive(N, M % 2 == 1):
        for J in _consecutive(M, (N - M + 1) % 2 == 1):
            e, r = _solve(L, N, M, u, I, J)
            if r <= max_residual:
                energies.append(t * e)
    if not energies:
        raise ValueError("no Bethe-ansatz candidate converged")
    return min(energies)
