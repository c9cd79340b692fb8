"""Ground-state energies with a closed form or a one-body reduction.

Part of the CPU oracle (test infrastructure only); each is a limit of Eq. (1).
"""
import math

import numpy as np


def dimer_energy(t, U):
    """Two sites, one bond, one electron of each spin: E0 = U/2 - sqrt(U^2/4 + 4 t^2)."""
    return U / 2.0 - math.sqrt(U * U / 4.0 + 4.0 * t * t)


def atomic_energy(ns, nup, ndn, U):
    """t = 0: H is diagonal; the fewest double occupancies are max(0, N_up + N_dn - Ns)."""
    return U * max(0, nup + ndn - ns)


def hopping_matrix(ns, bonds, t):
    """One-body matrix h with h_ij = h_ji = -t for every bond <ij>."""
    h = np.zeros((ns, ns))
    for i, j in bonds:
        h[i, j] -= t
        h[j, i] -= t
    return h


def free_energy(ns, bonds, nup, ndn, t):
    """U = 0: free fermions, E0 = sum of the lowest N_up plus lowest N_dn eigenvalues of h."""
    e = np.linalg.eigvalsh(hopping_matrix(ns, bonds, t))
    return float(e[:nup].sum() + e[:ndn].sum())
