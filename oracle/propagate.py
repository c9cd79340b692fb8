"""Time propagation psi(t) = exp(-i H t) v in one sector, for the CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names time propagation as the other main use of the H*v kernel
(Sec. 6, Conclusions) but gives no propagation algorithm, so the oracle
writes out the definition of the exact result:

  evolve_dense   expand v in the eigenvectors phi_k of the explicit H of
                 Eq. (1) (a dense symmetric eigendecomposition is the one
                 library step) and multiply each coefficient by its phase:
                 psi(t) = sum_k exp(-i E_k t) <phi_k|v> phi_k.
  evolve_sparse  the same product through scipy's expm_multiply (truncated
                 Taylor series with scaling, Al-Mohy & Higham 2011) on the
                 explicit sparse H, for sectors too large for a dense
                 eigendecomposition.

Independent routes that pin them (tests/test_oracle_propagate.py):

  evolve_taylor            the exponential series sum_k (-i tau H)^k v / k!
                           summed term by term until the terms vanish, in
                           steps tau small enough that no term exceeds the
                           vector (brute force, exact up to rounding);
  ring_onebody_propagator  U = 0, one electron of each spin on a ring:
                           H = h (x) 1 + 1 (x) h, so exp(-iHt) is the
                           Kronecker product of the one-body propagator,
                           whose plane-wave closed form is written out;
  dimer_evolution          two sites, one bond, N = (1, 1): the four-state
                           problem in closed form (cos / sin of the
                           singlet frequency);
  slater_evolution         U = 0 with several electrons per spin: a product
                           of Slater determinants stays one, its orbitals
                           propagated by the one-body exp(-i h t); the
                           amplitude of a basis state is the product of the
                           two determinants of its occupied rows (creators
                           in ascending site order, up before down).
"""
import math

import numpy as np
import scipy.sparse.linalg as spla

from oracle.basis import Sector


def evolve_dense(S, v, t):
    """exp(-i H t) v by the eigendecomposition of the dense H of sector S."""
    E, phi = np.linalg.eigh(S.dense())
    c = phi.T @ np.asarray(v, dtype=np.complex128)
    return phi @ (np.exp(-1j * E * t) * c)


def evolve_sparse(S, v, t):
    """exp(-i H t) v through scipy's expm_multiply on the explicit sparse H."""
    H = S.explicit().astype(np.complex128)
    return spla.expm_multiply(-1j * t * H, np.asarray(v, dtype=np.complex128))


def evolve_taylor(S, v, t):
    """exp(-i H t) v as the exponential series, summed term by term.

    The time is cut into n steps tau = t / n with |tau| * |H|_1 <= 1/2, so
    every term of the series is at most 2^-k of the vector it starts from and
    the sum of each step stops once a term is below 1e-18 of that vector.
    """
    H = S.explicit().tocsr()
    norm1 = float(abs(H).sum(axis=0).max()) if H.nnz else 0.0
    n = max(1, int(math.ceil(abs(t) * norm1 / 0.5)))
    tau = t / n
    psi = np.asarray(v, dtype=np.complex128).copy()
    for _ in range(n):
        term = psi.copy()
        acc = psi.copy()
        ref = max(np.abs(psi).max(), 1e-300)
        k = 0
        while True:
            k += 1
            term = (-1j * tau / k) * (H @ term)
            acc += term
            if np.abs(term).max() <= 1e-18 * ref:
                break
        psi = acc
    return psi


def ring_onebody_propagator(ns, t_hop, time):
    """exp(-i h time) for the ring hopping matrix h (h_{j,j+1} = h_{j+1,j} = -t_hop).

    Plane waves diagonalise h: h e_k = -2 t_hop cos(2 pi k / ns) e_k with
    (e_k)_j = exp(2 pi i k j / ns) / sqrt(ns), hence
    exp(-i h time)_{jl} = (1/ns) sum_k exp(2 pi i k (j - l) / ns) exp(2 i t_hop time cos(2 pi k / ns)).
    For ns = 2 the two bonds of the ring are one bond (unordered pairs) and
    h = -t_hop sigma_x, which this formula does not describe: ns >= 3.
    """
    if ns < 3:
        raise ValueError("ring_onebody_propagator needs ns >= 3")
    k = np.arange(ns)
    j = np.arange(ns)
    phase = np.exp(2j * t_hop * time * np.cos(2.0 * np.pi * k / ns))
    d = (j[:, None] - j[None, :])[:, :, None] * k[None, None, :]
    return (np.exp(2j * np.pi * d / ns) * phase[None, None, :]).sum(axis=2) / ns


def ring_one_pair_evolution(ns, t_hop, v, time):
    """U = 0, N = (1, 1) on a ring: exp(-iHt) v = P V P^T with P the one-body
    propagator and V the ns x ns matrix of v (row = up site, column = down
    site; with one electron per spin the basis rank of site j is j)."""
    P = ring_onebody_propagator(ns, t_hop, time)
    V = np.asarray(v, dtype=np.complex128).reshape(ns, ns)
    return (P @ V @ P.T).reshape(-1)


def dimer_evolution(t_hop, U, v, time):
    """Two sites, one bond (0, 1), N = (1, 1), in closed form.

    Basis J = 2 i_up + i_dn with site words 01, 10: J = 0 and 3 are the doubly
    occupied sites, J = 1, 2 the singly occupied pairs.  With
    a = (|0> + |3>)/sqrt2, d = (|0> - |3>)/sqrt2, s = (|1> + |2>)/sqrt2,
    r = (|1> - |2>)/sqrt2: H d = U d, H r = 0, and on (a, s)
    H = [[U, -2t], [-2t, 0]] = (U/2) 1 + W n.sigma with W = sqrt(U^2/4 + 4 t^2),
    so exp(-i H time) = exp(-i U time / 2) (cos(W time) 1 - i sin(W time) n.sigma)
    there, n.sigma = [[U/2, -2t], [-2t, -U/2]] / W.
    """
    v = np.asarray(v, dtype=np.complex128)
    r2 = math.sqrt(0.5)
    a = r2 * (v[0] + v[3])
    d = r2 * (v[0] - v[3])
    s = r2 * (v[1] + v[2])
    r = r2 * (v[1] - v[2])
    W = math.sqrt(U * U / 4.0 + 4.0 * t_hop * t_hop)
    c, sn = math.cos(W * time), math.sin(W * time)
    ph = np.exp(-0.5j * U * time)
    nx = np.array([[U / 2.0, -2.0 * t_hop], [-2.0 * t_hop, -U / 2.0]]) / W
    a2, s2 = ph * ((c * np.eye(2) - 1j * sn * nx) @ np.array([a, s]))
    d2 = np.exp(-1j * U * time) * d
    r2_ = r                                                  # energy 0: no phase
    out = np.empty(4, dtype=np.complex128)
    out[0] = r2 * (a2 + d2)
    out[3] = r2 * (a2 - d2)
    out[1] = r2 * (s2 + r2_)
    out[2] = r2 * (s2 - r2_)
    return out


def dimer_sector(t_hop, U):
    """The sector dimer_evolution describes, as an oracle Sector."""
    return Sector(2, [(0, 1)], 1, 1, t_hop, U)


def slater_state(ns, nup, ndn, phi_up, phi_dn):
    """The sector vector of the Slater determinant product with orbitals
    phi_up (ns x nup) and phi_dn (ns x ndn): amplitude of (up word, down word)
    = det(phi_up[up sites, :]) * det(phi_dn[down sites, :]), sites ascending."""
    from oracle.basis import spin_states
    ups, dns = spin_states(ns, nup), spin_states(ns, ndn)

    def dets(words, phi, n):
        out = np.empty(len(words), dtype=np.complex128)
        for k, wd in enumerate(words):
            rows = [i for i in range(ns) if (int(wd) >> i) & 1]
            out[k] = np.linalg.det(phi[rows, :]) if n > 0 else 1.0
        return out

    return np.outer(dets(ups, phi_up, nup), dets(dns, phi_dn, ndn)).reshape(-1)


def slater_evolution(ns, bonds, t_hop, nup, ndn, phi_up, phi_dn, time):
    """U = 0: exp(-iHt) of slater_state(phi_up, phi_dn) is slater_state of the
    orbitals exp(-i h t) phi (h the one-body hopping matrix of the bonds)."""
    from oracle.closed_forms import hopping_matrix
    e, u = np.linalg.eigh(hopping_matrix(ns, bonds, t_hop))
    P = (u * np.exp(-1j * e * time)) @ u.T
    return slater_state(ns, nup, ndn, P @ phi_up, P @ phi_dn)
