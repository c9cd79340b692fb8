"""Lanczos (Sec. 2.2, Algorithm 1) for the CPU oracle (test infrastructure only).

`lanczos_plain` is Algorithm 1 step by step in its two-vector form
(Eqs. split1): f_{j-1} <- -b_j f_{j-1}; f_{j-1} <- f_{j-1} + H f_j, then
a_j = q.f_j, q <- q - a_j f_j, b_{j+1} = |q|, f_{j+1} = q / b_{j+1}.
`lanczos_full` adds classical Gram-Schmidt against every stored Lanczos
vector, applied twice, after each step (full reorthogonalisation): slow,
but free of ghost eigenvalues.  Both return the a_j, b_{j+1} sequences;
the lowest eigenvalue of the tridiagonal T (Eq. Tmatrix) comes from
scipy's tridiagonal eigensolver.

Readings where the paper is silent:
  * "b_{j+1} = 0" (breakdown) is tested as
    b_{j+1} <= 1e-13 * max(1, max|a|, max b);
  * the stop test is either a fixed number of steps or the residual
    estimate rho = b_{m+1} * |s_m| < tol, with s the normalised
    eigenvector of T_m for its lowest eigenvalue.
"""
import numpy as np
from scipy.linalg import eigh_tridiagonal


def tridiag_lowest(a, b):
    """Lowest eigenvalue and eigenvector of T (a on the diagonal, b[1:] off it).

    `b` holds b_2..b_m (length m-1).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if len(a) == 1:
        return float(a[0]), np.ones(1)
    w, s = eigh_tridiagonal(a, b, select="i", select_range=(0, 0))
    return float(w[0]), s[:, 0]


def _breakdown(bnext, a, b):
    scale = max(1.0, max(abs(x) for x in a), max(b) if len(b) else 0.0)
    return bnext <= 1e-13 * scale


def lanczos_plain(hv, v0, max_iter, tol=None):
    """Algorithm 1 in the two-vector form (Eqs. split1).

    hv: callable returning H @ x (float64).  Stops after max_iter steps,
    on breakdown, or when tol is given and rho < tol.
    Returns dict(energy, a, b, iters, residual, breakdown).
    """
    f = np.array(v0, dtype=np.float64)
    f /= np.sqrt(np.dot(f, f))
    g = np.zeros_like(f)          # holds f_{j-1}; becomes q_j
    a, b = [], []                 # a_1..a_m and b_2..b_{m+1}
    bj = 0.0
    energy, rho, broke = None, None, False
    for j in range(max_iter):
        g *= -bj                  # f_{j-1} <- -b_j f_{j-1}
        g += hv(f)                # f_{j-1} <- f_{j-1} + H f_j   (= q_j)
        aj = float(np.dot(g, f))  # a_j = q_j . f_j
        g -= aj * f               # q_j <- q_j - a_j f_j
        bnext = float(np.sqrt(np.dot(g, g)))
        a.append(aj)
        energy, s = tridiag_lowest(a, b)
        rho = bnext * abs(s[-1])
        if _breakdown(bnext, a, b):
            broke = True
            b.append(bnext)
            break
        b.append(bnext)
        if tol is not None and rho < tol:
            break
        g /= bnext                # f_{j+1} = q_j / b_{j+1}
        f, g = g, f               # rename: the old f_j is the next step's f_{j-1}
        bj = bnext
    return dict(energy=energy, a=np.array(a), b=np.array(b), iters=len(a),
                residual=rho, breakdown=broke)


def lanczos_full(hv, v0, max_iter, tol=None):
    """Algorithm 1 with full reorthogonalisation (classical Gram-Schmidt, twice)."""
    f = np.array(v0, dtype=np.float64)
    f /= np.sqrt(np.dot(f, f))
    F = [f]
    a, b = [], []
    energy, rho, broke = None, None, False
    for j in range(max_iter):
        q = hv(F[-1])
        if j > 0:
            q -= b[-1] * F[-2]
        aj = float(np.dot(q, F[-1]))
        q -= aj * F[-1]
        Fm = np.array(F)
        for _ in range(2):
            q -= Fm.T @ (Fm @ q)
        bnext = float(np.sqrt(np.dot(q, q)))
        a.append(aj)
        energy, s = tridiag_lowest(a, b)
        rho = bnext * abs(s[-1])
        if _breakdown(bnext, a, b):
            broke = True
            b.append(bnext)
            break
        b.append(bnext)
        if tol is not None and rho < tol:
            break
        F.append(q / bnext)
    return dict(energy=energy, a=np.array(a), b=np.array(b), iters=len(a),
                residual=rho, breakdown=broke)


def ground_energy_dense(H):
    """Smallest eigenvalue of a dense symmetric matrix (numpy eigvalsh)."""
    return float(np.linalg.eigvalsh(np.asarray(H, dtype=np.float64))[0])
