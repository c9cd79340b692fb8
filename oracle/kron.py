"""Matrix-free Kronecker-sum H*v for large sectors (test infrastructure only).

Wraps oracle/kron_hv.c (built by `build()`, plain gcc + OpenMP) with the
oracle's own per-spin tables from `basis.Sector.spin_table`.  Used where
the explicit H of `basis.Sector.explicit` would not fit in memory: the
4x4 half-filled sector (D = 1.66e8) and the 18-site ring (D = 2.36e9), and
as the timed CPU baseline.  Cross-checked against the explicit H on every
sector where both fit (tests).
"""
import ctypes
import os
import subprocess

import numpy as np

from .basis import Sector
from .lanczos import tridiag_lowest, _breakdown

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_kron.so")
_lib = None


def build(force=False):
    """Compile kron_hv.c into oracle/_kron.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "kron_hv.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", src, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.kron_hv_acc.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                    ctypes.c_double, P, P]
        lib.kron_hv_acc.restype = None
        lib.kron_scale.argtypes = [ctypes.c_int64, ctypes.c_double, P]
        lib.kron_dot.argtypes = [ctypes.c_int64, P, P]
        lib.kron_dot.restype = ctypes.c_double
        lib.kron_axpy.argtypes = [ctypes.c_int64, ctypes.c_double, P, P]
        lib.kron_set_threads.argtypes = [ctypes.c_int]
        lib.kron_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def set_threads(n):
    """OpenMP threads of the C kernels (n > 0); returns the previous maximum."""
    return int(_load().kron_set_threads(int(n)))


class KronHamiltonian:
    """Eq. (1) in one sector as H_up (x) I + I (x) H_dn + H_int, applied matrix-free."""

    def __init__(self, ns, bonds, nup, ndn, t=1.0, U=0.0):
        self.sector = Sector(ns, bonds, nup, ndn, t, U)
        S = self.sector
        self.D, self.Dup, self.Ddn = S.D, S.Dup, S.Ddn
        self.U = float(U)
        self.tables = []
        for spin in (0, 1):
            states, rowptr, tgt, sign = S.spin_table(spin)
            # spin_table rows list <r'|H|r> for fixed r; H_sigma is symmetric,
            # so the same arrays are the CSR of H_sigma by output row.
            self.tables.append((states, rowptr, tgt, (-S.t * sign.astype(np.float64))))
        self._lib = _load()

    def hv_acc(self, x, y):
        """y <- y + H x (Eq. split1', second line)."""
        (su, ur, uc, uv), (sd, dr, dc, dv) = self.tables
        assert x.dtype == np.float64 and y.dtype == np.float64 and x.size == self.D == y.size
        self._lib.kron_hv_acc(self.Dup, self.Ddn, _p(ur), _p(uc), _p(uv), _p(dr), _p(dc), _p(dv),
                              _p(su), _p(sd), self.U, _p(x), _p(y))

    def hv(self, x):
        y = np.zeros(self.D)
        self.hv_acc(np.ascontiguousarray(x, dtype=np.float64), y)
        return y

    # vector helpers (parallel C loops; plain definitions)
    def dot(self, x, y):
        return self._lib.kron_dot(x.size, _p(x), _p(y))

    def axpy(self, a, x, y):
        self._lib.kron_axpy(x.size, float(a), _p(x), _p(y))

    def scale(self, a, y):
        self._lib.kron_scale(y.size, float(a), _p(y))


def lanczos_matrix_free(Hk, v0, max_iter, tol=None, on_step=None, inplace=False):
    """Algorithm 1, two-vector form (Eqs. split1), with the C helpers.

    Same steps as lanczos.lanczos_plain, written against KronHamiltonian so
    that two vectors of a 2.4e9-element sector fit in host memory (with
    inplace=True the start vector's own buffer becomes the first Lanczos
    vector).
    """
    f = v0 if (inplace and v0.dtype == np.float64) else np.array(v0, dtype=np.float64)
    Hk.scale(1.0 / np.sqrt(Hk.dot(f, f)), f)
    g = np.zeros_like(f)
    a, b = [], []
    bj = 0.0
    energy, rho, broke = None, None, False
    for j in range(max_iter):
        Hk.scale(-bj, g)                 # f_{j-1} <- -b_j f_{j-1}
        Hk.hv_acc(f, g)                  # f_{j-1} <- f_{j-1} + H f_j
        aj = Hk.dot(g, f)
        Hk.axpy(-aj, f, g)
        bnext = float(np.sqrt(Hk.dot(g, g)))
        a.append(aj)
        energy, s = tridiag_lowest(a, b)
        rho = bnext * abs(s[-1])
        if on_step is not None:
            on_step(j, energy, rho)
        if _breakdown(bnext, a, b):
            broke = True
            b.append(bnext)
            break
        b.append(bnext)
        if tol is not None and rho < tol:
            break
        Hk.scale(1.0 / bnext, g)
        f, g = g, f
        bj = bnext
    return dict(energy=energy, a=np.array(a), b=np.array(b), iters=len(a), residual=rho,
                breakdown=broke)
