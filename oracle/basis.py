"""Basis, ranking, signs and the explicit Hamiltonian, from Sec. 2.1.

Part of the CPU oracle (test infrastructure only).  Everything here is
float64 / exact integer NumPy, written to be checked against the paper by
eye rather than to be fast.

Conventions taken from the paper:
  * A spin configuration is an Ns-bit word, bit i set <=> site i occupied
    ("site indices run from right to left", Eq. binaryrep).
  * i_sigma = position of the word in the ascending list of all Ns-bit
    words with N_sigma bits set; J = i_up * C(Ns, N_dn) + i_dn
    (Eq. J-formula, Table 1).
  * A basis state is c+_{m1} c+_{m2} ... |O> with all up operators left
    of all down operators and ascending sites within a spin (Sec. 2.1,
    below Eq. basisstate).  We number the 2*Ns modes m = site for spin up
    and m = Ns + site for spin down, so a basis state is a product of
    creators in ascending mode order.
  * H = -t sum_<ij> sum_sigma (c+_i c_j + h.c.) + U sum_i n_i,up n_i,dn
    (Eq. 1).

Signs are computed with the generic Jordan-Wigner rule for c+_a c_b on the
whole 2*Ns-mode string (anticommute c_b to the front, then c+_a to its
place).  This never uses the paper's per-spin "electrons between origin
and destination" shortcut, so the tests that compare the two (and the
library's per-spin tables) are a real check.
"""
import math

import numpy as np
import scipy.sparse as sp


def spin_states(ns, n):
    """Ascending list of Ns-bit words with n bits set (Eq. J-formula)."""
    if n < 0 or n > ns:
        return np.zeros(0, dtype=np.int64)
    words = np.arange(1 << ns, dtype=np.int64)
    return words[np.bitwise_count(words) == n]


def sector_dim(ns, nup, ndn):
    """dim H = C(Ns, N_up) * C(Ns, N_dn) (Sec. 2.1)."""
    return math.comb(ns, nup) * math.comb(ns, ndn)


class Sector:
    """One fixed (N_up, N_dn) sector of Eq. (1) on a given bond list."""

    def __init__(self, ns, bonds, nup, ndn, t=1.0, U=0.0):
        self.ns, self.nup, self.ndn = int(ns), int(nup), int(ndn)
        self.bonds = [(int(i), int(j)) for i, j in bonds]
        self.t, self.U = float(t), float(U)
        self.up = spin_states(ns, nup)        # s_up[i_up]
        self.dn = spin_states(ns, ndn)        # s_dn[i_dn]
        self.Dup, self.Ddn = len(self.up), len(self.dn)
        self.D = self.Dup * self.Ddn

    # ---- labelling (Eq. J-formula) ------------------------------------
    def unrank(self, J):
        """J -> (up word, down word)."""
        J = np.asarray(J, dtype=np.int64)
        return self.up[J // self.Ddn], self.dn[J % self.Ddn]

    def rank(self, up, dn):
        """(up word, down word) -> J, by position in the ascending lists."""
        iu = np.searchsorted(self.up, up)
        idn = np.searchsorted(self.dn, dn)
        ok = (iu < self.Dup) & (idn < self.Ddn)
        ok &= self.up[np.minimum(iu, self.Dup - 1)] == up
        ok &= self.dn[np.minimum(idn, self.Ddn - 1)] == dn
        if not np.all(ok):
            raise ValueError("word not in this sector")
        return iu * self.Ddn + idn

    # ---- fermion algebra on the 2*Ns-mode string -----------------------
    def _modes(self, up, dn):
        """Occupation of modes 0..2Ns-1 as one integer: up sites low, down high."""
        return np.asarray(up, dtype=np.int64) | (np.asarray(dn, dtype=np.int64) << self.ns)

    @staticmethod
    def _below(occ, m):
        """Number of occupied modes with index < m."""
        return np.bitwise_count(occ & ((np.int64(1) << m) - 1))

    def _hop(self, occ, a, b):
        """Apply c+_a c_b (a != b) to product states `occ`.

        Returns (valid mask, new occupation, sign).  c_b meets the creators
        of all occupied modes < b on its way to c+_b; c+_a then passes the
        occupied modes < a of the intermediate state.
        """
        has_b = (occ >> b) & 1
        has_a = (occ >> a) & 1
        valid = (has_b == 1) & (has_a == 0)
        mid = occ & ~(np.int64(1) << b)
        n = self._below(occ, b) + self._below(mid, a)
        sign = np.where(n % 2 == 0, 1, -1).astype(np.int64)
        new = mid | (np.int64(1) << a)
        return valid, new, sign

    def _terms(self):
        """All (a, b) mode pairs of the hopping sum: both directions, both spins."""
        for i, j in self.bonds:
            for off in (0, self.ns):              # spin up, spin down
                yield i + off, j + off
                yield j + off, i + off

    # ---- explicit H ----------------------------------------------------
    def diagonal(self):
        """U * (number of doubly occupied sites) for every J (Sec. 2.1)."""
        J = np.arange(self.D, dtype=np.int64)
        up, dn = self.unrank(J)
        return self.U * np.bitwise_count(up & dn).astype(np.float64)

    def explicit(self):
        """H as a scipy CSR matrix: H[J', J] = <J'|H|J>."""
        J = np.arange(self.D, dtype=np.int64)
        up, dn = self.unrank(J)
        occ = self._modes(up, dn)
        rows, cols, vals = [J], [J], [self.diagonal()]
        mask_up = (np.int64(1) << self.ns) - 1
        for a, b in self._terms():
            valid, new, sign = self._hop(occ, a, b)
            if not np.any(valid):
                continue
            Jp = self.rank(new[valid] & mask_up, new[valid] >> self.ns)
            rows.append(Jp)
            cols.append(J[valid])
            vals.append(-self.t * sign[valid].astype(np.float64))
        H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.D, self.D))
        return H.tocsr()

    def dense(self):
        return self.explicit().toarray()

    def rows_of_hv(self, J, v):
        """(H v)[J] for the sampled indices J only: sum over <J|H|J'> v[J'].

        v is an array, or a callable returning v at an index array (so that
        sectors too large for host memory can be sampled).

        <J|H|J'> is nonzero for J' = J (diagonal) and for the states J'
        with c+_a c_b |J'> ~ |J>, i.e. |J'> ~ c+_b c_a |J>; the same sign
        appears both ways (the hopping matrix is real symmetric).
        """
        J = np.asarray(J, dtype=np.int64)
        vat = v if callable(v) else (lambda idx: v[idx])
        up, dn = self.unrank(J)
        occ = self._modes(up, dn)
        out = self.U * np.bitwise_count(up & dn).astype(np.float64) * vat(J)
        mask_up = (np.int64(1) << self.ns) - 1
        for a, b in self._terms():
            valid, new, sign = self._hop(occ, a, b)
            if not np.any(valid):
                continue
            Jp = self.rank(new[valid] & mask_up, new[valid] >> self.ns)
            out[valid] += -self.t * sign[valid] * vat(Jp)
        return out

    # ---- per-spin hopping tables (for bit-exact comparison) ------------
    def spin_table(self, spin):
        """Canonical per-spin table of H_sigma (Eq. H-Kroneckersum).

        Returns (states, rowptr, tgt, sign): row r lists every r' with
        <r'|H_sigma|r> != 0, sorted by r', and sign s with
        <r'|H_sigma|r> = -t * s.  Computed with the generic JW rule on the
        Ns modes of one species.
        """
        states = self.up if spin == 0 else self.dn
        D = len(states)
        rowptr = np.zeros(D + 1, dtype=np.int64)
        tg, sg = [], []
        for r in range(D):
            occ = np.int64(states[r])
            pairs = {}
            for i, j in self.bonds:
                for a, b in ((i, j), (j, i)):
                    if (occ >> b) & 1 and not (occ >> a) & 1:
                        mid = occ & ~(np.int64(1) << b)
                        n = self._below(occ, b) + self._below(mid, a)
                        new = mid | (np.int64(1) << a)
                        rp = int(np.searchsorted(states, new))
                        s = 1 if n % 2 == 0 else -1
                        pairs[rp] = pairs.get(rp, 0) + s
            for rp in sorted(pairs):
                if pairs[rp] != 0:
                    tg.append(rp)
                    sg.append(pairs[rp])
            rowptr[r + 1] = len(tg)
        return (states.astype(np.uint32), rowptr.astype(np.int32),
                np.asarray(tg, dtype=np.int32), np.asarray(sg, dtype=np.int8))

    def spin_matrix(self, spin):
        """H_sigma as a dense-free scipy CSR built from spin_table (values -t*sign)."""
        states, rowptr, tgt, sign = self.spin_table(spin)
        D = len(states)
        rows = np.repeat(np.arange(D), np.diff(rowptr))
        return sp.csr_matrix((-self.t * sign.astype(np.float64), (tgt, rows)), shape=(D, D))
