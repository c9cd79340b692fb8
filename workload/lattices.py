"""Bond lists for the lattices the paper studies (Sec. 5: a periodic ring and
a periodic square lattice) plus the two-site dimer used as a closed-form pin.

Conventions (the paper fixes none of them):
  * ring of Ns sites: bonds (i, i+1 mod Ns);
  * Lx x Ly square lattice: site index i = x + Lx*y, bonds to (x+1 mod Lx, y)
    and (x, y+1 mod Ly);
  * the nearest-neighbour sum <ij> of Eq. (1) runs over a *set* of unordered
    pairs, so a periodic direction of length 2 yields one bond per pair, not
    two, and a length-1 direction yields none.
Bonds are returned as a sorted list of (i, j) with i < j.
"""


def _dedup(pairs):
    out = set()
    for i, j in pairs:
        if i != j:
            out.add((min(i, j), max(i, j)))
    return sorted(out)


def ring(ns):
    """Periodic ring of ns sites."""
    return _dedup((i, (i + 1) % ns) for i in range(ns))


def square(lx, ly):
    """Periodic lx-by-ly square lattice, site i = x + lx*y."""
    pairs = []
    for y in range(ly):
        for x in range(lx):
            i = x + lx * y
            pairs.append((i, ((x + 1) % lx) + lx * y))
            pairs.append((i, x + lx * ((y + 1) % ly)))
    return _dedup(pairs)


def dimer():
    """Two sites joined by a single bond."""
    return [(0, 1)]


def lattice_by_name(name):
    """'ring12' -> (12, ring(12)); 'sq3x4' -> (12, square(3, 4)) (3 wide, 4 tall)."""
    if name.startswith("ring"):
        ns = int(name[4:])
        return ns, ring(ns)
    if name.startswith("sq"):
        lx, ly = (int(a) for a in name[2:].split("x"))
        return lx * ly, square(lx, ly)
    if name == "dimer":
        return 2, dimer()
    raise ValueError(f"unknown lattice {name!r}")
