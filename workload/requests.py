"""Seeded request lists for the batched and the serving workloads.

batch_sectors: many uneven small sectors (rings of 6..12 sites and the
2x3, 2x4, 3x3, 3x4 periodic lattices), fillings uniform in [1, Ns-1] per
spin, U uniform in [0, 12], t = 1.

serve_requests: Poisson arrivals (exponential gaps, mean 1/rate) of solve
requests over rings of 8..16 sites and the 3x3, 3x4, 4x4 lattices, fillings
and U drawn as above.
"""
import numpy as np

BATCH_LATTICES = [f"ring{n}" for n in range(6, 13)] + ["sq3x2", "sq4x2", "sq3x3", "sq4x3"]
SERVE_LATTICES = [f"ring{n}" for n in range(8, 17)] + ["sq3x3", "sq4x3", "sq4x4"]


def _ns(name):
    from .lattices import lattice_by_name
    return lattice_by_name(name)[0]


def batch_sectors(count=2048, seed=1234):
    """List of dicts {lattice, ns, nup, ndn, t, U, seed} for the batched workload."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        name = BATCH_LATTICES[int(rng.integers(len(BATCH_LATTICES)))]
        ns = _ns(name)
        nup = int(rng.integers(1, ns))
        ndn = int(rng.integers(1, ns))
        U = float(rng.uniform(0.0, 12.0))
        out.append(dict(lattice=name, ns=ns, nup=nup, ndn=ndn, t=1.0, U=U, seed=seed + 1 + k))
    return out


def serve_requests(count=5000, rate=500.0, seed=1234, lattices=None):
    """List of dicts {arrival_s, lattice, ns, nup, ndn, t, U, seed} (Poisson arrivals)."""
    rng = np.random.default_rng(seed)
    lats = SERVE_LATTICES if lattices is None else list(lattices)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        name = lats[int(rng.integers(len(lats)))]
        ns = _ns(name)
        nup = int(rng.integers(1, ns))
        ndn = int(rng.integers(1, ns))
        U = float(rng.uniform(0.0, 12.0))
        out.append(dict(arrival_s=t, lattice=name, ns=ns, nup=nup, ndn=ndn, t=1.0, U=U, seed=seed + 1 + k))
    return out
