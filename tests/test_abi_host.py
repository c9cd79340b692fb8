"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-built basis and hopping tables equal the oracle's bit for bit."""
import math
import os
import re

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
from workload import lattice_by_name, ring, square

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    import ctypes
    lib = ctypes.CDLL(hub.LIB_PATH)
    names = declared_functions()
    assert "hubbard_apply" in names and "lanczos_ground_state" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding knows every declared function
    assert set(names) <= set(hub.SIGNATURES), set(names) - set(hub.SIGNATURES)


CASES = [("ring4", 2), ("ring8", 4), ("ring8", 3), ("ring7", 3), ("sq4x4", 8), ("sq4x4", 5), ("sq3x3", 4),
         ("sq3x2", 3), ("sq4x2", 2), ("sq4x3", 6), ("ring12", 6), ("ring18", 9), ("ring6", 0), ("ring6", 6),
         ("dimer", 1)]


@pytest.mark.parametrize("name,n", CASES)
def test_host_tables_bit_exact(name, n):
    ns, bonds = lattice_by_name(name)
    if math.comb(ns, n) > 50000:
        pytest.skip("oracle table loop too slow")
    got = hub.hubbard_host_spin_tables(ns, bonds, n)
    ref = Sector(ns, bonds, n, 0).spin_table(0)
    for g, r in zip(got, ref):
        assert g.dtype == r.dtype
        assert np.array_equal(g, r)


def test_host_tables_ring18_sizes():
    ns, bonds = lattice_by_name("ring18")
    states, rowptr, tgt, sign = hub.hubbard_host_spin_tables(ns, bonds, 9)
    assert len(states) == 48620
    assert rowptr[-1] == 18 * 2 * math.comb(16, 8)       # = 463320
    assert np.all(np.diff(states.astype(np.int64)) > 0)
    # Hermiticity of the sign table: r -> r' with s  <=>  r' -> r with s
    rows = np.repeat(np.arange(len(states)), np.diff(rowptr))
    fwd = dict(zip(zip(rows.tolist(), tgt.tolist()), sign.tolist()))
    assert all(fwd[(b, a)] == s for (a, b), s in list(fwd.items())[:20000])


@pytest.mark.parametrize("args,msg", [
    ((0, [], 0), "Ns"), ((33, [], 0), "Ns"), ((4, [(0, 4)], 1), "range"), ((4, [(1, 1)], 1), "self"),
    ((4, [(0, 1), (1, 0)], 1), "duplicate"), ((4, ring(4), 5), "N_up"), ((4, ring(4), -1), "N_up"),
])
def test_host_tables_reject_bad_input(args, msg):
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_host_spin_tables(*args)
    assert ei.value.code == hub.HUB_EINVAL and msg in str(ei.value)


def test_sector_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_sector_create(4, ring(4), 2, 2, 1.0, 1.0)
    assert ei.value.code in (hub.HUB_ECUDA, hub.HUB_ENOMEM)
