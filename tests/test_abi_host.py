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
        text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M | re.S)       # function-pointer types
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


def _decode_row_table(boff, bcnt, ent, narrow):
    """entry[g][lane] = array of that lane's slots in slot order (the documented layout)."""
    out = []
    for g in range(len(boff)):
        nh = int(bcnt[g])
        nfull = nh // 2
        s = np.arange(4 * nh)
        lanes = np.arange(32)[:, None]
        pos = np.where(s < 8 * nfull,
                       boff[g] + ((s // 8) * 32 + lanes) * 8 + s % 8,
                       boff[g] + nfull * 256 + lanes * 4 + (s - 8 * nfull))
        out.append(ent[pos])
    return out


@pytest.mark.parametrize("name,n,eb", [
    ("ring12", 6, 8), ("ring12", 6, 16), ("sq4x4", 8, 16), ("sq4x4", 8, 8), ("sq3x3", 4, 4), ("ring18", 9, 4),
    ("sq4x3", 5, 8), ("dimer", 1, 16), ("ring6", 0, 8), ("ring6", 6, 4), ("ring10", 1, 8),
])
def test_row_table_layout(name, n, eb):
    """The coloured row-phase table (what the down-hop gathers walk) against the
    CSR hop table pinned to the oracle: every state's entries below D are exactly
    its hops (target and sign), every other entry points at a zero slot, each
    wavefront phase's entries of one slot fall in distinct bank groups (no
    shared-memory bank conflicts), and every group starts 16-byte aligned."""
    ns, bonds = lattice_by_name(name)
    states, rowptr, tgt, sign = hub.hubbard_host_spin_tables(ns, bonds, n)
    D = len(states)
    boff, bcnt, ent, narrow = hub.hubbard_host_row_table(ns, bonds, n, eb)
    assert len(boff) == (D + 31) // 32
    assert narrow == ((D + 31) // 32 * 32 + 32 <= 32767)
    assert np.all(boff % 128 == 0)
    assert np.array_equal(np.diff(np.append(boff, len(ent))), 128 * bcnt.astype(np.int64))
    negbit = 15 if narrow else 31
    idx = (ent & ((1 << negbit) - 1)).astype(np.int64)
    neg = ((ent >> negbit) & 1).astype(np.int64)
    ngroups = 128 // eb
    plane = min(32, ngroups)
    Dr = (D + 31) // 32 * 32
    tab = _decode_row_table(boff, bcnt, idx, narrow)
    sgn = _decode_row_table(boff, bcnt, neg, narrow)
    for g, (ix, sg) in enumerate(zip(tab, sgn)):
        pad = ix >= D
        assert np.all((ix[pad] >= Dr) & (ix[pad] < Dr + ngroups)) and np.all(sg[pad] == 0)
        for lane in range(32):
            r = 32 * g + lane
            real = ~pad[lane]
            got = sorted(zip(ix[lane][real].tolist(), (1 - 2 * sg[lane][real]).tolist()))
            if r >= D:
                assert got == []
                continue
            want = sorted(zip(tgt[rowptr[r]:rowptr[r + 1]].tolist(), sign[rowptr[r]:rowptr[r + 1]].tolist()))
            assert got == want, (g, lane)
        # [slot][phase][lane]: lanes reading the same slot index share the access
        # (broadcast); distinct indices must fall in distinct bank groups
        ph = ix.T.reshape(ix.shape[1], 32 // plane, plane)
        for s_ in range(ph.shape[0]):
            for p_ in range(ph.shape[1]):
                u = np.unique(ph[s_, p_])
                assert len(np.unique(u % ngroups)) == len(u), (g, s_, p_)


def test_row_table_rejects_bad_element_size():
    ns, bonds = lattice_by_name("ring8")
    with pytest.raises(hub.HubError) as ei:
        hub.hubbard_host_row_table(ns, bonds, 4, 12)
    assert ei.value.code == hub.HUB_EINVAL
