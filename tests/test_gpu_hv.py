"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * tables: bit-exact;
  * binary64 H*v: max-abs error <= 1e-12 * |v|_2 * max(1, |t|) (the hop sums are
    exact on a grid of 2^-48 max|v|, so the error is at most (W_up + W_dn + 1)
    grid steps times |t| plus one rounding of the result, far below this);
  * binary32 H*v: max-abs error <= 4e-7 * (W_up + W_dn + 1) * max(|t|, |U| Ns, 1) * max|v|;
  * ground-state energy: relative error <= 1e-9.
"""
import json
import math
import os

import numpy as np
import pytest

import paper_1204_3425_gb300 as hub
from oracle.basis import Sector
from oracle.lanczos import ground_energy_dense, lanczos_plain
from workload import lattice_by_name, start_vector

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1204_3425_gb300 import build
    build.build()
    hub.load_library()
    return torch.device("cuda:0")


# (lattice, N_up, N_dn, t, U): paper sizes, edge fillings, degenerate cases, ragged rows
SMALL = [
    ("ring8", 4, 4, 1.0, 4.0), ("ring4", 2, 3, 1.7, 0.0), ("sq3x2", 2, 4, 1.0, 3.0), ("sq3x3", 4, 5, 0.9, 7.0),
    ("sq4x2", 3, 5, 1.0, 2.0), ("ring6", 0, 3, 1.0, 2.0), ("ring6", 6, 2, 1.0, 2.0), ("ring5", 5, 5, 1.0, 2.0),
    ("ring6", 3, 3, 0.0, 4.0), ("ring7", 3, 2, 1.0, 0.0), ("dimer", 1, 1, 1.0, 4.0), ("ring10", 5, 4, 1.0, 5.0),
    ("sq4x3", 3, 2, 1.0, 6.0), ("ring9", 1, 8, 2.5, 1.5), ("sq4x4", 2, 1, 1.0, 8.0),
]


def _sector(name, nup, ndn, t, U):
    ns, bonds = lattice_by_name(name)
    return hub.hubbard_sector_create(ns, bonds, nup, ndn, t, U), Sector(ns, bonds, nup, ndn, t, U)


@pytest.mark.parametrize("case", SMALL[:6] + [("sq4x4", 8, 5, 1.0, 1.0)])
def test_device_tables_bit_exact(dev, case):
    H, S = _sector(*case)
    for spin in (0, 1):
        got = hub.hubbard_export_tables(H, spin)
        ref = S.spin_table(spin)
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("path", ["fast", "reference"])
def test_hv_f64(dev, case, path):
    H, S = _sector(*case)
    t = case[3]
    v = start_vector(S.D, seed=77)
    ref = S.explicit() @ v
    vd = torch.from_numpy(v).to(dev)
    w = torch.full_like(vd, np.nan)
    (hub.hubbard_apply if path == "fast" else hub.hubbard_apply_reference)(H, vd, w)
    got = w.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.linalg.norm(v) * max(1.0, abs(t))


@pytest.mark.parametrize("case", SMALL)
def test_hv_f32(dev, case):
    H, S = _sector(*case)
    name, nup, ndn, t, U = case
    v = start_vector(S.D, seed=78).astype(np.float32)
    ref = S.explicit() @ v.astype(np.float64)
    vd = torch.from_numpy(v).to(dev)
    w = torch.full_like(vd, np.nan)
    hub.hubbard_apply(H, vd, w)
    tol = 4e-7 * (H.Wup + H.Wdn + 1) * max(abs(t), abs(U) * S.ns, 1.0) * np.abs(v).max()
    assert np.abs(w.cpu().numpy() - ref).max() <= tol


@pytest.mark.parametrize("case", [("ring8", 4, 4, 1.0, 4.0), ("sq4x3", 3, 2, 1.0, 6.0), ("ring5", 5, 5, 1.0, 2.0)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_apply_host_buffers_vs_oracle(dev, case, dt):
    """hubbard_apply_host: page-locked host input and output, five calls in flight
    at once through the two staging slots, each result against the oracle's
    explicit H at the device path's tolerance and bit-identical to hubbard_apply."""
    H, S = _sector(*case)
    name, nup, ndn, t, U = case
    tdt = torch.float64 if dt == "f64" else torch.float32
    vs = [torch.from_numpy(start_vector(S.D, seed=300 + i)).to(tdt).pin_memory() for i in range(5)]
    ws = [torch.full((S.D,), float("nan"), dtype=tdt).pin_memory() for _ in range(5)]
    stream = torch.cuda.Stream()
    for v, w in zip(vs, ws):
        hub.hubbard_apply_host(H, v, w, stream=stream)
    stream.synchronize()
    for v, w in zip(vs, ws):
        vv = v.double().numpy()
        ref = S.explicit() @ vv
        if dt == "f64":
            tol = 1e-12 * np.linalg.norm(vv) * max(1.0, abs(t))
        else:
            tol = 4e-7 * (H.Wup + H.Wdn + 1) * max(abs(t), abs(U) * S.ns, 1.0) * np.abs(vv).max()
        assert np.abs(w.double().numpy() - ref).max() <= tol
        wd = torch.empty(S.D, dtype=tdt, device=dev)
        hub.hubbard_apply(H, v.to(dev), wd)
        assert torch.equal(wd.cpu(), w)
    # device pointers and overlapping buffers are refused by the C entry point
    lib = hub.load_library()
    vd = vs[0].to(dev)
    code = hub.HUB_F64 if dt == "f64" else hub.HUB_F32
    import ctypes
    assert lib.hubbard_apply_host(H.handle, ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(ws[0].data_ptr()),
                                  code, None) == hub.HUB_EINVAL
    assert lib.hubbard_apply_host(H.handle, ctypes.c_void_p(vs[0].data_ptr()), ctypes.c_void_p(vs[0].data_ptr()),
                                  code, None) == hub.HUB_EINVAL


@pytest.mark.parametrize("case", [("ring4", 2, 3, 1.7, 2.0), ("sq3x2", 2, 2, 1.0, 3.0), ("ring6", 2, 3, 0.8, 5.5)])
def test_hv_basis_vectors_exact(dev, case):
    # H e_J is column J of H; every entry is exactly -t*sign or U*n
    H, S = _sector(*case)
    Hd = S.dense()
    for J in range(S.D):
        e = torch.zeros(S.D, dtype=torch.float64, device=dev)     # fresh, 16-byte aligned
        e[J] = 1.0
        w = torch.empty(S.D, dtype=torch.float64, device=dev)
        hub.hubbard_apply(H, e, w)
        assert np.array_equal(w.cpu().numpy(), Hd[:, J]), J


def test_config1_hv_lanczos_and_alpha_beta(dev):
    """Ring 8, (4,4), t=1, U=4, binary64, 100 Lanczos steps from the seeded start."""
    H, S = _sector("ring8", 4, 4, 1.0, 4.0)
    Hx = S.explicit()
    v0 = start_vector(S.D, seed=1234)
    f = v0 / np.linalg.norm(v0)
    fd = torch.from_numpy(f).to(dev)
    w = torch.empty_like(fd)
    hub.hubbard_apply(H, fd, w)
    assert np.abs(w.cpu().numpy() - Hx @ f).max() <= 1e-12
    r = hub.lanczos_ground_state(H, torch.from_numpy(v0).to(dev), 100, 0.0)
    g = json.load(open(os.path.join(GOLD, "ring8_n4_4_U4.json")))
    assert r["iters"] == 100
    assert abs(r["energy"] - g["e0_dense"]) <= 1e-9 * abs(g["e0_dense"])
    ro = lanczos_plain(lambda x: Hx @ x, v0, 20)
    np.testing.assert_allclose(r["alpha"][:20], ro["a"], rtol=1e-10)
    np.testing.assert_allclose(r["beta"][:20], ro["b"], rtol=1e-10)


def test_lanczos_step_matches_oracle(dev):
    H, S = _sector("sq3x3", 3, 4, 1.0, 5.0)
    Hx = S.explicit()
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, S.D)
    f /= np.linalg.norm(f)
    g = rng.uniform(-1, 1, S.D)
    beta = 1.37
    q = Hx @ f - beta * g
    a = q @ f
    q -= a * f
    b = np.linalg.norm(q)
    fd, gd = torch.from_numpy(f).to(dev), torch.from_numpy(g).to(dev)
    ag, bg = hub.hubbard_lanczos_step(H, fd, gd, beta)
    assert ag == pytest.approx(a, rel=1e-12) and bg == pytest.approx(b, rel=1e-12)
    assert np.abs(gd.cpu().numpy() - q / b).max() <= 1e-12


@pytest.mark.parametrize("dt,norm_tol,ab_tol", [("f64", 1e-13, 1e-11), ("f32", 3e-6, 1e-4)])
def test_fused_lanczos_steps_keep_unit_norm(dev, dt, norm_tol, ab_tol):
    """120 steps with the reductions fused into H*v (beta^2 = <w,w> - 2a^2 + a^2 <f,f>):
    every f_j stays a unit vector (normalisation errors do not compound) and each
    (a, b) matches an explicit binary64 evaluation of the same update."""
    tdt = torch.float64 if dt == "f64" else torch.float32
    H, S = _sector("sq4x2", 3, 5, 1.0, 2.0)
    f = torch.from_numpy(start_vector(S.D, seed=11)).to(dev, tdt)
    f /= f.norm()
    g = torch.zeros_like(f)
    hf = torch.empty_like(f)
    beta = 0.0
    for j in range(120):
        hub.hubbard_apply(H, f, hf)
        q = hf.double() - beta * g.double()
        a_ref = float(q @ f.double())
        b_ref = float(torch.linalg.norm(q - a_ref * f.double()))
        a, b = hub.hubbard_lanczos_step(H, f, g, beta)
        assert abs(a - a_ref) <= ab_tol * max(1.0, abs(a_ref)), (j, a, a_ref)
        assert abs(b - b_ref) <= ab_tol * max(1.0, b_ref), (j, b, b_ref)
        assert abs(float(torch.linalg.norm(g.double())) - 1.0) <= norm_tol, j
        f, g = g, f
        beta = b


def test_deferred_update_matches_explicit_steps(dev):
    """lanczos_ground_state completes each f_{j+1} = (w - a_j f_j) / b_{j+1} inside
    the next step's row phase; driving the same recurrence through
    hubbard_lanczos_step (which normalises with a pass of its own) must give the
    same a_j, b_j: bit for bit in binary32 (same kernels, same roundings), to
    rounding in binary64 (the standalone step takes its fixed-point grid from
    max|f|, the solver the fixed 2^-47 grid of unit vectors).  Rows of 924
    elements: 28 full 32-lane groups and a ragged tail."""
    H, S = _sector("ring12", 6, 6, 1.0, 4.0)
    rng = np.random.default_rng(21)
    # 256 entries +-1: |v0| = 16 exactly, so f_0 = v0 / 16 is exact on both routes
    v0 = np.zeros(S.D)
    v0[rng.choice(S.D, 256, replace=False)] = rng.choice([-1.0, 1.0], 256)
    n = 40
    for tdt in (torch.float32, torch.float64):
        r = hub.lanczos_ground_state(H, torch.from_numpy(v0).to(dev, tdt), n, 0.0)
        assert r["iters"] == n
        f = torch.from_numpy(v0 / 16.0).to(dev, tdt)
        g = torch.zeros_like(f)
        a, b, beta = [], [], 0.0
        for _ in range(n):
            aj, bj = hub.hubbard_lanczos_step(H, f, g, beta)
            a.append(aj)
            b.append(bj)
            f, g = g, f
            beta = bj
        if tdt == torch.float32:
            assert np.array_equal(r["alpha"], np.array(a)) and np.array_equal(r["beta"], np.array(b))
        else:
            np.testing.assert_allclose(r["alpha"], a, rtol=1e-11, atol=1e-12)
            np.testing.assert_allclose(r["beta"], b, rtol=1e-11)


def test_lanczos_breakdown_tiny_sector(dev):
    # one electron on a 4-ring: eigenvalues -2, 0, 0, 2, so the Krylov space
    # of any start vector has dimension 3 and step 3 breaks down (b_4 ~ 0)
    H, S = _sector("ring4", 1, 0, 1.0, 2.0)
    r = hub.lanczos_ground_state(H, torch.from_numpy(start_vector(S.D, seed=5)).to(dev), 50, 0.0)
    assert r["breakdown"] and r["iters"] == 3
    assert r["energy"] == pytest.approx(-2.0, abs=1e-12)
    # a 16-state sector: iterations are capped at D, the energy is exact
    H, S = _sector("ring4", 1, 1, 1.0, 2.0)
    r = hub.lanczos_ground_state(H, torch.from_numpy(start_vector(S.D, seed=5)).to(dev), 50, 0.0)
    assert r["iters"] <= S.D
    assert r["energy"] == pytest.approx(ground_energy_dense(S.dense()), abs=1e-12)


@pytest.mark.parametrize("case", [("sq3x3", 4, 4, 1.0, 6.0), ("ring10", 5, 5, 1.0, 3.0), ("sq4x3", 2, 3, 1.0, 9.0)])
def test_lanczos_energy_small(dev, case):
    H, S = _sector(*case)
    from scipy.sparse.linalg import eigsh
    e_ref = float(eigsh(S.explicit(), k=1, which="SA", tol=1e-14, v0=start_vector(S.D, seed=9))[0][0])
    r = hub.lanczos_ground_state(H, torch.from_numpy(start_vector(S.D, seed=1234)).to(dev), 1000, 1e-10)
    assert r["status"] == hub.HUB_OK
    assert abs(r["energy"] - e_ref) <= 1e-9 * max(abs(e_ref), 1.0)


# ---- the 4x4 (8,8) sector: D = 1.66e8 ----------------------------------------
@pytest.fixture(scope="module")
def sq4x4(dev):
    H, S = _sector("sq4x4", 8, 8, 1.0, 8.0)
    v0 = start_vector(S.D, seed=1234)
    return H, S, v0


def test_config2_sampled_rows(dev, sq4x4):
    H, S, v0 = sq4x4
    f = v0 / np.linalg.norm(v0)
    fd = torch.from_numpy(f).to(dev)
    w = torch.empty_like(fd)
    hub.hubbard_apply(H, fd, w)
    rng = np.random.default_rng(1)
    J = np.concatenate([rng.integers(0, S.D, 4000), np.arange(64), S.D - 1 - np.arange(64)])
    ref = S.rows_of_hv(J, f)
    got = w.cpu().numpy()[J]
    assert np.abs(got - ref).max() <= 1e-12
    # the reference kernel over the whole vector (property: both GPU paths agree)
    w2 = torch.empty_like(fd)
    hub.hubbard_apply_reference(H, fd, w2)
    assert (w - w2).abs().max().item() <= 1e-12
    del fd, w, w2


def test_config2_whole_vector_vs_oracle(dev, sq4x4):
    """Every one of the 1.66e8 elements of one H*v on the 4x4 (8,8) sector
    against the oracle's Kronecker-sum H*v (plain C, Eq. H-Kroneckersum):
    binary64 within 1e-12 |v|_2, binary32 within its stated bound."""
    from oracle.kron import KronHamiltonian
    H, S, v0 = sq4x4
    K = KronHamiltonian(S.ns, S.bonds, S.nup, S.ndn, S.t, S.U)
    f = v0 / np.linalg.norm(v0)
    ref = K.hv(f)
    fd = torch.from_numpy(f).to(dev)
    w = torch.empty_like(fd)
    hub.hubbard_apply(H, fd, w)
    assert np.abs(w.cpu().numpy() - ref).max() <= 1e-12
    del fd, w
    f32 = f.astype(np.float32)
    ref32 = K.hv(f32.astype(np.float64))
    fd = torch.from_numpy(f32).to(dev)
    w = torch.empty_like(fd)
    hub.hubbard_apply(H, fd, w)
    tol = 4e-7 * (H.Wup + H.Wdn + 1) * max(1.0, abs(S.U) * S.ns) * np.abs(f32).max()
    assert np.abs(w.cpu().numpy().astype(np.float64) - ref32).max() <= tol
    del fd, w


def test_config2_ground_state(dev, sq4x4):
    H, S, v0 = sq4x4
    g = json.load(open(os.path.join(GOLD, "sq4x4_n8_8_U8.json")))
    r = hub.lanczos_ground_state(H, torch.from_numpy(v0).to(dev), 600, 1e-10)
    assert r["status"] == hub.HUB_OK and r["residual"] < 1e-10
    assert abs(r["energy"] - g["e0"]) <= 1e-9 * abs(g["e0"])


# ---- vector operations --------------------------------------------------------
@pytest.mark.parametrize("n", [1, 7, 1000, 1 << 20, 3_000_017])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_vec_ops(dev, n, dtype):
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = start_vector(n, seed=1).astype(np.float64)
    y = start_vector(n, seed=2).astype(np.float64)
    if dtype == "f32":
        x, y = x.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x).to(dev, tdt)
    yd = torch.from_numpy(y).to(dev, tdt)
    assert hub.hubbard_vec_dot(xd, yd) == pytest.approx(float(x @ y), rel=1e-12, abs=1e-12)
    assert hub.hubbard_vec_nrm2(xd) == pytest.approx(float(np.linalg.norm(x)), rel=1e-12)
    hub.hubbard_vec_axpy(-0.75, xd, yd)
    tol = 1e-15 if dtype == "f64" else 2e-7
    assert np.abs(yd.cpu().double().numpy() - (y - 0.75 * x)).max() <= tol * 2


def test_argument_errors(dev):
    H, S = _sector("ring6", 3, 3, 1.0, 2.0)
    buf = torch.zeros(S.D + 2, dtype=torch.float64, device=dev)
    w = torch.zeros(S.D, dtype=torch.float64, device=dev)
    with pytest.raises(hub.HubError) as e:
        hub.hubbard_apply(H, buf[1:S.D + 1], w)                     # 8-byte offset: misaligned
    assert e.value.code == hub.HUB_EINVAL
    with pytest.raises(hub.HubError) as e:
        hub.hubbard_apply(H, buf[:S.D], buf[2:S.D + 2])              # overlap
    assert e.value.code == hub.HUB_EINVAL
    with pytest.raises(hub.HubError):
        hub.hubbard_sector_create(4, [(0, 1), (1, 0)], 1, 1, 1.0, 1.0)
    with pytest.raises(hub.HubError):
        hub.hubbard_sector_create(4, [(0, 1)], 1, 1, float("nan"), 1.0)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_schedules_bit_identical_and_autotune(dev, dt):
    """Every H*v schedule (rows per block, row CTAs per SM, up-phase columns per
    lane, binary64 up-phase variant) gives the same bits; the autotuner keeps
    one of them."""
    tdt = torch.float64 if dt == "f64" else torch.float32
    ns, bonds = lattice_by_name("sq4x3")
    H = hub.hubbard_sector_create(ns, bonds, 6, 5, 1.0, 4.0)
    v = torch.from_numpy(start_vector(H.D, seed=17)).to(dev, tdt)
    w = torch.empty_like(v)
    ref = None
    vmax = 2 if dt == "f64" else 4
    for vr in (1, 2, 4):
        for vc in (1, 2, 4):
            if vr > vmax or vc > vmax:
                continue
            for cr in (1, 2):
                for cc in ((0, 1, 2) if dt == "f64" else (0,)):
                    hub.hubbard_set_schedule(H, vr, vc, cr, cc)
                    hub.hubbard_apply(H, v, w)
                    if ref is None:
                        ref = w.clone()
                    assert torch.equal(w, ref), (vr, vc, cr, cc)
    chosen = hub.hubbard_autotune_schedule(H, v, w)
    assert chosen[0] in (1, 2, 4) and chosen[1] in (1, 2, 4) and chosen[2] in (1, 2) and chosen[3] in (0, 1, 2)
    hub.hubbard_apply(H, v, w)
    assert torch.equal(w, ref)


def test_shared_tables_between_handles(dev):
    """Handles of the same lattice and fillings share one set of device tables
    (and N_up = N_dn shares it between the spins); each handle keeps its own
    t, U and scratch, and destroying one leaves the others intact."""
    ns, bonds = lattice_by_name("sq3x3")
    S1 = Sector(ns, bonds, 4, 4, 1.0, 3.0)
    S2 = Sector(ns, bonds, 4, 4, 0.5, 7.0)
    H1 = hub.hubbard_sector_create(ns, bonds, 4, 4, 1.0, 3.0)
    H2 = hub.hubbard_sector_create(ns, bonds, 4, 4, 0.5, 7.0)
    x = start_vector(S1.D, seed=8)
    v = torch.from_numpy(x).to(dev)
    w = torch.empty_like(v)
    hub.hubbard_apply(H1, v, w)
    assert np.abs(w.cpu().numpy() - S1.explicit() @ x).max() <= 1e-12 * np.linalg.norm(x)
    H1.close()
    hub.hubbard_apply(H2, v, w)
    assert np.abs(w.cpu().numpy() - S2.explicit() @ x).max() <= 1e-12 * np.linalg.norm(x)
    H3 = hub.hubbard_sector_create(ns, bonds, 4, 4, 1.0, 3.0)       # tables from the cache
    hub.hubbard_apply(H3, v, w)
    assert np.abs(w.cpu().numpy() - S1.explicit() @ x).max() <= 1e-12 * np.linalg.norm(x)
    for spin in (0, 1):
        for g, r in zip(hub.hubbard_export_tables(H3, spin), S1.spin_table(spin)):
            assert np.array_equal(g, r)
    H2.close()
    H3.close()


@pytest.mark.parametrize("scale", [2.0 ** 900, 2.0 ** -900, 1e-310, 3.7e12])
@pytest.mark.parametrize("case", [("sq3x3", 4, 5, 1.0, 6.0), ("ring6", 3, 3, 0.75, 2.5), ("ring8", 4, 3, 1.3, 7.0)])
def test_hv_f64_extreme_scales(dev, case, scale):
    """The fixed-point grid follows max|v| wherever it lies in the binary64
    range (huge, tiny, subnormal inputs), both in the standalone H*v and in a
    Lanczos step; an all-zero vector gives zero."""
    H, S = _sector(*case)
    t = case[3]
    u = start_vector(S.D, seed=79)
    v = u * scale
    ref = (S.explicit() @ u) * scale                   # no overflow in the reference
    vd = torch.from_numpy(v).to(dev)
    w = torch.full_like(vd, np.nan)
    hub.hubbard_apply(H, vd, w)
    got = w.cpu().numpy()
    assert np.all(np.isfinite(got))
    nrm = np.linalg.norm(u) * scale
    # subnormal inputs: the fixed-point grid cannot go below the smallest subnormal
    floor = 4.95e-324 * (S.D ** 0.5) * 64 * max(1.0, abs(t))
    err = np.abs(got - ref).max()
    tol = 1e-12 * nrm * max(1.0, abs(t)) + floor
    assert err <= tol, (err, tol, np.abs(ref).max())
    z = torch.zeros_like(vd)
    hub.hubbard_apply(H, z, w)
    assert torch.count_nonzero(w).item() == 0
