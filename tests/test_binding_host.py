"""Host tests of the binding's argument checks: the C entry points read and
write exactly D elements of the given dtype, so a vector of the wrong dtype or
length must be refused before any pointer reaches the library (no GPU needed:
the checks run before a device pointer is taken)."""
import types

import pytest

import paper_1204_3425_gb300 as hub

torch = pytest.importorskip("torch")


def _fake_sector(D):
    return types.SimpleNamespace(D=D, handle=None)


@pytest.mark.parametrize("fn", [hub.hubbard_apply, hub.hubbard_apply_reference, hub.hubbard_apply_noalloc,
                                hub.hubbard_autotune_schedule])
def test_wrong_length_refused(fn):
    H = _fake_sector(100)
    v = torch.zeros(99, dtype=torch.float64)
    w = torch.zeros(100, dtype=torch.float64)
    with pytest.raises(ValueError):
        fn(H, v, w)
    with pytest.raises(ValueError):
        fn(H, w, v)


@pytest.mark.parametrize("fn", [hub.hubbard_apply, hub.hubbard_apply_reference, hub.hubbard_autotune_schedule])
def test_mixed_or_unsupported_dtype_refused(fn):
    H = _fake_sector(8)
    with pytest.raises(TypeError):
        fn(H, torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float32))
    with pytest.raises(TypeError):
        fn(H, torch.zeros(8, dtype=torch.float16), torch.zeros(8, dtype=torch.float16))


def test_noalloc_accepts_only_binary64():
    H = _fake_sector(8)
    with pytest.raises(TypeError):
        hub.hubbard_apply_noalloc(H, torch.zeros(8, dtype=torch.float32), torch.zeros(8, dtype=torch.float32))
    with pytest.raises(TypeError):
        hub.hubbard_apply_noalloc(H, torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float32))


def test_apply_host_checks_before_the_library():
    H = _fake_sector(8)
    with pytest.raises(ValueError):                      # a device tensor is not a host buffer
        hub.hubbard_apply_host(H, types.SimpleNamespace(device=types.SimpleNamespace(type="cuda")),
                               torch.zeros(8, dtype=torch.float64))
    with pytest.raises(TypeError):
        hub.hubbard_apply_host(H, torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError):
        hub.hubbard_apply_host(H, torch.zeros(7, dtype=torch.float64), torch.zeros(8, dtype=torch.float64))


def test_queue_and_host_apply_c_entry_points_refuse_bad_arguments():
    """The queued solver's and the host-buffer product's argument checks run
    before any CUDA call (no GPU needed)."""
    import ctypes
    lib = hub.load_library()
    out = ctypes.c_void_p()
    assert lib.hubbard_queue_create(0, 100, 10, 1e-10, 0, ctypes.byref(out)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_create(4, 0, 10, 1e-10, 0, ctypes.byref(out)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_create(4, 100, 0, 1e-10, 0, ctypes.byref(out)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_create(4, 100, 10, -1.0, 0, ctypes.byref(out)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_create(4, 100, 10, 1e-10, -1, ctypes.byref(out)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_create(4, 100, 10, 1e-10, 0, None) == hub.HUB_EINVAL
    tk = ctypes.c_int64()
    assert lib.hubbard_queue_post(None, None, 1, ctypes.byref(tk)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_poll(None, 0, None) == hub.HUB_EINVAL
    n = ctypes.c_int()
    assert lib.hubbard_queue_collect(None, None, None, 0, ctypes.byref(n)) == hub.HUB_EINVAL
    assert lib.hubbard_queue_prepare(None, None) == hub.HUB_EINVAL
    lib.hubbard_queue_destroy(None)                      # a null queue is ignored
    buf = (ctypes.c_double * 8)()
    assert lib.hubbard_apply_host(None, buf, buf, hub.HUB_F64, None) == hub.HUB_EINVAL


def test_time_evolve_checks_before_the_library():
    """Host-side refusals of the propagator's binding and C entry point."""
    import ctypes
    H = _fake_sector(8)
    with pytest.raises(TypeError):
        hub.hubbard_time_evolve(H, torch.zeros(8, dtype=torch.float32), None, 0.5)
    with pytest.raises(ValueError):
        hub.hubbard_time_evolve(H, torch.zeros(7, dtype=torch.float64), None, 0.5)
    with pytest.raises(ValueError):                      # host tensors are not device vectors
        hub.hubbard_time_evolve(H, torch.zeros(8, dtype=torch.float64), None, 0.5,
                                workspace=torch.zeros(16, dtype=torch.uint8))
    lib = hub.load_library()
    info = hub.EvolveInfo()
    info.steps, info.norm = 7, 3.0
    assert lib.hubbard_time_evolve(None, None, None, 0.5, 10, 1e-10, None, 0, None, None, None,
                                   ctypes.byref(info)) == hub.HUB_EINVAL
    assert info.status == hub.HUB_EINVAL and info.steps == 0 and info.norm == 0.0
    assert lib.hubbard_evolve_workspace_bytes(None, 10, 1) == 0


def _expm_first_column(a, b, tau):
    import numpy as np
    from scipy.linalg import expm
    m = len(a)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1) if m > 1 else np.diag(a)
    return expm(-1j * tau * T)[:, 0]


@pytest.mark.parametrize("m,tau,seed", [(1, 0.7, 0), (2, -1.3, 1), (7, 2.5, 2), (40, 0.9, 3), (160, -4.0, 4),
                                        (64, 11.0, 5)])
def test_host_krylov_exp_matches_expm(m, tau, seed):
    """exp(-i T tau) e_1 of the host QR eigensolver against scipy's expm."""
    import numpy as np
    rng = np.random.default_rng(seed)
    a = rng.uniform(-5, 9, m)
    b = rng.uniform(0.05, 3, m - 1)
    y = hub.hubbard_host_krylov_exp(a, b, tau)
    assert np.abs(y - _expm_first_column(a, b, tau)).max() <= 1e-12


def test_host_krylov_exp_degenerate_and_split_tridiagonals():
    """Repeated eigenvalues (a Lanczos run repeats converged Ritz values),
    zero off-diagonals (a split matrix) and a zero matrix."""
    import numpy as np
    a = np.array([1.0, 1.0, 1.0, 2.0, 2.0, -3.0])
    b = np.array([1e-9, 0.0, 0.5, 1e-15, 0.25])
    for tau in (0.3, -2.2):
        assert np.abs(hub.hubbard_host_krylov_exp(a, b, tau) - _expm_first_column(a, b, tau)).max() <= 1e-12
    z = hub.hubbard_host_krylov_exp(np.zeros(5), np.zeros(4), 1.5)
    assert np.array_equal(z, np.eye(5)[:, 0].astype(complex))
    # a Lanczos tridiagonal of the ring 8 sector (clustered Ritz values after many steps)
    from oracle.basis import Sector
    from oracle.lanczos import lanczos_plain
    from workload import lattice_by_name, start_vector
    ns, bonds = lattice_by_name("ring8")
    S = Sector(ns, bonds, 4, 4, 1.0, 4.0)
    Hs = S.explicit()
    r = lanczos_plain(lambda x: Hs @ x, start_vector(S.D, seed=1), 120)
    al = np.asarray(r["a"])
    be = np.asarray(r["b"])[:len(al) - 1]
    assert len(al) == 120
    for tau in (0.5, 3.0):
        assert np.abs(hub.hubbard_host_krylov_exp(al, be, tau) - _expm_first_column(al, be, tau)).max() <= 1e-11


def test_host_krylov_exp_refuses_bad_input():
    import numpy as np
    lib = hub.load_library()
    y = np.zeros(4)
    a = np.ones(4)
    assert lib.hubbard_host_krylov_exp(a.ctypes.data, a.ctypes.data, 0, 1.0, y.ctypes.data, y.ctypes.data) == hub.HUB_EINVAL
    assert lib.hubbard_host_krylov_exp(a.ctypes.data, None, 4, 1.0, y.ctypes.data, y.ctypes.data) == hub.HUB_EINVAL
    assert lib.hubbard_host_krylov_exp(a.ctypes.data, a.ctypes.data, 4, float("nan"), y.ctypes.data,
                                       y.ctypes.data) == hub.HUB_EINVAL
    bad = np.array([1.0, float("inf"), 1.0, 1.0])
    assert lib.hubbard_host_krylov_exp(bad.ctypes.data, a.ctypes.data, 4, 1.0, y.ctypes.data, y.ctypes.data) == hub.HUB_EINVAL


def test_host_krylov_coefficients_propagate_a_lanczos_basis():
    """The library's host coefficients y = exp(-i T_m tau) e_1 applied to a
    Lanczos basis of the oracle's explicit H (the plain recurrence of
    Algorithm 1, written out here in numpy) reproduce exp(-iH tau) v of the
    oracle's eigendecomposition, and Saad's estimate b_{m+1} |y_{m-1}| is of
    the size of the actual error (the step-size rule of the propagator)."""
    import numpy as np
    from oracle import propagate as pr
    from oracle.basis import Sector
    from workload import lattice_by_name, start_vector
    ns, bonds = lattice_by_name("ring8")
    S = Sector(ns, bonds, 4, 4, 1.0, 4.0)
    Hx = S.explicit()
    v = start_vector(S.D, seed=5)
    v /= np.linalg.norm(v)
    F, a, b = [], [], []
    f, g, beta = v.copy(), np.zeros_like(v), 0.0
    for _ in range(30):
        w = Hx @ f - beta * g
        al = float(w @ f)
        w -= al * f
        be = float(np.linalg.norm(w))
        F.append(f)
        a.append(al)
        b.append(be)
        g, f, beta = f, w / be, be
    V = np.array(F).T
    for tau in (0.2, 0.6, -0.45):
        y = hub.hubbard_host_krylov_exp(np.array(a), np.array(b[:-1]), tau)
        err = np.abs(V @ y - pr.evolve_dense(S, v, tau)).max()
        est = b[-1] * abs(y[-1])
        assert err <= 1e-8 and err <= 10 * est + 1e-13, (tau, err, est)
