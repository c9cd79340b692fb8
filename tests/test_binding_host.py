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
