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
