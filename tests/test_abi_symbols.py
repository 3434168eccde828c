"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function include/tild.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tild.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:tild_status|const char\*)\s+(tild_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_02474_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tild_create", "tild_set_chains", "tild_set_interactions", "tild_step", "tild_compute",
                     "tild_get_positions", "tild_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2302_02474_gb300 import binding

    assert sorted(binding.declared_symbols()) == _declared()


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2302_02474_gb300 import binding as B

    lib = B.load()
    p = B.tild_params()
    p.L[:] = [10.0, 10.0, 12.0]
    p.n[:] = [16, 16, 16]
    p.pmeorder = 1
    ctx = ctypes.c_void_p()
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    assert b"cubic" in lib.tild_last_error(None)
    p.L[2] = 10.0
    p.n[:] = [3, 3, 3]  # below the smallest grid
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    p.n[:] = [300, 300, 300]  # above the largest 3D grid
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    p.n[:] = [16, 20, 16]  # not cubic
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    p.n[:] = [65, 64, 1]  # 2D grids are square
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    p.n[:] = [16, 16, 16]
    p.pmeorder = 5
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EINVAL
    p.pmeorder = 1
    p.precision = 1
    p.n[:] = [256, 256, 256]
    assert lib.tild_create(ctypes.byref(p), ctypes.byref(ctx)) == B.TILD_EUNSUPPORTED
    assert lib.tild_create(None, ctypes.byref(ctx)) == B.TILD_EINVAL
    assert lib.tild_destroy(None) == B.TILD_OK
    assert lib.tild_step(None, 1) == B.TILD_EINVAL
    # the variant, electrostatics and differentiable-form calls check their context first
    assert lib.tild_set_integrator_scheme(None, 0) == B.TILD_EINVAL
    assert lib.tild_set_force_method(None, 0) == B.TILD_EINVAL
    assert lib.tild_set_electrostatics(None, 1.0, -1.0, 1.0, 0.5) == B.TILD_EINVAL
    assert lib.tild_force_vjp(None, None, None, B.TILD_DTYPE_F64, B.TILD_HOST, None) == B.TILD_EINVAL
    assert lib.tild_trajectory_vjp(None, 1, 1, None, None, B.TILD_DTYPE_F64, B.TILD_HOST, None, None,
                                   None) == B.TILD_EINVAL
    best, ms = ctypes.c_int(), ctypes.c_double()
    assert lib.tild_autotune(None, 10, ctypes.byref(best), ctypes.byref(ms)) == B.TILD_EINVAL


def test_library_missing_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: a missing library is an error, not a silent path."""
    from paper_2302_02474_gb300 import binding as B

    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setenv("TILD_LIBRARY", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not found"):
        B.load()
