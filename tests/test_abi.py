"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function include/spca.h declares, and argument errors come back as
status codes with a message (no CUDA call is reached for them)."""
import ctypes
import os
import re

import pytest

import paper_1704_07669_gb300 as spca
from paper_1704_07669_gb300 import build as spca_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(spca_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    spca_build.build()
    return spca.lib()


def test_header_declares_the_core_calls():
    names = _declared_functions()
    for core in ("spca_create", "spca_update", "spca_finalize", "spca_destroy", "spca_merge"):
        assert core in names


def test_library_exports_every_declared_function(lib):
    raw = ctypes.CDLL(spca.lib_path())
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_default_options(lib):
    opt = spca.Options()
    lib.spca_default_options(ctypes.byref(opt))
    assert (opt.math, opt.center, opt.max_block_rows, opt.reserved) == (spca.SPCA_MATH_FP32, 1, 0, 0)
    assert not opt.cuda_stream


@pytest.mark.parametrize("n,k,p", [(0, 1, 0), (10, 0, 1), (10, 2, -1), (10, 8, 5), (1000, 200, 60)])
def test_create_rejects_bad_sizes_without_touching_the_gpu(lib, n, k, p):
    with pytest.raises(spca.SpcaError) as ei:
        spca.spca_create(n, k, p, 1)
    assert ei.value.status == 1
    assert spca.spca_last_error(None)


def test_create_rejects_bad_options(lib):
    opt = spca.Options()
    lib.spca_default_options(ctypes.byref(opt))
    opt.reserved = 7
    out = ctypes.c_void_p()
    assert lib.spca_create(100, 5, 5, 1, ctypes.byref(opt), ctypes.byref(out)) == 1
    assert out.value is None
    opt.reserved = 0
    opt.center = 3
    assert lib.spca_create(100, 5, 5, 1, ctypes.byref(opt), ctypes.byref(out)) == 1
    assert lib.spca_create(100, 5, 5, 1, ctypes.byref(opt), None) == 1


def test_null_session_calls_return_errors(lib):
    assert lib.spca_update(None, None, 1, 1, 0, None, 1, None) == 1
    assert lib.spca_finalize(None, None, None, 0) == 1
    assert lib.spca_left_vectors(None, None, 1, None, 0) == 1
    assert lib.spca_power_step(None) == 1
    assert lib.spca_state_bytes(None, None) == 1
    assert lib.spca_save_state(None, None, 0) == 1
    assert lib.spca_load_state(None, None, 0) == 1
    assert lib.spca_sync(None) == 1
    assert lib.spca_reset(None, 0) == 1
    assert lib.spca_merge(None, None) == 1
    assert lib.spca_destroy(None) == 0
    assert lib.spca_rows_seen(None) == -1
    assert lib.spca_set_profiling(None, 1) == 1
    assert lib.spca_omega_words(1, 0, 4, None) == 1
    assert lib.spca_omega(1, 10, 0, None) == 1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(spca, "_LIB", None)
    monkeypatch.setattr(spca_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        spca.lib()


def test_binding_rejects_layouts_the_library_cannot_see():
    """Checks the C ABI cannot make (it gets a pointer and a leading dimension): rows whose
    columns are not adjacent, and result buffers that are not float64, are refused before any
    library call (the handle below is never used)."""
    import numpy as np
    rows = np.zeros((8, 6), dtype=np.float32)
    with pytest.raises(ValueError):
        spca.spca_update(0, rows[:, ::2])                       # every other column
    with pytest.raises(ValueError):
        spca.spca_update(0, np.asfortranarray(rows))            # column-major
    with pytest.raises(ValueError):
        spca.spca_finalize(0, np.zeros(3, dtype=np.float32), np.zeros((3, 6)))
    with pytest.raises(ValueError):
        spca.spca_finalize(0, np.zeros(3), np.zeros((6, 3)).T)  # not contiguous
    with pytest.raises(ValueError):
        spca.spca_left_vectors(0, None, np.zeros((3, 8), dtype=np.float32))
