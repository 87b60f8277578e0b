"""The C-ABI library loads and exports every symbol include/nb.h declares; host-side
argument checks answer NB_EINVAL without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_06822_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = _declared()
    for f in ("nb_label", "nb_train_step", "nb_query", "nb_calibrate"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2310_06822_gb300 import nb
    names = _declared()
    assert sorted(nb.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_host_side_argument_errors(lib):
    lib.nb_label.restype = ctypes.c_int
    lib.nb_last_error.restype = ctypes.c_char_p
    # null shape
    assert lib.nb_label(None, 0, None, ctypes.c_int64(0), None, None, None) == 1
    assert b"shape" in lib.nb_last_error()
    # bad widths: last width must be 1; widths above 256 rejected
    h = ctypes.c_void_p()
    w = (ctypes.c_int32 * 3)(3, 16, 2)
    assert lib.nb_model_create(w, 2, 0, 0, ctypes.byref(h)) == 1
    w = (ctypes.c_int32 * 3)(3, 300, 1)
    assert lib.nb_model_create(w, 2, 0, 0, ctypes.byref(h)) == 1
    assert lib.nb_model_create(w, 9, 0, 0, ctypes.byref(h)) == 1
    # activations: unknown -> NB_EINVAL; sine networks with a BF16/FP8 path -> NB_EUNSUPPORTED
    w = (ctypes.c_int32 * 3)(3, 16, 1)
    assert lib.nb_model_create_act(w, 2, 0, 0, 2, ctypes.byref(h)) == 1
    assert lib.nb_model_create_act(w, 2, 0, 1, 1, ctypes.byref(h)) == 6   # sine, BF16 training
    assert lib.nb_model_create_act(w, 2, 2, 0, 1, ctypes.byref(h)) == 6   # sine, FP8 inference
    assert lib.nb_model_create_act(w, 2, 1, 0, 1, ctypes.byref(h)) == 6   # sine, BF16 inference
    # null model
    lib.nb_query.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.nb_query(None, None, 0, 0.0, None, None, None, None) == 1
    lib.nb_train_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.nb_train_step(None, None, None, 1, 1.0, 1.0, None, None) == 1


def test_selftest_argument_check_needs_no_device(lib):
    lib.nb_selftest_bounded_wait.restype = ctypes.c_int
    lib.nb_selftest_bounded_wait.argtypes = [ctypes.c_int32, ctypes.c_void_p]
    assert lib.nb_selftest_bounded_wait(0, None) == 1  # NB_EINVAL before any device work
    assert lib.nb_selftest_bounded_wait(1 << 21, None) == 1
