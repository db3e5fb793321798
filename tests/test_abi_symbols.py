"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import re

from paper_1609_07757_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"ISCSI_API\s+[\w\s\*]+?\b(iscsi_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_symbols()
    assert len(names) >= 18
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    src = open(os.path.join(ROOT, "paper_1609_07757_gb300", "_lib.py")).read()
    for n in declared_symbols():
        assert '"%s"' % n in src, n


def test_calls_without_context_fail_cleanly():
    lib = _lib.load()
    assert lib.iscsi_ndet() == -1
    assert lib.iscsi_ctx_current() == 0
    assert lib.iscsi_sigma(None, None, 1) == _lib.ISCSI_E_NOINIT
    assert lib.iscsi_density(None, None, None, None) == _lib.ISCSI_E_NOINIT
    assert lib.iscsi_set_gas(0, None, None, None, None) == _lib.ISCSI_E_NOINIT
    assert lib.iscsi_gas_mask(None) == _lib.ISCSI_E_NOINIT
    assert lib.iscsi_set_option(b"no_such_key", 1.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_set_option(b"precision", 16.0) == _lib.ISCSI_E_ARG
    assert b"precision" in lib.iscsi_last_error()
    assert lib.iscsi_batch_sigma(None, None, None, 0, 1) == _lib.ISCSI_E_ARG
    assert b"iscsi_batch_sigma" in lib.iscsi_last_error()


def test_init_rejects_bad_arguments_before_touching_the_gpu():
    lib = _lib.load()
    h = (ctypes.c_double * 4)()
    assert lib.iscsi_init(0, 1, 1, 2, h, None, 0.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_init(2, 1, 1, 2, h, None, -1.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_init(300, 1, 1, 2, h, None, 0.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_init(2, 3, 1, 2, h, None, 0.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_init(2, 1, 1, 2, None, None, 0.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_init(2, 1, 1, 2, h, None, float("nan")) == _lib.ISCSI_E_ARG
    # C(256, 16) ~ 1e25 strings: rejected by the string-space limit, not by an overflow
    assert lib.iscsi_init(256, 16, 16, 2, h, None, 0.0) == _lib.ISCSI_E_ARG
    assert b"string space" in lib.iscsi_last_error()


def test_init_gas_rejects_bad_limits_before_touching_the_gpu():
    lib = _lib.load()
    h = (ctypes.c_double * 4)()
    arr = lambda *v: (ctypes.c_int * len(v))(*v)
    # sizes not adding up to norb, cmin > cmax, cmax above the electrons, an empty subspace, 9 subspaces
    for sizes, cmin, cmax in [((1, 2), (0, 2), (2, 2)), ((1, 1), (2, 2), (1, 2)), ((1, 1), (0, 2), (2, 3)),
                              ((0, 2), (0, 2), (2, 2))]:
        assert lib.iscsi_init_gas(2, 1, 1, 2, arr(*sizes), arr(*cmin), arr(*cmax), h, None, 0.0) == _lib.ISCSI_E_ARG
    nine = arr(*([1] * 9))
    assert lib.iscsi_init_gas(9, 1, 1, 9, nine, arr(*([0] * 9)), arr(*([2] * 9)), h, None, 0.0) == _lib.ISCSI_E_ARG
    # a string space far too large (the enclosing space is chosen first, with saturated counts)
    big = arr(128, 128)
    assert lib.iscsi_init_gas(256, 16, 16, 2, big, arr(0, 32), arr(32, 32), h, None, 0.0) == _lib.ISCSI_E_ARG
    assert lib.iscsi_ctx_current() == 0
