"""The C ABI library builds, loads and exports every symbol include/tlr.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tlr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^int\s+(tlr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09137_gb300 import build as B
    from paper_1804_09137_gb300 import tlr as T

    B.build()
    return T.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ["tlr_create", "tlr_destroy", "tlr_matern_generate", "tlr_compress", "tlr_potrf", "tlr_loglik",
                 "tlr_loglik_grad", "tlr_predict"]:
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1804_09137_gb300 import tlr as T

    assert sorted(T.EXPORTS) == _declared()


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_1804_09137_gb300.tlr import TlrOpts

    h = C.c_void_p()
    opts = TlrOpts(64, 1e-9, 0, 0, 1, 0, 0.0)
    assert lib.tlr_create(0, None, None, C.byref(opts), None, C.byref(h)) == -1
    assert lib.tlr_create(10, None, None, C.byref(opts), None, C.byref(h)) == -2
    bad = TlrOpts(0, 1e-9, 0, 0, 1, 0, 0.0)
    one = C.c_double(0.0)
    assert lib.tlr_create(10, C.byref(one), C.byref(one), C.byref(bad), None, C.byref(h)) == -4
    assert lib.tlr_destroy(None) == -1
    assert lib.tlr_status(None, None) == -1
