"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol include/nm.h declares; host-only entry points agree with the oracle;
calls fail with status codes (never crash) when no device is usable."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nm():
    from paper_1906_11082_gb300 import _build
    _build.build()
    from paper_1906_11082_gb300 import nm as mod
    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "nm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|uint64_t|const\s+\w+\s*\*|const\s+char\s*\*)\s*(nm_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nm_assemble", "nm_set_interval", "nm_filter_apply", "nm_lanczos_slice", "nm_ritz"):
        assert required in names


def test_every_declared_symbol_is_exported(nm):
    lib = ctypes.CDLL(nm.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(nm.EXPORTS)


def test_filter_design_matches_oracle(nm):
    from oracle import filtlan
    for (lo, hi, xi, eta, d) in [(-1.0, 5000.0, 0.0, 9.0, 100), (0.0, 10.0, 2.0, 4.0, 30),
                                 (-3.0, 7.0, -2.0, 6.5, 7)]:
        g, c, e = nm.filter_design(lo, hi, xi, eta, d)
        g2, c2, e2 = filtlan.filter_coeffs(lo, hi, xi, eta, d)
        assert np.allclose(g, g2, rtol=1e-13, atol=1e-15)
        assert c == pytest.approx(c2) and e == pytest.approx(e2)


def test_invalid_arguments_return_status(nm):
    lib = nm.lib()
    g = np.empty(4)
    c, e = ctypes.c_double(), ctypes.c_double()
    # lam_hi <= lam_lo
    rc = lib.nm_filter_design(1.0, 0.0, 0.0, 1.0, 3, g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(c),
                              ctypes.byref(e))
    assert rc == nm.NM_EINVAL
    assert b"lam_lo" in lib.nm_last_error(None)
    assert lib.nm_set_interval(None, 0.0, 1.0, 0) == nm.NM_EINVAL
    assert lib.nm_filter_apply(None, None, None, 0, None, 0, 1, 0, None) == nm.NM_EINVAL


def test_ctx_create_without_gpu_fails_cleanly(nm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = nm.lib().nm_ctx_create(0, ctypes.byref(h))
    assert rc == nm.NM_ECUDA and not h.value
