"""nm_filter_apply_static, the filter entry point that allocates no device
memory, against nm_filter_apply (FP64) through the C ABI.

The file is named to be collected last: it has to pass in a fresh process,
where its first call sets up the static scratch on the device, and after
every other test, when the library, contexts and the problem-owned scratch
are already live. Two calls in a row with different widths check that the
array's left-over contents from one call do not leak into the next.
Tolerance: 1e-9 relative to the largest entry, the FP64 filter bound of the
parity tests (both entry points run the same kernels, so in practice they
agree to the bit).
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = "cuda:0"


def _nm():
    from paper_1906_11082_gb300 import _build
    _build.build()
    from paper_1906_11082_gb300 import nm
    return nm


def test_static_limit_matches_header():
    nm = _nm()
    src = open(os.path.join(ROOT, "include", "nm.h")).read()
    m = re.search(r"#define NM_STATIC_SCRATCH_BYTES \((\d+)u << (\d+)\)", src)
    assert m, "NM_STATIC_SCRATCH_BYTES not found in the header"
    assert nm.NM_STATIC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))
    assert hasattr(C.CDLL(nm.LIB_PATH), "nm_filter_apply_static")


@pytest.fixture(scope="module")
def planet():
    pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_11082_gb300 import nm
    from synth.model import layered_planet
    mesh, model = layered_planet(h=0.25, seed=7)
    ctx = nm.Context(0)
    P = nm.Problem(ctx, mesh, model)
    yield nm, ctx, P
    P.free()
    ctx.close()


def _filter(nm, P, d=12, k=8):
    lo, hi = P.spectrum_bounds(k_M=k)
    gam, c, e = nm.filter_design(lo, hi, 0.5, 9.0, d)
    gam = np.ascontiguousarray(gam, np.float64)
    f = nm.nm_filter(d, gam.ctypes.data_as(C.POINTER(C.c_double)), c, e, k, k, 0.0, 0.0)
    return f, gam, c, e, k


def _call_static(nm, ctx, P, f, Y, Z, stream):
    b = Y.shape[1]
    rc = nm.lib().nm_filter_apply_static(P.h, C.byref(f), C.c_void_p(Y.data_ptr()), Y.stride(0),
                                         C.c_void_p(Z.data_ptr()), Z.stride(0), b, C.c_void_p(stream))
    return rc, (nm.lib().nm_last_error(ctx.h) or b"").decode()


@pytest.mark.gpu
def test_static_matches_filter_apply_two_calls(planet):
    import torch
    nm, ctx, P = planet
    f, gam, c, e, k = _filter(nm, P)
    rng = np.random.default_rng(20)
    widths = (16, 8)               # the second call leaves part of the first call's scratch behind
    Ys = [torch.tensor(rng.standard_normal((P.n, b)), dtype=torch.float64, device=DEV) for b in widths]
    refs = []
    for Y in Ys:
        Zr = torch.empty_like(Y)
        P.filter_apply(gam, c, e, k, Y, Zr, k_P=k, prec=nm.NM_F64)
        refs.append(Zr)
    outs = [torch.full_like(Y, float("nan")) for Y in Ys]
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free_before = None
    for i, (Y, Z) in enumerate(zip(Ys, outs)):
        if i == 1:
            free_before = torch.cuda.mem_get_info()[0]
        rc, msg = _call_static(nm, ctx, P, f, Y, Z, stream)
        assert rc == nm.NM_OK, msg
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    # after the first call's set-up, a call takes no device memory
    assert free_before - free_after < (1 << 20)
    for Z, Zr in zip(outs, refs):
        z, zr = Z.cpu().numpy(), Zr.cpu().numpy()
        assert np.isfinite(z).all()
        assert np.abs(z - zr).max() <= 1e-9 * np.abs(zr).max()


@pytest.mark.gpu
def test_static_rejects_sizes_above_the_maximum(planet):
    import torch
    nm, ctx, P = planet
    f, *_ = _filter(nm, P, d=2, k=2)
    b = 64
    need = (5 * P.n + 3 * P.Np) * b * 8
    assert need > nm.NM_STATIC_SCRATCH_BYTES
    Y = torch.ones((P.n, b), dtype=torch.float64, device=DEV)
    Z = torch.full_like(Y, 7.0)
    torch.cuda.synchronize()
    rc, msg = _call_static(nm, ctx, P, f, Y, Z, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == nm.NM_EINVAL
    assert "static maximum" in msg and str(need) in msg
    assert bool((Z == 7.0).all())     # rejected before any launch
