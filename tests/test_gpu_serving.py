"""Serving: requests admitted while others run, overlapping on the device;
each result equals the same request solved alone (eigenvalues to 1e-8
relative, residuals <= 1e-6)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


_EDGES = {}


def _planet_edges():
    """Two slices of the test planet's seismic spectrum with edges in gaps."""
    if not _EDGES:
        from synth.model import layered_planet
        from oracle import fem, eig
        mesh, model = layered_planet(h=0.25, seed=7)
        S = fem.assemble(mesh, model)
        lam = eig.all_eigs(*eig.pencil_dense(S))[0]
        hi = np.sqrt(lam[lam > 0.5])
        _EDGES["a"] = (0.5 * (hi[3] + hi[4]), 0.5 * (hi[13] + hi[14]))
        _EDGES["b"] = (0.5 * (hi[10] + hi[11]), 0.5 * (hi[20] + hi[21]))
    return _EDGES["a"], _EDGES["b"]


def _requests():
    from synth.model import config_ball, layered_planet
    from paper_1906_11082_gb300 import nm
    pa, pb = _planet_edges()

    def ball():
        w = config_ball()
        return w.mesh, w.model

    def planet():
        return layered_planet(h=0.25, seed=7)

    opts_b = dict(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=3)
    opts_p = dict(block=8, degree=400, k_M=20, k_P=20, max_blocks=30, seed=2, check_every=2, prec=nm.NM_MIXED)
    return [("ball", ball, (0.0, 3.0), opts_b, 1899),
            ("planet", planet, pa, opts_p, 9627),
            ("ball", ball, (2.0, 2.9), opts_b, 1899),
            ("planet", planet, pb, opts_p, 9627)]


def test_serving_mix_equals_alone():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_11082_gb300 import nm
    from paper_1906_11082_gb300.serving import Request, SliceServer

    alone = []
    ctx = nm.Context(0)
    for key, build, iv, opts, _ in _requests():
        mesh, model = build()
        P = nm.Problem(ctx, mesh, model)
        P.set_interval(*iv)
        r = P.lanczos_slice(allow_unconverged=True, **opts)
        alone.append(r.lam.copy())
        r.free()
        P.free()
    ctx.close()

    srv = SliceServer(slots=3)
    reqs = []
    for i, (key, build, iv, opts, ndof) in enumerate(_requests()):
        reqs.append(srv.submit(Request(key=key, build=build, interval=iv, opts=opts), ndof))
        time.sleep(0.05 * i)           # staggered arrivals while earlier requests run
    srv.drain(timeout=600)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["errors"] == 0
    assert st["overlap_max"] >= 2
    for r, ref in zip(reqs, alone):
        assert len(r.lam) == len(ref) and len(ref) > 0
        assert np.allclose(r.lam, ref, rtol=1e-8, atol=1e-10 * max(1.0, np.abs(ref).max()))
        assert r.resid.max() <= 1e-6
    assert st["p99_s"] >= st["p50_s"] > 0
