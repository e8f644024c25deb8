"""Serving: requests admitted while others run, joining the running batch
of their mesh (continuous batching) or overlapping on the device in
another mesh's engine; each result equals the same request solved alone
(eigenvalues to 1e-8 relative, residuals <= 1e-6) and the dense oracle's
eigenvalues of its slice (1e-8)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


_REF = {}


def _oracle():
    """Dense spectra of the two test meshes and two slices of the planet's
    seismic spectrum with edges in gaps."""
    if not _REF:
        from synth.model import config_ball, layered_planet
        from oracle import fem, eig
        mesh, model = layered_planet(h=0.25, seed=7)
        lam = eig.all_eigs(*eig.pencil_dense(fem.assemble(mesh, model)))[0]
        hi = np.sqrt(lam[lam > 0.5])
        _REF["planet"] = lam
        _REF["a"] = (0.5 * (hi[3] + hi[4]), 0.5 * (hi[13] + hi[14]))
        _REF["b"] = (0.5 * (hi[10] + hi[11]), 0.5 * (hi[20] + hi[21]))
        w = config_ball()
        _REF["ball"] = eig.all_eigs(*eig.pencil_dense(fem.assemble(w.mesh, w.model)))[0]
    return _REF


def _requests():
    from synth.model import config_ball, layered_planet
    from paper_1906_11082_gb300 import nm
    ref = _oracle()

    def ball():
        w = config_ball()
        return w.mesh, w.model

    def planet():
        return layered_planet(h=0.25, seed=7)

    opts_b = dict(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=3)
    opts_p = dict(block=8, degree=400, k_M=20, k_P=20, max_blocks=30, check_every=2, prec=nm.NM_MIXED)
    return [("ball", ball, (0.0, 3.0), opts_b, 400),
            ("planet", planet, ref["a"], dict(opts_p, seed=2), 1980),
            ("ball", ball, (2.0, 2.9), dict(opts_b, seed=4), 400),
            ("planet", planet, ref["b"], dict(opts_p, seed=5), 1980),
            ("planet", planet, ref["a"], dict(opts_p, seed=6), 1980)]


def _reference(key, iv):
    lam = _oracle()[key]
    lo, hi = iv
    l = -1e-8 * lam[-1] if lo == 0 else lo * lo
    return lam[(lam >= l) & (lam <= hi * hi)], lam[-1]


def test_serving_mix_equals_alone_and_oracle():
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

    srv = SliceServer(slots=2)
    reqs = []
    for i, (key, build, iv, opts, tets) in enumerate(_requests()):
        reqs.append(srv.submit(Request(key=key, build=build, interval=iv, opts=opts), tets))
        time.sleep(0.3)                # staggered arrivals while earlier requests run
    srv.drain(timeout=900)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["errors"] == 0
    assert st["overlap_max"] >= 2
    assert st["joined_running_batch"] >= 1 and st["max_batch"] >= 2
    for (key, _, iv, _, _), r, ref_alone in zip(_requests(), reqs, alone):
        ref, lam_max = _reference(key, iv)
        assert len(r.lam) == len(ref_alone) == len(ref) > 0
        scale = 1e-10 * lam_max
        assert np.allclose(r.lam, ref_alone, rtol=1e-8, atol=scale)
        assert np.allclose(r.lam, ref, rtol=1e-8, atol=scale)
        assert r.resid.max() <= 1e-6
    assert st["p99_s"] >= st["p50_s"] > 0
