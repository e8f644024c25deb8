"""The stored oracle eigenvalues of tests/golden/planet_slice.json (the
reference of bench.py's per-eigenvalue precision report) are the oracle's:
recomputed by dense eigh, the slice edges sit in gaps of the spectrum."""
import json
import os

import numpy as np

from oracle import eig, fem
from synth.model import layered_planet

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "planet_slice.json")


def test_planet_slice_golden_matches_oracle():
    with open(GOLD) as f:
        gold = json.load(f)
    mesh, model = layered_planet(h=0.25, seed=7)
    lam = eig.all_eigs(*eig.pencil_dense(fem.assemble(mesh, model)))[0]
    lo, hi = gold["lambda_lo"], gold["lambda_hi"]
    ref = lam[(lam >= lo) & (lam <= hi)]
    assert len(ref) == len(gold["eigenvalues"]) == 13
    assert np.allclose(ref, gold["eigenvalues"], rtol=1e-12)
    # edges in gaps: no eigenvalue within 10% of the slice width of an edge
    width = hi - lo
    assert np.min(np.abs(lam - lo)) > 0.1 * width and np.min(np.abs(lam - hi)) > 0.1 * width
