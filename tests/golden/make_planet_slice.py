"""Writes planet_slice.json: the eigenvalues of one slice of the three-layer
planet's Cowling pencil (h = 0.25, seed 7; fluid core, reference gravity),
from the oracle's dense generalized symmetric eigensolver (FP64, eigh of
K_eff and M assembled by oracle/fem.py). The slice starts in the gap after
the third eigenvalue above 0.5 and ends in the widest gap after the 11th to
20th; both edges sit at gap midpoints. bench.py's precision leg reports the error of every eigenvalue of
each precision form against these values.
Run from the repository root: python tests/golden/make_planet_slice.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import eig, fem  # noqa: E402
from synth.model import layered_planet  # noqa: E402

mesh, model = layered_planet(h=0.25, seed=7)
K, M = eig.pencil_dense(fem.assemble(mesh, model))
lam = eig.all_eigs(K, M)[0]
above = lam[lam > 0.5]
lo = 0.5 * (above[2] + above[3])
k = 10 + int(np.argmax(np.diff(above[10:21])))
hi = 0.5 * (above[k] + above[k + 1])
out = {"source": "oracle dense eigh of (K_eff, M), layered_planet(h=0.25, seed=7), FP64",
       "lambda_lo": lo, "lambda_hi": hi, "lambda_max": float(lam[-1]),
       "eigenvalues": [float(x) for x in lam[(lam >= lo) & (lam <= hi)]]}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "planet_slice.json"), "w") as f:
    json.dump(out, f, indent=1)
