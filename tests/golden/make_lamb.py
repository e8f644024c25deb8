"""Writes lamb_ball.json: traction-free homogeneous-ball eigenfrequencies.

Closed-form equations (Lamb 1882; Dahlen & Tromp 1998, Sec. 8.7) solved by
root bracketing; calls only the oracle's closed-form module.
Run from the repository root: python tests/golden/make_lamb.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.lamb import lamb_modes  # noqa: E402

modes = lamb_modes(6.0, a=1.0, vp=1.7, vs=1.0)
out = {"source": "traction-free homogeneous ball, a=1, rho=1, Vp=1.7, Vs=1 "
                 "(Lamb 1882; Dahlen & Tromp 1998 Sec. 8.7)",
       "modes": [{"omega": w, "label": lab, "multiplicity": m} for w, lab, m in modes]}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lamb_ball.json"), "w") as f:
    json.dump(out, f, indent=1)
