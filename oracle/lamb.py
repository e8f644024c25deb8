"""Free oscillations of a homogeneous, non-gravitating elastic ball.

Test infrastructure (CPU oracle pin). Closed-form traction-free conditions
at r = a for a homogeneous isotropic ball (Lamb 1882; the textbook
treatment in Dahlen & Tromp 1998, Sec. 8.7), used as the h -> 0 limit of
the discrete spectrum of the homogeneous-ball workload:

  toroidal  l >= 1 : (l - 1) j_l(x) - x j_{l+1}(x) = 0,         x = w a / Vs
  radial    l = 0  : x cot x = 1 - x^2 Vp^2 / (4 Vs^2),          x = w a / Vp
  spheroidal l >= 1: det [[s_rr^P, s_rr^S], [t^P, t^S]] = 0 with
     s_rr = (lam + 2 mu) U' + lam (2 U - l(l+1) V) / r,
     t    = mu (V' - V / r + U / r),
     P solution: U = h j_l'(h r),         V = j_l(h r) / r,      h = w / Vp
     S solution: U = l(l+1) j_l(k r) / r,  V = j_l(k r) / r + k j_l'(k r),
                                                                 k = w / Vs
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn
from scipy.optimize import brentq


def _j(l, x):
    return spherical_jn(l, x)


def _jp(l, x):
    return spherical_jn(l, x, derivative=True)


def _jpp(l, x):
    # spherical Bessel equation: x^2 j'' + 2 x j' + (x^2 - l(l+1)) j = 0
    return -(2.0 / x) * _jp(l, x) - (1.0 - l * (l + 1) / x ** 2) * _j(l, x)


def toroidal_fn(l, w, a=1.0, vs=1.0):
    x = w * a / vs
    return (l - 1) * _j(l, x) - x * _j(l + 1, x)


def radial_fn(w, a=1.0, vp=1.7, vs=1.0):
    x = w * a / vp
    return x * np.cos(x) - np.sin(x) * (1.0 - x * x * vp * vp / (4.0 * vs * vs))


def spheroidal_fn(l, w, a=1.0, vp=1.7, vs=1.0, rho=1.0):
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    L = l * (l + 1)
    r = a
    h = w / vp
    k = w / vs
    # P solution
    U = h * _jp(l, h * r)
    Up = h * h * _jpp(l, h * r)
    V = _j(l, h * r) / r
    Vp = h * _jp(l, h * r) / r - _j(l, h * r) / r ** 2
    srr_p = (lam + 2 * mu) * Up + lam * (2 * U - L * V) / r
    t_p = mu * (Vp - V / r + U / r)
    # S solution
    U = L * _j(l, k * r) / r
    Up = L * (k * _jp(l, k * r) / r - _j(l, k * r) / r ** 2)
    V = _j(l, k * r) / r + k * _jp(l, k * r)
    Vp = k * _jp(l, k * r) / r - _j(l, k * r) / r ** 2 + k * k * _jpp(l, k * r)
    srr_s = (lam + 2 * mu) * Up + lam * (2 * U - L * V) / r
    t_s = mu * (Vp - V / r + U / r)
    return srr_p * t_s - srr_s * t_p


def _roots(f, wmax, step=4e-3, wmin=1e-2):
    w = np.arange(wmin, wmax, step)
    v = np.array([f(x) for x in w])
    out = []
    for i in np.nonzero(np.sign(v[1:]) * np.sign(v[:-1]) < 0)[0]:
        out.append(brentq(f, w[i], w[i + 1], xtol=1e-14))
    return out


def lamb_modes(wmax=6.0, a=1.0, vp=1.7, vs=1.0, lmax=8):
    """Sorted list of (omega, label, multiplicity 2l+1) below wmax."""
    modes = []
    for l in range(1, lmax + 1):
        # l = 1: the n = 0 toroidal branch is the rigid rotation (w = 0)
        base = 1 if l == 1 else 0
        for n, w in enumerate(_roots(lambda x: toroidal_fn(l, x, a, vs), wmax)):
            modes.append((w, f"{n + base}T{l}", 2 * l + 1))
    for n, w in enumerate(_roots(lambda x: radial_fn(x, a, vp, vs), wmax)):
        modes.append((w, f"{n}S0", 1))
    for l in range(1, lmax + 1):
        # l = 1: the n = 0 spheroidal branch is the rigid translation (w = 0)
        base = 1 if l == 1 else 0
        for n, w in enumerate(_roots(lambda x: spheroidal_fn(l, x, a, vp, vs), wmax)):
            modes.append((w, f"{n + base}S{l}", 2 * l + 1))
    return sorted(modes)
