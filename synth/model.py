"""Seeded synthetic planet models and workloads (inputs only).

Everything here is an *input* to the eigensolver: per-tet material
constants sampled at the tet centroid (the paper assigns element-wise
constants rho_k, c_k, kappa_k, N_k^2, Appendix A.1), the gravitational
constant, the rotation vector, and seeded random start blocks. No step of
the method (shape functions, integrals, operators, filters) lives here.

Units are nondimensional: radius a = 1, mean density 1, and G = 1/pi, so
the time unit is (pi G rho_mean)^(-1/2) = 1. Earth's rotation rate
7.2921e-5 rad/s in this unit (rho_mean = 5515 kg/m^3) is 0.06781.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .mesh import Mesh, layered_ball

G_NONDIM = 1.0 / np.pi
OMEGA_EARTH_NONDIM = 7.2921e-5 / np.sqrt(np.pi * 6.674e-11 * 5515.0)

SOLID, FLUID = 0, 1


@dataclasses.dataclass
class Model:
    rho: np.ndarray    # (nt,) density
    lam: np.ndarray    # (nt,) Lame lambda (fluid: kappa)
    mu: np.ndarray     # (nt,) shear modulus (0 in fluid)
    N2: np.ndarray     # (nt,) squared buoyancy frequency (used in fluid only)
    G: float           # gravitational constant (0: no reference gravity)
    Omega: np.ndarray  # (3,) rotation vector


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    model: Model
    interval: tuple    # (omega_lo, omega_hi), angular frequency
    degree: int        # Chebyshev filter degree
    block: int         # Lanczos block width
    nev: int           # eigenpairs expected in the slice (approximate)


def centroids(mesh: Mesh):
    return mesh.xyz[mesh.tet].mean(axis=1)


def homogeneous_ball(h=0.45, seed=1, rho=1.0, vp=1.7, vs=1.0):
    """Homogeneous non-rotating elastic unit ball without gravity."""
    mesh = layered_ball(radii=(1.0,), h=h, seed=seed)
    nt = mesh.nt
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return mesh, Model(rho=np.full(nt, rho), lam=np.full(nt, lam), mu=np.full(nt, mu),
                       N2=np.zeros(nt), G=0.0, Omega=np.zeros(3))


# Base three-layer profiles (inner core / fluid outer core / mantle), cubic in
# r per layer: value = c0 + c1 x + c2 x^2 + c3 x^3 with x = r / r_top. Shapes
# loosely follow a terrestrial planet scaled to mean density 1 and the
# nondimensional velocity unit (radius / time unit).
_RADII3 = (0.19, 0.55, 1.0)
_BASE = {
    # layer: (rho, vp, vs)
    0: ((2.42, 0.0, -0.10, 0.0), (1.63, 0.0, -0.04, 0.0), (0.53, 0.0, -0.03, 0.0)),
    1: ((2.30, -0.10, -0.35, 0.0), (1.51, 0.10, -0.45, 0.0), (0.0, 0.0, 0.0, 0.0)),
    2: ((1.00, 0.20, -0.55, 0.0), (2.00, 0.40, -1.20, 0.0), (1.07, 0.20, -0.62, 0.0)),
}


def layered_planet(h=0.05, seed=2, perturb=0.02, n2_level=4e-3, omega=0.0,
                   lateral=0.0, lateral_lmax=20):
    """Solid inner core / fluid outer core / solid mantle.

    perturb: relative seeded perturbation of the profile coefficients.
    n2_level: scale of the seeded, smooth, non-negative N^2 in the fluid
    (near-adiabatic core; the essential spectrum then sits in [0, n2_level]).
    omega: rotation rate about z. lateral: relative amplitude of a seeded
    spherical-harmonic perturbation (degree <= lateral_lmax) of rho, vp, vs
    in the solid layers only.
    """
    rng = np.random.default_rng(seed)
    mesh = layered_ball(radii=_RADII3, h=h, fluid_layers=(1,), seed=seed)
    c = centroids(mesh)
    r = np.linalg.norm(c, axis=1)
    nt = mesh.nt
    rho = np.empty(nt)
    vp = np.empty(nt)
    vs = np.empty(nt)
    for lay, (crho, cvp, cvs) in _BASE.items():
        sel = mesh.layer == lay
        x = r[sel] / _RADII3[lay]
        for out, coef in ((rho, crho), (vp, cvp), (vs, cvs)):
            cc = np.asarray(coef) * (1.0 + perturb * rng.uniform(-1, 1, 4))
            out[sel] = cc[0] + cc[1] * x + cc[2] * x ** 2 + cc[3] * x ** 3
    fluid = mesh.region == FLUID
    vs[fluid] = 0.0
    if lateral > 0.0:
        dl = _sh_field(c, lateral_lmax, rng)
        solid = ~fluid
        for arr in (rho, vp, vs):
            eps = lateral * rng.uniform(0.2, 1.0)
            arr[solid] *= 1.0 + eps * dl[solid]
    # rescale density to mean 1 over the meshed volume
    v = mesh.xyz[mesh.tet]
    vol = np.einsum('ij,ij->i', np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                    v[:, 3] - v[:, 0]) / 6.0
    rho *= vol.sum() / (rho * vol).sum()
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    # smooth seeded N^2 >= 0 in the fluid only
    ph = rng.uniform(0, 2 * np.pi, 2)
    xf = (r - _RADII3[0]) / (_RADII3[1] - _RADII3[0])
    N2 = np.where(fluid, n2_level * (0.6 + 0.4 * np.sin(2 * np.pi * xf + ph[0])
                                     * np.cos(np.pi * xf + ph[1])), 0.0)
    return mesh, Model(rho=rho, lam=lam, mu=mu, N2=N2, G=G_NONDIM,
                       Omega=np.array([0.0, 0.0, omega]))


def _sh_field(c, lmax, rng):
    """Seeded real spherical-harmonic field, degree 1..lmax, max |value| ~ 1."""
    from scipy.special import sph_harm_y
    r = np.linalg.norm(c, axis=1)
    th = np.arccos(np.clip(c[:, 2] / np.maximum(r, 1e-300), -1, 1))
    ph = np.arctan2(c[:, 1], c[:, 0])
    f = np.zeros(len(c))
    for l in range(1, lmax + 1):
        for m in range(0, l + 1):
            y = sph_harm_y(l, m, th, ph)
            a, b = rng.normal(size=2) / (l + 1)
            f += a * y.real + (b * y.imag if m > 0 else 0.0)
    return f / np.abs(f).max()


def start_block(n, b, seed):
    """Seeded Gaussian start block, row-major (n, b) float64."""
    return np.random.default_rng(seed).standard_normal((n, b))


def config_ball():
    """Homogeneous ball, ~400 tets, P2, all eigenpairs with omega in [0, 3]."""
    mesh, model = homogeneous_ball(h=0.45, seed=1)
    return Workload("ball-400tet", mesh, model, (0.0, 3.0), degree=100, block=8, nev=16)


def config_layered(h=0.05, omega=0.0, seed=2):
    """Three-layer planet, ~2.6e5 tets at h = 0.05 (about 1.1M dof)."""
    mesh, model = layered_planet(h=h, seed=seed, omega=omega)
    return Workload(f"layered-planet-h{h}", mesh, model, None, degree=100, block=32,
                    nev=100)
