"""Host part of the library's self-gravitation term (no GPU): the charge
points, their inverse self distances and the charge matrix C that libnm
builds at assembly (nm::self_gravity_host, selfgrav.cu) equal the oracle's
(oracle/selfgrav.py) on the homogeneous ball and on the layered planet with
its fluid-solid and density-jump faces. The two sides share no code: the
library integrates the self distances in its own polar closed form, the
oracle by the closed forms of the triangle and segment potentials.

The library's builder is a C++ function; a small harness, compiled here
against libnm.so, passes it the oracle's P2 numbering (it takes any
numbering) and returns flat arrays. Points are matched by position (the two
sides order the charged faces differently)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sps

from oracle import fem, selfgrav
from synth.model import homogeneous_ball, layered_planet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdint>
#include <cstring>
#include <vector>
namespace nm {
void self_gravity_host(const double* xyz, const int32_t* tet, const int64_t* tet10, const uint8_t* region,
                       const double* rho, int64_t nt, const int32_t* usol, const int32_t* uflu,
                       std::vector<double>& pts, std::vector<double>& invR, std::vector<int64_t>& erow,
                       std::vector<int32_t>& ecol, std::vector<double>& eval);
}
static std::vector<double> P, R, V;
static std::vector<int64_t> ER;
static std::vector<int32_t> EC;
extern "C" void sg_run(const double* xyz, const int32_t* tet, const int64_t* tet10, const uint8_t* region,
                       const double* rho, int64_t nt, const int32_t* usol, const int32_t* uflu, int64_t* sizes) {
    nm::self_gravity_host(xyz, tet, tet10, region, rho, nt, usol, uflu, P, R, ER, EC, V);
    sizes[0] = (int64_t)R.size();
    sizes[1] = (int64_t)V.size();
}
extern "C" void sg_get(double* p, double* r, int64_t* er, int32_t* ec, double* v) {
    std::memcpy(p, P.data(), P.size() * sizeof(double));
    std::memcpy(r, R.data(), R.size() * sizeof(double));
    std::memcpy(er, ER.data(), ER.size() * sizeof(int64_t));
    std::memcpy(ec, EC.data(), EC.size() * sizeof(int32_t));
    std::memcpy(v, V.data(), V.size() * sizeof(double));
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_1906_11082_gb300 import _build
    _build.build()
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("sg_harness")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    libdir = os.path.join(ROOT, "paper_1906_11082_gb300")
    out = d / "libsgharness.so"
    subprocess.run([gxx, "-O2", "-shared", "-fPIC", "-o", str(out), str(src), "-L", libdir, "-lnm",
                    "-Wl,-rpath," + libdir], check=True)
    return C.CDLL(str(out))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _library_charges(lib, mesh, model):
    xyz = np.ascontiguousarray(mesh.xyz, np.float64)
    tet = np.ascontiguousarray(mesh.tet, np.int32)
    reg = np.ascontiguousarray(mesh.region, np.uint8)
    rho = np.ascontiguousarray(model.rho, np.float64)
    dm = fem.dof_map(mesh.tet, mesh.region, len(xyz))
    t10 = np.ascontiguousarray(dm.tet10, np.int64)
    us = np.ascontiguousarray(dm.unode_solid, np.int32)
    uf = np.ascontiguousarray(dm.unode_fluid, np.int32)
    sizes = np.zeros(2, np.int64)
    lib.sg_run(_ptr(xyz), _ptr(tet), _ptr(t10), _ptr(reg), _ptr(rho), C.c_int64(len(tet)), _ptr(us), _ptr(uf),
               _ptr(sizes))
    npt, ne = int(sizes[0]), int(sizes[1])
    p, r = np.zeros(3 * npt), np.zeros(npt)
    er, ec, v = np.zeros(ne, np.int64), np.zeros(ne, np.int32), np.zeros(ne)
    lib.sg_get(_ptr(p), _ptr(r), _ptr(er), _ptr(ec), _ptr(v))
    Cm = sps.coo_matrix((v, (er, ec)), shape=(npt, 3 * dm.Nu)).tocsr()
    return p.reshape(-1, 3), r, Cm


@pytest.mark.parametrize("which", ["ball", "planet"])
def test_library_charges_match_oracle(harness, which):
    mesh, model = homogeneous_ball(h=0.45, seed=1) if which == "ball" else layered_planet(h=0.25, seed=7)
    pg, rg, Cg = _library_charges(harness, mesh, model)
    po, ro, Co = selfgrav.charges(mesh, model)
    assert len(rg) == len(ro) > mesh.nt
    kg = np.lexsort(np.round(pg, 12).T)
    ko = np.lexsort(np.round(po, 12).T)
    assert np.abs(pg[kg] - po[ko]).max() <= 1e-14
    assert np.abs(rg[kg] / ro[ko] - 1.0).max() <= 1e-12
    diff = (Cg[kg] - Co[ko]).tocsr()
    assert abs(diff).max() <= 1e-14 * abs(Co).max()
