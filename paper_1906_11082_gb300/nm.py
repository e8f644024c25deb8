"""Thin ctypes binding of libnm (include/nm.h): argument marshalling only.

Every computation runs inside libnm's CUDA kernels; this module converts
numpy host arrays and torch CUDA tensors into the plain pointers and sizes
of the C ABI and raises NMError on any non-zero status. There is no CPU
fallback: importing fails loudly when libnm.so cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnm.so")

NM_OK, NM_EINVAL, NM_ENOMEM, NM_ENOTCONV, NM_ECUDA, NM_ETIMEOUT, NM_EUNSUPPORTED = range(7)
NM_F64, NM_F32, NM_MIXED = 0, 1, 2
NM_UNIT_OMEGA, NM_UNIT_OMEGA2 = 0, 1
NM_RITZ_PENCIL, NM_RITZ_ROTATING = 0, 1
NM_GRAVITY, NM_CENTRIFUGAL, NM_SELF_GRAVITY = 1, 2, 4
NM_STATIC_SCRATCH_BYTES = 16 << 20     # size of the static scratch of nm_filter_apply_static

EXPORTS = (
    "nm_ctx_create", "nm_ctx_destroy", "nm_last_error", "nm_assemble", "nm_problem_free",
    "nm_problem_get_info", "nm_problem_unodes", "nm_problem_export", "nm_problem_gravity",
    "nm_apply_K", "nm_apply_M", "nm_solve_M", "nm_apply_R", "nm_set_interval",
    "nm_spectrum_bounds", "nm_filter_design", "nm_filter_apply", "nm_lanczos_slice", "nm_ritz",
    "nm_result_get_info", "nm_result_values", "nm_result_vectors", "nm_result_free",
    "nm_profile", "nm_profile_read", "nm_kernel_launches", "nm_set_option", "nm_autotune",
    "nm_lanczos_multi", "nm_filter_apply_static", "nm_lanczos_begin", "nm_lanczos_step",
    "nm_lanczos_get_info", "nm_lanczos_finish", "nm_lanczos_free", "nm_gemm_tn", "nm_gemm_nn",
    "nm_lanczos_add", "nm_lanczos_take",
)


class NMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnm error {code}: {msg}")
        self.code = code


class nm_mesh(C.Structure):
    _fields_ = [("nv", C.c_int64), ("xyz", C.POINTER(C.c_double)), ("nt", C.c_int64),
                ("tet", C.POINTER(C.c_int32)), ("region", C.POINTER(C.c_uint8))]


class nm_model(C.Structure):
    _fields_ = [("rho", C.POINTER(C.c_double)), ("lam", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("N2", C.POINTER(C.c_double)),
                ("gprime", C.POINTER(C.c_double)), ("G", C.c_double),
                ("Omega", C.c_double * 3), ("flags", C.c_uint32)]


class nm_problem_info(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("nv", "nt", "n_p2", "Nu", "n", "Np", "nnz_u", "nnz_p",
                                         "nnz_e", "n_fs", "n_charges")]


class nm_filter(C.Structure):
    _fields_ = [("degree", C.c_int32), ("gamma", C.POINTER(C.c_double)), ("c", C.c_double),
                ("e", C.c_double), ("k_M", C.c_int32), ("k_P", C.c_int32), ("m_lo", C.c_double),
                ("m_hi", C.c_double)]


class nm_slice_opts(C.Structure):
    _fields_ = [("block", C.c_int32), ("degree", C.c_int32), ("k_M", C.c_int32), ("k_P", C.c_int32),
                ("max_blocks", C.c_int32), ("check_every", C.c_int32), ("filter_prec", C.c_int32),
                ("tol", C.c_double), ("seed", C.c_uint64), ("start", C.c_void_p),
                ("bounds_steps", C.c_int32), ("log_every", C.c_int32)]


class nm_lanczos_info(C.Structure):
    _fields_ = [("blocks", C.c_int32), ("m", C.c_int32), ("active", C.c_int32), ("converged", C.c_int32),
                ("wanted", C.c_int32), ("ritz_converged", C.c_int32), ("seconds_filter", C.c_double)]


class nm_result_info(C.Structure):
    _fields_ = [("k", C.c_int64), ("n", C.c_int64), ("complex_vectors", C.c_int32),
                ("blocks", C.c_int32), ("m", C.c_int64), ("filter_applications", C.c_int64),
                ("lam_lo", C.c_double), ("lam_hi", C.c_double), ("seconds", C.c_double),
                ("seconds_filter", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libnm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "nm_ctx_create": [i32, C.POINTER(vp)],
        "nm_ctx_destroy": [vp],
        "nm_assemble": [vp, C.POINTER(nm_mesh), C.POINTER(nm_model), C.POINTER(vp)],
        "nm_problem_free": [vp],
        "nm_problem_get_info": [vp, C.POINTER(nm_problem_info)],
        "nm_problem_unodes": [vp, vp, vp, vp],
        "nm_problem_export": [vp, i32, C.POINTER(i64), C.POINTER(i64), vp, vp, vp],
        "nm_problem_gravity": [vp, vp],
        "nm_apply_K": [vp, vp, i64, vp, i64, i32, i32, i32, vp],
        "nm_apply_M": [vp, vp, i64, vp, i64, i32, i32, vp],
        "nm_apply_R": [vp, vp, i64, vp, i64, i32, i32, vp],
        "nm_solve_M": [vp, i32, dbl, dbl, vp, i64, vp, i64, i32, i32, vp],
        "nm_set_interval": [vp, dbl, dbl, i32],
        "nm_spectrum_bounds": [vp, i32, i32, C.c_uint64, C.POINTER(dbl), C.POINTER(dbl)],
        "nm_filter_design": [dbl, dbl, dbl, dbl, i32, vp, C.POINTER(dbl), C.POINTER(dbl)],
        "nm_filter_apply": [vp, C.POINTER(nm_filter), vp, i64, vp, i64, i32, i32, vp],
        "nm_lanczos_slice": [vp, C.POINTER(nm_slice_opts), C.POINTER(vp)],
        "nm_ritz": [vp, i32, vp, i64, i32, vp, C.POINTER(vp)],
        "nm_result_get_info": [vp, C.POINTER(nm_result_info)],
        "nm_result_values": [vp, vp, vp],
        "nm_result_vectors": [vp],
        "nm_result_free": [vp],
        "nm_profile": [vp, i32, i32],
        "nm_profile_read": [vp, i32, C.POINTER(i64), C.POINTER(dbl)],
        "nm_set_option": [vp, C.c_char_p, i64],
        "nm_autotune": [vp, i32, i32, i32, C.c_char_p, i32],
        "nm_lanczos_multi": [vp, C.POINTER(nm_slice_opts), i32, vp, vp, i32, vp],
        "nm_filter_apply_static": [vp, C.POINTER(nm_filter), vp, i64, vp, i64, i32, vp],
        "nm_lanczos_begin": [vp, C.POINTER(nm_slice_opts), i32, vp, vp, i32, C.POINTER(vp)],
        "nm_lanczos_step": [vp, C.POINTER(i32)],
        "nm_lanczos_get_info": [vp, i32, C.POINTER(nm_lanczos_info)],
        "nm_lanczos_finish": [vp, vp],
        "nm_lanczos_free": [vp],
        "nm_lanczos_add": [vp, dbl, dbl, i32, C.c_uint64, vp, C.POINTER(i32)],
        "nm_lanczos_take": [vp, i32, C.POINTER(vp)],
        "nm_gemm_tn": [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp],
        "nm_gemm_nn": [vp, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = vp if name == "nm_result_vectors" else i32
    lib.nm_kernel_launches.argtypes = []
    lib.nm_kernel_launches.restype = C.c_uint64
    lib.nm_last_error.argtypes = [vp]
    lib.nm_last_error.restype = C.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc, ctx=None):
    if rc != NM_OK:
        msg = _lib.nm_last_error(ctx)
        raise NMError(rc, msg.decode() if msg else "")


def _dptr(t):
    """Device pointer of a torch CUDA tensor (contiguous rows required)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _hp(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return NM_F64
    if t.dtype == torch.float32:
        return NM_F32
    raise TypeError("blocks must be float64 or float32")


def _ld(t, b):
    if t.dim() != 2 or t.stride(1) != 1 or t.shape[1] != b:
        raise ValueError("blocks must be 2-D row-major with unit column stride")
    return t.stride(0)


class Context:
    """An nm_ctx. Problems and results created under it are freed before it
    (the C ABI requires children to go first)."""

    def __init__(self, device=0):
        h = C.c_void_p()
        _check(_lib.nm_ctx_create(device, C.byref(h)))
        self.h = h
        self.device = device
        self._children = weakref.WeakSet()

    def _adopt(self, obj):
        self._children.add(obj)

    def gemm_tn(self, X, Y, C, alpha=1.0, beta=0.0, stream=None):
        """C (I x J, column-major: a torch tensor of shape (J, I)) = alpha X^T Y
        + beta C for row-major float64 device tensors X (K x I), Y (K x J)."""
        K, I = X.shape
        J = Y.shape[1]
        _check(_lib.nm_gemm_tn(self.h, I, J, K, alpha, _dptr(X), X.stride(0), _dptr(Y), Y.stride(0), beta, _dptr(C),
                               C.stride(0), _stream(stream)), self.h)

    def gemm_nn(self, X, Y, D, alpha=1.0, beta=0.0, stream=None):
        """D (I x J, row-major) = alpha X Y + beta D for row-major X (I x K) and
        column-major Y (K x J: a torch tensor of shape (J, K))."""
        I, K = X.shape
        J = Y.shape[0]
        _check(_lib.nm_gemm_nn(self.h, I, J, K, alpha, _dptr(X), X.stride(0), _dptr(Y), Y.stride(0), beta, _dptr(D),
                               D.stride(0), _stream(stream)), self.h)

    def close(self):
        if self.h:
            # runs before results before problems: a run borrows its problem
            order = {"LanczosRun": 0, "Result": 1}
            for ch in sorted(self._children, key=lambda o: order.get(type(o).__name__, 2)):
                ch.free()
            _lib.nm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h
        ctx._adopt(self)
        info = nm_result_info()
        _check(_lib.nm_result_get_info(h, C.byref(info)), ctx.h)
        self.info = {k: getattr(info, k) for k, _ in nm_result_info._fields_}
        k = info.k
        self.lam = np.zeros(k)
        self.resid = np.zeros(k)
        if k:
            _check(_lib.nm_result_values(h, _hp(self.lam, C.c_double), _hp(self.resid, C.c_double)), ctx.h)

    def vectors(self):
        """Copy of the eigenvector block (n x k) as a torch CUDA tensor."""
        import torch
        k, n = self.info["k"], self.info["n"]
        cplx = self.info["complex_vectors"]
        out = torch.empty((n, k), dtype=torch.complex128 if cplx else torch.float64,
                          device=f"cuda:{self.ctx.device}")
        if k:
            p = _lib.nm_result_vectors(self.h)
            torch.cuda.synchronize()
            _memcpy_d2d(out.data_ptr(), p, n * k * (16 if cplx else 8))
        return out

    def free(self):
        if self.h:
            if self.ctx.h:
                _lib.nm_result_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _memcpy_d2d(dst, src, nbytes):
    if _cudart is None:
        raise NMError(NM_ECUDA, "libcudart not found")
    rc = _cudart.cudaMemcpy(C.c_void_p(dst), C.c_void_p(src), C.c_size_t(nbytes), 3)
    if rc != 0:
        raise NMError(NM_ECUDA, f"cudaMemcpy failed ({rc})")


def _find_cudart():
    import glob
    for pat in ("/usr/local/cuda/lib64/libcudart.so*", "/usr/local/cuda/targets/*/lib/libcudart.so*"):
        for p in sorted(glob.glob(pat)):
            try:
                return C.CDLL(p)
            except OSError:
                continue
    try:
        return C.CDLL("libcudart.so")
    except OSError:
        return None


_cudart = _find_cudart()


class Problem:
    """An assembled pencil resident on the device (nm_assemble).

    self_gravity=True assembles the full operator K_eff - C^T S C (Sec. 5.2)
    instead of the Cowling approximation."""

    def __init__(self, ctx: Context, mesh, model, gprime=None, gravity=None, self_gravity=False):
        self.ctx = ctx
        self._keep = []
        xyz = np.ascontiguousarray(mesh.xyz, np.float64)
        tet = np.ascontiguousarray(mesh.tet, np.int32)
        reg = np.ascontiguousarray(mesh.region, np.uint8)
        m = nm_mesh(len(xyz), _hp(xyz, C.c_double), len(tet), _hp(tet, C.c_int32), _hp(reg, C.c_uint8))
        rho = np.ascontiguousarray(model.rho, np.float64)
        lam = np.ascontiguousarray(model.lam, np.float64)
        mu = np.ascontiguousarray(model.mu, np.float64)
        N2 = np.ascontiguousarray(model.N2, np.float64)
        gp = None if gprime is None else np.ascontiguousarray(gprime, np.float64).reshape(-1)
        if gravity is None:
            gravity = model.G != 0.0 or gprime is not None
        md = nm_model(_hp(rho, C.c_double), _hp(lam, C.c_double), _hp(mu, C.c_double), _hp(N2, C.c_double),
                      _hp(gp, C.c_double), float(model.G), (C.c_double * 3)(*[float(x) for x in model.Omega]),
                      (NM_GRAVITY if gravity else 0) | (NM_SELF_GRAVITY if self_gravity else 0))
        h = C.c_void_p()
        _check(_lib.nm_assemble(ctx.h, C.byref(m), C.byref(md), C.byref(h)), ctx.h)
        self.h = h
        ctx._adopt(self)
        info = nm_problem_info()
        _check(_lib.nm_problem_get_info(h, C.byref(info)), ctx.h)
        self.info = {k: getattr(info, k) for k, _ in nm_problem_info._fields_}
        self.n = self.info["n"]
        self.Nu = self.info["Nu"]
        self.Np = self.info["Np"]

    # -- maps and exports
    def unodes(self):
        canon = np.empty(self.Nu, np.int64)
        p2 = np.empty(self.Nu, np.int64)
        pc = np.empty(max(self.Np, 1), np.int64)
        _check(_lib.nm_problem_unodes(self.h, canon.ctypes.data_as(C.c_void_p), p2.ctypes.data_as(C.c_void_p),
                                      pc.ctypes.data_as(C.c_void_p)), self.ctx.h)
        return canon, p2, pc[:self.Np]

    def export(self, which):
        nr, nz = C.c_int64(), C.c_int64()
        _check(_lib.nm_problem_export(self.h, which, C.byref(nr), C.byref(nz), None, None, None), self.ctx.h)
        blk = {0: 9, 1: 1, 2: 1, 3: 3, 4: 3}[which]
        rp = np.empty(nr.value + 1, np.int64)
        col = np.empty(max(nz.value, 1), np.int32)
        val = np.empty(max(nz.value, 1) * blk, np.float64)
        _check(_lib.nm_problem_export(self.h, which, C.byref(nr), C.byref(nz), rp.ctypes.data_as(C.c_void_p),
                                      col.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p)), self.ctx.h)
        return rp, col[:nz.value], val[:nz.value * blk]

    def gravity(self):
        g = np.empty(3 * self.Nu)
        _check(_lib.nm_problem_gravity(self.h, g.ctypes.data_as(C.c_void_p)), self.ctx.h)
        return g.reshape(-1, 3)

    # -- operator pieces (torch CUDA tensors, row-major (rows x b))
    def apply_K(self, X, Y, k_P=0, stream=None, prec=None):
        b = X.shape[1]
        _check(_lib.nm_apply_K(self.h, _dptr(X), _ld(X, b), _dptr(Y), _ld(Y, b), b, k_P,
                               _prec_of(X) if prec is None else prec, _stream(stream)), self.ctx.h)

    def apply_M(self, X, Y, stream=None):
        b = X.shape[1]
        _check(_lib.nm_apply_M(self.h, _dptr(X), _ld(X, b), _dptr(Y), _ld(Y, b), b, _prec_of(X), _stream(stream)),
               self.ctx.h)

    def apply_R(self, X, Y, stream=None):
        b = X.shape[1]
        _check(_lib.nm_apply_R(self.h, _dptr(X), _ld(X, b), _dptr(Y), _ld(Y, b), b, _prec_of(X), _stream(stream)),
               self.ctx.h)

    def solve_M(self, W, X, k_M, m_lo=0.0, m_hi=0.0, stream=None, prec=None):
        b = W.shape[1]
        _check(_lib.nm_solve_M(self.h, k_M, m_lo, m_hi, _dptr(W), _ld(W, b), _dptr(X), _ld(X, b), b,
                               _prec_of(W) if prec is None else prec, _stream(stream)), self.ctx.h)

    def set_interval(self, lo, hi, unit=NM_UNIT_OMEGA):
        _check(_lib.nm_set_interval(self.h, lo, hi, unit), self.ctx.h)

    def spectrum_bounds(self, steps=40, k_M=57, seed=1):
        lo, hi = C.c_double(), C.c_double()
        _check(_lib.nm_spectrum_bounds(self.h, steps, k_M, seed, C.byref(lo), C.byref(hi)), self.ctx.h)
        return lo.value, hi.value

    def filter_apply(self, gamma, c, e, k_M, Y, Z, k_P=None, m_lo=0.0, m_hi=0.0, stream=None, prec=None):
        g = np.ascontiguousarray(gamma, np.float64)
        f = nm_filter(len(g) - 1, _hp(g, C.c_double), c, e, k_M, k_M if k_P is None else k_P, m_lo, m_hi)
        b = Y.shape[1]
        _check(_lib.nm_filter_apply(self.h, C.byref(f), _dptr(Y), _ld(Y, b), _dptr(Z), _ld(Z, b), b,
                                    _prec_of(Y) if prec is None else prec, _stream(stream)), self.ctx.h)

    def filter_apply_static(self, gamma, c, e, k_M, Y, Z, k_P=None, m_lo=0.0, m_hi=0.0, stream=None):
        """FP64 filter application with the library's fixed-size static
        scratch (no device allocation); Y, Z float64 device tensors."""
        g = np.ascontiguousarray(gamma, np.float64)
        f = nm_filter(len(g) - 1, _hp(g, C.c_double), c, e, k_M, k_M if k_P is None else k_P, m_lo, m_hi)
        b = Y.shape[1]
        _check(_lib.nm_filter_apply_static(self.h, C.byref(f), _dptr(Y), _ld(Y, b), _dptr(Z), _ld(Z, b), b,
                                           _stream(stream)), self.ctx.h)

    def lanczos_slice(self, block, degree, k_M=0, k_P=0, max_blocks=40, check_every=1, prec=NM_F64,
                      tol=1e-6, seed=1, start=None, bounds_steps=40, allow_unconverged=False, log_every=0):
        o = nm_slice_opts(block, degree, k_M, k_P, max_blocks, check_every, prec, tol, seed,
                          C.c_void_p(start.data_ptr()) if start is not None else None, bounds_steps, log_every)
        h = C.c_void_p()
        rc = _lib.nm_lanczos_slice(self.h, C.byref(o), C.byref(h))
        if rc != NM_OK and not (rc == NM_ENOTCONV and h.value and allow_unconverged):
            if h.value:
                _lib.nm_result_free(h)
            _check(rc, self.ctx.h)
        return Result(self.ctx, h)

    def lanczos_multi(self, slices, unit=NM_UNIT_OMEGA, block=16, degree=100, k_M=0, k_P=0, max_blocks=40,
                      check_every=1, prec=NM_F64, tol=1e-6, seed=1, bounds_steps=40, allow_unconverged=False,
                      log_every=0):
        """Solve several slices [(lo, hi), ...] in lockstep; returns a list of Results."""
        S = len(slices)
        lo = np.ascontiguousarray([s[0] for s in slices], np.float64)
        hi = np.ascontiguousarray([s[1] for s in slices], np.float64)
        o = nm_slice_opts(block, degree, k_M, k_P, max_blocks, check_every, prec, tol, seed, None, bounds_steps,
                          log_every)
        hs = (C.c_void_p * S)()
        rc = _lib.nm_lanczos_multi(self.h, C.byref(o), S, lo.ctypes.data_as(C.c_void_p),
                                   hi.ctypes.data_as(C.c_void_p), unit, C.cast(hs, C.c_void_p))
        res = [Result(self.ctx, C.c_void_p(h)) for h in hs if h]
        if rc != NM_OK and not (rc == NM_ENOTCONV and allow_unconverged and len(res) == S):
            for r in res:
                r.free()
            _check(rc, self.ctx.h)
        return res

    def lanczos_begin(self, slices=None, unit=NM_UNIT_OMEGA, block=16, degree=100, k_M=0, k_P=0, max_blocks=40,
                      check_every=1, prec=NM_F64, tol=1e-6, seed=1, start=None, bounds_steps=40, log_every=0):
        """Begin a resumable filtered block Lanczos run (nm_lanczos_begin):
        slices=None solves the interval of set_interval, else [(lo, hi), ...]."""
        o = nm_slice_opts(block, degree, k_M, k_P, max_blocks, check_every, prec, tol, seed,
                          C.c_void_p(start.data_ptr()) if start is not None else None, bounds_steps, log_every)
        if slices is None:
            S, lo, hi = 0, None, None
        else:
            S = len(slices)
            lo = np.ascontiguousarray([s[0] for s in slices], np.float64)
            hi = np.ascontiguousarray([s[1] for s in slices], np.float64)
        h = C.c_void_p()
        _check(_lib.nm_lanczos_begin(self.h, C.byref(o), S, lo.ctypes.data_as(C.c_void_p) if S else None,
                                     hi.ctypes.data_as(C.c_void_p) if S else None, unit, C.byref(h)), self.ctx.h)
        return LanczosRun(self, h, max(S, 1))

    def ritz(self, V, mode=NM_RITZ_PENCIL, lam_e=None):
        m = V.shape[1]
        le = None if lam_e is None else np.ascontiguousarray(lam_e, np.float64)
        h = C.c_void_p()
        _check(_lib.nm_ritz(self.h, mode, _dptr(V), V.stride(0), m,
                            le.ctypes.data_as(C.c_void_p) if le is not None else None, C.byref(h)), self.ctx.h)
        return Result(self.ctx, h)

    def set_option(self, key, value):
        _check(_lib.nm_set_option(self.h, key.encode(), int(value)), self.ctx.h)

    def autotune(self, b=32, prec=None, k_M=0):
        """Pick the fastest kernel variant for this problem; returns the report."""
        import json
        buf = C.create_string_buffer(16384)
        _check(_lib.nm_autotune(self.h, b, NM_MIXED if prec is None else prec, k_M, buf, len(buf)), self.ctx.h)
        return json.loads(buf.value.decode())

    def profile(self, enable=True, reset=True):
        _check(_lib.nm_profile(self.h, 1 if enable else 0, 1 if reset else 0), self.ctx.h)

    def profile_read(self, kind):
        """(launches, device milliseconds) of kernel kind 0 (mass steps) or 1 (K_eff)."""
        l, ms = C.c_int64(), C.c_double()
        _check(_lib.nm_profile_read(self.h, kind, C.byref(l), C.byref(ms)), self.ctx.h)
        return l.value, ms.value

    def free(self):
        if getattr(self, "h", None):
            if self.ctx.h:
                _lib.nm_problem_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class LanczosRun:
    """A resumable block Lanczos run (nm_lanczos_begin / step / add / take /
    finish). Slices are numbered in the order they were begun or added."""

    def __init__(self, prob, h, nslices):
        self.prob = prob
        self.h = h
        self.nslices = nslices
        prob.ctx._adopt(self)

    def step(self):
        """One block step; returns the number of slices still active."""
        a = C.c_int()
        _check(_lib.nm_lanczos_step(self.h, C.byref(a)), self.prob.ctx.h)
        return a.value

    def info(self, slice=0):
        st = nm_lanczos_info()
        _check(_lib.nm_lanczos_get_info(self.h, slice, C.byref(st)), self.prob.ctx.h)
        return {k: getattr(st, k) for k, _ in nm_lanczos_info._fields_}

    def add(self, lo, hi, unit=NM_UNIT_OMEGA, seed=1, start=None):
        """A slice joins the running batch; returns its slice number."""
        idx = C.c_int()
        _check(_lib.nm_lanczos_add(self.h, lo, hi, unit, seed, C.c_void_p(start.data_ptr()) if start is not None
                                   else None, C.byref(idx)), self.prob.ctx.h)
        self.nslices = max(self.nslices, idx.value + 1)
        return idx.value

    def take(self, slice, allow_unconverged=False):
        """The Result of one slice, which leaves the run."""
        h = C.c_void_p()
        rc = _lib.nm_lanczos_take(self.h, slice, C.byref(h))
        if rc != NM_OK and not (rc == NM_ENOTCONV and allow_unconverged and h.value):
            if h.value:
                _lib.nm_result_free(h)
            _check(rc, self.prob.ctx.h)
        return Result(self.prob.ctx, h)

    def finish(self, allow_unconverged=False):
        """Results of every slice not taken yet (list of Result, in slice
        order); frees the run."""
        hs = (C.c_void_p * self.nslices)()
        rc = _lib.nm_lanczos_finish(self.h, C.cast(hs, C.c_void_p))
        res = [Result(self.prob.ctx, C.c_void_p(h)) for h in hs if h]
        self.free()
        if rc != NM_OK and not (rc == NM_ENOTCONV and allow_unconverged):
            for r in res:
                r.free()
            _check(rc, self.prob.ctx.h)
        return res

    def free(self):
        if self.h:
            _lib.nm_lanczos_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kernel_launches():
    """Kernels libnm has launched in this process so far."""
    return int(_lib.nm_kernel_launches())


def filter_design(lam_lo, lam_hi, xi, eta, degree):
    g = np.empty(degree + 1)
    c, e = C.c_double(), C.c_double()
    _check(_lib.nm_filter_design(lam_lo, lam_hi, xi, eta, degree, g.ctypes.data_as(C.c_void_p),
                                 C.byref(c), C.byref(e)))
    return g, c.value, e.value
