"""Continuous-batching server for spectrum-slice requests on one GPU.

Requests (a mesh + model, a slice, solver options) arrive at any time. Each
mesh is served by an engine: a worker thread with its own libnm context
(CUDA stream, cuBLAS and cuSOLVER handles) holding the assembled problem
resident, and at most one running filtered-Lanczos batch (nm_lanczos_begin /
step / add / take). A request for a mesh joins its engine's running batch
at the next block step when the options agree (block width, filter degree,
inner steps, precision, limits) and the batch has room (64 columns); it
leaves the batch as soon as its slice converges, while the others keep
stepping. Requests that cannot join wait for the engine's next batch.
Engines of different meshes run concurrently, so their kernels overlap on
the device.

Admission is by device memory: the scheduler keeps a ledger of committed
bytes (resident problems with their filter scratch, and the Krylov bases
of admitted slices), reserved when a request is admitted and released when
its slice is taken or its problem evicted, and admits a request only when
it fits both the ledger (against the free memory at start, less a reserve)
and the device's current free memory. Problem sizes come from the
library's own counts (nm_problem_get_info) once a mesh has been assembled,
and from the mesh's tet count before. Idle engines are evicted least
recently used when memory is short. Every request records its arrival,
admission and completion times, from which the latency percentiles
follow.

The solves themselves are the library's; this module only schedules them.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Any, Callable, Optional

import numpy as np

from . import nm

# options that must agree for requests to share one batch
_BATCH_KEYS = ("block", "degree", "k_M", "k_P", "max_blocks", "check_every", "prec", "tol", "bounds_steps")
_MAX_COLS = 64


@dataclasses.dataclass
class Request:
    key: str                       # mesh identity (problems are cached by it)
    build: Callable[[], Any]       # returns (mesh, model) when the problem must be assembled
    interval: tuple                # (omega_lo, omega_hi)
    opts: dict                     # block, degree, k_M, k_P, max_blocks, check_every, prec, tol, seed
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    lam: Optional[np.ndarray] = None
    resid: Optional[np.ndarray] = None
    info: Optional[dict] = None
    error: Optional[str] = None
    done: threading.Event = dataclasses.field(default_factory=threading.Event)
    slot: int = -1                 # engine index that served it
    run_bytes: int = 0
    joined: bool = False           # joined a batch that was already running
    n_dof_hint: int = 0

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def _device_free_bytes(device):
    import torch
    free, _ = torch.cuda.mem_get_info(device)
    return free


def _batch_sig(opts):
    return tuple(opts.get(k) for k in _BATCH_KEYS)


def problem_bytes(info):
    """Device bytes of a resident problem from the library's counts: the
    FP64 matrices, their float and double-float copies, the reference field
    and the filter recurrence scratch of a full 64-column batch."""
    nnz_u, nnz_p, nnz_e = info["nnz_u"], info["nnz_p"], info["nnz_e"]
    n, Np, Nu = info["n"], info["Np"], info["Nu"]
    mats = nnz_u * (9 * 8 + 4 + 8 + 2 * 9 * 4 + 3 * 4) + nnz_p * (8 + 4 + 3 * 4) + 2 * nnz_e * (3 * 8 + 4)
    mats += 4 * (Nu + Np) * 8 + 3 * Nu * 8
    scratch = (n * _MAX_COLS) * (3 * 8 + 7 * 4) + Np * _MAX_COLS * 3 * 8
    return int(1.2 * (mats + scratch))


def slice_bytes(n, opts):
    """Device bytes of one slice in a batch: its Krylov basis, the block
    buffers, and the Rayleigh-Ritz products (K V, M V and the Ritz vectors)."""
    b = opts.get("block", 16)
    m = b * (opts.get("max_blocks", 40) + 1)
    return int(n * 8 * (m + 4 * b + 2 * m + m // 2))


class _Engine(threading.Thread):
    """One mesh: resident problem, at most one running batch."""

    def __init__(self, server, index, key):
        super().__init__(daemon=True, name=f"nm-engine-{index}")
        self.server = server
        self.index = index
        self.key = key
        self.queue = collections.deque()      # admitted requests not yet in a batch
        self.members = {}                     # slice number -> request of the running batch
        self.batch = None
        self.sig = None
        self.prob = None
        self.ctx = None
        self.info = None
        self.prob_bytes = 0                   # ledger entry of the resident problem
        self.last_used = time.perf_counter()
        self.max_batch = 0
        self._wake = threading.Event()
        self._halt = False

    # -- scheduler side (called under server._lock)
    def busy(self):
        return self.batch is not None or bool(self.queue) or bool(self.members)

    def post(self, req):
        self.queue.append(req)
        self.last_used = time.perf_counter()
        self._wake.set()

    def stop(self):
        self._halt = True
        self._wake.set()

    # -- engine thread
    def run(self):  # noqa: C901  (one loop: assemble, batch, step, take)
        import torch
        torch.cuda.set_device(self.server.device)
        self.ctx = nm.Context(self.server.device)
        while True:
            with self.server._lock:
                pending = list(self.queue)
                if self._halt and not pending and not self.members:
                    break
            if not pending and not self.members:
                self._wake.wait(0.05)
                self._wake.clear()
                continue
            try:
                self._ensure_problem(pending)
            except Exception as ex:  # the requests of this mesh fail, the server keeps serving
                self._fail_all(repr(ex))
                continue
            self._admit_pending()
            if not self.members:
                continue
            try:
                self.batch.step()
                self._take_finished()
            except Exception as ex:
                self._fail_members(repr(ex))
        self._release_problem()
        self.ctx.close()

    def _ensure_problem(self, pending):
        if self.prob is not None or not pending:
            return
        mesh, model = pending[0].build()
        self.prob = nm.Problem(self.ctx, mesh, model)
        self.info = dict(getattr(self.prob, "info", {}) or {})
        if self.info:
            with self.server._lock:
                exact = problem_bytes(self.info)
                self.server._known_sizes[self.key] = self.info
                self.prob_bytes = exact

    def _admit_pending(self):
        """Start a batch with the first queued request or let queued
        requests join the running one."""
        with self.server._lock:
            batch = []
            while self.queue:
                req = self.queue[0]
                b = req.opts.get("block", 16)
                if self.batch is None and not batch:
                    batch.append(self.queue.popleft())
                    continue
                sig = self.sig if self.batch is not None else _batch_sig(batch[0].opts)
                if _batch_sig(req.opts) != sig or (len(self.members) + len(batch) + 1) * b > _MAX_COLS:
                    break
                batch.append(self.queue.popleft())
        if not batch:
            return
        for req in batch:
            lo, hi = req.interval
            try:
                if self.batch is None:
                    o = {k: v for k, v in req.opts.items() if k not in ("seed",)}
                    self.batch = self.prob.lanczos_begin([(lo, hi)], seed=req.opts.get("seed", 1), **o)
                    self.sig = _batch_sig(req.opts)
                    q = 0
                else:
                    q = self.batch.add(lo, hi, seed=req.opts.get("seed", 1))
                    req.joined = True
                self.members[q] = req
                self.max_batch = max(self.max_batch, len(self.members))
            except Exception as ex:
                self._complete(req, error=repr(ex))

    def _take_finished(self):
        for q, req in list(self.members.items()):
            if self.batch.info(q)["active"]:
                continue
            del self.members[q]
            try:
                res = self.batch.take(q, allow_unconverged=True)
                self._complete(req, res=res)
            except Exception as ex:
                self._complete(req, error=repr(ex))
        if not self.members and self.batch is not None:
            self.batch.free()
            self.batch = None
            self.sig = None

    def _complete(self, req, res=None, error=None):
        if res is not None:
            req.lam, req.resid, req.info = res.lam.copy(), res.resid.copy(), dict(res.info)
            res.free()
        req.error = error
        req.t_done = time.perf_counter()
        with self.server._lock:
            self.server._slice_bytes -= req.run_bytes
            req.run_bytes = 0
        self.last_used = time.perf_counter()
        req.done.set()
        self.server._wake.set()

    def _fail_members(self, msg):
        for q, req in list(self.members.items()):
            del self.members[q]
            self._complete(req, error=msg)
        if self.batch is not None:
            try:
                self.batch.free()
            finally:
                self.batch = None
                self.sig = None

    def _fail_all(self, msg):
        with self.server._lock:
            pending = list(self.queue)
            self.queue.clear()
        for req in pending:
            self._complete(req, error=msg)
        self._fail_members(msg)
        self._release_problem()

    def _release_problem(self):
        if self.batch is not None:
            self.batch.free()
            self.batch = None
        if self.prob is not None:
            self.prob.free()
            self.prob = None
        with self.server._lock:
            self.prob_bytes = 0


class SliceServer:
    """Continuous batching over per-mesh engines, admission by device memory.

    slots: how many engines (meshes) may hold a resident problem at once;
    requests for a mesh without an engine wait for a free engine (idle
    engines are evicted least recently used)."""

    def __init__(self, slots=2, device=0, reserve_bytes=2 << 30):
        self.device = device
        self.reserve = reserve_bytes
        self.max_engines = slots
        self._budget = _device_free_bytes(device) - reserve_bytes
        self._slice_bytes = 0
        self._known_sizes = {}
        self.pending = collections.deque()
        self.all = []
        self.engines = {}          # key -> _Engine
        self._retired = []
        self._next_index = 0
        self._lock = threading.RLock()
        self._wake = threading.Event()
        self._stop = False
        self._sched = threading.Thread(target=self._loop, daemon=True, name="nm-scheduler")
        self._sched.start()

    # -- memory estimates (overridable)
    def estimate_bytes(self, req, resident):
        """(problem bytes, slice bytes) of a request: the problem's share is
        0 when its mesh is resident already."""
        info = self._known_sizes.get(req.key)
        if info is None:
            tets = max(int(req.n_dof_hint), 1)
            info = {"nnz_u": 40 * tets, "nnz_p": 12 * tets, "nnz_e": 10 * tets, "n": 5 * tets, "Np": tets,
                    "Nu": 2 * tets}
        prob = 0 if resident else problem_bytes(info)
        return prob, slice_bytes(info["n"], req.opts)

    def submit(self, req: Request, n_dof_hint: int):
        """Queue a request; n_dof_hint is the mesh's tet count (used until
        the mesh has been assembled once)."""
        req.t_arrival = time.perf_counter()
        req.n_dof_hint = n_dof_hint
        with self._lock:
            self.pending.append(req)
            self.all.append(req)
        self._wake.set()
        return req

    def _committed(self):
        return self._slice_bytes + sum(e.prob_bytes for e in self.engines.values())

    def _fits(self, need):
        return (self._committed() + need <= self._budget and
                need <= _device_free_bytes(self.device) - self.reserve)

    def _evict_idle(self, keep):
        """Retire the least recently used idle engine (not `keep`)."""
        idle = [e for k, e in self.engines.items() if k != keep and not e.busy()]
        if not idle:
            return False
        e = min(idle, key=lambda x: x.last_used)
        del self.engines[e.key]
        e.stop()
        self._retired.append(e)
        # the ledger drops its problem now; the device's free memory, also
        # checked at admission, follows once the engine has freed it
        e.prob_bytes = 0
        return True

    def _loop(self):
        while not self._stop:
            self._wake.wait(0.05)
            self._wake.clear()
            with self._lock:
                while self.pending:
                    req = self.pending[0]
                    eng = self.engines.get(req.key)
                    resident = eng is not None
                    prob, run = self.estimate_bytes(req, resident)
                    if eng is None and len(self.engines) >= self.max_engines:
                        if not self._evict_idle(keep=req.key):
                            break          # every engine busy: wait (FIFO)
                    while not self._fits(prob + run) and self._evict_idle(keep=req.key):
                        pass
                    if not self._fits(prob + run) and (self._slice_bytes > 0 or
                                                        any(e.busy() for e in self.engines.values())):
                        break              # wait for memory to be released by running slices
                    self.pending.popleft()
                    if eng is None:
                        eng = _Engine(self, self._next_index, req.key)
                        self._next_index += 1
                        eng.prob_bytes = prob
                        self.engines[req.key] = eng
                        eng.start()
                    self._slice_bytes += run
                    req.run_bytes = run
                    req.t_admit = time.perf_counter()
                    req.slot = eng.index
                    eng.post(req)

    def drain(self, timeout=None):
        for r in list(self.all):
            r.done.wait(timeout)

    def close(self):
        self.drain()
        self._stop = True
        self._wake.set()
        self._sched.join()
        with self._lock:
            engines = list(self.engines.values()) + self._retired
            self.engines.clear()
        for e in engines:
            e.stop()
        for e in engines:
            e.join()

    def stats(self):
        done = [r for r in self.all if r.done.is_set() and r.error is None]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        pairs = sum(int(np.sum(r.resid <= 1e-6)) for r in done if r.resid is not None)
        t0 = min(r.t_arrival for r in self.all) if self.all else 0.0
        t1 = max(r.t_done for r in done) if done else 0.0
        engines = list(self.engines.values()) + self._retired
        return {"requests": len(self.all), "completed": len(done),
                "errors": sum(1 for r in self.all if r.error is not None),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "eigenpairs": pairs, "eigenpairs_per_s": pairs / max(t1 - t0, 1e-9),
                "overlap_max": self.max_overlap(),
                "joined_running_batch": sum(1 for r in self.all if r.joined),
                "max_batch": max([e.max_batch for e in engines], default=0),
                "engines": len(engines)}

    def max_overlap(self):
        """Largest number of requests that were running at the same time."""
        ev = []
        for r in self.all:
            if r.t_admit and r.t_done:
                ev.append((r.t_admit, 1))
                ev.append((r.t_done, -1))
        cur = best = 0
        for _, d in sorted(ev):
            cur += d
            best = max(best, cur)
        return best
