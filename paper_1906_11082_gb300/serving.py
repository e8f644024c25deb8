"""Continuous-batching server for spectrum-slice requests on one GPU.

Requests (a mesh + model, a slice, solver options) arrive at any time. A
scheduler admits them FIFO as soon as a worker slot is idle and the
request's estimated device memory fits the free HBM; admitted requests run
concurrently, each slot on its own libnm context (own CUDA stream, cuBLAS
and cuSOLVER handles), so their kernels overlap on the device while later
arrivals wait. Assembled problems stay resident in the slot that built them
and are reused by later requests for the same mesh; the least recently used
ones are freed when memory is short. Every request records its arrival,
admission and completion times, from which the latency percentiles follow.

The solves themselves are the library's (nm_lanczos_slice); this module only
schedules them.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time
from typing import Any, Callable, Optional

import numpy as np

from . import nm


@dataclasses.dataclass
class Request:
    key: str                       # mesh identity (problems are cached by it)
    build: Callable[[], Any]       # returns (mesh, model) when the problem must be assembled
    interval: tuple                # (omega_lo, omega_hi)
    opts: dict                     # keyword arguments of Problem.lanczos_slice
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    lam: Optional[np.ndarray] = None
    resid: Optional[np.ndarray] = None
    info: Optional[dict] = None
    error: Optional[str] = None
    done: threading.Event = dataclasses.field(default_factory=threading.Event)
    slot: int = -1
    run_bytes: int = 0

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def _device_free_bytes(device):
    import torch
    free, _ = torch.cuda.mem_get_info(device)
    return free


class _Slot(threading.Thread):
    def __init__(self, server, index):
        super().__init__(daemon=True, name=f"nm-slot-{index}")
        self.server = server
        self.index = index
        self.inbox = queue.Queue()
        self.problems = collections.OrderedDict()   # key -> Problem (LRU)
        self.prob_bytes = {}                         # key -> bytes reserved for the resident problem
        self.ctx = None
        self.busy = False

    def run(self):
        import torch
        torch.cuda.set_device(self.server.device)
        self.ctx = nm.Context(self.server.device)
        while True:
            req = self.inbox.get()
            if req is None:
                break
            try:
                P = self.problems.get(req.key)
                if P is None:
                    mesh, model = req.build()
                    P = nm.Problem(self.ctx, mesh, model)
                    self.problems[req.key] = P
                self.problems.move_to_end(req.key)
                P.set_interval(*req.interval)
                res = P.lanczos_slice(allow_unconverged=True, **req.opts)
                req.lam, req.resid, req.info = res.lam.copy(), res.resid.copy(), dict(res.info)
                res.free()
            except Exception as ex:  # reported on the request, the slot keeps serving
                req.error = repr(ex)
            req.t_done = time.perf_counter()
            with self.server._lock:
                self.server._running_bytes -= req.run_bytes
            self.busy = False
            req.done.set()
            self.server._wake.set()
        for P in self.problems.values():
            P.free()
        self.ctx.close()

    def evict_one(self):
        """Free the least recently used resident problem of an idle slot."""
        if self.problems and not self.busy:
            key, P = self.problems.popitem(last=False)
            self.prob_bytes.pop(key, None)
            P.free()
            return True
        return False


class SliceServer:
    """FIFO admission by free slot and free HBM; concurrent execution.

    Admission keeps a ledger of committed bytes (the estimates of running
    solves and of resident problems), reserved when a request is admitted
    and released when it completes or its problem is evicted: a slot
    allocates only after admission, so the device's free memory alone would
    let several requests in on the same bytes. A request is admitted when
    it fits both the ledger (against the free memory at start, less the
    reserve) and the device's current free memory."""

    def __init__(self, slots=2, device=0, reserve_bytes=2 << 30):
        self.device = device
        self.reserve = reserve_bytes
        self._budget = _device_free_bytes(device) - reserve_bytes
        self._running_bytes = 0
        self.pending = collections.deque()
        self.all = []
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._stop = False
        self.slots = [_Slot(self, i) for i in range(slots)]
        for s in self.slots:
            s.start()
        self._sched = threading.Thread(target=self._loop, daemon=True, name="nm-scheduler")
        self._sched.start()

    @staticmethod
    def estimate_bytes(n_dof, opts, resident=False):
        """Device memory a request needs beyond a resident problem (basis,
        Rayleigh-Ritz products, filter scratch), plus the problem itself
        when it is not resident yet (about 80 B per dof for the matrices)."""
        b = opts.get("block", 16)
        m = b * (opts.get("max_blocks", 40) + 1)
        need = n_dof * 8 * (m + 2 * m + 8 * b)
        if not resident:
            need += 80 * n_dof * 30
        return need

    def submit(self, req: Request, n_dof_hint: int):
        req.t_arrival = time.perf_counter()
        req.n_dof_hint = n_dof_hint
        with self._lock:
            self.pending.append(req)
            self.all.append(req)
        self._wake.set()
        return req

    def _loop(self):
        while not self._stop:
            self._wake.wait(0.05)
            self._wake.clear()
            with self._lock:
                while self.pending:
                    req = self.pending[0]
                    idle = [s for s in self.slots if not s.busy]
                    if not idle:
                        break
                    # prefer an idle slot that already holds the problem
                    slot = next((s for s in idle if req.key in s.problems), idle[0])
                    resident = req.key in slot.problems
                    run = self.estimate_bytes(req.n_dof_hint, req.opts, True)
                    prob = 0 if resident else self.estimate_bytes(req.n_dof_hint, req.opts, False) - run
                    need = run + prob
                    while not self._fits(need) and any(s.evict_one() for s in self.slots if s is not slot or
                                                      not resident):
                        pass
                    if not self._fits(need) and any(s.busy for s in self.slots):
                        break        # wait for memory to be released by a running request
                    self.pending.popleft()
                    self._running_bytes += run
                    req.run_bytes = run
                    if prob:
                        slot.prob_bytes[req.key] = prob
                    req.t_admit = time.perf_counter()
                    req.slot = slot.index
                    slot.busy = True
                    slot.inbox.put(req)

    def _committed(self):
        return self._running_bytes + sum(sum(s.prob_bytes.values()) for s in self.slots)

    def _fits(self, need):
        return (self._committed() + need <= self._budget and
                need <= _device_free_bytes(self.device) - self.reserve)

    def drain(self, timeout=None):
        for r in list(self.all):
            r.done.wait(timeout)

    def close(self):
        self.drain()
        self._stop = True
        self._wake.set()
        self._sched.join()
        for s in self.slots:
            s.inbox.put(None)
        for s in self.slots:
            s.join()

    def stats(self):
        done = [r for r in self.all if r.done.is_set() and r.error is None]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        pairs = sum(int(np.sum(r.resid <= 1e-6)) for r in done if r.resid is not None)
        t0 = min(r.t_arrival for r in self.all) if self.all else 0.0
        t1 = max(r.t_done for r in done) if done else 0.0
        return {"requests": len(self.all), "completed": len(done),
                "errors": sum(1 for r in self.all if r.error is not None),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "eigenpairs": pairs, "eigenpairs_per_s": pairs / max(t1 - t0, 1e-9),
                "overlap_max": self.max_overlap()}

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
