"""Host logic of the continuous-batching server on CPU, with the library
replaced by a fake: FIFO admission by free device memory, one engine per
mesh with its problem resident, requests joining a running batch at a step
boundary, concurrent engines, least-recently-used eviction of idle engines,
errors reported per request with their reserved memory released, and the
latency statistics."""
import threading
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

GB = 1 << 30


class _Mem:
    """Device memory model: resident problems and slices in batches use it."""
    def __init__(self, total):
        self.total = total
        self.used = 0
        self.lock = threading.Lock()
        self.slices = 0
        self.peak_slices = 0
        self.runs = 0
        self.peak_runs = 0

    def free(self, device=0):
        with self.lock:
            return self.total - self.used


def _fake_nm(mem, prob_bytes, run_bytes, step_s, steps_needed=3):
    class Result:
        def __init__(self, n):
            self.lam = np.linspace(1.0, 2.0, n)
            self.resid = np.full(n, 1e-9)
            self.info = {"blocks": steps_needed}

        def free(self):
            pass

    class Run:
        def __init__(self, n_eigs):
            self.left = {}
            self.n = {}
            with mem.lock:
                mem.runs += 1
                mem.peak_runs = max(mem.peak_runs, mem.runs)
            self._add(n_eigs)

        def _add(self, n_eigs):
            q = len(self.left)
            self.left[q] = steps_needed
            self.n[q] = n_eigs
            with mem.lock:
                mem.used += run_bytes
                mem.slices += 1
                mem.peak_slices = max(mem.peak_slices, mem.slices)
            return q

        def add(self, lo, hi, seed=1, start=None):
            return self._add(4)

        def step(self):
            time.sleep(step_s)
            for q in self.left:
                if self.left[q] > 0:
                    self.left[q] -= 1
            return sum(1 for v in self.left.values() if v > 0)

        def info(self, q):
            return {"active": int(self.left[q] > 0), "blocks": steps_needed - self.left[q]}

        def take(self, q, allow_unconverged=False):
            self.left[q] = -1
            with mem.lock:
                mem.used -= run_bytes
                mem.slices -= 1
            return Result(self.n[q])

        def free(self):
            with mem.lock:
                mem.runs -= 1

    class Problem:
        def __init__(self, ctx, mesh, model):
            if getattr(model, "fail", False):
                raise RuntimeError("synthetic failure")
            with mem.lock:
                mem.used += prob_bytes
            self.alive = True
            self.info = {}

        def lanczos_begin(self, slices, seed=1, **opts):
            return Run(opts.get("n_eigs", 4))

        def free(self):
            if self.alive:
                with mem.lock:
                    mem.used -= prob_bytes
                self.alive = False

    class Context:
        def __init__(self, device):
            self.device = device

        def close(self):
            pass

    return types.SimpleNamespace(Context=Context, Problem=Problem)


@pytest.fixture
def server_factory(monkeypatch):
    from paper_1906_11082_gb300 import serving
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)

    def make(mem, slots, prob_bytes, run_bytes, step_s, reserve=0, steps_needed=3):
        monkeypatch.setattr(serving, "nm", _fake_nm(mem, prob_bytes, run_bytes, step_s, steps_needed))
        monkeypatch.setattr(serving, "_device_free_bytes", mem.free)
        monkeypatch.setattr(serving.SliceServer, "estimate_bytes",
                            lambda self, req, resident: (0 if resident else prob_bytes, run_bytes))
        return serving.SliceServer(slots=slots, device=0, reserve_bytes=reserve)
    return make


def _req(serving, key, fail=False, n=4, block=16):
    model = types.SimpleNamespace(fail=fail)
    return serving.Request(key=key, build=lambda: (None, model), interval=(1.0, 2.0),
                           opts={"n_eigs": n, "block": block, "degree": 10})


def test_concurrent_engines_and_stats(server_factory):
    from paper_1906_11082_gb300 import serving
    mem = _Mem(100 * GB)
    srv = server_factory(mem, slots=3, prob_bytes=GB, run_bytes=GB, step_s=0.05)
    reqs = [srv.submit(_req(serving, f"m{i % 3}"), 1000) for i in range(6)]
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["errors"] == 0
    assert mem.peak_runs == 3 and st["engines"] == 3       # one batch per mesh, all at once
    assert st["eigenpairs"] == 24 and st["overlap_max"] >= 3
    lat = sorted(r.latency for r in reqs)
    assert st["p50_s"] == pytest.approx(float(np.percentile(lat, 50)))
    assert st["p99_s"] == pytest.approx(float(np.percentile(lat, 99)))
    assert all(r.t_arrival <= r.t_admit <= r.t_done for r in reqs)
    assert mem.used == 0


def test_requests_join_a_running_batch(server_factory):
    """A request for a mesh whose batch is running joins it at the next
    step boundary (continuous batching) instead of waiting for it to end;
    one with other options waits for the next batch."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(100 * GB)
    srv = server_factory(mem, slots=2, prob_bytes=GB, run_bytes=GB, step_s=0.1, steps_needed=5)
    first = srv.submit(_req(serving, "planet"), 1000)
    time.sleep(0.25)                        # the first batch is stepping
    second = srv.submit(_req(serving, "planet"), 1000)
    other = srv.submit(_req(serving, "planet", block=8), 1000)
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 3 and st["errors"] == 0
    assert second.joined and not first.joined and not other.joined
    assert st["max_batch"] == 2 and st["joined_running_batch"] == 1
    assert second.t_done < other.t_admit + 0.45 + 5 * 0.1    # did not wait for a batch of its own
    assert other.t_done > first.t_done                      # incompatible options: next batch
    assert mem.used == 0


def test_admission_waits_for_memory_and_keeps_fifo(server_factory):
    """Room for one slice only: requests run one at a time, in arrival
    order, although engines are free."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(3 * GB)
    srv = server_factory(mem, slots=3, prob_bytes=GB, run_bytes=GB, step_s=0.05)
    reqs = [srv.submit(_req(serving, f"k{i}"), 1000) for i in range(4)]
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 4 and st["errors"] == 0
    assert mem.peak_slices == 1
    admits = [r.t_admit for r in reqs]
    assert admits == sorted(admits)                       # FIFO
    assert mem.used == 0


def test_eviction_frees_least_recently_used(server_factory):
    """Distinct meshes with room for one engine: each new mesh evicts the
    previous idle engine instead of failing."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(int(2.5 * GB))
    srv = server_factory(mem, slots=1, prob_bytes=GB, run_bytes=GB // 4, step_s=0.02)
    for i in range(4):
        srv.submit(_req(serving, f"mesh{i}"), 1000)
        srv.drain(timeout=30)
    st = srv.stats()
    live = len(srv.engines)
    srv.close()
    assert st["completed"] == 4 and st["errors"] == 0
    assert live == 1 and st["engines"] == 4
    assert mem.used == 0


def test_failing_request_is_reported_and_ledger_released(server_factory):
    """A mesh whose assembly raises: its request fails with the message,
    the bytes reserved for it return to the ledger, and other meshes are
    served."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(100 * GB)
    srv = server_factory(mem, slots=2, prob_bytes=GB, run_bytes=GB, step_s=0.02)
    before = srv._committed()
    bad = srv.submit(_req(serving, "bad", fail=True), 1000)
    good = srv.submit(_req(serving, "good"), 1000)
    srv.drain(timeout=30)
    st = srv.stats()
    time.sleep(0.2)
    after_slices = srv._slice_bytes
    bad_engine = srv.engines.get("bad")
    srv.close()
    assert bad.error and "synthetic failure" in bad.error
    assert good.error is None and len(good.lam) == 4
    assert st["completed"] == 1 and st["errors"] == 1
    assert after_slices == 0 and before == 0
    assert bad_engine is None or bad_engine.prob_bytes == 0
