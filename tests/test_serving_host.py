"""Host logic of the serving runtime on CPU, with the library replaced by a
fake: FIFO admission by free slot and free device memory, concurrent slots,
least-recently-used eviction of resident problems when memory is short,
errors reported per request, and the latency statistics."""
import threading
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

GB = 1 << 30


class _Mem:
    """Device memory model: resident problems and running solves use it."""
    def __init__(self, total):
        self.total = total
        self.used = 0
        self.lock = threading.Lock()
        self.running = 0
        self.peak_running = 0

    def free(self, device=0):
        with self.lock:
            return self.total - self.used


def _fake_nm(mem, prob_bytes, run_bytes, solve_s):
    class Result:
        def __init__(self, n):
            self.lam = np.linspace(1.0, 2.0, n)
            self.resid = np.full(n, 1e-9)
            self.info = {"blocks": 3}

        def free(self):
            pass

    class Problem:
        def __init__(self, ctx, mesh, model):
            self.fail = getattr(model, "fail", False)
            with mem.lock:
                mem.used += prob_bytes
            self.alive = True

        def set_interval(self, lo, hi):
            self.iv = (lo, hi)

        def lanczos_slice(self, allow_unconverged=True, **opts):
            if self.fail:
                raise RuntimeError("synthetic failure")
            with mem.lock:
                mem.used += run_bytes
                mem.running += 1
                mem.peak_running = max(mem.peak_running, mem.running)
            time.sleep(solve_s)
            with mem.lock:
                mem.used -= run_bytes
                mem.running -= 1
            return Result(opts.get("n_eigs", 4))

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

    def make(mem, slots, prob_bytes, run_bytes, solve_s, reserve=0):
        monkeypatch.setattr(serving, "nm", _fake_nm(mem, prob_bytes, run_bytes, solve_s))
        monkeypatch.setattr(serving, "_device_free_bytes", mem.free)
        monkeypatch.setattr(serving.SliceServer, "estimate_bytes",
                            staticmethod(lambda n, opts, resident=False: run_bytes + (0 if resident else prob_bytes)))
        return serving.SliceServer(slots=slots, device=0, reserve_bytes=reserve)
    return make


def _req(serving, key, fail=False, n=4):
    model = types.SimpleNamespace(fail=fail)
    return serving.Request(key=key, build=lambda: (None, model), interval=(1.0, 2.0), opts={"n_eigs": n})


def test_concurrent_slots_and_stats(server_factory):
    from paper_1906_11082_gb300 import serving
    mem = _Mem(100 * GB)
    srv = server_factory(mem, slots=3, prob_bytes=GB, run_bytes=GB, solve_s=0.2)
    reqs = [srv.submit(_req(serving, f"m{i % 2}"), 1000) for i in range(6)]
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["errors"] == 0
    assert st["overlap_max"] == 3 and mem.peak_running == 3     # never more than the slots
    assert st["eigenpairs"] == 24
    lat = sorted(r.latency for r in reqs)
    assert st["p50_s"] == pytest.approx(float(np.percentile(lat, 50)))
    assert st["p99_s"] == pytest.approx(float(np.percentile(lat, 99)))
    assert all(r.t_arrival <= r.t_admit <= r.t_done for r in reqs)


def test_admission_waits_for_memory_and_keeps_fifo(server_factory):
    """Room for one running solve only: requests run one at a time, in
    arrival order, although three slots are idle."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(3 * GB)
    srv = server_factory(mem, slots=3, prob_bytes=GB, run_bytes=GB, solve_s=0.15)
    reqs = [srv.submit(_req(serving, f"k{i}"), 1000) for i in range(4)]
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 4 and st["errors"] == 0
    assert mem.peak_running == 1
    admits = [r.t_admit for r in reqs]
    assert admits == sorted(admits)                       # FIFO
    assert mem.used <= 3 * GB


def test_eviction_frees_least_recently_used(server_factory):
    """Distinct meshes on one slot with room for one resident problem:
    each new mesh evicts the previous one instead of failing."""
    from paper_1906_11082_gb300 import serving
    mem = _Mem(int(2.5 * GB))
    srv = server_factory(mem, slots=1, prob_bytes=GB, run_bytes=GB // 4, solve_s=0.05)
    for i in range(4):
        srv.submit(_req(serving, f"mesh{i}"), 1000)
        srv.drain(timeout=30)
    st = srv.stats()
    resident = len(srv.slots[0].problems)
    srv.close()
    assert st["completed"] == 4 and st["errors"] == 0
    assert resident <= 2


def test_failing_request_is_reported_and_slot_survives(server_factory):
    from paper_1906_11082_gb300 import serving
    mem = _Mem(100 * GB)
    srv = server_factory(mem, slots=1, prob_bytes=GB, run_bytes=GB, solve_s=0.05)
    bad = srv.submit(_req(serving, "bad", fail=True), 1000)
    good = srv.submit(_req(serving, "good"), 1000)
    srv.drain(timeout=30)
    st = srv.stats()
    srv.close()
    assert bad.error and "synthetic failure" in bad.error
    assert good.error is None and len(good.lam) == 4
    assert st["completed"] == 1 and st["errors"] == 1
