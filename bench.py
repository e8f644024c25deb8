"""Benchmark: eigenpairs/s of a filtered-Lanczos spectrum-slice sweep on GB300.

Workload (default): the three-layer planet (solid inner core, fluid outer
core, solid mantle; seeded smooth profiles; reference gravity by direct
summation; Cowling operator), P2 on 263,760 tets (1.15M dof), slices of
the low-frequency spectrum above the fluid band, block width 32, filter
degree 600 (the configured degree 100 cannot keep the fluid core's
essential spectrum near lambda = 0 out of the slice on this mesh).

A step is ONE BLOCK STEP of a continuous sweep over adjacent slices
(nm_lanczos_step): the degree-600 filter of the current 32-vector block
(K_eff SpMMs and inner mass / pressure solves), two-pass CGS and
Cholesky-QR in the M inner product, the projected matrix and, every
second block, the convergence test; the step in which a slice converges
also runs its FP64 Rayleigh-Ritz and residuals, and the next slice of the
sweep begins in the following step. Matrices are resident; assembly and
the spectrum bounds of P_M K_eff (shared by every slice of the problem)
run before the timed region. The timed region starts on a fresh slice.
value = eigenpairs with residual <= 1e-6 accepted during the timed steps,
summed over ranks, divided by the max-over-ranks timed seconds.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|f64|f32]
       [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s per slice"
UNIT = "eigenpairs/s"

# Adjacent slices (angular frequency) of the layered-planet workload. A
# rank sweeps its own slices in order: r, r + N, r + 2N, ... (mod the list).
# The first slice holds 90 eigenpairs above the fluid band; later slices
# continue upward.
SLICES_OMEGA = [(4.0, 6.5), (6.5, 7.6), (7.6, 8.4), (8.4, 9.0), (9.0, 9.6), (9.6, 10.1), (10.1, 10.5),
                (10.5, 10.9)]
H_MESH = 0.05
# The configured degree is 100; on this mesh (lambda_max ~ 3.4e5) a
# degree-100 filter passes the fluid core's ~8e4-dimensional essential
# spectrum near lambda = 0 as strongly as the slice. Degree 600 holds it
# below 0.7% of the slice's filter value.
DEGREE_CONFIG = 100
DEGREE = 600
BLOCK = 32
# Inner Chebyshev steps per solve. Mixed form: 18 converges the benchmark
# slice in 18 blocks with residuals <= 2.0e-7; 17 reaches 5.9e-7, too close
# to the 1e-6 gate; 16 stalls (residual 3.3 at the 24-block limit). The
# serving leg's meshes and slices keep the measured 20.
K_INNER = {"f64": 38, "mixed": 18, "f32": 28}
K_SERVING = 20
SEED = 11

# Serving leg: layered planets of three sizes with the spectrum upper bound
# the library's bounds estimate gives on each (lambda_max sets the filter
# degree), and three slices of width 1.5 in omega. Near the bottom of the
# spectrum a slice of width dw spans dw sqrt(2/e) in Chebyshev angle
# (e = lambda_max / 2), so the degree is 1.7 pi sqrt(lambda_max) / (2 dw),
# the ratio the benchmark slice runs at. Requests arrive as a seeded
# Poisson stream.
SERVING_MESHES = [(0.25, 58954.0), (0.15, 45045.0), (0.1, 85700.0)]
SERVING_SLICES = [(4.0, 5.5), (4.5, 6.0), (3.5, 5.0)]

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the
# float mass-step kernel (kron_v4_kernel<3, 1, 32>) on this workload (same
# matrices, b = 32; mean of two launches), captured with
#   ncu --kernel-name-base demangled --metrics gpu__time_duration.sum,\
#       dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k 'regex:kron_v4_kernel<\(int\)3' -s 4 -c 2 --csv \
#       python bench.py --profile-case filter
# and the SHA-256 of kernels.cu when it was taken: once the kernel source
# changes the figure no longer describes it and the bench reports traffic
# null.
TRAFFIC_CAPTURE = {"kernel": "kron_v4_kernel<3, 1, 32>", "bytes": 543_591_808 + 121_877_248,
                   "kernels_cu_sha256": "2d86c3f12eacd75a3d36d4645078875c2e42d76cb1c6fc99cd683f8038ef0bf0"}

# FP64 peak of GB300 (NVIDIA's published B300 figure, 1.25 TFLOP/s; equal to
# 152 SMs x ~2.05 GHz x 2 FP64 FMA per SM per clock x 2 flop).
FP64_PEAK_TFLOPS = 1.25


def serving_degree(lam_max, lo, hi):
    return int(np.ceil(1.7 * np.pi * np.sqrt(lam_max) / (2.0 * (hi - lo))))


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prec", choices=("mixed", "f64", "f32"), default="mixed")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--h", type=float, default=H_MESH)
    ap.add_argument("--max-blocks", type=int, default=24)
    ap.add_argument("--degree", type=int, default=DEGREE)
    ap.add_argument("--k-m", type=int, default=0)
    ap.add_argument("--profile-case", nargs="?", const="filter", choices=("filter", "gemm", "selfgrav"),
                    default=None,
                    help="a short case for ncu captures: 'filter' = two mixed filter applications of degree 10 "
                         "on the full matrices; 'gemm' = the tensor-core dense products of a 576-column basis "
                         "on 200,003 rows; 'selfgrav' = K_eff products with and without the self-gravitation "
                         "term on a planet of --sg-h (timed, one JSON line)")
    ap.add_argument("--sg-h", type=float, default=0.15, help="mesh size of the 'selfgrav' profile case")
    ap.add_argument("--rotating", action="store_true",
                    help="instead of the bench line: the rotating layered planet (Omega of the Earth), "
                         "ROTATING_SLICES solved as one batched run (b = 16 each, one 64-column "
                         "recurrence, mixed filter), then the rotating projection of all their Ritz "
                         "vectors (eq. sublinear0); one JSON line")
    ap.add_argument("--rot-h", type=float, default=0.1, help="mesh size of the --rotating run")
    ap.add_argument("--rot-degree", type=int, default=800, help="filter degree of the --rotating run")
    ap.add_argument("--heterogeneous", action="store_true",
                    help="instead of the bench line: the rotating planet with a seeded spherical-harmonic "
                         "perturbation (degree 20, 3%% in the solid layers) and HETERO_SLICES, 16 adjacent "
                         "slices solved as one batched run (b = 4 each, one 64-column recurrence), then the "
                         "rotating projection of all their Ritz vectors; one JSON line")
    ap.add_argument("--het-degree", type=int, default=3000, help="filter degree of the --heterogeneous run")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="problem option (nm_set_option), repeatable")
    ap.add_argument("--chunk", type=int, default=None,
                    help="chunked row schedule of the semi-iteration SpMMs (threads per CTA; 0 = off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f64-leg", action="store_true")
    ap.add_argument("--f64-steps", type=int, default=2)
    ap.add_argument("--cpu-workers", type=int, default=0, help="0: all host cores (up to the block width)")
    return ap.parse_args(argv)


def rank_slice(rank):
    """The first slice rank r solves: the units (slices) are sharded over
    ranks, so the data path needs no collective."""
    return SLICES_OMEGA[rank % len(SLICES_OMEGA)]


def rank_sweep(rank, world, count):
    """The first `count` slices of rank r's sweep: r, r + N, r + 2N, ..."""
    return [SLICES_OMEGA[(rank + i * world) % len(SLICES_OMEGA)] for i in range(count)]


def reduce_over_ranks(t_ms, pairs, world, device):
    """Whole-job figures: the max over ranks of the timed region and the
    sum over ranks of converged eigenpairs (one all-reduce each, after the
    timed region)."""
    if world <= 1:
        return float(t_ms), int(pairs)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pp = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(pp, op=dist.ReduceOp.SUM)
    return float(tt.item()), int(pp.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.out = ""

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm_, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def kernels_sha256():
    with open(os.path.join(ROOT, "paper_1906_11082_gb300", "csrc", "kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def mass_step_bytes(info, b, s):
    """Algorithmic bytes of one mass-solve step launch (read M_rho, gather
    x_k once, read x_{k-1} and the right-hand side, write x_{k+1})."""
    nnz, Nu, n = info["nnz_u"], info["Nu"], info["n"]
    return nnz * (s + 4) + 4 * (Nu + 1) + s * Nu + 4 * n * b * s


def mass_step_flops(info, b):
    return 2 * info["nnz_u"] * 3 * b + 6 * info["n"] * b


def workload(h):
    from synth.model import config_layered
    return config_layered(h=h)


# ------------------------------------------------------------------ CPU legs
# The oracle as it stands, on a bounded sample: one filter degree (K_eff +
# inner mass solve) for the 32 vectors of a block on the octant x, y, z > 0
# of the mesh, scaled to the full mesh by stored blocks. All cores: the 32
# columns are split over worker processes (the operator acts on each column
# on its own), each worker assembling the octant itself; one core: one
# worker with all 32 columns. Workers are started with `spawn` and run with
# one BLAS / OpenMP thread each, so `cores` is the number of processes.

def _octant_operator(h, prec, k_M):
    import copy
    from synth.mesh import Mesh
    from oracle import fem, filtlan
    w = workload(h)
    m = w.mesh
    c = m.xyz[m.tet].mean(axis=1)
    sel = np.nonzero((c > 0).all(axis=1))[0]
    sub = Mesh(xyz=m.xyz, tet=m.tet[sel], region=m.region[sel], layer=m.layer[sel], radii=m.radii)
    mdl = copy.copy(w.model)
    for k in ("rho", "lam", "mu", "N2"):
        setattr(mdl, k, getattr(w.model, k)[sel])
    S = fem.assemble(sub, mdl)
    op = filtlan.Operator(S, k_M=k_M, k_P=k_M, refine=(prec == "mixed"))
    return op, S, len(sel)


def _cpu_worker(conn, h, prec, k_M, c0, c1):
    try:
        op, S, nt = _octant_operator(h, prec, k_M)
        Y = np.ascontiguousarray(np.random.default_rng(0).standard_normal((S.n, BLOCK))[:, c0:c1])
        if prec == "f32":
            Y = Y.astype(np.float32)
        conn.send(("ready", S.n, nt, S.A_G.nnz / 9))
        while True:
            msg = conn.recv()
            if msg == "stop":
                break
            t0 = time.time()
            op.B(Y)
            conn.send((t0, time.time()))
    except Exception as ex:  # reported to the parent, which raises
        conn.send(("error", repr(ex)))
    finally:
        conn.close()


class CpuPool:
    """`workers` spawned oracle processes holding the octant operator, each
    with its share of the block's columns."""

    def __init__(self, h, prec, k_M, workers):
        ctx = mp.get_context("spawn")
        env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env_keep:
            os.environ[k] = "1"
        self.procs, self.conns = [], []
        try:
            cuts = np.linspace(0, BLOCK, workers + 1).round().astype(int)
            for i in range(workers):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_cpu_worker, args=(b, h, prec, k_M, int(cuts[i]), int(cuts[i + 1])),
                                daemon=True)
                p.start()
                self.procs.append(p)
                self.conns.append(a)
        finally:
            for k, v in env_keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.info = None
        for c in self.conns:
            r = c.recv()
            if r[0] != "ready":
                self.close()
                raise RuntimeError(f"oracle worker failed: {r[1]}")
            self.info = r[1:]
        self.workers = workers

    def degree(self):
        """Wall seconds of one filter degree with every worker on its columns."""
        for c in self.conns:
            c.send("go")
        spans = [c.recv() for c in self.conns]
        for s in spans:
            if s[0] == "error":
                raise RuntimeError(f"oracle worker failed: {s[1]}")
        return max(s[1] for s in spans) - min(s[0] for s in spans)

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except (OSError, BrokenPipeError):
                pass
        for p in self.procs:
            p.join(timeout=30)


def cpu_workers(requested):
    n = os.cpu_count() or 1
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    return max(1, min(requested or n, BLOCK))


def _graph_blocks(mesh):
    from oracle import fem
    dm = fem.dof_map(mesh.tet, mesh.region, mesh.nv)
    un = dm.elem_unodes(np.asarray(mesh.region))
    a = np.repeat(un, 10, axis=1).ravel()
    b = np.tile(un, (1, 10)).ravel()
    key = np.unique(a.astype(np.int64) * dm.Nu + b)
    return len(key)


def cpu_baseline(h, prec, k_M, pairs, blocks, degree, blocks_full, workers, reps=2):
    """The oracle's eigenpairs/s on all cores and on one core, scaled from
    one timed filter degree on the octant sample to the benchmark slice."""
    out = {}
    for label, nw in (("all", workers), ("one", 1)):
        pool = CpuPool(h, prec, k_M, nw)
        try:
            pool.degree()   # warm
            t = min(pool.degree() for _ in range(reps))
        finally:
            pool.close()
        n_sub, nt_sub, blocks_sub = pool.info
        t_deg = t * blocks_full / blocks_sub
        out[label] = {"value": pairs / (t_deg * degree * blocks), "cores": nw, "sample_degree_s": t,
                      "full_degree_s": t_deg, "sample_tets": int(nt_sub), "sample_dof": int(n_sub)}
    a, o = out["all"], out["one"]
    sample = (f"one filter degree (K_eff + {k_M}-step inner solves, {'refined ' if prec == 'mixed' else ''}"
              f"FP64) on {BLOCK} vectors over the octant x,y,z>0 ({a['sample_tets']} tets, {a['sample_dof']} "
              f"dof; {a['sample_degree_s']:.2f} s on {a['cores']} processes, {o['sample_degree_s']:.2f} s on "
              f"one), scaled by stored blocks to the full mesh and by degree {degree} x {blocks} Lanczos "
              f"blocks to the {pairs}-pair slice")
    return {"value": a["value"], "unit": UNIT, "cores": a["cores"], "kind": "oracle", "sample": sample,
            "one_core": {"value": o["value"], "unit": UNIT, "cores": 1},
            "nproc": os.cpu_count()}


# Pairs and blocks of the benchmark slice (4.0, 6.5) as the mixed-form
# sweep converges it (90 eigenpairs with residual <= 1e-6 in 18 blocks of
# 32); the reference arm scales its timed oracle degree by these.
SLICE_PAIRS = 90
SLICE_BLOCKS = 18


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    k_M = args.k_m or K_INNER[args.prec]
    w = workload(args.h)
    blocks_full = _graph_blocks(w.mesh)
    workers = cpu_workers(args.cpu_workers)
    pool = CpuPool(args.h, args.prec, k_M, workers)
    try:
        for _ in range(args.warmup):
            pool.degree()
        times = [pool.degree() for _ in range(args.steps)]
    finally:
        pool.close()
    n_sub, nt_sub, blocks_sub = pool.info
    t_step = float(np.mean(times))
    t_deg = t_step * blocks_full / blocks_sub
    value = SLICE_PAIRS / (t_deg * args.degree * SLICE_BLOCKS)
    sample = (f"each step: one filter degree (K_eff + {k_M}-step inner solves) on {BLOCK} vectors over the "
              f"octant x,y,z>0 ({nt_sub} tets, {n_sub} dof) on {workers} oracle processes; value scales the "
              f"mean step by stored blocks to the full mesh and by degree {args.degree} x {SLICE_BLOCKS} blocks "
              f"to the {SLICE_PAIRS}-pair benchmark slice")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "tets": int(w.mesh.nt), "degree": args.degree, "block": BLOCK},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
class Sweep:
    """A continuous sweep over a rank's slices, one block step per call."""

    def __init__(self, P, slices, opts):
        self.P = P
        self.slices = slices
        self.opts = opts
        self.i = 0
        self.run = None
        self.done = []   # (slice, pairs passing 1e-6, blocks, max resid)

    def _begin(self):
        self.run = self.P.lanczos_begin([self.slices[self.i % len(self.slices)]], **self.opts)

    def step(self):
        if self.run is None:
            self._begin()
        if self.run.step() == 0:
            info = self.run.info(0)
            res = self.run.finish(allow_unconverged=True)[0]
            good = int(np.sum(res.resid <= 1e-6))
            self.done.append((self.slices[self.i % len(self.slices)], good, int(info["blocks"]),
                              float(res.resid.max()) if len(res.lam) else 0.0))
            res.free()
            self.run = None
            self.i += 1
            return good
        return 0

    def close(self):
        if self.run is not None:
            self.run.free()
            self.run = None


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_11082_gb300 import nm

    if args.profile_case == "gemm":
        gemm_case(nm, local)
        return
    if args.profile_case == "selfgrav":
        selfgrav_case(nm, local, args.sg_h)
        return
    if args.rotating:
        rotating_case(nm, local, args.rot_h, args.rot_degree)
        return
    if args.heterogeneous:
        rotating_case(nm, local, args.rot_h, args.het_degree, b=4, slices=HETERO_SLICES, lateral=0.03)
        return
    w = workload(args.h)
    ctx = nm.Context(local)
    torch.cuda.synchronize()
    t_asm = time.perf_counter()
    P = nm.Problem(ctx, w.mesh, w.model)
    t_asm = time.perf_counter() - t_asm
    if args.chunk is not None:
        P.set_option("chunk", args.chunk)
    for kv in args.option:
        key, val = kv.split("=", 1)
        P.set_option(key, int(val))
    prec = {"f64": nm.NM_F64, "f32": nm.NM_F32, "mixed": nm.NM_MIXED}[args.prec]
    k_M = args.k_m or K_INNER[args.prec]
    opts = dict(block=BLOCK, degree=args.degree, k_M=k_M, k_P=k_M, max_blocks=args.max_blocks, check_every=2,
                prec=prec, seed=SEED + rank)
    lo, hi = rank_slice(rank)
    P.set_interval(lo, hi)
    if args.profile_case:
        lo_b, hi_b = P.spectrum_bounds(steps=40, k_M=k_M)
        g, c, e = nm.filter_design(lo_b, hi_b, lo * lo, hi * hi, 10)
        Y = torch.randn((P.n, BLOCK), dtype=torch.float64, device="cuda")
        Z = torch.empty_like(Y)
        P.filter_apply(g, c, e, k_M, Y, Z, prec=nm.NM_MIXED)
        torch.cuda.synchronize()
        P.filter_apply(g, c, e, k_M, Y, Z, prec=nm.NM_MIXED)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "mixed filter, degree 10, b = 32", "n": P.n}))
        return

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # Warm-up: W block steps of the rank's first slice (this also computes
    # the spectrum bounds the problem keeps for every later slice); the run
    # is then dropped, so the timed sweep starts on a fresh slice.
    warm = P.lanczos_begin([rank_slice(rank)], **opts)
    for _ in range(args.warmup):
        warm.step()
    warm.free()

    P.profile(True, reset=True)
    sweep = Sweep(P, rank_sweep(rank, world, len(SLICES_OMEGA)), opts)
    lat = []
    pairs = 0
    barrier()
    launches0 = nm.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            t = time.perf_counter()
            pairs += sweep.step()
            lat.append(time.perf_counter() - t)
        ev1.record()
        barrier()
    launches = nm.kernel_launches() - launches0
    t_ms = ev0.elapsed_time(ev1)
    partial = sweep.run.info(0) if sweep.run is not None else None
    sweep.close()
    ml, mms = P.profile_read(0)
    kl, kms = P.profile_read(1)
    # the dominant kernel's own launches: the float M_rho semi-iteration
    # steps (kind 2) in the mixed form, the mass-step launches (kind 0) else
    dl, dms = P.profile_read(2) if args.prec == "mixed" else (ml, mms)
    P.profile(False, reset=True)
    t_ms, tot_pairs = reduce_over_ranks(t_ms, pairs, world, "cuda")
    value = tot_pairs / (t_ms / 1e3)
    done = sweep.done
    if rank != 0:
        return
    info = P.info
    first = done[0] if done else None
    slice_pairs = first[1] if first else 0
    slice_blocks = first[2] if first else 0

    # end to end through the public API: one full slice solve of the first
    # slice (nm_lanczos_slice) with its start block copied from pinned host
    # memory and eigenvalues, residuals and eigenvectors copied back
    e2e = None
    if not args.no_e2e:
        host_start = torch.from_numpy(np.random.default_rng(SEED).standard_normal((P.n, BLOCK))).pin_memory()
        dev_start = torch.empty((P.n, BLOCK), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dev_start.copy_(host_start, non_blocking=True)
        torch.cuda.synchronize()
        r = P.lanczos_slice(**dict(opts, start=dev_start), allow_unconverged=True)
        X = r.vectors()
        host_out = torch.empty(X.shape, dtype=X.dtype).pin_memory()
        host_out.copy_(X)
        torch.cuda.synchronize()
        lam = r.lam.copy()
        e2e_pairs = int(np.sum(r.resid <= 1e-6))
        dt = time.perf_counter() - t0
        e2e = {"value": e2e_pairs / dt, "unit": UNIT, "h2d_bytes_per_step": int(host_start.numel() * 8),
               "d2h_bytes_per_step": int(X.numel() * 8 + 2 * lam.size * 8), "steps": 1,
               "step": "one nm_lanczos_slice call on the first slice (host start block in, eigenpairs out)",
               "eigenpairs": e2e_pairs, "seconds": dt}
        r.free()
        del X, dev_start

    # the plain FP64 form on the same slice: block steps of its own run
    # (FP64 filter, k = 38 inner steps), timed with CUDA events, after one
    # untimed step (its spectrum bounds and start)
    f64 = None
    if not args.no_f64_leg and args.prec != "f64" and args.f64_steps > 0:
        k64 = K_INNER["f64"]
        run = P.lanczos_begin([rank_slice(rank)], **dict(opts, prec=nm.NM_F64, k_M=k64, k_P=k64))
        run.step()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(args.f64_steps):
            run.step()
        a1.record()
        torch.cuda.synchronize()
        run.free()
        ms64 = a0.elapsed_time(a1) / args.f64_steps
        ms_mixed = t_ms / args.steps
        f64 = {"ms_per_block_step": ms64, "steps_timed": args.f64_steps, "k_inner": k64,
               "mixed_ms_per_block_step": ms_mixed,
               "speedup_mixed_over_f64": ms64 / ms_mixed}
        if slice_blocks:
            f64["eigenpairs_per_s_at_same_blocks"] = slice_pairs / (ms64 / 1e3 * slice_blocks)

    s = 8 if args.prec == "f64" else 4   # the dominant mass-step kernel's value size
    peak_hbm, peak_src = peaks()
    # average duration of one launch of the dominant kernel, from CUDA
    # events around its back-to-back launches on the problem's stream
    # during the timed steps
    avg_launch_s = (dms / 1e3) / max(dl, 1)
    mbytes = mass_step_bytes(info, BLOCK, s)
    mflops = mass_step_flops(info, BLOCK)
    gbs = mbytes / avg_launch_s / 1e9 if dl else None
    tfl = mflops / avg_launch_s / 1e12 if dl else None
    traffic = None
    if (s == 4 and args.h == H_MESH and TRAFFIC_CAPTURE["kernels_cu_sha256"] == kernels_sha256()):
        traffic = TRAFFIC_CAPTURE["bytes"]
    if args.prec == "f64" and tfl is not None and tfl / FP64_PEAK_TFLOPS > gbs / peak_hbm:
        roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "kron_warp_kernel<double, 3, 1, 1>",
                "peak_source": "GB300 FP64 nominal (152 SM x 2 FMA/clk x 2.05 GHz)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": (gbs / peak_hbm) if gbs else None, "traffic": traffic,
                "kernel": "kron_warp_kernel<double, 3, 1, 1>" if s == 8 else TRAFFIC_CAPTURE["kernel"],
                "peak_source": f"{peak_src} copy bandwidth"}
    roof["bytes_per_launch"] = mbytes
    roof["flops_per_launch"] = mflops
    roof["avg_launch_us"] = avg_launch_s * 1e6
    roof["launches"] = dl
    filt_ms = mms + kms
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f64+f32", "f64": "f64", "f32": "f32+f64"}[args.prec], "data": "synthetic",
            "config": {"workload": w.name, "tets": int(w.mesh.nt), "dof": int(info["n"]),
                       "pressure_dof": int(info["Np"]), "degree": args.degree, "degree_config": DEGREE_CONFIG,
                       "block": BLOCK, "k_inner": k_M, "filter_prec": args.prec,
                       "step": "one block step of a slice sweep (filter, CGS2, Cholesky-QR; Rayleigh-Ritz "
                               "in the step a slice converges)",
                       "sweep_omega": rank_sweep(rank, world, max(len(done) + 1, 1)),
                       "parallelism": f"slices x{world}",
                       "l2": "inputs larger than L2 (A_G %.2f GB resident)" % (info["nnz_u"] * 76 / 1e9),
                       "untimed_prologue": "assembly (%.1f s) and the spectrum bounds shared by every slice"
                                           % t_asm},
            "slices_completed": [{"omega": list(sl), "eigenpairs": g, "blocks": bk, "max_resid": mr}
                                 for sl, g, bk, mr in done],
            "slice_in_progress": partial,
            "gpu_launches": int(launches),
            "roofline": roof,
            "filter_apply": {"mass_steps_ms": mms, "k_apply_ms": kms, "share_of_step": filt_ms / max(t_ms, 1e-9)},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "of": "block steps"},
            "f64_form": f64,
            "e2e": e2e, "clocks": clk.summary()}
    if not args.no_serving and world == 1:
        P.free()
        try:
            line["serving"] = run_serving(args, local)
        except Exception as ex:  # the serving leg must not cost the slice measurement
            line["serving"] = {"error": repr(ex)}
    if not args.no_precision and rank == 0:
        try:
            line["precision"] = precision_leg(nm, local)
        except Exception as ex:
            line["precision"] = {"error": repr(ex)}
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args.h, args.prec, k_M, max(slice_pairs, 1),
                                                max(slice_blocks, 1), args.degree, int(info["nnz_u"]),
                                                cpu_workers(args.cpu_workers))
        except Exception as ex:
            line["cpu_baseline"] = {"error": repr(ex)}
    print(json.dumps(line))


def precision_leg(nm, device):
    """The error of every eigenvalue of each precision form against the FP64
    dense oracle: one slice of the three-layer planet at h = 0.25 (the
    stored oracle eigenvalues of tests/golden/planet_slice.json, written by
    tests/golden/make_planet_slice.py), solved in FP64, mixed and float-filter
    form with the same filter (degree 400, b = 8)."""
    import torch
    from synth.model import layered_planet
    with open(os.path.join(ROOT, "tests", "golden", "planet_slice.json")) as f:
        gold = json.load(f)
    ref = np.asarray(gold["eigenvalues"])
    mesh, model = layered_planet(h=0.25, seed=7)
    ctx = nm.Context(device)
    P = nm.Problem(ctx, mesh, model)
    P.set_interval(gold["lambda_lo"], gold["lambda_hi"], unit=nm.NM_UNIT_OMEGA2)
    out = {"workload": "layered-planet-h0.25 (%d tets, %d dof), lambda in [%.4f, %.4f], %d eigenvalues"
                       % (mesh.nt, P.n, gold["lambda_lo"], gold["lambda_hi"], len(ref)),
           "oracle": "dense FP64 eigh (tests/golden/planet_slice.json)", "forms": {}}
    for name, prec, k in (("f64", nm.NM_F64, 40), ("mixed", nm.NM_MIXED, 20), ("f32_filter", nm.NM_F32, 40)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.lanczos_slice(block=8, degree=400, k_M=k, k_P=k, max_blocks=30, check_every=2, prec=prec, seed=2,
                            allow_unconverged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lam = np.sort(r.lam)
        entry = {"found": int(len(lam)), "seconds": dt, "blocks": int(r.info["blocks"]),
                 "max_resid": float(r.resid.max()) if len(lam) else None}
        if len(lam) == len(ref):
            err = np.abs(lam - ref) / np.abs(ref)
            entry["rel_error"] = [float(e) for e in err]
            entry["max_rel_error"] = float(err.max())
        else:
            entry["count_mismatch"] = True
        out["forms"][name] = entry
        r.free()
    ctx.close()
    return out


def gemm_case(nm, device):
    """The dense products of the Lanczos and Ritz steps on a 200,003-row,
    576-column basis: V^T W (576 x 32), V C (200,003 x 32), four of each."""
    import torch
    ctx = nm.Context(device)
    g = torch.Generator(device="cuda").manual_seed(0)
    n, m, b = 200003, 576, 32
    V = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g)
    W = torch.randn((n, b), dtype=torch.float64, device="cuda", generator=g)
    C = torch.empty((b, m), dtype=torch.float64, device="cuda")
    D = torch.empty((n, b), dtype=torch.float64, device="cuda")
    for _ in range(4):
        ctx.gemm_tn(V, W, C)
        ctx.gemm_nn(V, C, D)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "gemm", "n": n, "m": m, "b": b}))


def selfgrav_case(nm, device, h, b=32, reps=5):
    """K_eff X with and without -C^T S C (FP64, b columns) on the layered
    planet of mesh size h, timed with CUDA events on the launching stream.
    The N-body sum over the np charge points dominates the term; its
    algorithmic FP64 work per product is np^2 (9 + 2 b) flops (distance
    and 1/r once per pair, one FMA per pair and column)."""
    import torch
    from synth.model import layered_planet
    mesh, model = layered_planet(h=h, seed=2)
    ctx = nm.Context(device)
    P0 = nm.Problem(ctx, mesh, model)
    P1 = nm.Problem(ctx, mesh, model, self_gravity=True)
    X = torch.randn((P0.n, b), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()
    out = {}
    for key, P in (("cowling", P0), ("self_gravity", P1)):
        for _ in range(2):
            P.apply_K(X, Y, k_P=20)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            P.apply_K(X, Y, k_P=20)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[key] = ev[0].elapsed_time(ev[1]) / reps
    n_pts = P1.info["n_charges"]
    tet = np.asarray(mesh.tet)
    sg_ms = out["self_gravity"] - out["cowling"]
    flops = float(n_pts) ** 2 * (9 + 2 * b)
    print(json.dumps({"profile_case": "selfgrav", "h": h, "tets": len(tet), "n": P0.n, "points": n_pts, "b": b,
                      "k_eff_ms": out["cowling"], "full_ms": out["self_gravity"], "selfgrav_ms": sg_ms,
                      "nbody_tflops": flops / (sg_ms * 1e-3) / 1e12 if sg_ms > 0 else None,
                      "fp64_peak_tflops": FP64_PEAK_TFLOPS}))
    ctx.close()


# Four adjacent slices of the rotating planet's seismic band (angular
# frequency), about 200 eigenpairs together.
ROTATING_SLICES = [(4.0, 5.0), (5.0, 6.0), (6.0, 7.0), (7.0, 8.0)]
# Sixteen adjacent slices of width 0.25 over the same band.
HETERO_SLICES = [(4.0 + 0.25 * i, 4.25 + 0.25 * i) for i in range(16)]


def rotating_case(nm, device, h, degree, b=16, slices=None, lateral=0.0):
    """The rotating layered planet: the slices solved in one batched run
    (their blocks filtered as one 64-column recurrence, the mixed form), then
    the rotating reduction (eq. sublinear0) on all their Ritz vectors at
    once. Phases timed by host clocks around device synchronisations;
    eigenpairs/s counts the pencil pairs with residual <= 1e-6."""
    import torch
    from synth.model import OMEGA_EARTH_NONDIM, layered_planet
    slices = slices or ROTATING_SLICES
    mesh, model = layered_planet(h=h, seed=2, omega=OMEGA_EARTH_NONDIM, lateral=lateral, lateral_lmax=20)
    ctx = nm.Context(device)
    t0 = time.perf_counter()
    P = nm.Problem(ctx, mesh, model)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = P.lanczos_multi(slices, block=b, degree=degree, k_M=20, k_P=20, max_blocks=40, check_every=2,
                          prec=nm.NM_MIXED, seed=SEED, allow_unconverged=True)
    torch.cuda.synchronize()
    t_lanczos = time.perf_counter() - t0
    good = [int(np.sum(r.resid <= 1e-6)) for r in res]
    lam_e = np.concatenate([r.lam for r in res])
    t0 = time.perf_counter()
    Xe = torch.cat([r.vectors() for r in res], dim=1).contiguous()
    P.set_interval(slices[0][0], slices[-1][1])
    rot = P.ritz(Xe, mode=nm.NM_RITZ_ROTATING, lam_e=lam_e)
    torch.cuda.synchronize()
    t_rot = time.perf_counter() - t0
    print(json.dumps({
        "workload": ("rotating-heterogeneous-planet-h%g" if lateral else "rotating-layered-planet-h%g") % h,
        "lateral_perturbation": {"amplitude": lateral, "lmax": 20} if lateral else None,
        "tets": int(mesh.nt), "dof": int(P.n),
        "pressure_dof": int(P.Np), "omega_rotation": OMEGA_EARTH_NONDIM, "slices_omega": slices,
        "block": b, "degree": degree, "filter_prec": "mixed", "batched_columns": b * len(slices),
        "eigenpairs": int(sum(good)),
        "per_slice": [{"pairs": g, "found": len(r.lam), "blocks": int(r.info["blocks"]),
                       "max_resid": float(r.resid.max()) if len(r.lam) else None} for g, r in zip(good, res)],
        "assembly_s": t_asm, "lanczos_s": t_lanczos, "rotating_projection_s": t_rot,
        "eigenpairs_per_s": sum(good) / t_lanczos,
        "rotating": {"m_e": int(Xe.shape[1]), "frequencies_in_band": int(len(rot.lam)),
                     "max_quadratic_resid": float(rot.resid.max()) if len(rot.lam) else None},
    }))
    for r in res:
        r.free()
    rot.free()
    ctx.close()


def run_serving(args, device):
    """Continuous-batching serving leg: a seeded Poisson stream of slice
    requests over three mesh sizes, admitted by free slot and free HBM,
    overlapping on the device. Latency counts from arrival to result and
    includes each mesh's assembly in the slot that first serves it."""
    from paper_1906_11082_gb300 import nm
    from paper_1906_11082_gb300.serving import Request, SliceServer
    from synth.model import layered_planet

    rng = np.random.default_rng(5)
    meshes = {}

    def builder(h):
        def build():
            if h not in meshes:
                meshes[h] = layered_planet(h=h, seed=7)
            return meshes[h]
        return build

    srv = SliceServer(slots=3, device=device)
    sizes = {}
    for i in range(args.serving_requests):
        h, lam_max = SERVING_MESHES[int(rng.integers(len(SERVING_MESHES)))]
        iv = SERVING_SLICES[int(rng.integers(len(SERVING_SLICES)))]
        opts = dict(block=16, degree=serving_degree(lam_max, *iv), k_M=K_SERVING, k_P=K_SERVING,
                    max_blocks=30, check_every=2, prec=nm.NM_MIXED, seed=100 + i)
        if h not in sizes:
            m, _ = builder(h)()
            sizes[h] = int(m.nt)
        srv.submit(Request(key=f"planet-h{h}", build=builder(h), interval=iv, opts=opts), 5 * sizes[h])
        time.sleep(float(rng.exponential(1.0)))
    srv.drain(timeout=1800)
    st = srv.stats()
    srv.close()
    st.update({"slots": 3, "arrivals": "Poisson, mean gap 1.0 s", "block": 16, "filter_prec": "mixed",
               "meshes": [{"h": h, "tets": sizes.get(h), "lambda_max": lm,
                           "degrees": [serving_degree(lm, *iv) for iv in SERVING_SLICES]} for h, lm in SERVING_MESHES],
               "slices_omega": SERVING_SLICES, "latency_includes": "queueing and first assembly per slot"})
    return st


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
