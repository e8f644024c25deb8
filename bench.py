"""Benchmark: eigenpairs/s of one filtered-Lanczos spectrum slice on GB300.

Workload (default): the three-layer planet (solid inner core, fluid outer
core, solid mantle; seeded smooth profiles; reference gravity by direct
summation; Cowling operator), P2 on ~2.6e5 tets (~1.1M dof), one
low-frequency slice holding ~100 eigenpairs, block width 32. A step is one full slice solve: spectrum bounds, filtered block
Lanczos, FP64 Rayleigh-Ritz and FP64 residuals (matrices resident,
assembly excluded). The filter degree is 600, not the configured 100: on
this mesh a degree-100 filter cannot keep the fluid core's essential
spectrum near lambda = 0 out of the slice. value = eigenpairs with residual <= 1e-6 per second,
summed over ranks (each rank solves its own slice; no collective).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|f64|f32]
       [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
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

# Slice edges (angular frequency) of the layered-planet workload; rank r of
# N solves slice r. The first slice holds ~100 eigenpairs above the fluid
# band; later slices continue upward.
SLICES_OMEGA = [(4.0, 6.5), (6.5, 7.6), (7.6, 8.4), (8.4, 9.0), (9.0, 9.6), (9.6, 10.1), (10.1, 10.5),
                (10.5, 10.9)]
H_MESH = 0.05
# The configured degree is 100; on this mesh (lambda_max ~ 3.4e5) a
# degree-100 filter passes the fluid core's ~8e4-dimensional essential
# spectrum near lambda = 0 as strongly as the slice. Degree 600 holds it
# below 0.7% of the slice's filter value.
DEGREE_CONFIG = 100
DEGREE = 600
# The benchmark slice as the filtered Lanczos solves it: 90 eigenpairs with
# residual <= 1e-6 after 18 blocks of 32 (measured); the reference arm
# scales one timed CPU filter degree by degree x blocks of this slice.
SLICE_PAIRS = 90
SLICE_BLOCKS = 18
BLOCK = 32
K_INNER = {"f64": 38, "mixed": 20, "f32": 28}

# Serving leg: layered planets of three sizes with the spectrum upper bound
# the library's bounds estimate gives on each (lambda_max sets the filter
# degree), and three slices of width 1.5 in omega. Near the bottom of the
# spectrum a slice of width dw spans dw sqrt(2/e) in Chebyshev angle
# (e = lambda_max / 2), so the degree is 1.7 pi sqrt(lambda_max) / (2 dw),
# the ratio the benchmark slice runs at. Requests arrive as a seeded
# Poisson stream.
SERVING_MESHES = [(0.25, 58954.0), (0.15, 45045.0), (0.1, 85700.0)]
SERVING_SLICES = [(4.0, 5.5), (4.5, 6.0), (3.5, 5.0)]


def serving_degree(lam_max, lo, hi):
    return int(np.ceil(1.7 * np.pi * np.sqrt(lam_max) / (2.0 * (hi - lo))))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=("mixed", "f64", "f32"), default="mixed")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--h", type=float, default=H_MESH)
    ap.add_argument("--max-blocks", type=int, default=24)
    ap.add_argument("--degree", type=int, default=DEGREE)
    ap.add_argument("--k-m", type=int, default=0)
    ap.add_argument("--profile-case", action="store_true",
                    help="one short mixed filter application on the full matrices (for ncu captures)")
    ap.add_argument("--chunk", type=int, default=None,
                    help="chunked row schedule of the semi-iteration SpMMs (threads per CTA; 0 = off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def rank_slice(rank):
    """The slice rank r solves: the units (slices) are sharded over ranks,
    so the data path needs no collective."""
    return SLICES_OMEGA[rank % len(SLICES_OMEGA)]


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


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the float
# mass-step kernel (kron_v4_kernel<3, 1, 32>) on this workload, from the ncu
# capture summarised in profiles/kron_v4_mass_step_planet_h0.05_b32.md
# (same matrices and block width as the timed launches).
V4_TRAFFIC_BYTES = 543_801_344 + 123_877_376

# FP64 peak of GB300 (NVIDIA's published B300 figure, 1.25 TFLOP/s; equal to
# 152 SMs x ~2.05 GHz x 2 FP64 FMA per SM per clock x 2 flop).
FP64_PEAK_TFLOPS = 1.25


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


def cpu_sample(w, prec, b, k_M, warm=0, steps=1):
    """The oracle as it stands, on a bounded sample: one filter degree
    (K_eff + mass solve) for b vectors on the octant x, y, z > 0 of the mesh.
    The mixed form's oracle counterpart applies the refined solves in FP64.
    Returns (seconds per step, stored blocks of the sample, tets, dof)."""
    import copy
    from synth.mesh import Mesh
    from oracle import fem, filtlan
    m = w.mesh
    c = m.xyz[m.tet].mean(axis=1)
    sel = np.nonzero((c > 0).all(axis=1))[0]
    sub = Mesh(xyz=m.xyz, tet=m.tet[sel], region=m.region[sel], layer=m.layer[sel], radii=m.radii)
    mdl = copy.copy(w.model)
    for k in ("rho", "lam", "mu", "N2"):
        setattr(mdl, k, getattr(w.model, k)[sel])
    S = fem.assemble(sub, mdl)
    op = filtlan.Operator(S, k_M=k_M, k_P=k_M, refine=(prec == "mixed"))
    Y = np.random.default_rng(0).standard_normal((S.n, b))
    if prec == "f32":
        Y = Y.astype(np.float32)
    times = []
    for i in range(warm + steps):
        t = time.perf_counter()
        op.B(Y)
        if i >= warm:
            times.append(time.perf_counter() - t)
    blocks_sub = S.A_G.nnz / 9
    return float(np.mean(times)), blocks_sub, len(sel), S.n


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    w = workload(args.h)
    k_M = args.k_m or K_INNER[args.prec]
    t_step, blocks_sub, nt_sub, n_sub = cpu_sample(w, args.prec, BLOCK, k_M, warm=args.warmup, steps=args.steps)
    # full-mesh scale from the stored-block count of the full graph
    from oracle import fem
    dm = fem.dof_map(w.mesh.tet, w.mesh.region, w.mesh.nv)
    blocks_full = _graph_blocks(w.mesh, dm)
    t_deg = t_step * blocks_full / blocks_sub
    nev, nblocks = SLICE_PAIRS, SLICE_BLOCKS
    value = nev / (t_deg * args.degree * nblocks)
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "tets": int(w.mesh.nt), "degree": args.degree, "block": BLOCK},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one filter degree (K_eff + {k_M}-step mass solve) on {BLOCK} vectors "
                                       f"over the octant x,y,z>0 ({nt_sub} tets, {n_sub} dof), scaled by "
                                       f"stored blocks to the full mesh and by degree {args.degree} x {nblocks} "
                                       f"blocks to the {nev}-pair benchmark slice (the same algorithm "
                                       f"converges it in {nblocks} blocks)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _graph_blocks(mesh, dm):
    un = dm.elem_unodes(np.asarray(mesh.region))
    a = np.repeat(un, 10, axis=1).ravel()
    b = np.tile(un, (1, 10)).ravel()
    key = np.unique(a.astype(np.int64) * dm.Nu + b)
    return len(key)


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

    w = workload(args.h)
    ctx = nm.Context(local)
    P = nm.Problem(ctx, w.mesh, w.model)
    if args.chunk is not None:
        P.set_option("chunk", args.chunk)
    lo, hi = rank_slice(rank)
    P.set_interval(lo, hi)
    prec = {"f64": nm.NM_F64, "f32": nm.NM_F32, "mixed": nm.NM_MIXED}[args.prec]
    k_M = args.k_m or K_INNER[args.prec]
    opts = dict(block=BLOCK, degree=args.degree, k_M=k_M, k_P=k_M, max_blocks=args.max_blocks, check_every=2,
                prec=prec, seed=11 + rank, allow_unconverged=True)
    if args.profile_case:
        lo_b, hi_b = P.spectrum_bounds(steps=40, k_M=k_M)
        g, c, e = nm.filter_design(lo_b, hi_b, lo * lo, hi * hi, 10)
        Y = torch.randn((P.n, BLOCK), dtype=torch.float64, device="cuda")
        Z = torch.empty_like(Y)
        P.filter_apply(g, c, e, k_M, Y, Z, prec=nm.NM_MIXED)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("filter")
        P.filter_apply(g, c, e, k_M, Y, Z, prec=nm.NM_MIXED)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": "mixed filter, degree 10, b = 32", "n": P.n}))
        return

    def step():
        return P.lanczos_slice(**opts)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def e2e_steps(count):
        """`count` steps end to end through the public API: every step copies
        its start block from pinned host memory to the device, solves the
        slice, and copies eigenvectors and eigenvalues back to the host."""
        n = P.n
        host_start = torch.randn((n, BLOCK), dtype=torch.float64).pin_memory()
        dev_start = torch.empty((n, BLOCK), dtype=torch.float64, device="cuda")
        host_out = None
        barrier()
        t0 = time.perf_counter()
        pairs = h2d = d2h = 0
        for _ in range(count):
            dev_start.copy_(host_start, non_blocking=True)
            torch.cuda.synchronize()
            r = P.lanczos_slice(**dict(opts, start=dev_start))
            X = r.vectors()
            if host_out is None or host_out.shape != X.shape:
                host_out = torch.empty(X.shape, dtype=X.dtype).pin_memory()
            host_out.copy_(X)
            lam = r.lam.copy()
            pairs += int(np.sum(r.resid <= 1e-6))
            h2d += host_start.numel() * 8
            d2h += X.numel() * 8 + 2 * lam.size * 8
            r.free()
            del X
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"value": pairs / dt, "unit": UNIT, "h2d_bytes_per_step": h2d // count,
                "d2h_bytes_per_step": d2h // count, "steps": count}

    # Warm-up: the first step plain; with W >= 2 the remaining W - 1 warm-up
    # steps are the end-to-end measurement (warm, untimed for `value`).
    e2e = None
    n_e2e_warm = args.warmup - 1 if (not args.no_e2e and args.warmup >= 2) else 0
    for _ in range(args.warmup - n_e2e_warm):
        r = step()
        r.free()
    if n_e2e_warm:
        e2e = e2e_steps(n_e2e_warm)
        e2e["note"] = "measured on warm-up steps 2..W"

    P.profile(True, reset=True)
    launches0 = nm.kernel_launches()
    lat = []
    results = []
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            t = time.perf_counter()
            r = step()
            lat.append(time.perf_counter() - t)
            results.append((int(np.sum(r.resid <= 1e-6)), float(r.resid.max()) if len(r.lam) else 0.0,
                            dict(r.info, found=len(r.lam))))
            r.free()
        ev1.record()
        barrier()
    launches = nm.kernel_launches() - launches0
    t_ms = ev0.elapsed_time(ev1)
    good = sum(k for k, _, _ in results)
    k_last, res_last, info_last = results[-1]
    ml, mms = P.profile_read(0)
    kl, kms = P.profile_read(1)
    # the dominant kernel's own launches: the float M_rho semi-iteration
    # steps (kind 2) in the mixed form, the mass-step launches (kind 0) else
    dl, dms = P.profile_read(2) if args.prec == "mixed" else (ml, mms)
    P.profile(False, reset=True)
    t_ms, tot_pairs = reduce_over_ranks(t_ms, good, world, "cuda")
    value = tot_pairs / (t_ms / 1e3)

    # end to end through the public API with host buffers, when the warm-up
    # was too short to carry it
    if e2e is None and not args.no_e2e:
        e2e = e2e_steps(args.steps)

    if rank != 0:
        return
    info = P.info
    # per-degree cost of the plain FP64 filter (same slice, k = 38) for the
    # FP64-form comparison; measured outside the timed region
    lo_b, hi_b = P.spectrum_bounds(steps=40, k_M=K_INNER["f64"])
    g4, c4, e4 = nm.filter_design(lo_b, hi_b, lo * lo, hi * hi, 4)
    Yb = torch.randn((P.n, BLOCK), dtype=torch.float64, device="cuda")
    Zb = torch.empty_like(Yb)
    per_deg = {}
    for name, pr, kk in (("f64", nm.NM_F64, K_INNER["f64"]), ("mixed", nm.NM_MIXED, K_INNER["mixed"])):
        P.filter_apply(g4, c4, e4, kk, Yb, Zb, prec=pr)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        P.filter_apply(g4, c4, e4, kk, Yb, Zb, prec=pr)
        a1.record()
        torch.cuda.synchronize()
        per_deg[name] = a0.elapsed_time(a1) / 4.0
    blocks_used = max(int(info_last["blocks"]), 1)
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
    if args.prec == "f64" and tfl is not None and tfl / FP64_PEAK_TFLOPS > gbs / peak_hbm:
        roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "kron_warp_kernel<double, 3, 1, 1>",
                "peak_source": "GB300 FP64 nominal (152 SM x 2 FMA/clk x 2.05 GHz)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": (gbs / peak_hbm) if gbs else None,
                "traffic": V4_TRAFFIC_BYTES if (s == 4 and args.h == H_MESH) else None,
                "kernel": "kron_warp_kernel<double, 3, 1, 1>" if s == 8 else "kron_v4_kernel<3, 1, 32>",
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
                       "block": BLOCK, "k_inner": k_M,
                       "slice_omega": [lo, hi], "eigenpairs": int(k_last), "max_resid": res_last,
                       "lanczos_blocks": int(info_last["blocks"]), "filter_prec": args.prec,
                       "parallelism": f"slices x{world}",
                       "l2": "inputs larger than L2 (A_G %.2f GB resident)" % (info["nnz_u"] * 76 / 1e9)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "filter_apply": {"mass_steps_ms": mms, "k_apply_ms": kms, "share_of_step":
                             filt_ms / max(t_ms, 1e-9)},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
            "forms_ms_per_degree_b32": per_deg,
            "f64_form_estimate": {"value": k_last / (per_deg["f64"] / 1e3 * args.degree * blocks_used),
                                  "unit": UNIT, "basis": "plain FP64 filter ms/degree x degree x the Lanczos "
                                                         "blocks of this run (filter time only)"},
            "e2e": e2e, "clocks": clk.summary()}
    if not args.no_serving and world == 1:
        P.free()
        try:
            line["serving"] = run_serving(args, local)
        except Exception as ex:  # the serving leg must not cost the slice measurement
            line["serving"] = {"error": repr(ex)}
    if not args.no_cpu_baseline:
        t_step, blocks_sub, nt_sub, n_sub = cpu_sample(w, args.prec, BLOCK, k_M)
        blocks_full = info["nnz_u"]
        t_deg = t_step * blocks_full / blocks_sub
        cpu_val = max(k_last, 1) / (t_deg * args.degree * max(int(info_last["blocks"]), 1))
        line["cpu_baseline"] = {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one filter degree (K_eff + {k_M}-step mass solve) on {BLOCK} vectors "
                                          f"over the octant x,y,z>0 ({nt_sub} tets, {n_sub} dof, "
                                          f"{t_step:.1f} s), scaled by stored blocks to the full mesh and by "
                                          f"degree x Lanczos blocks of the GPU run"}
    print(json.dumps(line))


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
    reqs = []
    sizes = {}
    for i in range(args.serving_requests):
        h, lam_max = SERVING_MESHES[int(rng.integers(len(SERVING_MESHES)))]
        iv = SERVING_SLICES[int(rng.integers(len(SERVING_SLICES)))]
        opts = dict(block=16, degree=serving_degree(lam_max, *iv), k_M=K_INNER["mixed"], k_P=K_INNER["mixed"],
                    max_blocks=30, check_every=2, prec=nm.NM_MIXED, seed=100 + i)
        if h not in sizes:
            m, _ = builder(h)()
            sizes[h] = int(m.nt)
        reqs.append(srv.submit(Request(key=f"planet-h{h}", build=builder(h), interval=iv, opts=opts),
                               5 * sizes[h]))
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
