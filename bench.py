"""Benchmark: eigenpairs/s of one filtered-Lanczos spectrum slice on GB300.

Workload (default): the three-layer planet (solid inner core, fluid outer
core, solid mantle; seeded smooth profiles; reference gravity by direct
summation; Cowling operator), P2 on ~2.6e5 tets (~1.1M dof), Chebyshev
degree 100, one low-frequency slice holding ~100 eigenpairs, block width
32. A step is one full slice solve: spectrum bounds, filtered block
Lanczos, FP64 Rayleigh-Ritz and FP64 residuals (matrices resident,
assembly excluded). value = eigenpairs with residual <= 1e-6 per second,
summed over ranks (each rank solves its own slice; no collective).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f64|f32]
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

# Slice edges (angular frequency) of the layered-planet workload, placed in
# spectral gaps; rank r of N solves slice r (adjacent slices, ~100 pairs).
SLICES_OMEGA = [(0.5, 3.0), (3.0, 3.8), (3.8, 4.4), (4.4, 4.9), (4.9, 5.3), (5.3, 5.7), (5.7, 6.0),
                (6.0, 6.3)]
H_MESH = 0.05
DEGREE = 100
BLOCK = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=("f64", "f32"), default="f64")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--h", type=float, default=H_MESH)
    ap.add_argument("--max-blocks", type=int, default=16)
    ap.add_argument("--k-m", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


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
    Returns (seconds per step, scale factor to the full mesh, description)."""
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
    op = filtlan.Operator(S, k_M=k_M, k_P=k_M)
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
    k_M = args.k_m or (57 if args.prec == "f64" else 28)
    t_step, blocks_sub, nt_sub, n_sub = cpu_sample(w, args.prec, BLOCK, k_M, warm=args.warmup, steps=args.steps)
    # full-mesh scale from the stored-block count of the full graph
    from oracle import fem
    dm = fem.dof_map(w.mesh.tet, w.mesh.region, w.mesh.nv)
    blocks_full = _graph_blocks(w.mesh, dm)
    t_deg = t_step * blocks_full / blocks_sub
    nev, nblocks = 100, 8
    value = nev / (t_deg * DEGREE * nblocks)
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": w.name, "tets": int(w.mesh.nt), "degree": DEGREE, "block": BLOCK},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one filter degree (K_eff + {k_M}-step mass solve) on {BLOCK} vectors "
                                       f"over the octant x,y,z>0 ({nt_sub} tets, {n_sub} dof), scaled by "
                                       f"stored blocks to the full mesh and by degree {DEGREE} x {nblocks} "
                                       f"blocks to a {nev}-pair slice"},
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
    lo, hi = SLICES_OMEGA[rank % len(SLICES_OMEGA)]
    P.set_interval(lo, hi)
    prec = nm.NM_F64 if args.prec == "f64" else nm.NM_F32
    k_M = args.k_m or (57 if args.prec == "f64" else 28)
    opts = dict(block=BLOCK, degree=DEGREE, k_M=k_M, k_P=k_M, max_blocks=args.max_blocks, check_every=1,
                prec=prec, seed=11 + rank, allow_unconverged=True)

    def step():
        return P.lanczos_slice(**opts)

    for _ in range(args.warmup):
        r = step()
        r.free()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

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
            results.append((len(r.lam), float(r.resid.max()) if len(r.lam) else 0.0, r.info))
            r.free()
        ev1.record()
        barrier()
    launches = nm.kernel_launches() - launches0
    t_ms = ev0.elapsed_time(ev1)
    good = sum(int(np.sum(np.asarray([k]))) for k, _, _ in results)
    k_last, res_last, info_last = results[-1]
    ml, mms = P.profile_read(0)
    kl, kms = P.profile_read(1)
    P.profile(False, reset=True)
    # max over ranks of the timed region; eigenpairs summed over ranks
    tot_pairs = good
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        pp = torch.tensor([float(good)], device="cuda")
        dist.all_reduce(pp, op=dist.ReduceOp.SUM)
        tot_pairs = int(pp.item())
    value = tot_pairs / (t_ms / 1e3)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        n = P.n
        host_start = torch.randn((n, BLOCK), dtype=torch.float64).pin_memory()
        dev_start = torch.empty((n, BLOCK), dtype=torch.float64, device="cuda")
        host_out = None
        barrier()
        t0 = time.perf_counter()
        pairs_e2e = 0
        h2d = d2h = 0
        for _ in range(args.steps):
            dev_start.copy_(host_start, non_blocking=True)
            torch.cuda.synchronize()
            r = P.lanczos_slice(**dict(opts, start=dev_start))
            X = r.vectors()
            if host_out is None or host_out.shape != X.shape:
                host_out = torch.empty(X.shape, dtype=X.dtype).pin_memory()
            host_out.copy_(X)
            lam = r.lam.copy()
            pairs_e2e += int(np.sum(r.resid <= 1e-6))
            h2d += host_start.numel() * 8
            d2h += X.numel() * 8 + 2 * lam.size * 8
            r.free()
            del X
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": pairs_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
               "d2h_bytes_per_step": d2h // args.steps}

    if rank != 0:
        return
    info = P.info
    s = 8 if args.prec == "f64" else 4
    peak_hbm, peak_src = peaks()
    avg_launch_s = (mms / 1e3) / max(ml, 1)
    mbytes = mass_step_bytes(info, BLOCK, s)
    mflops = mass_step_flops(info, BLOCK)
    gbs = mbytes / avg_launch_s / 1e9 if ml else None
    tfl = mflops / avg_launch_s / 1e12 if ml else None
    if args.prec == "f64" and tfl is not None and tfl / FP64_PEAK_TFLOPS > gbs / peak_hbm:
        roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "kron_kernel<double,3,CHEB>",
                "peak_source": "GB300 FP64 nominal (152 SM x 2 FMA/clk x 2.05 GHz)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": (gbs / peak_hbm) if gbs else None, "traffic": None,
                "kernel": f"kron_kernel<{'double' if s == 8 else 'float'},3,CHEB>",
                "peak_source": f"{peak_src} copy bandwidth"}
    roof["bytes_per_launch"] = mbytes
    roof["flops_per_launch"] = mflops
    roof["avg_launch_us"] = avg_launch_s * 1e6
    roof["launches"] = ml
    filt_ms = mms + kms
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": w.name, "tets": int(w.mesh.nt), "dof": int(info["n"]),
                       "pressure_dof": int(info["Np"]), "degree": DEGREE, "block": BLOCK, "k_M": k_M,
                       "slice_omega": [lo, hi], "eigenpairs": int(k_last), "max_resid": res_last,
                       "lanczos_blocks": int(info_last["blocks"]), "filter_prec": args.prec,
                       "parallelism": f"slices x{world}",
                       "l2": "inputs larger than L2 (A_G %.2f GB resident)" % (info["nnz_u"] * 76 / 1e9)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "filter_apply": {"mass_steps_ms": mms, "k_apply_ms": kms, "share_of_step":
                             filt_ms / max(t_ms, 1e-9)},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
            "e2e": e2e, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        t_step, blocks_sub, nt_sub, n_sub = cpu_sample(w, args.prec, BLOCK, k_M)
        blocks_full = info["nnz_u"]
        t_deg = t_step * blocks_full / blocks_sub
        cpu_val = max(k_last, 1) / (t_deg * DEGREE * max(int(info_last["blocks"]), 1))
        line["cpu_baseline"] = {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one filter degree (K_eff + {k_M}-step mass solve) on {BLOCK} vectors "
                                          f"over the octant x,y,z>0 ({nt_sub} tets, {n_sub} dof, "
                                          f"{t_step:.1f} s), scaled by stored blocks to the full mesh and by "
                                          f"degree x Lanczos blocks of the GPU run"}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
