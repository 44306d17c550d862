#!/usr/bin/env python3
"""Benchmark of the Galerkin-FFT solver on one GB300 (or N replicas).

Step = one Galerkin-operator apply y = G(K : x) (Eq. newlinop) at 128^3 voxels
in FP64 with the continuous projection, K = the rotated cubic stiffness of a
500-grain periodic Voronoi polycrystal (the tangent at F = I), x ~ N(0, 1).
value = applies/s over all ranks.  The JSON line also carries the FP32 and
discrete-projection variants, the per-kernel roofline of the dominant kernel,
the end-to-end rate with host buffers, the CPU-oracle baseline, SM clocks
sampled during the timed region, and the seconds per crystal-plasticity load
increment (64^3, 200 grains, +-1 % strain cycles) in FP64, in mixed precision,
and in mixed precision started from the extrapolated last increment.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gff|reference]
"""

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Galerkin-operator applies/s at 128^3; s per cyclic increment, mixed vs FP64"
UNIT = "applies/s"
N_GRID = 128
N_GRAINS = 500
SEED_MS = 5
SEED_X = 7
FP64_PEAK_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 (vector and tensor), nominal


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["gff", "reference"], default="gff")
    p.add_argument("--increments", type=int, default=12,
                   help="CP increments timed per variant: FP64, mixed, mixed + extrapolated start (0: skip)")
    p.add_argument("--cpu-applies", type=int, default=3, help="oracle applies in the CPU baseline sample")
    p.add_argument("--batch-increments", type=int, default=2,
                   help="increments of the 32-RVE batch, batched and one by one (0: skip)")
    p.add_argument("--grid", type=int, default=N_GRID, help="grid size (smaller grids only for profiling runs)")
    a = p.parse_args()
    return a


# --------------------------------------------------------------------------- distributed plumbing
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() and args.impl == "gff" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available() and args.impl == "gff":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- roofline model
def kernel_bytes_per_voxel(n, elem):
    """Algorithmic DRAM bytes per voxel of the three apply kernels: each
    field read or written once.  elem = 8 (FP64) or 4 (FP32); a complex
    half-spectrum value has 2 elem bytes and there are (n/2+1)/n of them per
    real value."""
    half = 9 * 2 * elem * (n // 2 + 1) / n
    return [81 * elem + 9 * elem + half,  # K, x in; half spectrum out
            2 * half,                      # half spectrum in and out
            half + 9 * elem]               # half spectrum in; y out


def kernel_flops_per_voxel(n):
    """Algorithmic floating-point operations per voxel (5 n log2 n per complex
    FFT of length n, the usual convention): forward plane pass = K:x (162) +
    9 x (x real transform 2.5 log2 n + y transform 5 log2 n (n/2+1)/n);
    z pass = 9 x 2 x 5 log2 n (n/2+1)/n + projection (~56 per frequency);
    inverse plane pass = 9 x (same transforms)."""
    import math

    lg = math.log2(n)
    fr = (n // 2 + 1) / n
    plane = 9 * (2.5 * lg + 5 * lg * fr)
    return [162 + plane, 9 * 2 * 5 * lg * fr + 56 * fr, plane]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hbm_peak(peaks):
    for k in ("hbm_gbs", "hbm_GBs", "hbm"):
        if k in peaks and isinstance(peaks[k], (int, float)):
            return float(peaks[k])
    return 6800.0


# --------------------------------------------------------------------------- CPU oracle
def oracle_inputs(n=N_GRID):
    import numpy as np

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import materials as omat
    from rve_inputs import polycrystal, standard_normal

    ms = polycrystal(n, N_GRAINS, SEED_MS)
    R = omat.quat_to_rot(ms.quat)
    Cc = omat.cubic_stiffness(168.4e9, 121.4e9, 75.4e9)
    Cg = np.stack([omat.rotate4(Cc, R[g]) for g in range(ms.ngrains)])  # tangent at F = I
    K = np.ascontiguousarray(np.moveaxis(Cg[ms.grain_id], (0, 1, 2), (4, 5, 6)))
    x = standard_normal(SEED_X, 9 * ms.n_voxels).reshape((3, 3) + ms.grain_id.shape)
    return K, x


def oracle_apply_rate(napplies, n=N_GRID):
    """Oracle applies/s on this host (numpy FFT and einsum: 1 thread)."""
    from oracle import spectral as sp

    K, x = oracle_inputs(n)
    sp.GK(K, x)  # warm-up
    t0 = time.perf_counter()
    for _ in range(napplies):
        sp.GK(K, x)
    dt = time.perf_counter() - t0
    return napplies / dt, dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import spectral as sp

    K, x = oracle_inputs(args.grid)
    for _ in range(args.warmup):
        sp.GK(K, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sp.GK(K, x)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args.grid),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d oracle applies at %d^3 (numpy FP64, one thread)" % (args.steps, args.grid)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(n=N_GRID):
    return {
        "workload": "Galerkin operator apply y = G(K:x) at %d^3 voxels, FP64, continuous projection; "
                    "K = rotated cubic C (168.4/121.4/75.4 GPa) per voxel of a 500-grain periodic Voronoi "
                    "polycrystal (seed 5); x ~ N(0,1) (seed 7)" % n,
        "grid": [n] * 3, "grains": N_GRAINS, "projection": "continuous", "precision": "fp64",
        "l2": "inputs larger than L2 (K alone is %.2f GB)" % (81 * 8 * n ** 3 / 1e9),
        "parallelism": "independent replicas",
    }


def measured_traffic(n):
    """DRAM bytes per launch of the FP64 k_plane_fwd at 128^3 from the committed ncu summary, or None when
    the grid differs or the kernel source changed since the counters were taken."""
    if n != 128:
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", "k_plane_fwd_fp64_64cube.md")).read()
        src = open(os.path.join(ROOT, "paper_1806_10599_gb300", "csrc", "fft_proj.cu"), "rb").read()
    except OSError:
        return None
    sha = re.search(r"sha1 ([0-9a-f]{40})", txt)
    val = re.search(r"traffic_bytes_per_launch_128: ([0-9.eE+]+)", txt)
    if not sha or not val or sha.group(1) != hashlib.sha1(src).hexdigest():
        return None
    return float(val.group(1))


# --------------------------------------------------------------------------- GPU arm
def time_applies(torch, g, h, prec, X, Y, steps, warmup, world, mask=None):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        g.gff_apply_operator(h, prec, mask, X, Y)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.gff_apply_operator(h, prec, mask, X, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    return max_over_ranks(ms, world)


def per_kernel_ms(g, h, prec, X, Y, reps):
    acc = [0.0, 0.0, 0.0]
    for _ in range(reps):
        t = g.gff_apply_operator_timed(h, prec, None, X, Y)
        acc = [a + b for a, b in zip(acc, t)]
    return [a / reps for a in acc]


def time_increments(g, torch, nsteps, precision, warm=0):
    try:
        return _time_increments(g, torch, nsteps, precision, warm)
    except Exception as e:  # report, do not lose the apply measurement
        return {"error": str(e)}


def _time_increments(g, torch, nsteps, precision, warm):
    from rve_inputs import cyclic_history, polycrystal

    ms = polycrystal(64, 200, 2)
    hist = cyclic_history(0.01, 1).head(nsteps)
    opts = g.make_options(precision=precision, newton_tol=1e-6, cg_tol=1e-3 if precision == 0 else 1e-3)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_CP_FCC)}, opts)
    try:
        if warm:
            g.gff_set_warm_start(h, None, warm)
        g.gff_autotune(h)  # outside the timed region
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Pm, reps = g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        g.gff_destroy(h)
    return {"s_per_increment": dt / nsteps, "newton": [r.newton_iters for r in reps],
            "cp_local_iters_per_voxel": [round(r.cp_local_iters, 2) for r in reps],
            "cp_fallbacks": [r.cp_fallbacks for r in reps],
            "s_each": [round(r.seconds, 4) for r in reps],
            "cg": [r.cg_iters for r in reps], "P11_MPa_last": Pm[-1][0] / 1e6,
            "s_constitutive": sum(r.t_constitutive for r in reps) / nsteps,
            "s_residual": sum(r.t_residual for r in reps) / nsteps,
            "s_linear": sum(r.t_linear for r in reps) / nsteps}


def time_batch(g, torch, nsteps, precision):
    """32 RVEs of 32^3 ... 96^3 voxels (10,956,800 in all), crystal plasticity,
    first `nsteps` increments of a +-1 % cycle: gff_batch_run against running
    the same RVEs one handle after the other."""
    try:
        from rve_inputs import batch_rves, cyclic_history, polycrystal

        specs = batch_rves()
        hist = cyclic_history(0.01, 1).head(nsteps)
        opts = g.make_options(precision=precision, newton_tol=1e-6, cg_tol=1e-3)
        out = {"rves": len(specs), "voxels": int(sum(n ** 3 for n, _, _ in specs)), "increments": nsteps}
        for mode in ("batched", "one_by_one"):
            hs = [g.create_rve(polycrystal(n, ng, seed), {0: g.make_material(g.GFF_MAT_CP_FCC)}, opts)
                  for n, ng, seed in specs]
            try:
                for h in hs:
                    g.gff_autotune(h)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode == "batched":
                    Pm, reps, stat = g.gff_batch_run(hs, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
                    newton = [r[-1].newton_iters for r in reps]
                else:
                    newton = []
                    for h in hs:
                        _, rp = g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
                        newton.append(rp[-1].newton_iters)
                torch.cuda.synchronize()
                out["s_per_increment_" + mode] = (time.perf_counter() - t0) / nsteps
                out["newton_last_" + mode] = newton
            finally:
                for h in hs:
                    g.gff_destroy(h)
        return out
    except Exception as e:  # report, do not lose the apply measurement
        return {"error": str(e)}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1806_10599_gb300 import build as b

    if not os.path.exists(b.LIB):
        if rank == 0:
            b.build()
        barrier(world)
    from paper_1806_10599_gb300 import gff as g
    from rve_inputs import polycrystal, standard_normal

    ms = polycrystal(args.grid, N_GRAINS, SEED_MS)
    N = ms.n_voxels
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options())
    hd = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(projection=g.GFF_PROJ_DISCRETE))
    tiles = g.gff_autotune(h)
    g.gff_autotune(hd)
    g.gff_constitutive(h, 1.0)
    g.gff_constitutive(hd, 1.0)
    x = standard_normal(SEED_X, 9 * N).reshape(9, N)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    X32 = X.float()
    Y32 = torch.empty_like(X32)

    vis = [d for d in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if d.strip()]
    clocks = ClockSampler(vis[local].strip() if local < len(vis) else str(local))
    if rank == 0:
        clocks.start()
    ms64 = time_applies(torch, g, h, g.GFF_PREC_FP64, X, Y, args.steps, args.warmup, world)
    clk = clocks.stop() if rank == 0 else None
    ms32 = time_applies(torch, g, h, g.GFF_PREC_MIXED, X32, Y32, args.steps, args.warmup, world)
    msd = time_applies(torch, g, hd, g.GFF_PREC_FP64, X, Y, args.steps, args.warmup, world)
    k64 = per_kernel_ms(g, h, g.GFF_PREC_FP64, X, Y, max(5, args.steps // 2))
    k32 = per_kernel_ms(g, h, g.GFF_PREC_MIXED, X32, Y32, max(5, args.steps // 2))

    # end to end: pinned host x -> device, apply, device -> pinned host y, every step
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(args.warmup):
        X.copy_(xh, non_blocking=True)
        g.gff_apply_operator(h, g.GFF_PREC_FP64, None, X, Y)
        yh.copy_(Y, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        X.copy_(xh, non_blocking=True)
        g.gff_apply_operator(h, g.GFF_PREC_FP64, None, X, Y)
        yh.copy_(Y, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    barrier(world)

    inc = None
    if args.increments > 0 and rank == 0:
        inc = {"workload": ("64^3, 200-grain periodic Voronoi (seed 2), FCC crystal plasticity, R=-1 +-1 pct "
                            "strain cycles, first %d increments (dt 0.05 s), Newton tol 1e-6") % args.increments,
               "fp64": time_increments(g, torch, args.increments, 0),
               "mixed": time_increments(g, torch, args.increments, 1),
               "mixed_extrapolated": time_increments(g, torch, args.increments, 1, g.GFF_WARM_EXTRAPOLATE)}
    g.gff_destroy(h)
    g.gff_destroy(hd)
    batch = None
    if args.batch_increments > 0 and rank == 0:
        batch = {"workload": "32 RVEs (7x32^3, 7x48^3, 6x64^3, 6x80^3, 6x96^3; 50-300 grains, seeds 4000+i), FCC "
                             "crystal plasticity, +-1 pct cycle, mixed precision, Newton tol 1e-6",
                 "mixed": time_batch(g, torch, args.batch_increments, 1)}

    if rank != 0:
        return
    cpu = None
    if world == 1 and args.cpu_applies > 0:
        rate, secs = oracle_apply_rate(args.cpu_applies, args.grid)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d oracle applies at %d^3 (numpy FP64, one thread), %.1f s"
                         % (args.cpu_applies, args.grid, secs)}
    raw = {"ms64": ms64, "ms32": ms32, "msd": msd, "k64": k64, "k32": k32, "e2e_s": e2e_s,
           "xbytes": int(x.nbytes), "clocks": clk, "increment": inc, "cpu": cpu, "tiles": tiles,
           "batch": batch}
    print(json.dumps(build_line(args, world, raw, *measured_peaks())), flush=True)


def build_line(args, world, raw, peaks, src):
    """The benchmark's JSON line from the measured numbers (pure function)."""
    peak = hbm_peak(peaks)
    nvox = args.grid ** 3
    k64, k32 = raw["k64"], raw["k32"]
    b64 = kernel_bytes_per_voxel(args.grid, 8)
    b32 = kernel_bytes_per_voxel(args.grid, 4)
    fl = kernel_flops_per_voxel(args.grid)
    names = ["k_plane_fwd (K:x + forward x/y transforms)", "k_zproj (z transforms + projection)",
             "k_plane_inv (inverse y/x transforms)"]
    dom = max(range(3), key=lambda i: k64[i])
    gbs = [b64[i] * nvox / (k64[i] * 1e-3) / 1e9 for i in range(3)]
    gfl = [fl[i] * nvox / (k64[i] * 1e-3) / 1e9 for i in range(3)]
    hbm_frac = gbs[dom] / peak
    alu_frac = gfl[dom] / FP64_PEAK_NOMINAL_GFLOPS
    if alu_frac > hbm_frac:
        roof = {"bound": "alu", "kernel": names[dom], "achieved": gfl[dom], "peak": FP64_PEAK_NOMINAL_GFLOPS,
                "unit": "GFLOP/s", "frac": alu_frac, "peak_source": "nominal GB300 FP64 rate",
                "hbm_achieved_gbs": gbs[dom], "hbm_frac": hbm_frac, "hbm_peak_source": src}
    else:
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": gbs[dom], "peak": peak, "unit": "GB/s",
                "frac": hbm_frac, "peak_source": src}
    roof["traffic"] = measured_traffic(args.grid) if dom == 0 else None
    roof["algorithmic_bytes_per_launch"] = b64[dom] * nvox
    roof["kernel_ms"] = k64
    dom32 = max(range(3), key=lambda i: k32[i])
    gbs32 = [b32[i] * nvox / (k32[i] * 1e-3) / 1e9 for i in range(3)]
    roof32 = {"bound": "hbm", "kernel": names[dom32], "achieved": gbs32[dom32], "peak": peak, "unit": "GB/s",
              "frac": gbs32[dom32] / peak, "peak_source": src, "kernel_ms": k32, "all_kernels_gbs": gbs32,
              "apply_gbs": sum(b32) * nvox / (sum(k32) * 1e-3) / 1e9, "traffic": None,
              "algorithmic_bytes_per_launch": b32[dom32] * nvox}
    steps = args.steps
    return {
        "metric": METRIC, "value": world * steps / (raw["ms64"] * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": raw["ms64"] / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.grid), "roofline": roof, "cpu_baseline": raw["cpu"],
        "e2e": {"value": world * steps / raw["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": raw["xbytes"],
                "d2h_bytes_per_step": raw["xbytes"]},
        "gpu_launches": 3 * steps, "clocks": raw["clocks"],
        "variants": {
            "fp32_apply": {"value": world * steps / (raw["ms32"] * 1e-3), "unit": UNIT, "dtype": "f32",
                           "roofline": roof32},
            "discrete_projection_fp64": {"value": world * steps / (raw["msd"] * 1e-3), "unit": UNIT,
                                         "dtype": "f64"},
        },
        "increment": raw["increment"],
        "autotuned_tiles": raw.get("tiles"),
        "batch": raw.get("batch"),
    }


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
