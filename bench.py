#!/usr/bin/env python3
"""Benchmark of the Galerkin-FFT solver on one GB300 (or N replicas).

Step = one Galerkin-operator apply y = G(K : x) (Eq. newlinop) at 128^3 voxels
in FP64 with the continuous projection, K = the rotated cubic stiffness of a
500-grain periodic Voronoi polycrystal (the tangent at F = I), x ~ N(0, 1).
value = applies/s over all ranks.  The JSON line also carries:
  * the FP32 and discrete-projection variants and the per-kernel roofline of
    the dominant kernel, against the measured HBM copy bandwidth or the FP64
    FMA throughput measured here (gff_measure_fp64_peak);
  * the CG vector kernels' bandwidth at 128^3 (FP64 and FP32);
  * the end-to-end rate through gff_apply_operator_host (pinned host x in,
    host y out, copies inside the call);
  * seconds per cyclic load increment over one full +-1 % strain cycle
    (80 increments, Newton tolerance 1e-6) for the 64^3 / 200-grain RVE
    (FP64, mixed, mixed + extrapolated start, and the latter with the
    FP64-only return map; continuous and discrete projection; the
    constitutive time split into return maps and tangents) and the
    128^3 / 500-grain RVE (FP64 zero start, mixed zero
    start, mixed + extrapolated start, mixed + learned U-Net start trained
    inside the run), each with its macroscopic-P error against the FP64 arm
    and the SM clocks sampled over the arm;
  * the 32-RVE batch; the CPU oracle (one thread, all host cores, and per
    load increment).

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
    p.add_argument("--increments", type=int, default=80,
                   help="load increments per arm of the cyclic-increment measurements (80 = one cycle; 0: skip)")
    p.add_argument("--config5", type=int, default=1, help="1: also the 128^3 / 500-grain arms")
    p.add_argument("--unet-train-steps", type=int, default=400, help="Adam steps of the in-run U-Net training")
    p.add_argument("--unet-train-rves", type=int, default=2, help="64^3 RVEs whose increments train the U-Net")
    p.add_argument("--cpu-applies", type=int, default=3, help="oracle applies in the CPU baseline sample")
    p.add_argument("--cpu-increments", type=int, default=1, help="1: time the oracle per load increment too")
    p.add_argument("--batch-cycle", type=int, default=80,
                   help="increments of the 32-RVE batch run (80 = one cycle; 0: skip)")
    p.add_argument("--batch-increments", type=int, default=8,
                   help="increments of the 32-RVE batch compared with one handle after the other (0: skip)")
    p.add_argument("--grid", type=int, default=N_GRID, help="grid size (smaller grids only for profiling runs)")
    p.add_argument("--tiles", default="", help="12 comma-separated launch-shape ints (FP64 then FP32, the layout "
                   "gff_autotune returns) to use instead of the tuned ones in the apply measurement; write "
                   "--tiles=... (the values may be negative)")
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
    z pass = 6 x 2 x 5 log2 n (n/2+1)/n (each tensor row packed into two
    fields, transformed both ways) + packing, projection and unpacking (~72
    per frequency); inverse plane pass = 9 x (same transforms)."""
    import math

    lg = math.log2(n)
    fr = (n // 2 + 1) / n
    plane = 9 * (2.5 * lg + 5 * lg * fr)
    return [162 + plane, 6 * 2 * 5 * lg * fr + 72 * fr, plane]


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


def _oracle_apply_worker(napplies, n):
    return oracle_apply_rate(napplies, n)


def host_info():
    """Host core count and CPU model (for the CPU-baseline record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    mem = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable"):
                mem = int(line.split()[1]) * 1024
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "mem_available_bytes": mem}


def oracle_apply_rate_all_cores(napplies, n, info):
    """Independent oracle applies in a spawn process pool, one per core (one
    BLAS/FFT thread each), as many processes as the host memory allows
    (about 3 GB each at 128^3).  Aggregate applies/s and processes used."""
    import concurrent.futures
    import multiprocessing

    procs = info["nproc"] or 1
    if info["mem_available_bytes"]:
        procs = max(1, min(procs, int(0.5 * info["mem_available_bytes"] / (3.0 * (n / 128.0) ** 3 * 1e9))))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    ctx = multiprocessing.get_context("spawn")
    t0 = time.perf_counter()
    with concurrent.futures.ProcessPoolExecutor(max_workers=procs, mp_context=ctx) as ex:
        res = list(ex.map(_oracle_apply_worker, [napplies] * procs, [n] * procs))
    wall = time.perf_counter() - t0
    # each worker's timed loop excludes its start-up and input generation; the rate is the sum of theirs
    return sum(r for r, _ in res), procs, wall


def oracle_increment_seconds():
    """Oracle seconds per load increment on one host thread: config 1 (16^3,
    cubic SVK, mixed control, all 5 steps) and the first 20 increments of the
    config-2 loading on a 16^3 / 8-grain crystal-plasticity RVE (the 64^3 /
    200-grain RVE's grain density), extrapolated to 64^3 by the voxel count."""
    from oracle.solver import CP_FCC, SVK_CUBIC, Material, OracleRVE, Options
    from rve_inputs import cyclic_history, polycrystal, ramp_history

    out = {}
    o = OracleRVE(polycrystal(16, 8, 1), {0: Material(SVK_CUBIC)}, Options(newton_tol=1e-8, cg_tol=1e-8))
    h1 = ramp_history()
    t0 = time.perf_counter()
    o.run(h1)
    out["config1_16cube_s_per_increment"] = (time.perf_counter() - t0) / h1.nsteps
    o = OracleRVE(polycrystal(16, 8, 2), {0: Material(CP_FCC)}, Options(newton_tol=1e-6, cg_tol=1e-3))
    h2 = cyclic_history(0.01, 1).head(20)
    t0 = time.perf_counter()
    o.run(h2)
    s16 = (time.perf_counter() - t0) / h2.nsteps
    out["config2_loading_16cube_s_per_increment"] = s16
    out["config2_64cube_s_per_increment_extrapolated"] = s16 * 64
    out["note"] = "64^3 figure extrapolated from the 16^3 sample by the voxel count (64x); one thread"
    return out


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


PASS1_END = b"// ---------------------------------------------------------------- pass 2:"
PLAN_START = b"template <int R1, int R2> struct Inv2Plan {"
PLAN_END = b"template <typename T, int R1, int R2>\n__device__ __forceinline__ void inv2_x1("
FWD2_START = b"// ---------------------------------------------------------------- pass 1 for two-stage plans, register-staged"
FWD2_END = b"template <typename T> constexpr int zproj_width()"
# the parts of fft_proj.cu each profiled forward kernel is built from: everything before the pass-2
# marker (complex arithmetic, butterflies, radix stages, line transforms, the contraction, pass 1),
# and for the register-staged pass also the plan constants, swizzle and row-pair mapping it shares
# with the register-staged inverse, and its own section
SOURCE_REGIONS = {"k_plane_fwd": [(None, PASS1_END)],
                  "k_plane_fwd2": [(None, PASS1_END), (PLAN_START, PLAN_END), (FWD2_START, FWD2_END)]}
PROFILE_FILES = {"k_plane_fwd": "k_plane_fwd_fp64_64cube.md", "k_plane_fwd2": "k_plane_fwd2_fp64_64cube.md"}


def kernel_source_sha1(kernel):
    """sha1 of the source regions of fft_proj.cu that `kernel` is built from."""
    src = open(os.path.join(ROOT, "paper_1806_10599_gb300", "csrc", "fft_proj.cu"), "rb").read()
    parts = []
    for a, b in SOURCE_REGIONS[kernel]:
        i = 0 if a is None else src.find(a)
        j = src.find(b, max(i, 0))
        if i < 0 or j < 0:
            return None
        parts.append(src[i:j])
    return hashlib.sha1(b"".join(parts)).hexdigest()


def pass1_source_sha1():
    return kernel_source_sha1("k_plane_fwd")


def measured_traffic(n, kernel="k_plane_fwd"):
    """DRAM bytes per launch of the FP64 forward kernel at 128^3 from its committed ncu summary, or None when
    the grid differs, no summary exists, or the kernel source changed since the counters were taken."""
    if n != 128 or kernel not in PROFILE_FILES:
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", PROFILE_FILES[kernel])).read()
        src_sha = kernel_source_sha1(kernel)
    except OSError:
        return None
    sha = re.search(r"source sha1 ([0-9a-f]{40})", txt)
    val = re.search(r"traffic_bytes_per_launch_128: ([0-9.eE+]+)", txt)
    if not sha or not val or sha.group(1) != src_sha:
        return None
    return float(val.group(1))


def pass_names(tiles):
    """Names of the three apply kernels the tuned launch shapes select (fwd threads < 0, inv blocks -1 and
    TMA z blocks < 0 are the register-staged variants)."""
    fwd, _, _, _, invb, zb = tiles if tiles else (1, 0, 0, 0, 0, 0)
    f = ("k_plane_fwd2 (K:x + register-staged forward x/y transforms)" if fwd < 0
         else "k_plane_fwd (K:x + forward x/y transforms)")
    z = ("k_zproj_tma (register-staged strip: z transforms + projection)" if zb < 0
         else "k_zproj_tma (z transforms + projection)" if zb > 0 else "k_zproj (z transforms + projection)")
    i = ("k_plane_inv2 (register-staged inverse y/x transforms)" if invb == -1
         else "k_plane_inv_stream (inverse y/x transforms)" if invb > 0 else "k_plane_inv (inverse y/x transforms)")
    return [f, z, i], ("k_plane_fwd2" if fwd < 0 else "k_plane_fwd")


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


def time_arm(g, torch, ms, hist, precision, projection=0, warm=0, unet=None, clock_index=None, return_map=None):
    """One arm of the cyclic-increment measurement: the whole history through
    gff_run_history on a fresh handle, timed on the host around the call (the
    launch shapes are tuned before).  Returns seconds per increment, the
    macroscopic P of every increment and per-increment diagnostics."""
    try:
        opts = g.make_options(precision=precision, projection=projection, newton_tol=1e-6, cg_tol=1e-3)
        h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_CP_FCC)}, opts)
        try:
            if warm:
                g.gff_set_warm_start(h, unet, warm)
            if return_map is not None:
                g.gff_set_return_map(h, return_map)
            g.gff_autotune(h)  # outside the timed region
            torch.cuda.synchronize()
            clk = ClockSampler(clock_index) if clock_index is not None else None
            if clk:
                clk.start()
            t0 = time.perf_counter()
            Pm, reps = g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            clocks = clk.stop() if clk else None
        finally:
            g.gff_destroy(h)
    except Exception as e:  # report, do not lose the other measurements
        return {"error": str(e)}
    n = len(reps)
    return {"s_per_cyclic_increment": dt / n, "increments": n, "seconds": dt,
            "newton_mean": sum(r.newton_iters for r in reps) / n, "cg_mean": sum(r.cg_iters for r in reps) / n,
            "cuts": sum(r.cuts for r in reps), "residual_max": max(r.residual for r in reps),
            "residual_first_mean": sum(r.residual_first for r in reps) / n,
            "cp_local_iters_per_voxel_mean": sum(r.cp_local_iters for r in reps) / n,
            "cp_fallbacks": sum(r.cp_fallbacks for r in reps),
            "s_constitutive": sum(r.t_constitutive for r in reps) / n,
            "s_tangent": sum(r.t_tangent for r in reps) / n,
            "s_residual": sum(r.t_residual for r in reps) / n, "s_linear": sum(r.t_linear for r in reps) / n,
            "P11_MPa_peak": max(p[0] for p in Pm) / 1e6, "P11_MPa_min": min(p[0] for p in Pm) / 1e6,
            "clocks": clocks, "_Pm": Pm.tolist()}


def macro_errors(arms, ref_key):
    """Each arm's largest relative macroscopic-P deviation from the reference arm over the history."""
    import numpy as np

    ref = arms.get(ref_key, {}).get("_Pm")
    for k, a in arms.items():
        if "_Pm" not in a:
            continue
        if ref is not None and len(a["_Pm"]) == len(ref):
            P, R = np.array(a["_Pm"]), np.array(ref)
            a["macroP_rel_err_vs_" + ref_key] = float(max(np.linalg.norm(P[i] - R[i]) / np.linalg.norm(R[i])
                                                          for i in range(len(R))))
    for a in arms.values():
        a.pop("_Pm", None)
    return arms


def train_unet(g, torch, rves, steps, increments):
    """The learned warm start, trained inside the run on the solver's own load
    increments of `rves` 64^3 / 200-grain RVEs (seeds 5000+i, one +-1 % cycle,
    mixed precision): a bounded data collection plus `steps` Adam steps."""
    from paper_1806_10599_gb300 import warmstart

    u = g.gff_unet_create(1)
    t0 = time.perf_counter()
    warmstart.collect(u, [5000 + i for i in range(rves)], increments=increments)
    t1 = time.perf_counter()
    g.gff_unet_set_sampling(u, 1)
    losses = g.gff_unet_train(u, steps, 1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    k = max(1, min(50, steps // 4))
    info = {"rves": rves, "increments_per_rve": increments, "samples": g.gff_unet_num_samples(u), "steps": steps,
            "data_s": t1 - t0, "train_s": t2 - t1, "loss_first": float(sum(losses[:k]) / k),
            "loss_last": float(sum(losses[-k:]) / k)}
    return u, info


def cyclic_increments(g, torch, args, clock_index):
    """Seconds per cyclic increment, mixed vs FP64 (the metric's second half)."""
    from rve_inputs import cyclic_history, polycrystal

    hist = cyclic_history(0.01, 1).head(args.increments)
    out = {}
    ms2 = polycrystal(64, 200, 2)
    arms = {}
    for proj, pname in ((0, "continuous"), (1, "discrete")):
        arms["fp64_" + pname] = time_arm(g, torch, ms2, hist, 0, proj, clock_index=clock_index)
        arms["mixed_" + pname] = time_arm(g, torch, ms2, hist, 1, proj, clock_index=clock_index)
        arms["mixed_extrapolated_" + pname] = time_arm(g, torch, ms2, hist, 1, proj, g.GFF_WARM_EXTRAPOLATE,
                                                       clock_index=clock_index)
        # the mixed arms run the default return map (FP32 pre-iteration, then FP64); this one the FP64
        # iteration alone, which shows what the pre-iteration saves
        arms["mixed_extrapolated_fp64map_" + pname] = time_arm(g, torch, ms2, hist, 1, proj,
                                                               g.GFF_WARM_EXTRAPOLATE, clock_index=clock_index,
                                                               return_map=g.GFF_RETURN_MAP_FP64)
    macro_errors({k: v for k, v in arms.items() if k.endswith("continuous")}, "fp64_continuous")
    macro_errors({k: v for k, v in arms.items() if k.endswith("discrete")}, "fp64_discrete")
    out["config2"] = {"workload": "64^3, 200-grain periodic Voronoi (seed 2), FCC crystal plasticity, R=-1 +-1 pct "
                                  "strain cycle, %d increments (dt 0.05 s), Newton tol 1e-6, CG tol 1e-3"
                                  % hist.nsteps, "arms": arms}
    if args.config5:
        ms5 = polycrystal(128, 500, 5)
        arms5 = {"fp64_zero": time_arm(g, torch, ms5, hist, 0, clock_index=clock_index),
                 "mixed_zero": time_arm(g, torch, ms5, hist, 1, clock_index=clock_index),
                 "mixed_extrapolated": time_arm(g, torch, ms5, hist, 1, 0, g.GFF_WARM_EXTRAPOLATE,
                                                clock_index=clock_index)}
        unet_info = None
        if args.unet_train_steps > 0:
            try:
                u, unet_info = train_unet(g, torch, args.unet_train_rves, args.unet_train_steps, 80)
                try:
                    arms5["mixed_unet"] = time_arm(g, torch, ms5, hist, 1, 0, g.GFF_WARM_NET, unet=u,
                                                   clock_index=clock_index)
                finally:
                    g.gff_unet_destroy(u)
            except Exception as e:
                unet_info = {"error": str(e)}
        macro_errors(arms5, "fp64_zero")
        f64 = arms5["fp64_zero"].get("s_per_cyclic_increment")
        target = {}
        for k in ("mixed_unet", "mixed_extrapolated"):
            v = arms5.get(k, {}).get("s_per_cyclic_increment")
            if f64 and v:
                target[k + "_speedup_vs_fp64_zero"] = f64 / v
        if "mixed_unet_speedup_vs_fp64_zero" in target:
            # mixed precision with the learned start faster per cyclic increment than FP64 at residual <= 1e-6
            target["mixed_unet_faster_than_fp64_at_1e-6"] = (target["mixed_unet_speedup_vs_fp64_zero"] > 1.0
                                                            and arms5["mixed_unet"].get("residual_max", 1.0) <= 1e-6)
        out["config5"] = {"workload": "128^3, 500-grain periodic Voronoi (seed 5), FCC crystal plasticity, R=-1 "
                                      "+-1 pct strain cycle, %d increments, Newton tol 1e-6, CG tol 1e-3; U-Net "
                                      "trained in this run" % hist.nsteps,
                          "arms": arms5, "unet_training": unet_info, "target": target}
    return out


def time_batch(g, torch, cycle_increments, compare_increments, precision, world=1, rank=0):
    """32 RVEs of 32^3 ... 96^3 voxels (10,956,800 in all), crystal plasticity,
    +-1 % strain cycle, mixed precision, extrapolated warm start: one full
    cycle through gff_batch_run (one graph launch per increment) with the
    per-grain Fatemi-Socie parameter at its end, and the first
    `compare_increments` increments batched against running the same RVEs one
    handle after the other.  With several ranks the RVEs are spread over them
    (shard.assign; each rank runs its share as one batch, no collective on the
    data path), the time is the slowest rank's and the per-RVE results are
    gathered on rank 0 once at the end."""
    from paper_1806_10599_gb300 import shard
    from rve_inputs import batch_rves, cyclic_history, polycrystal

    specs = batch_rves()
    parts = shard.assign([n for n, _, _ in specs], world)
    mine = parts[rank]
    full = cyclic_history(0.01, 1).head(cycle_increments)
    out = {"rves": len(specs), "voxels": int(sum(n ** 3 for n, _, _ in specs))}
    if world > 1:
        out["ranks"] = world
        out["rves_per_rank"] = [len(p) for p in parts]
    errors = []

    def make():
        opts = g.make_options(precision=precision, newton_tol=1e-6, cg_tol=1e-3, warm_start=g.GFF_WARM_EXTRAPOLATE)
        hs = []
        for i in mine:
            n, ng, seed = specs[i]
            hs.append(g.create_rve(polycrystal(n, ng, seed), {0: g.make_material(g.GFF_MAT_CP_FCC)}, opts))
        for h in hs:
            g.gff_set_warm_start(h, None, g.GFF_WARM_EXTRAPOLATE)
            g.gff_autotune(h)
        torch.cuda.synchronize()
        return hs

    def timed(run):
        """Local run on this rank's RVEs between barriers; seconds of the slowest rank (collectives always run)."""
        secs, res = float("nan"), None
        hs = []
        try:
            hs = make()
            barrier(world)
            t0 = time.perf_counter()
            res = run(hs)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        except Exception as e:  # report, do not lose the apply measurement (nor hang the other ranks)
            errors.append(str(e))
            if world > 1 and not hs:
                barrier(world)
        finally:
            for h in hs:
                g.gff_destroy(h)
        return max_over_ranks(secs, world), res

    if cycle_increments > 0:
        def cycle(hs):
            Pm, reps, stat = g.gff_batch_run(hs, full.dt, full.Fbar, full.mask, full.Pbar, full.cycle_start,
                                             raise_on_error=False)
            torch.cuda.synchronize()
            return [{"status": int(stat[j]), "fs_max": float(max(g.gff_get_fips(h, specs[i][1])[2])),
                     "newton": int(sum(r.newton_iters for r in reps[j])), "cuts": int(sum(r.cuts for r in reps[j]))}
                    for j, (i, h) in enumerate(zip(mine, hs))]

        secs, res = timed(cycle)
        got = shard.gather_to_rank0(res if res is not None else [None] * len(mine), world)
        if rank == 0:
            per = shard.merge(got, parts, len(specs))
            ok = all(p is not None for p in per)
            out["cycle"] = {"increments": full.nsteps, "s_per_increment_batched": secs / full.nsteps,
                            "status": [p["status"] if p else None for p in per],
                            "newton_mean": (sum(p["newton"] for p in per) / (len(per) * full.nsteps)) if ok else None,
                            "cuts": sum(p["cuts"] for p in per) if ok else None,
                            "fatemi_socie_max_per_rve": [p["fs_max"] if p else None for p in per]}
    if compare_increments > 0:
        part = full.head(compare_increments) if cycle_increments > 0 else \
            cyclic_history(0.01, 1).head(compare_increments)
        for mode in ("batched", "one_by_one"):
            if mode == "batched":
                def run(hs):
                    return g.gff_batch_run(hs, part.dt, part.Fbar, part.mask, part.Pbar, part.cycle_start)
            else:
                def run(hs):
                    return [g.gff_run_history(h, part.dt, part.Fbar, part.mask, part.Pbar, part.cycle_start)
                            for h in hs]
            secs, _ = timed(run)
            out["s_per_increment_%s_first_%d" % (mode, part.nsteps)] = secs / part.nsteps
        a1 = out.get("s_per_increment_batched_first_%d" % part.nsteps)
        a2 = out.get("s_per_increment_one_by_one_first_%d" % part.nsteps)
        if a1 and a2 and a1 == a1 and a2 == a2:
            out["batched_speedup_first_%d" % part.nsteps] = a2 / a1
    if errors:
        out["error"] = "; ".join(errors)
    return out


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
    if args.tiles:  # pinned launch shapes (profiling runs: timings under a profiler would mislead the tuner)
        t = [int(v) for v in args.tiles.split(",")]
        tiles = {"fp64": t[:6], "fp32": t[6:12]}
        for hh in (h, hd):
            g.gff_set_tiles(hh, tiles["fp64"], tiles["fp32"])
    g.gff_constitutive(h, 1.0)
    g.gff_constitutive(hd, 1.0)
    x = standard_normal(SEED_X, 9 * N).reshape(9, N)
    X = torch.from_numpy(x).cuda()
    Y = torch.empty_like(X)
    X32 = X.float()
    Y32 = torch.empty_like(X32)

    vis = [d for d in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if d.strip()]
    clock_index = vis[local].strip() if local < len(vis) else str(local)
    clocks = ClockSampler(clock_index)
    if rank == 0:
        clocks.start()
    ms64 = time_applies(torch, g, h, g.GFF_PREC_FP64, X, Y, args.steps, args.warmup, world)
    clk = clocks.stop() if rank == 0 else None
    ms32 = time_applies(torch, g, h, g.GFF_PREC_MIXED, X32, Y32, args.steps, args.warmup, world)
    msd = time_applies(torch, g, hd, g.GFF_PREC_FP64, X, Y, args.steps, args.warmup, world)
    k64 = per_kernel_ms(g, h, g.GFF_PREC_FP64, X, Y, max(5, args.steps // 2))
    k32 = per_kernel_ms(g, h, g.GFF_PREC_MIXED, X32, Y32, max(5, args.steps // 2))
    fp64_peak = g.gff_measure_fp64_peak()
    g.gff_destroy(hd)

    # end to end through the C ABI with host buffers: pinned x in, y out, copies inside the call
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(args.warmup):
        g.gff_apply_operator_host(h, g.GFF_PREC_FP64, None, xh, yh)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.gff_apply_operator_host(h, g.GFF_PREC_FP64, None, xh, yh)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    barrier(world)
    # the CG vector kernels on the same grid (the handle's work vectors)
    cg64 = g.gff_cg_kernels_timed(h, g.GFF_PREC_FP64, 20)
    cg32 = g.gff_cg_kernels_timed(h, g.GFF_PREC_MIXED, 20)
    g.gff_destroy(h)
    del X, Y, X32, Y32
    torch.cuda.empty_cache()

    inc = None
    if args.increments > 0 and rank == 0:
        inc = cyclic_increments(g, torch, args, clock_index)
    batch = None
    if args.batch_cycle > 0 or args.batch_increments > 0:  # every rank: the RVEs are spread over the ranks
        batch = {"workload": "32 RVEs (7x32^3, 7x48^3, 6x64^3, 6x80^3, 6x96^3; 50-300 grains, seeds 4000+i), FCC "
                             "crystal plasticity, +-1 pct cycle, mixed precision, Newton tol 1e-6, extrapolated "
                             "warm start",
                 "mixed": time_batch(g, torch, args.batch_cycle, args.batch_increments, 1, world, rank)}

    if rank != 0:
        return
    cpu = None
    if world == 1 and args.cpu_applies > 0:
        info = host_info()
        rate, secs = oracle_apply_rate(args.cpu_applies, args.grid)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d oracle applies at %d^3 (numpy FP64, one thread), %.1f s"
                         % (args.cpu_applies, args.grid, secs), "host": info}
        try:
            rall, procs, wall = oracle_apply_rate_all_cores(args.cpu_applies, args.grid, info)
            cpu["all_cores"] = {"value": rall, "unit": UNIT, "cores": procs,
                                "sample": "%d independent oracle processes x %d applies at %d^3, %.1f s wall"
                                          % (procs, args.cpu_applies, args.grid, wall)}
        except Exception as e:
            cpu["all_cores"] = {"error": str(e)}
        if args.cpu_increments:
            try:
                cpu["increments"] = oracle_increment_seconds()
            except Exception as e:
                cpu["increments"] = {"error": str(e)}
    raw = {"ms64": ms64, "ms32": ms32, "msd": msd, "k64": k64, "k32": k32, "e2e_s": e2e_s,
           "xbytes": int(x.nbytes), "clocks": clk, "increment": inc, "cpu": cpu, "tiles": tiles,
           "batch": batch, "fp64_peak_gflops": fp64_peak[0], "cg64": cg64, "cg32": cg32}
    print(json.dumps(build_line(args, world, raw, *measured_peaks())), flush=True)


def cg_kernel_roofline(ms3, n_elems, elem, peak):
    """GB/s and HBM fraction of the CG vector kernels: p.Ap reads 2 vectors;
    the update reads x, p, r, Ap and writes x, r; p = r + beta p reads 2 and
    writes 1 (each vector n_elems values of elem bytes)."""
    accesses = [2, 6, 3]
    names = ["dot p.Ap with alpha (k_cg_alpha)", "x, r update + r.r with beta (k_cg_update_dev)",
             "p = r + beta p (k_xpby_dev)"]
    out = {}
    for nm, a, ms in zip(names, accesses, ms3):
        gbs = a * n_elems * elem / (ms * 1e-3) / 1e9 if ms > 0 else None
        out[nm] = {"ms": ms, "bytes": a * n_elems * elem, "gbs": gbs, "frac": gbs / peak if gbs else None}
    return out


def build_line(args, world, raw, peaks, src):
    """The benchmark's JSON line from the measured numbers (pure function)."""
    peak = hbm_peak(peaks)
    nvox = args.grid ** 3
    k64, k32 = raw["k64"], raw["k32"]
    b64 = kernel_bytes_per_voxel(args.grid, 8)
    b32 = kernel_bytes_per_voxel(args.grid, 4)
    fl = kernel_flops_per_voxel(args.grid)
    fp64_peak = raw.get("fp64_peak_gflops")
    fp64_src = "measured here (FP64 FMA chains, gff_measure_fp64_peak)" if fp64_peak else "nominal GB300 FP64 rate"
    fp64_peak = fp64_peak or FP64_PEAK_NOMINAL_GFLOPS
    tiles = raw.get("tiles") or {}
    names, fwd_id = pass_names(tiles.get("fp64"))
    names32, _ = pass_names(tiles.get("fp32"))
    dom = max(range(3), key=lambda i: k64[i])
    gbs = [b64[i] * nvox / (k64[i] * 1e-3) / 1e9 for i in range(3)]
    gfl = [fl[i] * nvox / (k64[i] * 1e-3) / 1e9 for i in range(3)]
    hbm_frac = gbs[dom] / peak
    alu_frac = gfl[dom] / fp64_peak
    if alu_frac > hbm_frac:
        roof = {"bound": "alu", "kernel": names[dom], "achieved": gfl[dom], "peak": fp64_peak,
                "unit": "GFLOP/s", "frac": alu_frac, "peak_source": fp64_src,
                "hbm_achieved_gbs": gbs[dom], "hbm_frac": hbm_frac, "hbm_peak_source": src}
    else:
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": gbs[dom], "peak": peak, "unit": "GB/s",
                "frac": hbm_frac, "peak_source": src}
    roof["traffic"] = measured_traffic(args.grid, fwd_id) if dom == 0 else None
    roof["algorithmic_bytes_per_launch"] = b64[dom] * nvox
    roof["kernel_ms"] = k64
    roof["all_kernels_gflops"] = gfl
    roof["all_kernels_gbs"] = gbs
    dom32 = max(range(3), key=lambda i: k32[i])
    gbs32 = [b32[i] * nvox / (k32[i] * 1e-3) / 1e9 for i in range(3)]
    roof32 = {"bound": "hbm", "kernel": names32[dom32], "achieved": gbs32[dom32], "peak": peak, "unit": "GB/s",
              "frac": gbs32[dom32] / peak, "peak_source": src, "kernel_ms": k32, "all_kernels_gbs": gbs32,
              "all_kernels_frac": [v / peak for v in gbs32],
              "apply_gbs": sum(b32) * nvox / (sum(k32) * 1e-3) / 1e9, "traffic": None,
              "algorithmic_bytes_per_launch": b32[dom32] * nvox}
    steps = args.steps
    cg = None
    if raw.get("cg64") and raw.get("cg32"):
        cg = {"grid": [args.grid] * 3, "fp64": cg_kernel_roofline(raw["cg64"], 9 * nvox, 8, peak),
              "fp32": cg_kernel_roofline(raw["cg32"], 9 * nvox, 4, peak)}
    return {
        "metric": METRIC, "value": world * steps / (raw["ms64"] * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": raw["ms64"] / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.grid), "roofline": roof, "cpu_baseline": raw["cpu"],
        "e2e": {"value": world * steps / raw["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": raw["xbytes"],
                "d2h_bytes_per_step": raw["xbytes"],
                "how": "gff_apply_operator_host per step: pinned host x -> device in chunks of z-planes that overlap the forward plane pass, z pass, pinned host y <- device in chunks that overlap the inverse plane pass"},
        "gpu_launches": 3 * steps, "clocks": raw["clocks"],
        "fp64_tflops_measured": (raw.get("fp64_peak_gflops") or 0) / 1e3 or None,
        "variants": {
            "fp32_apply": {"value": world * steps / (raw["ms32"] * 1e-3), "unit": UNIT, "dtype": "f32",
                           "roofline": roof32},
            "discrete_projection_fp64": {"value": world * steps / (raw["msd"] * 1e-3), "unit": UNIT,
                                         "dtype": "f64"},
        },
        "cg_kernels": cg,
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
