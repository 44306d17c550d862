"""Train and evaluate the learned warm start through the C ABI.

Training data are the solver's own load increments on 64^3 polycrystals
(crystal plasticity, fully reversed +-1 % strain cycles, mixed precision);
evaluation runs the same kind of history on a larger RVE from the zero
fluctuation start (mode 0), from the extrapolated last increment (mode 3)
and from the network's guess (modes 1 and 2), and reports Newton and CG
iterations, the first residual and the wall time per increment.

    python -m paper_1806_10599_gb300.warmstart [--train-rves 4] [--steps 2000] ...
"""

import argparse
import json
import time

import numpy as np

from . import gff as g


def _rve(n, ngrains, seed, precision=1, tol=1e-6):
    from rve_inputs import polycrystal

    opts = g.make_options(precision=precision, newton_tol=tol, cg_tol=1e-3)
    return g.create_rve(polycrystal(n, ngrains, seed), {0: g.make_material(g.GFF_MAT_CP_FCC)}, opts)


def collect(u, seeds, n=64, ngrains=200, increments=80, eps=0.01):
    """Run each RVE through `increments` increments and keep every one as a sample."""
    from rve_inputs import cyclic_history

    hist = cyclic_history(eps, max(1, (increments + 79) // 80)).head(increments)
    for s in seeds:
        h = _rve(n, ngrains, s)
        try:
            for k in range(hist.nsteps):
                g.gff_step(h, hist.dt[k], hist.Fbar[k], hist.mask[k], hist.Pbar[k])
                g.gff_unet_add_sample(u, h)
        finally:
            g.gff_destroy(h)


def evaluate(u, n=128, ngrains=500, seed=5, increments=20, eps=0.01, modes=(0, 3, 1, 2)):
    """Per warm-start mode: mean Newton/CG iterations, first residual and seconds per increment."""
    import torch

    from rve_inputs import cyclic_history

    hist = cyclic_history(eps, max(1, (increments + 79) // 80)).head(increments)
    out = {}
    for mode in modes:
        h = _rve(n, ngrains, seed)
        reps, Pm = [], []
        try:
            if mode:
                g.gff_set_warm_start(h, u, mode)
            g.gff_autotune(h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(hist.nsteps):
                reps.append(g.gff_step(h, hist.dt[k], hist.Fbar[k], hist.mask[k], hist.Pbar[k]))
                Pm.append(np.array(reps[-1].Pmacro))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        except g.GffError as e:
            out["mode%d" % mode] = {"failed_at": len(reps), "error": str(e)}
            continue
        finally:
            g.gff_destroy(h)
        out["mode%d" % mode] = {
            "s_per_increment": dt / hist.nsteps,
            "newton_mean": float(np.mean([r.newton_iters for r in reps])),
            "cg_mean": float(np.mean([r.cg_iters for r in reps])),
            "cuts": int(sum(r.cuts for r in reps)),
            "residual_first_mean": float(np.mean([r.residual_first for r in reps])),
            "warm_used": int(sum(r.warm_start_used for r in reps)),
            "P11_MPa_last": float(Pm[-1][0] / 1e6),
            "newton_per_increment": [r.newton_iters for r in reps],
            "residual_first": [r.residual_first for r in reps],
        }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-rves", type=int, default=4)
    ap.add_argument("--train-increments", type=int, default=80)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-n", type=int, default=128)
    ap.add_argument("--eval-grains", type=int, default=500)
    ap.add_argument("--eval-increments", type=int, default=20)
    ap.add_argument("--weights", default=None, help="save the trained weights here")
    ap.add_argument("--sampling", type=int, default=1,
                    help="0: shuffled epochs; 1: samples drawn in proportion to their target energy (half uniform)")
    a = ap.parse_args()
    u = g.gff_unet_create(1)
    try:
        t0 = time.perf_counter()
        collect(u, [5000 + i for i in range(a.train_rves)], increments=a.train_increments)
        t1 = time.perf_counter()
        g.gff_unet_set_sampling(u, a.sampling)
        losses = g.gff_unet_train(u, a.steps, a.lr)
        t2 = time.perf_counter()
        if a.weights:
            g.gff_unet_save(u, a.weights)
        print(json.dumps({"samples": g.gff_unet_num_samples(u), "data_s": t1 - t0, "train_s": t2 - t1,
                          "loss_curve": [float(np.mean(c)) for c in np.array_split(losses, 10)]}), flush=True)
        ev = evaluate(u, a.eval_n, a.eval_grains, increments=a.eval_increments)
        print(json.dumps({
            "samples": g.gff_unet_num_samples(u), "data_s": t1 - t0, "train_s": t2 - t1,
            "train_steps": a.steps, "loss_first": float(np.mean(losses[:50])), "loss_last": float(np.mean(losses[-50:])),
            "loss_curve": [float(np.mean(c)) for c in np.array_split(losses, 10)],
            "eval": ev,
        }))
    finally:
        g.gff_unet_destroy(u)


if __name__ == "__main__":
    main()
