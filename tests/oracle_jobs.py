"""Oracle runs of the long GPU parity tests, executed in worker processes.

TEST INFRASTRUCTURE ONLY: this module calls oracle/ and rve_inputs/ and
nothing else (no torch, no CUDA).  The tests start a process pool with the
`spawn` method before their first GPU call and submit every run at once, so
the slow CPU runs overlap each other and the GPU work.

A case is described by plain tuples so that it pickles:
  ms    ("poly", n, ngrains, seed) | ("particles", n, ngrains, seed)
        (n an int or (nz, ny, nx); particles: radius 3, 5 % volume)
  kinds {phase: oracle material kind}
  hist  ("cyclic", eps, cycles, incr_per_quarter, nsteps)
  proj  oracle projection kind
  snaps increments after which the per-grain FIPs are recorded
"""

import concurrent.futures
import multiprocessing
import os

import numpy as np


def microstructure(spec):
    from rve_inputs import polycrystal, polycrystal_with_particles

    kind, n, ngrains, seed = spec
    if kind == "poly":
        return polycrystal(n, ngrains, seed)
    if kind == "particles":
        return polycrystal_with_particles(n, ngrains, seed, radius=3, frac=0.05)
    raise ValueError(spec)


def history(spec):
    from rve_inputs import cyclic_history

    kind, eps, cycles, ipq, nsteps = spec
    assert kind == "cyclic"
    return cyclic_history(eps, cycles, incr_per_quarter=ipq).head(nsteps)


BAND_WIDTHS = (1.0, 2.5)  # band widths of the W_cyc^b comparisons, in voxel spacings along x


def run_case(ms_spec, kinds, hist_spec, proj, snaps=(), newton_tol=1e-11):
    """The oracle's run of one case: macroscopic P per increment, the final
    fields, the per-grain FIPs after the increments in `snaps` and the
    band-averaged W_cyc (Eq. Wmax) of the final state for BAND_WIDTHS."""
    from oracle.solver import Material, OracleRVE, Options

    ms = microstructure(ms_spec)
    hist = history(hist_spec)
    o = OracleRVE(ms, {ph: Material(k) for ph, k in kinds.items()},
                  Options(projection=proj, newton_tol=newton_tol, cg_tol=newton_tol))
    fips = {}

    def snap(k, rep):
        if k in snaps:
            fips[k] = o.grain_fips()

    reps = o.run(hist, on_step=snap)
    N = ms.n_voxels
    return {
        "Pmacro": np.array([r["Pmacro"] for r in reps]),
        "newton": [r["newton"] for r in reps],
        "F": o.F.reshape(9, N),
        "P": o.P.reshape(9, N),
        "Fpi": o.Fpi.transpose(1, 2, 0).reshape(9, N),
        "chi": o.chi.T.copy(),
        "fips": fips,
        "band": {k: o.band_fips(k * ms.L[0] / ms.nx) for k in BAND_WIDTHS},
    }


def start_pool(jobs, max_workers=None):
    """Submits {name: (fn, args)} to a spawn process pool; returns the pool
    and {name: future}.  Worker BLAS threads are limited to one each."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    workers = max_workers or max(1, min(len(jobs), os.cpu_count() or 1))
    pool = concurrent.futures.ProcessPoolExecutor(max_workers=workers,
                                                  mp_context=multiprocessing.get_context("spawn"))
    futures = {name: pool.submit(fn, *args) for name, (fn, args) in jobs.items()}
    return pool, futures
