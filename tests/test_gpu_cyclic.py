"""Parity with the oracle across the load reversals of fatigue cycles.

Fully reversed strain cycles (R = -1, Eq. eqFt with the triangular history
of reading R8) at 3 increments per quarter cycle: every run crosses a load
reversal, so elastic unloading, reversed slip against a non-zero
Armstrong-Frederick backstress (Sect. 3.2) and, over two cycles, the restart
of the per-cycle FIP accumulators (Sect. 3.3) and the gamma_max - gamma_min
range of the Fatemi-Socie parameter are all compared element by element.

  * 8^3, 2 cycles (24 increments), continuous and discrete projection, FP64
    and mixed precision; FIPs after cycle 1 and after cycle 2;
  * 8^3 with the exact-Newton return map alone (the fallback path);
  * 16^3, 15 increments (cycle 1 and the start of cycle 2), FP64 and mixed;
  * 32^3 two-phase (5 % stiff spheres), discrete projection, 5 increments
    across the first reversal;
  * gff_batch_run against the oracle: 12^3, 20^3 and a 40 x 24 x 16 RVE over
    the first reversal (radix plans 4x3, 4x5, 8x5, 8x3),
    and 48^3 with 24^3 for the first increment.

Tolerances (both sides to Newton tolerance 1e-11 in FP64): macroscopic P
relative 1e-10 (FP64) / 1e-5 (mixed); voxel fields relative L2 1e-8 /
1e-4 (Fp^-1 - I and chi, which start at zero, 1e-7); per-grain FIPs 1e-3.

The oracle runs in a spawn process pool started before this module's first
GPU call; every run is submitted at once and each test waits for its own.
"""

import numpy as np
import pytest

from gpu_helpers import gff, gpu_materials, rel_l2, torch_cuda
from oracle import spectral as sp
from oracle.solver import CP_FCC, SVK_CUBIC, SVK_ISO
from oracle_jobs import BAND_WIDTHS, history, microstructure, run_case, start_pool

pytestmark = pytest.mark.gpu

TOL = 1e-11
CONT, DISC = sp.KIND_CONTINUOUS, sp.KIND_DISCRETE
CYC2 = ("cyclic", 0.005, 2, 3, 24)  # peaks at increments 3 and 9, cycle 2 starts at 12

CASES = {
    "c8_cont": (("poly", 8, 4, 21), {0: CP_FCC}, CYC2, CONT, (11, 23)),
    "c8_disc": (("poly", 8, 4, 21), {0: CP_FCC}, CYC2, DISC, (11, 23)),
    "c16": (("poly", 16, 6, 25), {0: CP_FCC}, ("cyclic", 0.005, 2, 3, 15), CONT, (11, 14)),
    "p32": (("particles", 32, 8, 3), {0: CP_FCC, 1: SVK_ISO}, ("cyclic", 0.003, 1, 3, 5), DISC, (4,)),
    "bA0": (("poly", 12, 3, 31), {0: CP_FCC}, ("cyclic", 0.004, 1, 3, 5), CONT, (4,)),
    "bA1": (("poly", 20, 5, 32), {0: CP_FCC}, ("cyclic", 0.004, 1, 3, 5), CONT, (4,)),
    "bA2": (("poly", (16, 24, 40), 6, 33), {0: CP_FCC}, ("cyclic", 0.004, 1, 3, 5), CONT, (4,)),
    "bB0": (("poly", 48, 20, 34), {0: CP_FCC}, ("cyclic", 0.005, 1, 3, 1), CONT, (0,)),
    "bB1": (("poly", 24, 8, 35), {0: CP_FCC}, ("cyclic", 0.005, 1, 3, 1), CONT, (0,)),
}


@pytest.fixture(scope="module")
def oracle_runs():
    # the slowest runs first, so that they start at once
    order = sorted(CASES, key=lambda k: -int(np.prod(microstructure(CASES[k][0]).grain_id.shape)) *
                   history(CASES[k][2]).nsteps)
    pool, futures = start_pool({k: (run_case, CASES[k]) for k in order})
    yield futures
    pool.shutdown(wait=False, cancel_futures=True)


def _gpu_run(case, precision=0, exact=False, newton_tol=TOL, cg_tol=TOL, return_map=None):
    """The library's run of a case, in segments ending at the FIP snapshots."""
    torch_cuda()
    g = gff()
    ms_spec, kinds, hist_spec, proj, snaps = CASES[case]
    ms, hist = microstructure(ms_spec), history(hist_spec)
    h = g.create_rve(ms, gpu_materials(kinds),
                     g.make_options(projection=proj, precision=precision, newton_tol=newton_tol, cg_tol=cg_tol))
    try:
        if exact:
            g.gff_set_return_map(h, g.GFF_RETURN_MAP_EXACT)
        if return_map is not None:
            g.gff_set_return_map(h, return_map)
        Pm, reps, fips, a = [], [], {}, 0
        for b in sorted(snaps):
            sl = slice(a, b + 1)
            P, r = g.gff_run_history(h, hist.dt[sl], hist.Fbar[sl], hist.mask[sl], hist.Pbar[sl],
                                     hist.cycle_start[sl])
            Pm.append(P)
            reps += r
            fips[b] = g.gff_get_fips(h, ms.ngrains)
            a = b + 1
        N = ms.n_voxels
        fields = {w: g.gff_get_field(h, w, N) for w in (g.GFF_FIELD_F, g.GFF_FIELD_P, g.GFF_FIELD_FP_INV,
                                                        g.GFF_FIELD_CHI)}
        fields["band"] = {k: g.gff_get_band_fips(h, k * ms.L[0] / ms.nx, ms.ngrains)[0] for k in BAND_WIDTHS}
    finally:
        g.gff_destroy(h)
    return np.concatenate(Pm), reps, fields, fips


def _macro_err(Pm, ref):
    return max(np.linalg.norm(Pm[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(len(ref)))


def _compare(case, ref, Pm, reps, f, fips, mixed):
    g = gff()
    N = ref["F"].shape[1]
    assert all(r.cuts == 0 for r in reps), ("the GPU cut an increment the oracle took whole",
                                           [(k, r.cuts, r.newton_iters, r.cp_fallbacks, r.residual)
                                            for k, r in enumerate(reps) if r.cuts])
    assert _macro_err(Pm, ref["Pmacro"]) <= (1e-5 if mixed else 1e-10)
    ftol = 1e-4 if mixed else 1e-8
    assert rel_l2(f[g.GFF_FIELD_F], ref["F"]) <= ftol
    assert rel_l2(f[g.GFF_FIELD_P], ref["P"]) <= ftol
    I9 = np.eye(3).reshape(9, 1)
    itol = 1e-4 if mixed else 1e-7
    assert rel_l2(f[g.GFF_FIELD_FP_INV].reshape(9, N) - I9, ref["Fpi"] - I9) <= itol
    assert rel_l2(f[g.GFF_FIELD_CHI].reshape(12, N), ref["chi"]) <= itol
    for k, (pc, w, fs) in ref["fips"].items():
        gp, gw, gf = fips[k]
        assert rel_l2(gp, pc) <= 1e-3, (case, k)
        assert rel_l2(gw, w) <= 1e-3, (case, k)
        assert rel_l2(gf, fs) <= 1e-3, (case, k)
    if "band" in f:  # band-averaged W_cyc (Eq. Wmax) of the final state
        for k in BAND_WIDTHS:
            assert rel_l2(f["band"][k], ref["band"][k]) <= 1e-3, (case, k)
            assert (ref["band"][k] >= 0).all()


def _crosses_reversal(ref):
    """The macroscopic P11 rises to a peak and then falls: plastic loading,
    then unloading and reversed loading (an interior local maximum)."""
    p = ref["Pmacro"][:, 0]
    return bool(np.any((p[1:-1] > p[:-2]) & (p[1:-1] > p[2:])))


@pytest.mark.parametrize("case", ["c8_cont", "c8_disc"])
@pytest.mark.parametrize("precision", [0, 1])
def test_two_cycles_8cube(oracle_runs, case, precision):
    mixed = precision == 1
    Pm, reps, f, fips = _gpu_run(case, precision, newton_tol=1e-9 if mixed else TOL, cg_tol=1e-6 if mixed else TOL)
    ref = oracle_runs[case].result()
    assert _crosses_reversal(ref)
    p11 = ref["Pmacro"][:, 0]
    assert p11.min() < -0.5 * p11.max()  # reversed yielding in compression
    _compare(case, ref, Pm, reps, f, fips, mixed)
    # the second cycle restarted the accumulators: its P_cyc differs from the first's
    assert not np.allclose(fips[11][0], fips[23][0])
    # Fatemi-Socie needs a slip range; after a reversal every grain has one
    assert (fips[23][2] > 0).all()


def test_exact_return_map_matches_oracle(oracle_runs):
    """The exact-Newton return map from zero slip -- the library's fallback,
    run for every voxel -- reaches the oracle's root across both cycles."""
    Pm, reps, f, fips = _gpu_run("c8_cont", exact=True)
    assert all(r.cp_fallbacks >= 512 for r in reps)
    _compare("c8_cont", oracle_runs["c8_cont"].result(), Pm, reps, f, fips, False)


@pytest.mark.parametrize("precision", [0, 1])
def test_fp32_pre_iteration_reaches_the_oracle_root(oracle_runs, precision):
    """Return maps that iterate in FP32 first and finish in FP64 reach the
    oracle's roots across both cycles (the FP64 residual decides)."""
    mixed = precision == 1
    g = gff()
    Pm, reps, f, fips = _gpu_run("c8_cont", precision, newton_tol=1e-9 if mixed else TOL,
                                 cg_tol=1e-6 if mixed else TOL, return_map=g.GFF_RETURN_MAP_F32_FIRST)
    _compare("c8_cont", oracle_runs["c8_cont"].result(), Pm, reps, f, fips, mixed)


@pytest.mark.parametrize("precision", [0, 1])
def test_default_return_map_is_f32_first_in_mixed_and_fp64_in_fp64(precision):
    """GFF_RETURN_MAP_DEFAULT runs the FP32 pre-iteration in mixed precision and
    the FP64 iteration alone in FP64: bit for bit the explicit modes."""
    g = gff()
    mixed = precision == 1
    kw = dict(newton_tol=1e-9 if mixed else TOL, cg_tol=1e-6 if mixed else TOL)
    a = _gpu_run("c8_cont", precision, **kw)
    b = _gpu_run("c8_cont", precision, return_map=g.GFF_RETURN_MAP_F32_FIRST if mixed else g.GFF_RETURN_MAP_FP64,
                 **kw)
    c = _gpu_run("c8_cont", precision, return_map=g.GFF_RETURN_MAP_FP64 if mixed else g.GFF_RETURN_MAP_F32_FIRST,
                 **kw)
    F, FPI = g.GFF_FIELD_F, g.GFF_FIELD_FP_INV
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[2][F], b[2][F]) and np.array_equal(a[2][FPI], b[2][FPI])
    # the other mode iterates differently: the same root to the tolerances, not the same bits
    assert not np.array_equal(a[2][FPI], c[2][FPI])
    assert np.abs(a[0] - c[0]).max() <= 1e-6 * np.abs(a[0]).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_cycle_and_restart_16cube(oracle_runs, precision):
    mixed = precision == 1
    Pm, reps, f, fips = _gpu_run("c16", precision, newton_tol=1e-9 if mixed else TOL, cg_tol=1e-6 if mixed else TOL)
    ref = oracle_runs["c16"].result()
    assert _crosses_reversal(ref)
    _compare("c16", ref, Pm, reps, f, fips, mixed)


def test_two_phase_32cube_across_reversal(oracle_runs):
    Pm, reps, f, fips = _gpu_run("p32")
    ref = oracle_runs["p32"].result()
    assert _crosses_reversal(ref)
    _compare("p32", ref, Pm, reps, f, fips, False)
    pc = fips[4][0]
    assert pc[-1] == 0.0 and ref["fips"][4][0][-1] == 0.0  # the particle phase carries no FIP


def _batch_vs_oracle(oracle_runs, cases):
    torch_cuda()
    g = gff()
    hs = []
    try:
        for c in cases:
            ms_spec, kinds, _, proj, _ = CASES[c]
            hs.append(g.create_rve(microstructure(ms_spec), gpu_materials(kinds),
                                   g.make_options(projection=proj, newton_tol=TOL, cg_tol=TOL)))
        hist = history(CASES[cases[0]][2])
        Pm, reps, stat = g.gff_batch_run(hs, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        assert (stat == 0).all()
        for r, c in enumerate(cases):
            ms = microstructure(CASES[c][0])
            N = ms.n_voxels
            ref = oracle_runs[c].result()
            f = {w: g.gff_get_field(hs[r], w, N) for w in (g.GFF_FIELD_F, g.GFF_FIELD_P, g.GFF_FIELD_FP_INV,
                                                           g.GFF_FIELD_CHI)}
            k = max(CASES[c][4])
            fips = {k: g.gff_get_fips(hs[r], ms.ngrains)}
            _compare(c, ref, Pm[r], reps[r], f, fips, False)
    finally:
        for h in hs:
            g.gff_destroy(h)


def test_batch_matches_oracle_across_reversal(oracle_runs):
    _batch_vs_oracle(oracle_runs, ["bA0", "bA1", "bA2"])


def test_batch_matches_oracle_48cube(oracle_runs):
    _batch_vs_oracle(oracle_runs, ["bB0", "bB1"])
