"""Parity of whole load increments (Sect. 2.1 Newton-CG, Sect. 3.2 material
update, Sect. 3.3 FIPs) between the CUDA library and the oracle, on the
same seeded microstructures and loading histories.

Tolerances: macroscopic P relative 1e-10 (FP64) / 1e-5 (mixed), voxel
fields relative L2 1e-8 (FP64) / 1e-4 (mixed), FIPs relative 1e-3.  Both
sides run Newton to 1e-11 so that the comparison measures the solution, not
the stopping point."""

import os

import numpy as np
import pytest

from gpu_helpers import gff, gpu_materials, oracle_materials, rel_l2, torch_cuda
from oracle import spectral as sp
from oracle.solver import OracleRVE, Options, SVK_CUBIC, SVK_ISO, CP_FCC
from rve_inputs import cyclic_history, polycrystal, polycrystal_with_particles, ramp_history

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _run_pair(ms, kinds, hist, kind=sp.KIND_CONTINUOUS, precision=0, newton_tol=TOL, cg_tol=TOL):
    torch_cuda()
    g = gff()
    o = OracleRVE(ms, oracle_materials(kinds), Options(projection=kind, newton_tol=newton_tol, cg_tol=cg_tol))
    orep = o.run(hist)
    h = g.create_rve(ms, gpu_materials(kinds),
                     g.make_options(projection=kind, precision=precision, newton_tol=newton_tol, cg_tol=cg_tol))
    try:
        Pm, reps = g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        N = ms.n_voxels
        fields = {w: g.gff_get_field(h, w, N) for w in (g.GFF_FIELD_F, g.GFF_FIELD_P, g.GFF_FIELD_FP_INV,
                                                        g.GFF_FIELD_CHI)}
        fips = g.gff_get_fips(h, ms.ngrains)
    finally:
        g.gff_destroy(h)
    return o, orep, Pm, reps, fields, fips


def _macro_err(Pm, orep):
    ref = np.array([r["Pmacro"] for r in orep])
    return max(np.linalg.norm(Pm[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(len(orep)))


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_config1_svk_mixed_control_fp64(kind):
    """16^3, 8 Voronoi grains, cubic SVK, F11 ramped to 1.01 in 5 steps with
    zero average stress on the other components."""
    ms = polycrystal(16, 8, 1)
    o, orep, Pm, reps, f, _ = _run_pair(ms, {0: SVK_CUBIC}, ramp_history(), kind)
    g = gff()
    assert _macro_err(Pm, orep) <= 1e-10
    assert rel_l2(f[g.GFF_FIELD_F], o.F.reshape(9, -1)) <= 1e-8
    assert rel_l2(f[g.GFF_FIELD_P], o.P.reshape(9, -1)) <= 1e-8
    assert all(r.residual <= TOL for r in reps)
    # the stress-controlled averages are zero, F32 stays at its prescribed 0
    assert np.abs(Pm[-1][1:7]).max() <= 1e-6 * abs(Pm[-1][0])
    assert abs(reps[-1].Fmacro[7]) < 1e-14


def test_config1_mixed_precision():
    ms = polycrystal(16, 8, 1)
    o, orep, Pm, reps, f, _ = _run_pair(ms, {0: SVK_CUBIC}, ramp_history(), precision=1, newton_tol=1e-9,
                                        cg_tol=1e-6)
    g = gff()
    assert _macro_err(Pm, orep) <= 1e-5
    assert rel_l2(f[g.GFF_FIELD_F], o.F.reshape(9, -1)) <= 1e-4
    assert rel_l2(f[g.GFF_FIELD_P], o.P.reshape(9, -1)) <= 1e-4


def test_homogeneous_medium_converges_without_newton_correction():
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 1, 3)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(newton_tol=1e-12))
    try:
        Fbar = np.eye(3) + np.array([[0.01, 0.002, 0], [0.001, -0.003, 0.004], [0, 0.002, 0.005]])
        rep = g.gff_step(h, 1.0, Fbar.reshape(9), np.zeros(9, np.uint8), np.zeros(9))
        assert rep.newton_iters == 0
        F = g.gff_get_field(h, g.GFF_FIELD_F, 512).reshape(9, -1)
        assert np.abs(F - Fbar.reshape(9, 1)).max() < 1e-15
    finally:
        g.gff_destroy(h)


CP_HIST = cyclic_history(0.01, 1).head(14)  # through yield, 14 of the 20 increments up to the first peak


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_crystal_plasticity_increments_fp64(kind):
    ms = polycrystal(8, 4, 21)
    o, orep, Pm, reps, f, fips = _run_pair(ms, {0: CP_FCC}, CP_HIST, kind)
    g = gff()
    assert _macro_err(Pm, orep) <= 1e-10
    assert rel_l2(f[g.GFF_FIELD_F], o.F.reshape(9, -1)) <= 1e-8
    assert rel_l2(f[g.GFF_FIELD_P], o.P.reshape(9, -1)) <= 1e-8
    Fpi_ref = o.Fpi.transpose(1, 2, 0).reshape(9, -1)
    I9 = np.eye(3).reshape(9, 1)
    assert rel_l2(f[g.GFF_FIELD_FP_INV].reshape(9, -1) - I9, Fpi_ref - I9) <= 1e-7
    assert rel_l2(f[g.GFF_FIELD_CHI].reshape(12, -1), o.chi.T) <= 1e-7
    pc, w, fs = o.grain_fips()
    assert rel_l2(fips[0], pc) <= 1e-3
    assert rel_l2(fips[1], w) <= 1e-3
    assert rel_l2(fips[2], fs) <= 1e-3
    assert (pc > 0).all()


def test_crystal_plasticity_mixed_precision():
    ms = polycrystal(8, 4, 21)
    o, orep, Pm, reps, f, fips = _run_pair(ms, {0: CP_FCC}, CP_HIST, precision=1, newton_tol=1e-9, cg_tol=1e-6)
    g = gff()
    assert _macro_err(Pm, orep) <= 1e-5
    assert rel_l2(f[g.GFF_FIELD_F], o.F.reshape(9, -1)) <= 1e-4
    pc, w, fs = o.grain_fips()
    assert rel_l2(fips[0], pc) <= 1e-3


def test_two_phase_particles_discrete_projection():
    ms = polycrystal_with_particles(16, 6, 3, radius=3, frac=0.05)
    assert (ms.grain_id == ms.ngrains - 1).sum() >= 0.05 * ms.n_voxels
    hist = cyclic_history(0.008, 1).head(8)
    o, orep, Pm, reps, f, fips = _run_pair(ms, {0: CP_FCC, 1: SVK_ISO}, hist, sp.KIND_DISCRETE)
    g = gff()
    assert _macro_err(Pm, orep) <= 1e-10
    assert rel_l2(f[g.GFF_FIELD_F], o.F.reshape(9, -1)) <= 1e-8
    pc, w, fs = o.grain_fips()
    assert fips[0][-1] == 0.0 and pc[-1] == 0.0  # the particle phase carries no FIP
    assert rel_l2(fips[0], pc) <= 1e-3


def test_save_load_resume_is_bitwise(tmp_path):
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 4, 21)
    hist = CP_HIST
    mats = gpu_materials({0: CP_FCC})

    def run(h, a, b):
        return g.gff_run_history(h, hist.dt[a:b], hist.Fbar[a:b], hist.mask[a:b], hist.Pbar[a:b])[0]

    h1 = g.create_rve(ms, mats, g.make_options(newton_tol=1e-9))
    h2 = g.create_rve(ms, mats, g.make_options(newton_tol=1e-9))
    try:
        run(h1, 0, 6)
        path = os.path.join(str(tmp_path), "state.bin")
        g.gff_save_state(h1, path)
        a = run(h1, 6, 9)
        g.gff_load_state(h2, path)
        b = run(h2, 6, 9)
        assert np.array_equal(a, b)
        for w in (g.GFF_FIELD_F, g.GFF_FIELD_FP_INV, g.GFF_FIELD_CHI):
            assert np.array_equal(g.gff_get_field(h1, w, 512), g.gff_get_field(h2, w, 512))
    finally:
        g.gff_destroy(h1)
        g.gff_destroy(h2)


def test_cut_back_reaches_the_uncut_solution():
    """A hyperelastic increment too large for a small Newton budget is split
    into halves; the elastic solution does not depend on the path, so the cut
    step must end where one generous uncut step ends.  Without cuts the same
    step fails and leaves the committed state unchanged."""
    torch_cuda()
    g = gff()
    ms = polycrystal(16, 6, 41)
    mats = gpu_materials({0: SVK_CUBIC})
    N = ms.n_voxels
    Fbar = np.eye(3).ravel().copy()
    Fbar[0] += 0.08
    Fbar[4] -= 0.03
    mask = np.zeros(9, np.uint8)
    Pbar = np.zeros(9)

    def run(newton_max, max_cuts):
        h = g.create_rve(ms, mats, g.make_options(newton_tol=1e-10, cg_tol=1e-4, newton_max=newton_max,
                                                  max_cuts=max_cuts))
        try:
            try:
                rep = g.gff_step(h, 1.0, Fbar, mask, Pbar)
            except g.GffError as e:
                return e.status, None, g.gff_get_field(h, g.GFF_FIELD_F, N)
            return 0, rep, g.gff_get_field(h, g.GFF_FIELD_F, N)
        finally:
            g.gff_destroy(h)

    st, ref, F_ref = run(60, 0)
    assert st == 0 and ref.cuts == 0
    for m in range(ref.newton_iters - 1, 0, -1):
        st0, _, F0 = run(m, 0)
        assert st0 == g.GFF_ERR_NO_CONVERGENCE
        assert np.array_equal(F0, np.tile(np.eye(3).reshape(9, 1), (1, N)).ravel())  # nothing committed
        st, rep, F = run(m, 4)
        if st == 0:
            assert rep.cuts >= 1
            assert np.allclose(rep.Fmacro, Fbar, rtol=0, atol=1e-12)
            assert rel_l2(F, F_ref) <= 1e-8
            assert np.linalg.norm(np.array(rep.Pmacro) - ref.Pmacro) <= 1e-8 * np.linalg.norm(ref.Pmacro)
            break
    else:
        pytest.fail("no Newton budget below %d iterations was rescued by cut-back" % ref.newton_iters)
