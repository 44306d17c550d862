"""Automatic time incrementation (gff_run_auto; Sect. 2.3 names an automatic
incrementation algorithm, the rule is the FE-style one stated in gff.h).

  * The controller: on an elastic path every accepted increment follows the
    stated rule (grow after an easy increment, never across a knot, clamped
    to dt_max), the knots are hit exactly and the path ends at its last knot.
  * Parity: the increments the controller picks on a crystal-plasticity
    cycle (+-0.5 %, one load reversal per half cycle) are run by the oracle;
    macroscopic P agrees to 1e-10 at every increment and the fields to 1e-8.
"""

import numpy as np
import pytest

from gpu_helpers import gff, gpu_materials, oracle_materials, rel_l2, torch_cuda
from oracle.solver import CP_FCC, SVK_CUBIC, OracleRVE, Options
from rve_inputs import polycrystal
from rve_inputs.loading import isochoric

pytestmark = pytest.mark.gpu


def _path(amplitudes, period=4.0):
    """Knots of a triangular F11 history: F11 = 1 + e at t = k period / 4."""
    e = np.asarray(amplitudes, dtype=np.float64)
    t = np.arange(len(e)) * period / 4
    return t, np.stack([isochoric(1.0 + x) for x in e])


def _targets(t, tk, Fk):
    return np.stack([np.interp(t, tk, Fk[:, c]) for c in range(9)], axis=1)


def test_controller_follows_its_rule_on_an_elastic_path():
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 4, 7)
    # (an elastic path ending back at F = I would end at P = 0, where the relative residual
    # ||b|| / ||P|| of the stopping test has no meaning; this one ends at 0.2 %)
    tk, Fk = _path([0.0, 0.004, 0.002])
    h = g.create_rve(ms, gpu_materials({0: SVK_CUBIC}), g.make_options(newton_tol=1e-10, cg_tol=1e-8))
    try:
        ao = g.gff_auto_options_default(dt_initial=0.05, dt_max=0.4, grow=1.5, easy_newton=3, hard_newton=8)
        t, Pm, reps = g.gff_run_auto(h, tk, Fk, np.zeros(9, np.uint8), np.zeros_like(Fk), options=ao)
        Fm = np.array(reps[-1].Fmacro)
    finally:
        g.gff_destroy(h)
    assert abs(t[-1] - tk[-1]) < 1e-12 and np.any(np.abs(t - tk[1]) < 1e-12)
    assert np.all(np.diff(np.r_[0.0, t]) > 0)
    assert np.allclose(Fm, Fk[-1], rtol=0, atol=1e-13)
    # replay the rule on the reported Newton counts
    dt, prev = 0.05, 0.0
    for k, r in enumerate(reps):
        seg_end = tk[1] if prev < tk[1] - 1e-12 else tk[2]
        want = min(prev + dt, seg_end)
        assert abs(t[k] - want) < 1e-12, (k, t[k], want)
        taken = t[k] - prev
        assert r.cuts == 0
        if r.newton_iters <= 3 and taken >= 0.999 * dt:
            dt = min(dt * 1.5, 0.4)
        elif r.newton_iters >= 8:
            dt = dt * 0.75
        prev = t[k]
    assert len(reps) < 2 / 0.05  # fewer increments than a fixed dt_initial would take


def test_auto_increments_match_the_oracle_on_a_plastic_cycle():
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 4, 21)
    tk, Fk = _path([0.0, 0.005, 0.0, -0.005, 0.0])
    tol = 1e-11
    h = g.create_rve(ms, gpu_materials({0: CP_FCC}), g.make_options(newton_tol=tol, cg_tol=tol))
    try:
        ao = g.gff_auto_options_default(dt_initial=0.05, dt_max=1.0 / 3.0, easy_newton=3, hard_newton=8)
        cs = np.array([1, 0, 0, 0, 0], np.uint8)
        t, Pm, reps = g.gff_run_auto(h, tk, Fk, np.zeros(9, np.uint8), np.zeros_like(Fk), cs, ao)
        N = ms.n_voxels
        F = g.gff_get_field(h, g.GFF_FIELD_F, N)
        P = g.gff_get_field(h, g.GFF_FIELD_P, N)
    finally:
        g.gff_destroy(h)
    assert all(r.cuts == 0 for r in reps)
    assert len(reps) < 80  # the fixed-increment history of this cycle takes 80
    dts = np.diff(np.r_[0.0, t])
    assert dts.max() > 2 * dts.min()  # the controller did change the step
    o = OracleRVE(ms, oracle_materials({0: CP_FCC}), Options(newton_tol=tol, cg_tol=tol))
    targets = _targets(t, tk, Fk)
    ref = []
    for k in range(len(t)):
        ref.append(o.step(dts[k], targets[k], np.zeros(9, np.uint8), np.zeros(9))["Pmacro"])
    ref = np.array(ref)
    err = max(np.linalg.norm(Pm[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(len(t)))
    assert err <= 1e-10
    assert rel_l2(F, o.F.reshape(9, -1)) <= 1e-8
    assert rel_l2(P, o.P.reshape(9, -1)) <= 1e-8
