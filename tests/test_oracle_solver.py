"""Pins of the oracle's Newton-CG increment (Sect. 2.1) and of its FIPs
(Sect. 3.3): exact solutions (homogeneous medium, laminate), a 0-D solve of
the mixed macroscopic control, quadratic Newton convergence (Sect. 2, the
consistent tangent), Voigt/Reuss bounds, and hand-computed FIP values."""

import numpy as np
import pytest

from oracle import materials as mat
from oracle import spectral as sp
from oracle import fips
from oracle.solver import OracleRVE, Material, Options, SVK_CUBIC, SVK_ISO, CP_FCC
from rve_inputs import Microstructure, polycrystal

C11, C12, C44 = 168.4e9, 121.4e9, 75.4e9


def _ms(gid, quats, phase=None):
    nz, ny, nx = gid.shape
    ng = quats.shape[0]
    ph = np.zeros(ng, dtype=np.int32) if phase is None else np.asarray(phase, dtype=np.int32)
    return Microstructure(nx, ny, nz, (1.0, 1.0, 1.0), gid.astype(np.int32), quats, ph)


def test_homogeneous_medium_is_affine_and_converged_at_iteration_zero():
    q = np.array([[0.8, 0.2, -0.4, 0.4]])
    q /= np.linalg.norm(q)
    rve = OracleRVE(_ms(np.zeros((4, 6, 8), dtype=int), q), {0: Material(SVK_CUBIC)}, Options(newton_tol=1e-12))
    Fbar = np.eye(3) + np.array([[0.01, 0.002, 0], [0.001, -0.003, 0.004], [0, 0.002, 0.005]])
    rep = rve.step(1.0, Fbar.reshape(9), np.zeros(9), np.zeros(9))
    assert rep["newton"] == 0
    assert np.abs(rve.F - Fbar[:, :, None, None, None]).max() < 1e-15
    C = mat.rotate4(mat.cubic_stiffness(C11, C12, C44), mat.quat_to_rot(q[0]))
    P, _ = mat.svk(Fbar[None], C)
    assert np.abs(rep["Pmacro"] - P.reshape(9)).max() <= 1e-14 * np.abs(P).max()


def _laminate_exact(Fbar, CA, CB):
    """Two equal layers normal to x: F = Fbar +- a (x) e1, traction P.e1
    continuous.  Solved by an independent 3-unknown Newton with a
    finite-difference Jacobian."""
    def traction_jump(a):
        FA = Fbar + np.outer(a, [1, 0, 0])
        FB = Fbar - np.outer(a, [1, 0, 0])
        return mat.svk(FA[None], CA)[0][0][:, 0] - mat.svk(FB[None], CB)[0][0][:, 0]

    a = np.zeros(3)
    for _ in range(50):
        r = traction_jump(a)
        J = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-7
            J[:, k] = (traction_jump(a + e) - traction_jump(a - e)) / 2e-7
        da = np.linalg.solve(J, -r)
        a += da
        if np.abs(da).max() < 1e-16:
            break
    return a


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_laminate_closed_form(kind):
    nz, ny, nx = 4, 4, 16
    gid = np.zeros((nz, ny, nx), dtype=int)
    gid[:, :, 8:] = 1  # layers of width 8 starting at even index: no Nyquist content
    quats = np.array([[1.0, 0, 0, 0], [np.cos(0.4), 0.3 * np.sin(0.4), 0.5 * np.sin(0.4), np.sqrt(0.66) * np.sin(0.4)]])
    rve = OracleRVE(_ms(gid, quats), {0: Material(SVK_CUBIC)}, Options(projection=kind, newton_tol=1e-13, cg_tol=1e-14))
    Fbar = np.eye(3) + np.array([[0.006, 0.001, 0.0], [0.0, -0.002, 0.001], [0.002, 0.0, -0.002]])
    rve.step(1.0, Fbar.reshape(9), np.zeros(9), np.zeros(9))
    Rb = mat.quat_to_rot(quats[1])
    CA = mat.cubic_stiffness(C11, C12, C44)
    CB = mat.rotate4(CA, Rb)
    a = _laminate_exact(Fbar, CA, CB)
    assert np.abs(a).max() > 1e-4
    FA = Fbar + np.outer(a, [1, 0, 0])
    FB = Fbar - np.outer(a, [1, 0, 0])
    exact = np.where((gid == 0)[None, None], FA[:, :, None, None, None], FB[:, :, None, None, None])
    assert np.abs(rve.F - exact).max() <= 1e-11


def test_mixed_control_matches_zero_dimensional_solve():
    q = np.array([[0.9, 0.1, 0.3, 0.2]])
    q /= np.linalg.norm(q)
    rve = OracleRVE(_ms(np.zeros((4, 4, 4), dtype=int), q), {0: Material(SVK_CUBIC)},
                    Options(newton_tol=1e-12, cg_tol=1e-11))
    mask = np.ones(9)
    mask[0] = 0
    mask[7] = 0  # F32 held: removes the free rotation about the loading axis
    Fbar = np.eye(3).reshape(9).copy()
    Fbar[0] = 1.01
    rep = rve.step(1.0, Fbar, mask, np.zeros(9))
    C = mat.rotate4(mat.cubic_stiffness(C11, C12, C44), mat.quat_to_rot(q[0]))
    # 0-D: find the 8 free components with P_c = 0 for every stress-controlled c
    free = np.nonzero(mask)[0]
    F = np.eye(3).reshape(9).copy()
    F[0] = 1.01

    def r(F):
        return mat.svk(F.reshape(1, 3, 3), C)[0].reshape(9)[free]

    for _ in range(30):
        J = np.zeros((7, 7))
        for k, c in enumerate(free):
            e = np.zeros(9)
            e[c] = 1e-7
            J[:, k] = (r(F + e) - r(F - e)) / 2e-7
        F[free] -= np.linalg.solve(J, r(F))
    assert np.abs(rep["Fmacro"] - F).max() <= 1e-10
    P0 = mat.svk(F.reshape(1, 3, 3), C)[0].reshape(9)
    assert np.abs(rep["Pmacro"] - P0).max() <= 1e-8 * abs(P0[0])
    # uniaxial: the held component carries no stress either
    assert abs(P0[7]) <= 1e-8 * abs(P0[0]) and abs(rep["Pmacro"][7]) <= 1e-8 * abs(P0[0])


def test_newton_converges_quadratically_with_the_consistent_tangent():
    ms = polycrystal(8, 6, 11)
    rve = OracleRVE(ms, {0: Material(SVK_CUBIC)}, Options(newton_tol=1e-11, cg_tol=1e-11))
    Fbar = np.eye(3).reshape(9).copy()
    Fbar[0] = 1.08
    Fbar[4] = Fbar[8] = 1.08 ** -0.5
    rep = rve.step(1.0, Fbar, np.zeros(9), np.zeros(9))
    r = [x for x in rep["res"] if x > 1e-10]
    assert len(r) >= 3
    ratios = [r[i + 1] / r[i] ** 2 for i in range(len(r) - 1)]
    assert max(ratios) < 20.0, ratios


def _mandel(C):
    idx = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    w = [1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)]
    return np.array([[C[a + b] * w[i] * w[j] for j, b in enumerate(idx)] for i, a in enumerate(idx)])


def test_effective_stiffness_within_voigt_and_reuss_bounds():
    ms = polycrystal(8, 8, 12)
    rve = OracleRVE(ms, {0: Material(SVK_CUBIC)}, Options(newton_tol=1e-10, cg_tol=1e-10))
    eps = 1e-4  # small enough for the linear bounds, large enough that E = (F^T F - I)/2 keeps 12 digits
    Fbar = np.eye(3).reshape(9).copy()
    Fbar[0] += eps
    rep = rve.step(1.0, Fbar, np.zeros(9), np.zeros(9))
    ceff = rep["Pmacro"][0] / eps
    R = mat.quat_to_rot(ms.quat)
    Cc = mat.cubic_stiffness(C11, C12, C44)
    vol = np.bincount(ms.grain_id.ravel(), minlength=ms.ngrains) / ms.n_voxels
    Ms = [_mandel(mat.rotate4(Cc, R[g])) for g in range(ms.ngrains)]
    CV = sum(v * M for v, M in zip(vol, Ms))
    CR = np.linalg.inv(sum(v * np.linalg.inv(M) for v, M in zip(vol, Ms)))
    assert CR[0, 0] * (1 - 1e-3) <= ceff <= CV[0, 0] * (1 + 1e-3)
    assert CV[0, 0] - CR[0, 0] > 0.05 * CV[0, 0]  # the bounds are not trivially tight
    # the polycrystal is stiffer than the compliant bound by a clear margin
    assert ceff > CR[0, 0] * 1.001 and ceff < CV[0, 0] * 0.999


def test_fip_single_slip_values():
    s, m = mat.fcc_slip_systems()
    S0 = np.einsum("ai,aj->aij", s, m)
    acc = fips.new_accumulators(1)
    fips.reset(acc)
    dg = np.zeros((1, 12))
    dg[0, 4] = 3e-4
    tau = np.full((1, 12), 60e6)
    P = np.diag([200e6, 0, 0])[None]
    F = np.eye(3)[None]
    fips.accumulate(acc, np.array([0]), dg, tau, S0, m, P, F)
    # |sym(s (x) m)|^2 = 1/2 for orthonormal s, m  ->  sqrt(2/3 * dg^2 / 2) = dg / sqrt(3)
    assert abs(acc["pcyc"][0] - 3e-4 / np.sqrt(3)) < 1e-18
    assert abs(acc["w"][0, 4] - 60e6 * 3e-4) < 1e-6 and acc["w"][0, 0] == 0
    # sigma = P for F = I: normal stress on the (111)-type plane = 200 MPa * m_x^2 = 200/3 MPa
    assert np.allclose(acc["sn"][0], 200e6 / 3)
    fips.accumulate(acc, np.array([0]), -2 * dg, tau, S0, m, P, F)
    assert abs(acc["gmax"][0, 4] - 3e-4) < 1e-18 and abs(acc["gmin"][0, 4] + 3e-4) < 1e-18
    pc, w, fs = fips.grain_fips(acc, np.array([0]), 1, np.array([True]), fs_k=0.5, fs_sigma_y=100e6)
    # FS = (dgamma/2)(1 + k sn/sigma_y) on the system with the largest value
    assert abs(fs[0] - 0.5 * 6e-4 * (1 + 0.5 * (200e6 / 3) / 100e6)) < 1e-15
    assert abs(pc[0] - 3 * 3e-4 / np.sqrt(3)) < 1e-15


@pytest.mark.slow
def test_cp_polycrystal_increment_runs_and_conserves_macro_strain():
    ms = polycrystal(8, 4, 21)
    rve = OracleRVE(ms, {0: Material(CP_FCC)}, Options(newton_tol=1e-9, cg_tol=1e-10))
    from rve_inputs import cyclic_history

    h = cyclic_history(0.01, 1).head(12)
    reps = rve.run(h)
    assert all(r["converged"] for r in reps)
    assert np.abs(reps[-1]["Fmacro"] - h.Fbar[11]).max() < 1e-13
    pc, w, fs = rve.grain_fips()
    assert (pc > 0).all() and (fs > 0).all()


def _one_voxel_cycles(hist, S0, C, normals, cp, fs_k, fs_sigma_y, reset_each_cycle=True):
    """The same single crystal as one voxel: its return map driven by the
    prescribed F history directly (no spectral solve), with its own FIP
    accumulators (cleared at each cycle start when asked)."""
    Fpi, chi = np.eye(3)[None].copy(), np.zeros((1, 12))
    acc = fips.new_accumulators(1)
    fips.reset(acc)
    P_hist = []
    for k in range(hist.nsteps):
        if reset_each_cycle and hist.cycle_start[k]:
            fips.reset(acc)
        F = hist.Fbar[k].reshape(1, 3, 3)
        out = mat.cp_return_map(F, Fpi, chi, hist.dt[k], S0, C, cp)
        assert out["conv"].all()
        Fpi, chi = out["Fpi"], out["chi"]
        fips.accumulate(acc, np.array([0]), out["dg"], out["tau"], S0, normals, out["P"], F)
        P_hist.append(out["P"][0].reshape(9))
    pc, w, fs = fips.grain_fips(acc, np.array([0]), 1, np.array([True]), fs_k=fs_k, fs_sigma_y=fs_sigma_y)
    return np.array(P_hist), pc[0], w[0], fs[0]


def test_single_orientation_polycrystal_is_one_crystal_over_two_cycles():
    """Sect. 2.1 (the Newton-CG increment), Sect. 3.2 (Eq. gamma_dot) and
    Sect. 3.3 (FIPs accumulated over a loading cycle).
    Grains that all share one orientation make a single crystal: under two
    full strain cycles (both reversals, the accumulators cleared again at the
    second cycle start) every increment of the RVE is affine and converged at
    Newton iteration 0, its macro P is the one-voxel return map's P driven by
    the same F, and every grain's FIPs are the one-voxel FIPs of the second
    cycle alone (with the first cycle's kept they differ)."""
    from rve_inputs import cyclic_history

    rng = np.random.default_rng(5)
    gid = rng.integers(0, 3, size=(4, 4, 4))
    q = np.array([0.9, 0.3, -0.2, 0.25])
    q /= np.linalg.norm(q)
    ms = _ms(gid, np.tile(q, (3, 1)))
    opt = Options(newton_tol=1e-9, cg_tol=1e-10)
    rve = OracleRVE(ms, {0: Material(CP_FCC)}, opt)
    hist = cyclic_history(0.01, 2, incr_per_quarter=3)
    reps = rve.run(hist)
    assert all(r["converged"] and r["newton"] == 0 for r in reps)
    Fv = rve.F.reshape(9, -1)
    assert np.abs(Fv - hist.Fbar[-1][:, None]).max() < 1e-13  # uniform: the sum of the increments
    g = rve.grains[0]
    P1, pc1, w1, fs1 = _one_voxel_cycles(hist, g["S0"], g["C"], g["normals"], g["mat"].cp, opt.fs_k, opt.fs_sigma_y)
    Pm = np.array([r["Pmacro"] for r in reps])
    assert np.abs(Pm - P1).max() <= 1e-9 * np.abs(P1).max()
    assert np.abs(P1[:, 0]).max() > 1e8  # plastic: well past the elastic range, both signs
    assert P1[:, 0].min() < -1e8
    pc, w, fs = rve.grain_fips()
    assert pc1 > 0 and fs1 > 0
    assert np.allclose(pc, pc1, rtol=1e-9, atol=0) and np.allclose(fs, fs1, rtol=1e-9, atol=0)
    assert np.allclose(w, w1, rtol=1e-9, atol=1e-9 * np.abs(w1).max())
    _, pc2, _, fs2 = _one_voxel_cycles(hist, g["S0"], g["C"], g["normals"], g["mat"].cp, opt.fs_k, opt.fs_sigma_y,
                                       reset_each_cycle=False)
    assert pc2 > 1.5 * pc1  # the reset matters: two cycles' plastic strain against one
