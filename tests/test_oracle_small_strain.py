"""Pins of the oracle's small-strain variant (the paper's solver runs at small
and finite strains, Sect. 2.3): the projection G^s onto compatible symmetric
strain fields and the linear-elastic solve built on it.

  * G^s is idempotent, self-adjoint and returns symmetric fields;
  * it keeps a compatible strain sym(a (x) grad) cos(2 pi k.x) of one Fourier
    mode and removes a symmetric field whose rows are orthogonal to k (a
    divergence-free stress);
  * a two-phase isotropic laminate reaches the closed-form solution
    eps_p = eps_bar + sym(a_p (x) e1), sum f_p a_p = 0, continuous traction
    sigma e1 (acoustic tensors Q_p,ik = C_p,i1k1);
  * uniaxial stress on a homogeneous isotropic body gives eps22 = eps33 =
    -nu eps11 and sigma11 = E eps11 after one linear solve;
  * a homogeneous body under a prescribed strain needs no correction at all.
"""

import numpy as np

from oracle import materials as mat
from oracle import spectral as sp
from oracle.solver import SVK_CUBIC, SVK_ISO, Material, OracleRVE, Options
from rve_inputs import Microstructure, polycrystal, standard_normal


def _sym_field(seed, shape):
    a = standard_normal(seed, 9 * int(np.prod(shape))).reshape((3, 3) + shape)
    return 0.5 * (a + a.transpose(1, 0, 2, 3, 4))


def test_projection_is_a_symmetric_orthogonal_projector():
    shape = (6, 8, 10)
    L = (1.0, 2.0, 0.5)
    for kind in (sp.KIND_CONTINUOUS, sp.KIND_DISCRETE):
        A, B = _sym_field(1, shape), _sym_field(2, shape)
        PA = sp.G_sym(A, L, kind)
        assert np.abs(PA - PA.transpose(1, 0, 2, 3, 4)).max() <= 1e-14 * np.abs(PA).max()
        assert np.abs(sp.G_sym(PA, L, kind) - PA).max() <= 1e-13 * np.abs(PA).max()
        assert abs(np.vdot(B, PA) - np.vdot(sp.G_sym(B, L, kind), A)) <= 1e-12 * abs(np.vdot(B, PA))


def test_compatible_strain_kept_and_divergence_free_stress_removed():
    n = 8
    shape = (n, n, n)
    idx = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    k = np.array([1, 2, -1])  # mode numbers along x, y, z (box of length 1)
    th = 2 * np.pi * (k[0] * x + k[1] * y + k[2] * z)
    grad = 2 * np.pi * k.astype(float)
    a = np.array([0.3, -0.7, 0.2])
    eps = 0.5 * (np.outer(a, grad) + np.outer(grad, a))[:, :, None, None, None] * np.cos(th)
    assert np.abs(sp.G_sym(eps) - eps).max() <= 1e-12 * np.abs(eps).max()
    b = np.cross(k, [1.0, 0, 0])
    c = np.cross(k, b)
    sig = (np.outer(b, c) + np.outer(c, b))[:, :, None, None, None] * np.cos(th)
    assert np.abs(sp.G_sym(sig)).max() <= 1e-13 * np.abs(sig).max()


def _laminate(n, E, nu):
    gid = np.zeros((n, n, n), dtype=np.int32)
    gid[:, :, n // 2:] = 1  # layers normal to x, each n/2 wide (even widths: no Nyquist content)
    ms = Microstructure(n, n, n, (1.0, 1.0, 1.0), gid, np.tile([1.0, 0, 0, 0], (2, 1)), np.array([0, 1]))
    mats = {ph: Material(SVK_ISO, E=E[ph], nu=nu[ph]) for ph in (0, 1)}
    return ms, mats


def test_two_phase_laminate_matches_the_closed_form():
    E, nu = (100e9, 400e9), (0.3, 0.2)
    ms, mats = _laminate(8, E, nu)
    eps_bar = np.array([[0.002, 0.0005, -0.0003], [0.0005, -0.001, 0.0007], [-0.0003, 0.0007, 0.0004]])
    for kind in (sp.KIND_CONTINUOUS, sp.KIND_DISCRETE):
        o = OracleRVE(ms, mats, Options(projection=kind, newton_tol=1e-12, cg_tol=1e-12, small_strain=True))
        o.step(1.0, eps_bar.reshape(9), np.zeros(9, np.uint8), np.zeros(9))
        C = [mat.isotropic_stiffness(E[p], nu[p]) for p in (0, 1)]
        Q = [C[p][:, 0, :, 0] for p in (0, 1)]  # acoustic tensors along e1
        rhs = (np.einsum("ijkl,kl->ij", C[1] - C[0], eps_bar))[:, 0]
        a0 = np.linalg.solve(Q[0] + Q[1], rhs)  # equal volume fractions: a1 = -a0
        e1 = np.array([1.0, 0, 0])
        for p, ap in ((0, a0), (1, -a0)):
            want = eps_bar + 0.5 * (np.outer(ap, e1) + np.outer(e1, ap))
            got = o.F[:, :, :, :, :4] if p == 0 else o.F[:, :, :, :, 4:]
            assert np.abs(got - want[:, :, None, None, None]).max() <= 1e-12 * np.abs(want).max()


def test_uniaxial_stress_on_a_homogeneous_body():
    E, nuv = 200e9, 0.3
    ms = polycrystal(4, 1, 1)
    o = OracleRVE(ms, {0: Material(SVK_ISO, E=E, nu=nuv)}, Options(newton_tol=1e-12, small_strain=True))
    mask = np.ones(9, np.uint8)
    mask[0] = 0
    Fbar = np.zeros(9)
    Fbar[0] = 1e-3
    rep = o.step(1.0, Fbar, mask, np.zeros(9))
    e = rep["Fmacro"]
    assert abs(e[4] + nuv * 1e-3) < 1e-15 and abs(e[8] + nuv * 1e-3) < 1e-15
    assert abs(rep["Pmacro"][0] - E * 1e-3) < 1e-6 * E * 1e-3
    # the prescribed stresses are reached from the strain start once the linear solve is done
    assert rep["newton"] <= 1


def test_homogeneous_medium_needs_no_correction():
    """One rotated cubic grain filling the box: the uniform strain is the solution."""
    ms1 = polycrystal(6, 1, 2)
    o = OracleRVE(ms1, {0: Material(SVK_CUBIC)}, Options(newton_tol=1e-12, small_strain=True))
    eb = np.array([1e-3, 2e-4, 0, 2e-4, -5e-4, 1e-4, 0, 1e-4, 3e-4])
    rep = o.step(1.0, eb, np.zeros(9, np.uint8), np.zeros(9))
    assert rep["newton"] == 0
    assert np.abs(o.F.reshape(9, -1) - eb[:, None]).max() < 1e-18
