"""The small-strain variant on the GPU (Sect. 2.3: the solver runs at small
and finite strains): the symmetric projection G^s against the oracle on the
same seeded fields, and linear-elastic solves -- a cubic polycrystal under
uniaxial stress and the two-phase laminate of known closed form -- against
the oracle.  Tolerances as the finite-strain tests: projection relative L2
1e-12 (FP64) / 2e-6 (FP32); solves macroscopic 1e-10, fields 1e-8 (FP64),
1e-5 / 1e-4 (mixed)."""

import numpy as np
import pytest

from gpu_helpers import gff, rel_l2, torch_cuda
from oracle import spectral as sp
from oracle.solver import SVK_CUBIC, SVK_ISO, Material, OracleRVE, Options
from rve_inputs import Microstructure, polycrystal, ramp_history, standard_normal

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (6, 10, 12), (12, 48, 20), (32, 32, 32), (48, 40, 64)]  # (nz, ny, nx)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_symmetric_projection_matches_oracle(shape, kind):
    torch = torch_cuda()
    g = gff()
    nz, ny, nx = shape
    L = (1.0, 2.0, 0.5) if shape == (12, 48, 20) else (1.0, 1.0, 1.0)
    h = g.gff_create(g.make_grid(nx, ny, nz, L), g.make_options(projection=kind))
    try:
        g.gff_set_strain_measure(h, g.GFF_STRAIN_SMALL)
        x = standard_normal(17, 9 * nx * ny * nz).reshape((3, 3) + (nz, ny, nx))
        x = 0.5 * (x + x.transpose(1, 0, 2, 3, 4))
        for mask in (None, np.array([0, 1, 1, 1, 1, 1, 1, 1, 1], dtype=np.uint8)):
            ref = sp.G_sym(x, L, kind, None if mask is None else mask.astype(np.float64))
            X = torch.from_numpy(x.reshape(9, -1).copy()).cuda()
            Y = torch.empty_like(X)
            g.gff_project(h, g.GFF_PREC_FP64, mask, X, Y)
            Y32 = torch.empty_like(X.float())
            g.gff_project(h, g.GFF_PREC_MIXED, mask, X.float(), Y32)
            torch.cuda.synchronize()
            assert rel_l2(Y.cpu().numpy(), ref) <= 1e-12
            assert rel_l2(Y32.cpu().numpy(), ref) <= 2e-6
    finally:
        g.gff_destroy(h)


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
@pytest.mark.parametrize("precision", [0, 1])
def test_polycrystal_uniaxial_stress_matches_oracle(kind, precision):
    """16^3, 8 cubic grains, eps11 ramped to 1e-3 in 3 steps with zero
    average stress on the other eight components (small strains carry no
    rotation, so no component needs holding; the skew part stays 0)."""
    torch_cuda()
    g = gff()
    ms = polycrystal(16, 8, 1)
    hist = ramp_history(1.001, 3)
    hist.mask[:, :] = 1
    hist.mask[:, 0] = 0
    Ebar = np.zeros((3, 9))
    Ebar[:, 0] = 1e-3 * np.arange(1, 4) / 3
    tol = 1e-11 if precision == 0 else 1e-9
    o = OracleRVE(ms, {0: Material(SVK_CUBIC)}, Options(projection=kind, newton_tol=1e-11, cg_tol=1e-11,
                                                        small_strain=True))
    orep = [o.step(hist.dt[k], Ebar[k], hist.mask[k], hist.Pbar[k]) for k in range(hist.nsteps)]
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)},
                     g.make_options(projection=kind, precision=precision, newton_tol=tol,
                                    cg_tol=tol if precision == 0 else 1e-6), small_strain=True)
    try:
        Pm, reps = g.gff_run_history(h, hist.dt, Ebar, hist.mask, hist.Pbar)
        eps = g.gff_get_field(h, g.GFF_FIELD_F, ms.n_voxels)
        sig = g.gff_get_field(h, g.GFF_FIELD_P, ms.n_voxels)
    finally:
        g.gff_destroy(h)
    ref = np.array([r["Pmacro"] for r in orep])
    err = max(np.linalg.norm(Pm[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(hist.nsteps))
    assert err <= (1e-10 if precision == 0 else 1e-5)
    ftol = 1e-8 if precision == 0 else 1e-4
    assert rel_l2(eps, o.F.reshape(9, -1)) <= ftol
    assert rel_l2(sig, o.P.reshape(9, -1)) <= ftol
    assert np.abs(Pm[-1][1:7]).max() <= 1e-6 * abs(Pm[-1][0])  # stress-controlled averages vanish
    e = eps.reshape(3, 3, -1)
    # strains stay symmetric (to rounding: FP32 corrections in mixed precision)
    assert np.abs(e - e.transpose(1, 0, 2)).max() <= (1e-12 if precision == 0 else 1e-5) * np.abs(e).max()


def test_laminate_closed_form_on_the_gpu():
    from oracle import materials as mat

    torch_cuda()
    g = gff()
    n = 16
    E, nu = (100e9, 400e9), (0.3, 0.2)
    gid = np.zeros((n, n, n), dtype=np.int32)
    gid[:, :, n // 2:] = 1
    ms = Microstructure(n, n, n, (1.0, 1.0, 1.0), gid, np.tile([1.0, 0, 0, 0], (2, 1)), np.array([0, 1]))
    mats = {p: g.make_material(g.GFF_MAT_SVK_ISO, E=E[p], nu=nu[p]) for p in (0, 1)}
    eb = np.array([[0.002, 0.0005, -0.0003], [0.0005, -0.001, 0.0007], [-0.0003, 0.0007, 0.0004]])
    h = g.create_rve(ms, mats, g.make_options(newton_tol=1e-12, cg_tol=1e-12), small_strain=True)
    try:
        g.gff_step(h, 1.0, eb.reshape(9), np.zeros(9, np.uint8), np.zeros(9))
        eps = g.gff_get_field(h, g.GFF_FIELD_F, ms.n_voxels).reshape(3, 3, n, n, n)
    finally:
        g.gff_destroy(h)
    C = [mat.isotropic_stiffness(E[p], nu[p]) for p in (0, 1)]
    Q = [C[p][:, 0, :, 0] for p in (0, 1)]
    a0 = np.linalg.solve(Q[0] + Q[1], np.einsum("ijkl,kl->ij", C[1] - C[0], eb)[:, 0])
    e1 = np.array([1.0, 0, 0])
    for p, ap in ((0, a0), (1, -a0)):
        want = eb + 0.5 * (np.outer(ap, e1) + np.outer(e1, ap))
        got = eps[..., : n // 2] if p == 0 else eps[..., n // 2:]
        assert np.abs(got - want[:, :, None, None, None]).max() <= 1e-11 * np.abs(want).max()


def test_small_strain_rejects_plastic_phases_and_batches():
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 2, 3)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_CP_FCC)}, g.make_options(), small_strain=True)
    try:
        with pytest.raises(g.GffError) as e:
            g.gff_step(h, 1.0, np.zeros(9), np.zeros(9, np.uint8), np.zeros(9))
        assert e.value.status == g.GFF_ERR_ARG
    finally:
        g.gff_destroy(h)
    a = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(), small_strain=True)
    b = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(), small_strain=True)
    try:
        with pytest.raises(g.GffError) as e:
            g.gff_batch_run([a, b], np.ones(1), np.zeros((1, 9)), np.zeros((1, 9), np.uint8), np.zeros((1, 9)))
        assert e.value.status == g.GFF_ERR_ARG
    finally:
        g.gff_destroy(a)
        g.gff_destroy(b)
