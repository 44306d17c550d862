"""Appendix A on the GPU: the conversion of a user material's Cauchy stress
and Jaumann-rate tangent C^ab (Eq. ABAtang) into P = J sigma F^-T (Eq. fPK)
and K = dP/dF, against the oracle's conversion element by element, and a
finite-strain solve with a material evaluated through that interface (a
compressible neo-Hookean solid in two phases) against the oracle.

Tolerances: the conversion relative L2 1e-13 (FP64, same formula, different
rounding order); the solve as the other FP64 parity tests (macroscopic P
1e-10, fields 1e-8) and mixed precision 1e-5 / 1e-4."""

import numpy as np
import pytest

from gpu_helpers import gff, rel_l2, torch_cuda
from oracle import materials as omat
from oracle import spectral as sp
from oracle.solver import NEO_HOOKE, Material, OracleRVE, Options
from rve_inputs import polycrystal_with_particles, ramp_history, standard_normal

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    F = np.eye(3)[None] + 0.1 * standard_normal(seed, 9 * n).reshape(n, 3, 3)
    s = standard_normal(seed + 1, 9 * n).reshape(n, 3, 3) * 1e8
    sig = 0.5 * (s + s.transpose(0, 2, 1))
    A = standard_normal(seed + 2, 81 * n).reshape(n, 3, 3, 3, 3) * 1e11
    C = 0.5 * (A + A.transpose(0, 1, 2, 4, 3))
    C = 0.5 * (C + C.transpose(0, 2, 1, 3, 4))
    return F, sig, C


@pytest.mark.parametrize("n", [1000, 777, 1])
def test_umat_conversion_matches_oracle(n):
    torch = torch_cuda()
    g = gff()
    F, sig, C = _inputs(n, 40 + n)
    P_ref, K_ref = omat.umat_to_PK(F, sig, C)

    def dev(a, comps):  # [V][...] -> SoA [comps][V] on the device
        return torch.from_numpy(np.ascontiguousarray(a.reshape(n, comps).T)).cuda()

    Fd, Sd, Cd = dev(F, 9), dev(sig, 9), dev(C, 81)
    Pd = torch.empty(9, n, dtype=torch.float64, device="cuda")
    Kd = torch.empty(81, n, dtype=torch.float64, device="cuda")
    g.gff_umat_tangent(n, Fd, Sd, Cd, Pd, Kd, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rel_l2(Pd.cpu().numpy().T, P_ref.reshape(n, 9)) <= 1e-13
    assert rel_l2(Kd.cpu().numpy().T, K_ref.reshape(n, 81)) <= 1e-13


def test_umat_conversion_rejects_bad_arguments():
    torch_cuda()
    g = gff()
    g.gff_umat_tangent(0, 0, 0, 0, 0, 0)  # nothing to do
    with pytest.raises(g.GffError) as e:
        g.gff_umat_tangent(-1, 0, 0, 0, 0, 0)
    assert e.value.status == g.GFF_ERR_ARG
    with pytest.raises(g.GffError):
        g.gff_umat_tangent(5, 0, 0, 0, 0, 0)


PHASES = {0: (100e9, 0.3), 1: (400e9, 0.2)}  # soft matrix, stiff spheres: (E, nu)


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
@pytest.mark.parametrize("precision", [0, 1])
def test_neo_hookean_two_phase_finite_strain_solve(kind, precision):
    """F11 ramped to 1.05 with zero average stress on the other components:
    a finite-strain two-phase solve whose stresses and tangents all come
    through the Appendix-A conversion, against the oracle's solve."""
    torch_cuda()
    g = gff()
    ms = polycrystal_with_particles(16, 4, 3, radius=3, frac=0.05)
    hist = ramp_history(1.05, 4)
    tol = 1e-11 if precision == 0 else 1e-9
    o = OracleRVE(ms, {ph: Material(NEO_HOOKE, E=E, nu=nu) for ph, (E, nu) in PHASES.items()},
                  Options(projection=kind, newton_tol=1e-11, cg_tol=1e-11))
    orep = o.run(hist)
    mats = {ph: g.make_material(g.GFF_MAT_NEOHOOKE, E=E, nu=nu) for ph, (E, nu) in PHASES.items()}
    h = g.create_rve(ms, mats, g.make_options(projection=kind, precision=precision, newton_tol=tol,
                                              cg_tol=tol if precision == 0 else 1e-6))
    try:
        Pm, reps = g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        N = ms.n_voxels
        F = g.gff_get_field(h, g.GFF_FIELD_F, N)
        P = g.gff_get_field(h, g.GFF_FIELD_P, N)
    finally:
        g.gff_destroy(h)
    ref = np.array([r["Pmacro"] for r in orep])
    err = max(np.linalg.norm(Pm[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(hist.nsteps))
    assert err <= (1e-10 if precision == 0 else 1e-5)
    ftol = 1e-8 if precision == 0 else 1e-4
    assert rel_l2(F, o.F.reshape(9, -1)) <= ftol
    assert rel_l2(P, o.P.reshape(9, -1)) <= ftol
    assert all(r.cuts == 0 for r in reps)
    if precision == 0:
        # exact tangents keep Newton's quadratic convergence: a few corrections per increment
        assert max(r.newton_iters for r in reps) <= 6
