"""Batched RVEs of uneven sizes (gff_batch_run): every RVE's result must be
bitwise the result of running its handle alone (the batched launches keep
each RVE's arithmetic and reduction order), in FP64 and in mixed precision,
with crystal plasticity and with a stiff second phase."""

import numpy as np
import pytest

from gpu_helpers import gff, gpu_materials, torch_cuda
from oracle.solver import CP_FCC, SVK_CUBIC, SVK_ISO
from rve_inputs import cyclic_history, polycrystal, polycrystal_with_particles

pytestmark = pytest.mark.gpu


def _rves():
    return [
        (polycrystal((8, 8, 8), 4, 21), {0: CP_FCC}),
        (polycrystal((12, 8, 16), 6, 22), {0: CP_FCC}),
        (polycrystal_with_particles(16, 5, 23, radius=3, frac=0.05), {0: CP_FCC, 1: SVK_ISO}),
        (polycrystal((6, 10, 20), 3, 24), {0: CP_FCC}),
    ]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_one_by_one_bitwise(precision):
    torch_cuda()
    g = gff()
    hist = cyclic_history(0.01, 1).head(7)
    opts = dict(precision=precision, newton_tol=1e-9 if precision == 0 else 1e-7, cg_tol=1e-6)
    rves = _rves()
    singles, batch = [], []
    try:
        for ms, kinds in rves:
            singles.append(g.create_rve(ms, gpu_materials(kinds), g.make_options(**opts)))
            batch.append(g.create_rve(ms, gpu_materials(kinds), g.make_options(**opts)))
        ref = [g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start) for h in singles]
        Pm, reps, stat = g.gff_batch_run(batch, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        assert (stat == 0).all()
        for r, (ms, kinds) in enumerate(rves):
            assert np.array_equal(Pm[r], ref[r][0]), r
            assert [x.newton_iters for x in reps[r]] == [x.newton_iters for x in ref[r][1]]
            assert [x.cg_iters for x in reps[r]] == [x.cg_iters for x in ref[r][1]]
            for w in (g.GFF_FIELD_F, g.GFF_FIELD_P, g.GFF_FIELD_FP_INV, g.GFF_FIELD_CHI):
                a = g.gff_get_field(batch[r], w, ms.n_voxels)
                b = g.gff_get_field(singles[r], w, ms.n_voxels)
                assert np.array_equal(a, b), (r, w)
            fa = g.gff_get_fips(batch[r], ms.ngrains)
            fb = g.gff_get_fips(singles[r], ms.ngrains)
            for x, y in zip(fa, fb):
                assert np.allclose(x, y, rtol=1e-12, atol=0)
    finally:
        for h in singles + batch:
            g.gff_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_accepts_persistent_launch_shapes(precision):
    """The batched passes have no persistent variants: handles whose launch
    shapes select the TMA z pass (512 threads) or the streamed inverse pass
    (up to 1024 threads) still batch, with the bits of the one-by-one run."""
    torch_cuda()
    g = gff()
    hist = cyclic_history(0.01, 1).head(2)
    opts = dict(precision=precision, newton_tol=1e-9 if precision == 0 else 1e-7, cg_tol=1e-6)
    rves = _rves()
    singles, batch = [], []
    try:
        for ms, kinds in rves:
            singles.append(g.create_rve(ms, gpu_materials(kinds), g.make_options(**opts)))
            h = g.create_rve(ms, gpu_materials(kinds), g.make_options(**opts))
            batch.append(h)
            # (threads fwd, W, threads z, threads inv, inverse blocks, z blocks)
            g.gff_set_tiles(h, (512, 8, 512, 512, 7, 3), (256, 16, 512, 1024, 5, 3))
        ref = [g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start) for h in singles]
        Pm, reps, stat = g.gff_batch_run(batch, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        assert (stat == 0).all()
        for r in range(len(rves)):
            assert np.array_equal(Pm[r], ref[r][0]), r
    finally:
        for h in singles + batch:
            g.gff_destroy(h)


def test_batch_rejects_mismatched_options():
    torch_cuda()
    g = gff()
    ms = polycrystal(8, 3, 1)
    a = g.create_rve(ms, gpu_materials({0: CP_FCC}), g.make_options(precision=0))
    b = g.create_rve(ms, gpu_materials({0: CP_FCC}), g.make_options(precision=1))
    try:
        hist = cyclic_history(0.01, 1).head(1)
        with pytest.raises(g.GffError) as e:
            g.gff_batch_run([a, b], hist.dt, hist.Fbar, hist.mask, hist.Pbar)
        assert e.value.status == g.GFF_ERR_ARG
        with pytest.raises(g.GffError):
            g.gff_batch_run([a, a], hist.dt, hist.Fbar, hist.mask, hist.Pbar)
    finally:
        g.gff_destroy(a)
        g.gff_destroy(b)


def test_batch_with_extrapolated_warm_start_equals_one_by_one():
    """Warm-start mode 3 (extrapolated last increment) applied per RVE inside
    the batch gives each RVE the bits of its own gff_run_history."""
    torch_cuda()
    g = gff()
    hist = cyclic_history(0.01, 1).head(6)
    opts = dict(precision=1, newton_tol=1e-7, cg_tol=1e-6)
    rves = _rves()
    singles, batch = [], []
    try:
        for ms, kinds in rves:
            for lst in (singles, batch):
                h = g.create_rve(ms, gpu_materials(kinds), g.make_options(**opts))
                g.gff_set_warm_start(h, None, g.GFF_WARM_EXTRAPOLATE)
                lst.append(h)
        ref = [g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start) for h in singles]
        Pm, reps, stat = g.gff_batch_run(batch, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)
        assert (stat == 0).all()
        for r, (ms, kinds) in enumerate(rves):
            assert np.array_equal(Pm[r], ref[r][0]), r
            assert [x.warm_start_used for x in reps[r]] == [x.warm_start_used for x in ref[r][1]]
            assert sum(x.warm_start_used for x in reps[r]) >= 4
            for w in (g.GFF_FIELD_F, g.GFF_FIELD_FP_INV):
                assert np.array_equal(g.gff_get_field(batch[r], w, ms.n_voxels),
                                      g.gff_get_field(singles[r], w, ms.n_voxels)), (r, w)
    finally:
        for h in singles + batch:
            g.gff_destroy(h)


def test_failed_batch_increments_are_cut_back_per_rve():
    """A hyperelastic increment too large for the Newton budget fails inside the
    batched graph; each RVE is then redone on its own handle with cut-backs and
    ends exactly where gff_step with cut-backs ends."""
    torch_cuda()
    g = gff()
    shapes = [(8, 8, 8), (12, 8, 16), (16, 16, 16)]
    Fbar = np.eye(3).ravel().copy()
    Fbar[0] += 0.12
    Fbar[4] -= 0.04
    dt, F1, mk, P0 = np.ones(1), Fbar[None, :], np.zeros((1, 9), np.uint8), np.zeros((1, 9))
    mss = [polycrystal(sh, 4, 50 + i) for i, sh in enumerate(shapes)]
    # Tight CG: the Newton iteration count is then set by the nonlinearity, and a
    # smaller increment needs fewer corrections.  (With a loose CG tolerance the
    # relative residual of a first increment from F = I is limited by the CG
    # tolerance whatever the increment's size, and no cut-back helps.)  On the
    # oracle at 8^3 the residual after two corrections falls about 7x per halving
    # (1.8e-6 for the whole increment, 8.3e-9 for an eighth of it).
    base = dict(newton_tol=1e-8, cg_tol=1e-11)
    # the Newton corrections each RVE needs for the whole increment; a budget below the
    # smallest of them makes every RVE fail in the graph
    need = []
    for ms in mss:
        h = g.create_rve(ms, gpu_materials({0: SVK_CUBIC}), g.make_options(newton_max=60, max_cuts=0, **base))
        try:
            need.append(g.gff_step(h, 1.0, Fbar, mk[0], P0[0]).newton_iters)
        finally:
            g.gff_destroy(h)
    assert min(need) >= 2, need
    # the smallest such budget at which the one-by-one runs succeed through cut-backs
    opts = None
    for nm in range(1, min(need)):
        o = dict(newton_max=nm, max_cuts=6, **base)
        hs = [g.create_rve(ms, gpu_materials({0: SVK_CUBIC}), g.make_options(**o)) for ms in mss]
        ok = True
        try:
            for h in hs:
                try:
                    g.gff_run_history(h, dt, F1, mk, P0)
                except g.GffError:
                    ok = False
                    break
        finally:
            for h in hs:
                g.gff_destroy(h)
        if ok:
            opts = o
            break
    assert opts is not None, need
    singles, batch = [], []
    try:
        for ms in mss:
            singles.append(g.create_rve(ms, gpu_materials({0: SVK_CUBIC}), g.make_options(**opts)))
            batch.append(g.create_rve(ms, gpu_materials({0: SVK_CUBIC}), g.make_options(**opts)))
        ref = [g.gff_run_history(h, dt, F1, mk, P0) for h in singles]
        assert all(r[1][0].cuts >= 1 for r in ref)  # the increment does need cutting
        Pm, reps, stat = g.gff_batch_run(batch, dt, F1, mk, P0)
        assert (stat == 0).all()
        for r, sh in enumerate(shapes):
            assert reps[r][0].cuts == ref[r][1][0].cuts
            assert np.array_equal(Pm[r], ref[r][0])
            N = int(np.prod(sh))
            assert np.array_equal(g.gff_get_field(batch[r], g.GFF_FIELD_F, N),
                                  g.gff_get_field(singles[r], g.GFF_FIELD_F, N))
    finally:
        for h in singles + batch:
            g.gff_destroy(h)
