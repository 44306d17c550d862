"""Warm starts.  The network on the GPU against the FP64 oracle
(oracle/unet.py) with the same bfloat16 rounding points: forward output,
loss and every parameter gradient; training lowers the loss; the solver
reaches the same solution from the learned start and from the extrapolated
start as from the zero-fluctuation start, and extrapolation lowers the first
residual of monotone increments.

Tolerance: a bfloat16 network is chaotic at the rounding level -- weights
perturbed by 1e-6 (relative) move the oracle's own output by ~0.6 % and its
deepest gradients by several % -- and the GPU accumulates in FP32 where the
oracle uses FP64.  So each comparison is held to three times the oracle's
own spread under such perturbations (plus a small floor), and every
gradient must point the same way (cosine >= 0.995)."""

import numpy as np
import pytest

from gpu_helpers import gff, gpu_materials, rel_l2, torch_cuda
from oracle import unet as U
from oracle.solver import CP_FCC
from rve_inputs import cyclic_history, polycrystal

pytestmark = pytest.mark.gpu


def flat(p):
    parts = []
    for name, ci, co in U.LAYERS:
        W, b = p[name]
        parts += [W.ravel(), b]
    W, b = p["head"]
    parts += [W.ravel(), b]
    return np.concatenate(parts)


def unflat(w):
    p, k = {}, 0
    for name, ci, co in U.LAYERS + [U.HEAD]:
        shape = (27, co, ci) if name != "head" else (co, ci)
        m = int(np.prod(shape))
        p[name] = (w[k:k + m].reshape(shape), w[k + m:k + m + co])
        k += m + co
    return p


@pytest.mark.parametrize("n", [8, 32])  # 32^3: several voxel chunks per weight-gradient tap
def test_forward_and_gradients_match_oracle(n):
    torch_cuda()
    g = gff()
    V = n ** 3
    p = U.init_params(5)
    rng = np.random.default_rng(6)
    for name in p:  # non-zero biases exercise the bias paths
        p[name] = (p[name][0], 0.1 * rng.standard_normal(p[name][1].shape))
    x = rng.standard_normal((U.IN_CH, n, n, n))
    t = 0.5 * rng.standard_normal((9, n, n, n))
    u = g.gff_unet_create(1)
    try:
        assert g.gff_unet_num_params(u) == flat(p).size
        g.gff_unet_set_params(u, flat(p).astype(np.float32))
        assert np.array_equal(g.gff_unet_get_params(u), flat(p).astype(np.float32))
        p32 = unflat(flat(p).astype(np.float32).astype(np.float64))
        y, loss, grads = g.gff_unet_eval_host(u, n, x.reshape(U.IN_CH, V).T, t.reshape(9, V).T)
        yo, cache = U.forward(p32, x, round_bf16=True)
        lo, dy = U.mse(yo, t)
        go = U.backward(p32, cache, dy, round_bf16=True)
        # the oracle's own spread under 1e-6 relative weight perturbations
        spread_y, spread = 0.0, {}
        for k in range(3):
            w = flat(p32)
            pe = unflat(w * (1 + 1e-6 * np.random.default_rng(100 + k).standard_normal(w.size)))
            ye, ce = U.forward(pe, x, round_bf16=True)
            le, dye = U.mse(ye, t)
            ge = U.backward(pe, ce, dye, round_bf16=True)
            spread_y = max(spread_y, rel_l2(ye, yo))
            for name in ge:
                spread[name] = max(spread.get(name, 0.0), rel_l2(ge[name][0], go[name][0]),
                                   rel_l2(ge[name][1], go[name][1]))
        assert spread_y < 0.05  # sanity of the calibration itself
        assert rel_l2(y.T.reshape(9, n, n, n), yo) <= 3 * spread_y + 1e-3
        assert abs(loss - lo) <= (3 * spread_y + 1e-3) * lo
        gg = unflat(grads.astype(np.float64))
        for name, _, _ in U.LAYERS + [U.HEAD]:
            for part in (0, 1):
                a, b = gg[name][part].ravel(), go[name][part].ravel()
                assert rel_l2(a, b) <= 3 * spread[name] + 2e-3, (name, part, rel_l2(a, b), spread[name])
                assert a @ b >= 0.995 * np.linalg.norm(a) * np.linalg.norm(b), (name, part)
    finally:
        g.gff_unet_destroy(u)


def test_one_training_step_is_adam():
    """First Adam step from fresh moments: every parameter with a clear
    gradient moves by -lr sign(g) (moment ratios are exactly g and g^2 after
    bias correction; clipping rescales g, not its sign)."""
    torch_cuda()
    g = gff()
    n, lr = 8, 1e-3
    V = n ** 3
    p = U.init_params(7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((V, U.IN_CH)).astype(np.float32)
    t = (0.5 * rng.standard_normal((V, 9))).astype(np.float32)
    u = g.gff_unet_create(1)
    try:
        w0 = flat(p).astype(np.float32)
        g.gff_unet_set_params(u, w0)
        _, _, grad = g.gff_unet_eval_host(u, n, x, t)
        g.gff_unet_add_sample_host(u, n, x, t)
        g.gff_unet_train(u, 1, lr)
        w1 = g.gff_unet_get_params(u)
        clear = np.abs(grad) > 1e-3 * np.abs(grad).max()
        assert clear.sum() > 0.5 * grad.size
        step = (w1 - w0)[clear].astype(np.float64)
        assert np.allclose(step, -lr * np.sign(grad[clear]), rtol=1e-3, atol=1e-6)
    finally:
        g.gff_unet_destroy(u)


def test_training_fits_a_learnable_target():
    """The target is a fixed periodic 3x3x3 smoothing of the inputs mixed by a
    fixed matrix: the network (head starting at zero) must fit it."""
    torch_cuda()
    g = gff()
    n = 16
    rng = np.random.default_rng(9)
    x = rng.standard_normal((U.IN_CH, n, n, n))
    smooth = sum(U.shift(x, d) for d in U.TAPS) / 27.0
    A = rng.standard_normal((9, U.IN_CH)) / np.sqrt(U.IN_CH)
    t = np.einsum("oi,i...->o...", A, smooth)
    u = g.gff_unet_create(4)
    try:
        g.gff_unet_add_sample_host(u, n, x.reshape(U.IN_CH, -1).T, t.reshape(9, -1).T)
        losses = g.gff_unet_train(u, 300, 2e-3)
        assert np.isfinite(losses).all()
        assert losses[-20:].mean() < 0.3 * losses[:5].mean(), (losses[:5], losses[-20:])
    finally:
        g.gff_unet_destroy(u)


def _solve(g, ms, hist, u=None, mode=0, tol=1e-10):
    h = g.create_rve(ms, gpu_materials({0: CP_FCC}), g.make_options(newton_tol=tol, cg_tol=1e-8))
    if mode:
        g.gff_set_warm_start(h, u, mode)
    return h, g.gff_run_history(h, hist.dt, hist.Fbar, hist.mask, hist.Pbar, hist.cycle_start)


def test_training_lowers_the_loss_and_warm_start_keeps_the_solution(tmp_path):
    torch_cuda()
    g = gff()
    hist = cyclic_history(0.01, 1).head(6)
    u = g.gff_unet_create(3)
    hs = []
    try:
        # training samples from the solver's own increments (two 16^3 RVEs)
        for seed in (31, 32):
            h = g.create_rve(polycrystal(16, 6, seed), gpu_materials({0: CP_FCC}), g.make_options(newton_tol=1e-8))
            hs.append(h)
            for k in range(hist.nsteps):
                g.gff_step(h, hist.dt[k], hist.Fbar[k], hist.mask[k], hist.Pbar[k])
                g.gff_unet_add_sample(u, h)
        assert g.gff_unet_num_samples(u) == 12
        losses = g.gff_unet_train(u, 120, 1e-3)
        assert np.isfinite(losses).all()
        # the last epoch sees the same 12 samples as the first
        assert losses[-12:].sum() < losses[:12].sum()
        path = tmp_path / "w.bin"
        g.gff_unet_save(u, path)
        u2 = g.gff_unet_create(99)
        g.gff_unet_load(u2, path)
        assert np.array_equal(g.gff_unet_get_params(u2), g.gff_unet_get_params(u))
        g.gff_unet_destroy(u2)

        ms = polycrystal(16, 6, 33)  # held-out RVE
        h0, (P0, r0) = _solve(g, ms, hist)
        h2, (P2, r2) = _solve(g, ms, hist, u, mode=2)
        h1, (P1, r1) = _solve(g, ms, hist, u, mode=1)
        h3, (P3, r3) = _solve(g, ms, hist, None, mode=g.GFF_WARM_EXTRAPOLATE)
        hs += [h0, h2, h1, h3]
        assert all(r.warm_start_used == 1 for r in r2)
        # The measured relation (the same one the 128^3 benchmark shows over a full cycle): the
        # network's guess keeps the extrapolation's gain over the zero start, and its trained
        # correction moves the first residual by little either way -- it does not beat the
        # extrapolation it is added to.
        f0 = np.mean([r.residual_first for r in r0[1:]])
        f2 = np.mean([r.residual_first for r in r2[1:]])
        f3 = np.mean([r.residual_first for r in r3[1:]])
        assert f2 <= 0.6 * f0, (f2, f0)
        assert 0.8 <= f2 / f3 <= 1.25, (f2, f3)
        # same increments solved to tolerance: same solution
        for k in range(hist.nsteps):
            assert np.linalg.norm(P2[k] - P0[k]) <= 1e-7 * np.linalg.norm(P0[k])
        F0 = g.gff_get_field(h0, g.GFF_FIELD_F, ms.n_voxels)
        F2 = g.gff_get_field(h2, g.GFF_FIELD_F, ms.n_voxels)
        assert rel_l2(F2, F0) <= 1e-7
        # mode 1: where the guess was not kept, the increment is the plain one (the return maps of
        # the re-evaluated zero start begin from other slip increments: equal to their tolerance)
        for k in range(hist.nsteps):
            if r1[k].warm_start_used == 0 and all(r.warm_start_used == 0 for r in r1[:k]):
                assert np.linalg.norm(P1[k] - P0[k]) <= 1e-12 * np.linalg.norm(P0[k])
            assert r1[k].residual_first <= r0[k].residual_first * (1 + 1e-12) or r1[k].warm_start_used == 0
    finally:
        for h in hs:
            g.gff_destroy(h)
        g.gff_unet_destroy(u)


def test_extrapolation_keeps_the_solution_and_lowers_the_first_residual():
    torch_cuda()
    g = gff()
    ms = polycrystal(16, 6, 34)
    hist = cyclic_history(0.01, 1).head(12)  # monotone: elastic, then plastic
    hs = []
    try:
        h0, (P0, r0) = _solve(g, ms, hist)
        h3, (P3, r3) = _solve(g, ms, hist, None, mode=g.GFF_WARM_EXTRAPOLATE)
        hs += [h0, h3]
        assert r3[0].warm_start_used == 0  # no history yet
        assert all(r.warm_start_used == 1 for r in r3[1:])
        for k in range(hist.nsteps):
            assert np.linalg.norm(P3[k] - P0[k]) <= 1e-7 * np.linalg.norm(P0[k])
        N = ms.n_voxels
        assert rel_l2(g.gff_get_field(h3, g.GFF_FIELD_F, N), g.gff_get_field(h0, g.GFF_FIELD_F, N)) <= 1e-7
        ratio = np.mean([a.residual_first / b.residual_first for a, b in zip(r3[1:], r0[1:])])
        assert ratio < 0.5, ratio
        assert sum(r.newton_iters for r in r3) <= sum(r.newton_iters for r in r0)
    finally:
        for h in hs:
            g.gff_destroy(h)
