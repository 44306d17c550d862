"""Parity of the CUDA Galerkin operator with the oracle (Eqs. eql_discrete3,
newlinop; G^ of Eq. G and G^' of Sect. 2.2), element by element on seeded
inputs.  Tolerances: FP64 relative L2 1e-12 (the transforms differ only in
rounding order), FP32 relative L2 2e-6 (single-precision rounding of
~log2(N) butterfly stages and the K contraction)."""

import numpy as np
import pytest

from gpu_helpers import gff, rel_l2, torch_cuda, voxel_K_oracle
from oracle import spectral as sp
from rve_inputs import polycrystal, standard_normal

pytestmark = pytest.mark.gpu

# (nz, ny, nx): radix plans 16, 4x3 / 2x5 / 4x3, 4x3 / 16x3 / 4x5, 8x5 / 8 / 2x5x3, 8x4, and the
# batch sizes 80 (16x5) and 96 (16x2x3, generic stages) with 48 (16x3)
SHAPES = [(16, 16, 16), (6, 10, 12), (12, 48, 20), (40, 8, 30), (32, 32, 32), (96, 80, 48), (80, 80, 80)]
MASKS = [None, np.array([0, 1, 1, 1, 1, 1, 1, 0, 1], dtype=np.uint8)]


def _field(seed, shape):
    nz, ny, nx = shape
    return standard_normal(seed, 9 * nz * ny * nx).reshape(3, 3, nz, ny, nx)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
@pytest.mark.parametrize("mi", [0, 1])
def test_project_matches_oracle(shape, kind, mi):
    torch = torch_cuda()
    g = gff()
    nz, ny, nx = shape
    L = (1.0, 2.0, 0.5) if shape == (12, 48, 20) else (1.0, 1.0, 1.0)
    h = g.gff_create(g.make_grid(nx, ny, nz, L), g.make_options(projection=kind))
    try:
        x = _field(7, shape)
        mask = MASKS[mi]
        ref = sp.G(x, L, kind, None if mask is None else mask.astype(np.float64))
        X = torch.from_numpy(x.reshape(9, -1).copy()).cuda()
        Y = torch.empty_like(X)
        g.gff_project(h, g.GFF_PREC_FP64, mask, X, Y)
        torch.cuda.synchronize()
        assert rel_l2(Y.cpu().numpy(), ref) <= 1e-12
        X32, Y32 = X.float(), torch.empty_like(X.float())
        g.gff_project(h, g.GFF_PREC_MIXED, mask, X32, Y32)
        torch.cuda.synchronize()
        assert rel_l2(Y32.cpu().numpy(), ref) <= 2e-6
    finally:
        g.gff_destroy(h)


def _svk_handle(shape, ngrains, seed, kind=sp.KIND_CONTINUOUS):
    g = gff()
    ms = polycrystal(shape, ngrains, seed)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(projection=kind))
    return g, ms, h


@pytest.mark.parametrize("shape", [(16, 16, 16), (6, 10, 12), (40, 8, 30), (48, 96, 80)])
@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_apply_matches_oracle(shape, kind):
    torch = torch_cuda()
    g, ms, h = _svk_handle(shape, 5, 3, kind)
    try:
        N = ms.n_voxels
        F = np.eye(3).reshape(3, 3, 1, 1, 1) + 0.02 * _field(11, shape)
        g.gff_set_field(h, g.GFF_FIELD_F, F.reshape(9, N))
        g.gff_constitutive(h, 1.0)
        P_ref, K_ref = voxel_K_oracle(ms, F)
        K_gpu = g.gff_get_field(h, g.GFF_FIELD_K, N).reshape(3, 3, 3, 3, *shape)
        P_gpu = g.gff_get_field(h, g.GFF_FIELD_P, N).reshape(3, 3, *shape)
        assert rel_l2(K_gpu, K_ref) <= 1e-14
        assert rel_l2(P_gpu, P_ref) <= 1e-13
        x = _field(12, shape)
        mask = MASKS[1]
        ref = sp.GK(K_ref, x, (1.0, 1.0, 1.0), kind, mask.astype(np.float64))
        X = torch.from_numpy(x.reshape(9, -1).copy()).cuda()
        Y = torch.empty_like(X)
        g.gff_apply_operator(h, g.GFF_PREC_FP64, mask, X, Y)
        torch.cuda.synchronize()
        assert rel_l2(Y.cpu().numpy(), ref) <= 1e-12
        Y32 = torch.empty_like(X.float())
        g.gff_apply_operator(h, g.GFF_PREC_MIXED, mask, X.float(), Y32)
        torch.cuda.synchronize()
        assert rel_l2(Y32.cpu().numpy(), ref) <= 2e-6
    finally:
        g.gff_destroy(h)


def _bench_case(n, ngrains, seed_x):
    """Apply-benchmark inputs: K = rotated cubic C per voxel (the tangent at
    F = I), x ~ N(0, 1) per component."""
    ms = polycrystal(n, ngrains, 5)
    x = standard_normal(seed_x, 9 * ms.n_voxels)
    return ms, x


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_apply_full_size_128_matches_oracle(kind):
    """The benchmark's 128^3 case, same launch configuration, every output
    element compared with the oracle."""
    torch = torch_cuda()
    g = gff()
    ms, x = _bench_case(128, 500, 7)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options(projection=kind))
    try:
        g.gff_constitutive(h, 1.0)
        X = torch.from_numpy(x.reshape(9, -1)).cuda()
        Y = torch.empty_like(X)
        g.gff_apply_operator(h, g.GFF_PREC_FP64, None, X, Y)
        Y32 = torch.empty_like(X.float())
        g.gff_apply_operator(h, g.GFF_PREC_MIXED, None, X.float(), Y32)
        torch.cuda.synchronize()
        F = np.broadcast_to(np.eye(3).reshape(3, 3, 1, 1, 1), (3, 3, 128, 128, 128))
        _, K_ref = voxel_K_oracle(ms, F)
        ref = sp.GK(K_ref, x.reshape(3, 3, 128, 128, 128), (1.0, 1.0, 1.0), kind)
        del K_ref
        assert rel_l2(Y.cpu().numpy(), ref) <= 1e-12
        assert rel_l2(Y32.cpu().numpy(), ref) <= 2e-6
    finally:
        g.gff_destroy(h)


def test_invalid_sizes_are_rejected():
    torch_cuda()
    g = gff()
    for n in [(7, 8, 8), (8, 8, 14), (8, 8, 256), (2, 8, 8), (8, 8, 22)]:
        with pytest.raises(g.GffError) as e:
            g.gff_create(g.make_grid(*n))
        assert e.value.status == g.GFF_ERR_ARG


def test_apply_without_tangent_is_a_state_error():
    torch = torch_cuda()
    g = gff()
    h = g.gff_create(g.make_grid(8, 8, 8))
    try:
        X = torch.zeros(9 * 512, dtype=torch.float64, device="cuda")
        with pytest.raises(g.GffError) as e:
            g.gff_apply_operator(h, g.GFF_PREC_FP64, None, X, torch.empty_like(X))
        assert e.value.status == g.GFF_ERR_STATE
    finally:
        g.gff_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_launch_shapes_give_identical_results(prec):
    """Every launch shape -- one block per z strip or the persistent TMA z pass,
    one block per plane or the persistent bulk-copy inverse pass, with few blocks
    so that each walks several strips / planes -- computes the same operations in
    the same order: results equal bit for bit, and match the oracle."""
    torch = torch_cuda()
    g = gff()
    shape = (32, 32, 32)
    nz, ny, nx = shape
    ms = polycrystal(nx, 6, 9)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options())
    try:
        g.gff_constitutive(h, 1.0)
        x = _field(11, shape).reshape(9, -1)
        X = torch.from_numpy(x.copy()).cuda()
        if prec == 1:
            X = X.float()
        outs = []
        # (fwd threads, W, z threads, inv threads, inv blocks, TMA z blocks)
        shapes = [(512, 8, 256, 512, 0, 0), (256, 8, 256, 256, 0, 7), (512, 16, 512, 512, 5, 3),
                  (256, 16, 128, 512, 0, 0)]
        for s in shapes:
            g.gff_set_tiles(h, s, s)
            Y = torch.empty_like(X)
            g.gff_apply_operator(h, prec, None, X, Y)
            torch.cuda.synchronize()
            outs.append(Y.double().cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        F = np.tile(np.eye(3).reshape(3, 3, 1, 1, 1), (1, 1) + shape)
        _, K = voxel_K_oracle(ms, F)
        ref = sp.GK(K, x.reshape(3, 3, nz, ny, nx), ms.L, sp.KIND_CONTINUOUS)
        assert rel_l2(outs[0], ref.reshape(9, -1)) <= (1e-12 if prec == 0 else 2e-6)
        with pytest.raises(g.GffError):
            g.gff_set_tiles(h, (512, 4, 256, 512, 0, 5), (512, 4, 256, 512, 0, 5))  # no TMA at W = 4
    finally:
        g.gff_destroy(h)


@pytest.mark.parametrize("shape", [(64, 64, 64), (12, 128, 128), (128, 16, 32)])
@pytest.mark.parametrize("prec", [0, 1])
def test_register_staged_passes_are_bit_identical(shape, prec):
    """The register-staged passes of the two-stage plans -- the forward and the
    inverse plane passes for nx = ny = 64 (8 x 8) or 128 (16 x 8), tiles fwd
    threads -256 / -512 and inv blocks = -1 with 256 or 512 threads, and the TMA
    z pass's strip for nz = 64 or 128, TMA z blocks < 0 -- perform the
    operations of the generic passes in the same order: y equal bit for bit,
    with and without the mixed-control mask, and the oracle's."""
    torch = torch_cuda()
    nz, ny, nx = shape
    g, ms, h = _svk_handle(shape, 12, 21)
    inv2 = nx == ny and nx in (64, 128)
    z2 = nz in (64, 128)
    shapes = [(512, 8, 256, 512, 0, 0)]
    if inv2:
        shapes += [(512, 8, 256, 256, -1, 0), (512, 8, 256, 512, -1, 0), (256, 16, 256, 512, -1, 7),
                   (-256, 8, 256, 512, 0, 0), (-512, 8, 256, 256, -1, 0)]
        # persistent register-staged inverse (two plane buffers: FP32, and FP64 at n = 64), few blocks
        # so that each walks several planes
        if prec == 1:
            shapes += [(512, 8, 256, 512, -5, 0), (512, 8, 256, 1024, -3, 0)]
        elif nx == 64:
            shapes += [(512, 8, 256, 512, -6, 0)]
    if z2:
        shapes += [(512, 16, 256, 512, 0, -5), (256, 8, 256, 256, 0, -3)]
        if prec == 1:  # 384 threads: FP32 only
            shapes += [(512, 16, 384, 512, 0, -4)]
    if inv2 and z2:
        shapes += [(512, 16, 256, 512, -1, -11), (-256, 16, 256, 256, -1, -7)]
    try:
        g.gff_constitutive(h, 1.0)
        x = _field(13, shape).reshape(9, -1)
        X = torch.from_numpy(x.copy()).cuda()
        if prec == 1:
            X = X.float()
        outs = []
        base = (512, 8, 256, 512, 0, 0)
        for s in shapes:
            g.gff_set_tiles(h, s if prec == 0 else base, s if prec == 1 else base)
            for mask in (None, MASKS[1]):
                Y = torch.empty_like(X)
                g.gff_apply_operator(h, prec, mask, X, Y)
                g.gff_sync(h)
                outs.append(Y.double().cpu().numpy())
            Y = torch.empty_like(X)  # projection alone (the forward pass without K)
            g.gff_project(h, prec, MASKS[1], X, Y)
            g.gff_sync(h)
            outs.append(Y.double().cpu().numpy())
        for i in range(3, len(outs)):
            assert np.array_equal(outs[i], outs[i % 3]), (i // 3, i % 3)
        refG = sp.G(x.reshape(3, 3, nz, ny, nx), ms.L, sp.KIND_CONTINUOUS, MASKS[1].astype(np.float64))
        assert rel_l2(outs[2], refG.reshape(9, -1)) <= (1e-12 if prec == 0 else 2e-6)
        F = np.tile(np.eye(3).reshape(3, 3, 1, 1, 1), (1, 1) + shape)
        _, K = voxel_K_oracle(ms, F)
        ref = sp.GK(K, x.reshape(3, 3, nz, ny, nx), ms.L, sp.KIND_CONTINUOUS)
        assert rel_l2(outs[0], ref.reshape(9, -1)) <= (1e-12 if prec == 0 else 2e-6)
        refused = [(512, 8, 256, 1024, -1, 0), (-384, 8, 256, 512, 0, 0),  # not shapes of the passes
                   (512, 8, 256, 256, -5, 0)]
        if not inv2:
            refused += [(512, 8, 256, 512, -1, 0), (-256, 8, 256, 512, 0, 0)]
        if not z2:
            refused.append((512, 16, 256, 512, 0, -5))
        refused.append((512, 16, 192, 512, 0, -5))  # the register-staged strip runs 256 (or 384 in FP32) threads
        for s in refused:
            with pytest.raises(g.GffError):
                g.gff_set_tiles(h, s, s)
    finally:
        g.gff_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_bounded_wait_timeout_is_reported_and_recoverable(prec):
    """The inverse FFT pass waits on an asynchronous (TMA) copy with a bounded
    budget.  With the budget set to 0 every such wait gives up at once: the
    pass records it, lets its copies land and leaves its planes of y as NaN;
    gff_sync reports GFF_ERR_TIMEOUT once and clears the record.  With the
    default budget restored the same handle computes the oracle's result."""
    torch = torch_cuda()
    shape = (16, 16, 16)
    g, ms, h = _svk_handle(shape, 5, 3)
    try:
        g.gff_autotune(h)
        g.gff_constitutive(h, 1.0)
        x = _field(12, shape)
        X = torch.from_numpy(x.reshape(9, -1).copy()).cuda()
        if prec == 1:
            X = X.float()
        Y = torch.zeros_like(X)
        g.gff_set_wait_limit(h, 0)
        g.gff_apply_operator(h, prec, None, X, Y)  # queued: the device reports through gff_sync
        with pytest.raises(g.GffError) as e:
            g.gff_sync(h)
        assert e.value.status == g.GFF_ERR_TIMEOUT
        assert torch.isnan(Y).all()
        g.gff_sync(h)  # the record was cleared
        g.gff_set_wait_limit(h, -1)
        g.gff_apply_operator(h, prec, None, X, Y)
        g.gff_sync(h)
        F = np.tile(np.eye(3).reshape(3, 3, 1, 1, 1), (1, 1) + shape)
        _, K = voxel_K_oracle(ms, F)
        ref = sp.GK(K, x, ms.L, sp.KIND_CONTINUOUS)
        assert rel_l2(Y.double().cpu().numpy(), ref) <= (1e-12 if prec == 0 else 2e-6)
    finally:
        g.gff_destroy(h)


@pytest.mark.parametrize("tiles", [(512, 8, 256, 256, -1, 0), (512, 16, 256, 512, -5, -7)])
def test_bounded_wait_timeout_of_the_register_staged_passes(tiles):
    """The same error path in the register-staged passes (64^3, FP32): the
    inverse pass one block per plane (inv blocks -1, bulk copy) or persistent
    with two plane buffers (inv blocks -5), with the TMA z pass's register-
    staged strip (z blocks -7).  A zero budget leaves every plane of y NaN and
    gff_sync reports GFF_ERR_TIMEOUT once; the default budget then gives the
    bits of the generic passes."""
    torch = torch_cuda()
    shape = (64, 64, 64)
    g, ms, h = _svk_handle(shape, 12, 21)
    try:
        g.gff_constitutive(h, 1.0)
        X = torch.from_numpy(_field(14, shape).reshape(9, -1).copy()).cuda().float()
        base = (512, 8, 256, 512, 0, 0)
        g.gff_set_tiles(h, base, base)
        Yref = torch.empty_like(X)
        g.gff_apply_operator(h, 1, None, X, Yref)
        g.gff_sync(h)
        g.gff_set_tiles(h, base, tiles)
        Y = torch.zeros_like(X)
        g.gff_set_wait_limit(h, 0)
        g.gff_apply_operator(h, 1, None, X, Y)
        with pytest.raises(g.GffError) as e:
            g.gff_sync(h)
        assert e.value.status == g.GFF_ERR_TIMEOUT
        assert torch.isnan(Y).all()
        g.gff_sync(h)
        g.gff_set_wait_limit(h, -1)
        g.gff_apply_operator(h, 1, None, X, Y)
        g.gff_sync(h)
        assert torch.equal(Y, Yref)
    finally:
        g.gff_destroy(h)


def test_timeout_fails_the_increment_and_keeps_the_state():
    """A load increment whose residual evaluation meets a timed-out wait
    returns GFF_ERR_TIMEOUT (no cut-back: it is not a convergence failure)
    and commits nothing; the next increment at the default budget runs."""
    torch_cuda()
    g, ms, h = _svk_handle((8, 8, 8), 3, 4)
    try:
        g.gff_autotune(h)
        N = ms.n_voxels
        Fbar = np.eye(3).ravel() + np.array([0.004, 0, 0, 0, -0.002, 0, 0, 0, -0.002])
        zero9 = np.zeros(9)
        g.gff_set_wait_limit(h, 0)
        with pytest.raises(g.GffError) as e:
            g.gff_step(h, 1.0, Fbar, np.zeros(9, np.uint8), zero9)
        assert e.value.status == g.GFF_ERR_TIMEOUT
        F = g.gff_get_field(h, g.GFF_FIELD_F, N)
        assert np.array_equal(F, np.tile(np.eye(3).reshape(9, 1), (1, N)).ravel())
        g.gff_set_wait_limit(h, -1)
        rep = g.gff_step(h, 1.0, Fbar, np.zeros(9, np.uint8), zero9)
        assert rep.residual <= 1e-8 and np.allclose(rep.Fmacro, Fbar, rtol=0, atol=1e-14)
    finally:
        g.gff_destroy(h)


# 64^3 takes 8 chunks of 8 planes; 36 planes split 4 / 5 unevenly; the persistent inverse
# passes (streamed with 5 blocks, register-staged with 4) are replaced per chunk
HOST_CASES = [((64, 64, 64), None), ((36, 48, 64), None), ((64, 64, 64), (512, 8, 256, 512, 5, 0)),
              ((64, 64, 64), (-256, 8, 256, 512, -4, 0)), ((8, 16, 16), None)]


@pytest.mark.parametrize("shape,tiles", HOST_CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_host_buffer_apply_equals_device_apply(shape, tiles, prec):
    """gff_apply_operator_host copies x in and y out in chunks of z-planes that
    overlap the plane passes of the other chunks: the same kernels on the same
    planes as gff_apply_operator, so y is bitwise the same -- from pageable and
    from pinned host buffers, on repeated calls."""
    torch = torch_cuda()
    g = gff()
    ms = polycrystal(shape, 6, 9)
    h = g.create_rve(ms, {0: g.make_material(g.GFF_MAT_SVK_CUBIC)}, g.make_options())
    try:
        g.gff_constitutive(h, 1.0)
        if tiles is not None:
            g.gff_set_tiles(h, tiles, tiles)
        dt = np.float64 if prec == 0 else np.float32
        xh = np.ascontiguousarray(_field(13, shape).reshape(9, -1).astype(dt))
        X = torch.from_numpy(xh.copy()).cuda()
        Y = torch.empty_like(X)
        g.gff_apply_operator(h, prec, MASKS[1], X, Y)
        torch.cuda.synchronize()
        ref = Y.cpu().numpy()
        yh = np.full_like(xh, np.nan)
        g.gff_apply_operator_host(h, prec, MASKS[1], xh, yh)
        assert np.array_equal(yh, ref)
        xp = torch.from_numpy(xh.copy()).pin_memory()
        yp = torch.empty_like(xp).pin_memory()
        for _ in range(2):
            yp.fill_(float("nan"))
            g.gff_apply_operator_host(h, prec, MASKS[1], xp, yp)
            assert np.array_equal(yp.numpy(), ref)
    finally:
        g.gff_destroy(h)
