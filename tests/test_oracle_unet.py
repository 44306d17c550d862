"""Pins of the oracle's U-Net pieces: brute-force convolution, adjoint
identities of every linear map and its gradient, finite-difference
gradients of the whole network, and bfloat16 rounding."""

import numpy as np
import pytest

from oracle import unet as U


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_brute_force():
    x = _rand((3, 4, 5, 6), 1)
    W = _rand((27, 2, 3), 2)
    b = _rand(2, 3)
    y = U.conv(x, W, b)
    C, nz, ny, nx = x.shape
    ref = np.zeros((2, nz, ny, nx))
    for o in range(2):
        for z in range(nz):
            for yy in range(ny):
                for xx in range(nx):
                    s = b[o]
                    for t, (dz, dy, dx) in enumerate(U.TAPS):
                        for i in range(C):
                            s += W[t, o, i] * x[i, (z + dz) % nz, (yy + dy) % ny, (xx + dx) % nx]
                    ref[o, z, yy, xx] = s
    assert np.abs(y - ref).max() < 1e-12


def test_linear_maps_and_their_adjoints():
    x = _rand((3, 4, 6, 8), 4)
    W = _rand((27, 5, 3), 5)
    dy = _rand((5, 4, 6, 8), 6)
    lhs = np.sum(U.conv(x, W) * dy)
    assert abs(lhs - np.sum(x * U.conv_grad_input(dy, W))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * U.conv_grad_weight(x, dy))) < 1e-10 * abs(lhs)
    p = _rand((3, 2, 3, 4), 7)
    assert abs(np.sum(U.pool(x) * p) - np.sum(x * U.pool_grad(p))) < 1e-12
    q = _rand((3, 8, 12, 16), 8)
    assert abs(np.sum(U.up(x) * q) - np.sum(x * U.up_grad(q))) < 1e-10
    assert np.allclose(U.pool(U.up(x)), x)


def test_network_gradient_matches_finite_differences():
    p = U.init_params(3)
    x = _rand((U.IN_CH, 8, 8, 8), 9)
    t = _rand((9, 8, 8, 8), 10)
    y, cache = U.forward(p, x)
    loss, dy = U.mse(y, t)
    g = U.backward(p, cache, dy)
    rng = np.random.default_rng(11)
    h = 1e-6
    floor = 4 * np.finfo(float).eps * loss / h  # round-off of the central difference
    for name in ("e1a", "e3b", "e4a", "d3a", "d1b", "head"):
        W, b = p[name]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in W.shape)
            W0 = W[idx]
            W[idx] = W0 + h
            lp, _ = U.mse(U.forward(p, x)[0], t)
            W[idx] = W0 - h
            lm, _ = U.mse(U.forward(p, x)[0], t)
            W[idx] = W0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][0][idx]) <= 1e-6 * abs(fd) + floor, (name, idx)
        j = rng.integers(0, b.shape[0])
        b0 = b[j]
        b[j] = b0 + h
        lp, _ = U.mse(U.forward(p, x)[0], t)
        b[j] = b0 - h
        lm, _ = U.mse(U.forward(p, x)[0], t)
        b[j] = b0
        assert abs((lp - lm) / (2 * h) - g[name][1][j]) <= 1e-6 * abs((lp - lm) / (2 * h)) + floor


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1e-3, 3.0e38])
    r = U.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # tie -> even
    assert r[2] == 1.0 + 2 * 2.0 ** -7  # tie -> even (odd mantissa rounds up)
    assert r[3] == -2.5
    assert abs(r[4] - 1e-3) <= 2.0 ** -8 * 1e-3
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(12).standard_normal(1000) * 10.0 ** np.random.default_rng(13).integers(-5, 5, 1000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x), ref)
