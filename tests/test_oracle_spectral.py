"""Pins of the oracle's transforms and projection operators (Sect. 2.1-2.2).

Every check below is independent of the formula it pins: brute-force DFT
sums, fields built in real space from analytic derivatives or explicit
finite-difference stencils, and algebraic invariants of a projector."""

import numpy as np
import pytest

from oracle import spectral as sp


def brute_dft(A):
    """Definition of the unnormalised 3D DFT, exp(-2 pi i k.x / n), on a
    (..., nz, ny, nx) array, written as explicit sums."""
    nz, ny, nx = A.shape[-3:]
    out = np.zeros(A.shape, dtype=complex)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for kz in range(nz):
        for ky in range(ny):
            for kx in range(nx):
                ph = np.exp(-2j * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz))
                out[..., kz, ky, kx] = (A * ph).sum(axis=(-3, -2, -1))
    return out


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 5, 4), (10, 3, 6)])
def test_fft_matches_brute_force_dft(shape):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3) + shape)
    ref = brute_dft(A)
    got = sp.fft3(A)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    back = sp.ifft3(got)
    assert np.abs(back - A).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("n", [4, 5, 8, 9, 16, 15])
def test_axis_frequencies_are_the_paper_set(n):
    # Eq. xis: q_i = 2 pi (n/2 - i)/n (n even), 2 pi ((n+1)/2 - i)/n (n odd), i = 1..n
    i = np.arange(1, n + 1)
    paper = 2 * np.pi * ((n / 2 - i) if n % 2 == 0 else ((n + 1) / 2 - i)) / n
    q, nyq = sp.axis_frequencies(n)
    assert np.allclose(np.sort(q), np.sort(paper), atol=1e-15)
    # FFT index k carries exp(-2 pi i k x / n) = exp(-i q x): q = 2 pi k / n mod 2 pi
    k = np.arange(n)
    assert np.allclose(np.exp(1j * q), np.exp(2j * np.pi * k / n))
    assert nyq.sum() == (1 if n % 2 == 0 else 0)
    if n % 2 == 0:
        assert abs(abs(q[nyq][0]) - np.pi) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_gamma_hat_is_symmetric_idempotent_projector(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(3)
    G = sp.gamma_hat_tensor(q).reshape(9, 9)
    assert np.allclose(G, G.T, atol=1e-15)
    assert np.allclose(G @ G, G, atol=1e-14)
    assert abs(np.trace(G) - 3.0) < 1e-13  # rank 3: one free vector a in a (x) q
    # compatible tensors a (x) q are kept, equilibrated ones (B q = 0) are removed
    a = rng.standard_normal(3)
    comp = np.outer(a, q).reshape(9)
    assert np.allclose(G @ comp, comp, atol=1e-13 * np.abs(comp).max())
    B = rng.standard_normal((3, 3))
    B = B - np.outer(B @ q, q) / (q @ q)
    assert np.allclose(B @ q, 0, atol=1e-13)
    assert np.allclose(G @ B.reshape(9), 0, atol=1e-13)


def _grid_centres(shape, L):
    nz, ny, nx = shape
    h = np.array(L) / np.array([nx, ny, nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (x + 0.5) * h[0], (y + 0.5) * h[1], (z + 0.5) * h[2]


@pytest.mark.parametrize("L", [(1.0, 1.0, 1.0), (1.0, 2.0, 0.5)])
def test_continuous_projection_keeps_gradients_and_kills_divergence_free(L):
    shape = (8, 12, 10)
    nz, ny, nx = shape
    X = _grid_centres(shape, L)
    rng = np.random.default_rng(3)
    F = np.zeros((3, 3) + shape)
    Pdiv = np.zeros((3, 3) + shape)
    for _ in range(6):
        kap = np.array([rng.integers(-nx // 2 + 1, nx // 2), rng.integers(-ny // 2 + 1, ny // 2),
                        rng.integers(-nz // 2 + 1, nz // 2)])
        kvec = 2 * np.pi * kap / np.array(L)
        ph = kvec[0] * X[0] + kvec[1] * X[1] + kvec[2] * X[2] + rng.uniform(0, 2 * np.pi)
        a = rng.standard_normal(3)
        # u = a cos(k.x + phi): grad u_ij = -a_i k_j sin(.)
        F += -np.einsum("i,j,...->ij...", a, kvec, np.sin(ph))
        # P_ij = eps_jmn d_m psi_in with psi_in = b_in cos(k.x + phi): divergence free rows
        b = rng.standard_normal((3, 3))
        eps = np.zeros((3, 3, 3))
        eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
        eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
        Pdiv += -np.einsum("jmn,m,in,...->ij...", eps, kvec, b, np.sin(ph))
    GF = sp.G(F, L, sp.KIND_CONTINUOUS)
    assert np.abs(GF - F).max() <= 1e-12 * np.abs(F).max()
    GP = sp.G(Pdiv, L, sp.KIND_CONTINUOUS)
    assert np.abs(GP).max() <= 1e-12 * np.abs(Pdiv).max()
    # the discrete operator is a different projector: it does not keep this field
    GdF = sp.G(F, L, sp.KIND_DISCRETE)
    assert np.abs(GdF - F).max() > 1e-3 * np.abs(F).max()


def rotated_fd_gradient(u, L):
    """Rotated centred difference of corner displacements u (3, nz, ny, nx):
    u[:, k, j, i] sits at corner (i h_x, j h_y, k h_z); the gradient at voxel
    centre (i+1/2, j+1/2, k+1/2) averages the four edge differences along
    each axis."""
    nz, ny, nx = u.shape[1:]
    h = np.array(L) / np.array([nx, ny, nz])

    def sh(a, dz, dy, dx):
        return np.roll(a, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))

    F = np.zeros((3, 3, nz, ny, nx))
    for b in (0, 1):
        for c in (0, 1):
            F[:, 0] += sh(u, c, b, 1) - sh(u, c, b, 0)
            F[:, 1] += sh(u, c, 1, b) - sh(u, c, 0, b)
            F[:, 2] += sh(u, 1, c, b) - sh(u, 0, c, b)
    F[:, 0] /= 4 * h[0]
    F[:, 1] /= 4 * h[1]
    F[:, 2] /= 4 * h[2]
    return F


def rotated_fd_divergence_adjoint(P, L):
    """Adjoint (w.r.t. the plain sum over voxels) of rotated_fd_gradient,
    mapping a centre field P (3,3,...) to a corner vector field; a stress is
    discretely equilibrated iff this vanishes."""
    nz, ny, nx = P.shape[2:]
    h = np.array(L) / np.array([nx, ny, nz])

    def sh(a, dz, dy, dx):
        return np.roll(a, shift=(dz, dy, dx), axis=(-3, -2, -1))

    out = np.zeros((3, nz, ny, nx))
    for b in (0, 1):
        for c in (0, 1):
            out += (sh(P[:, 0], c, b, 1) - sh(P[:, 0], c, b, 0)) / (4 * h[0])
            out += (sh(P[:, 1], c, 1, b) - sh(P[:, 1], c, 0, b)) / (4 * h[1])
            out += (sh(P[:, 2], 1, c, b) - sh(P[:, 2], 0, c, b)) / (4 * h[2])
    return out


@pytest.mark.parametrize("L", [(1.0, 1.0, 1.0), (1.0, 2.0, 0.5)])
def test_discrete_projection_matches_rotated_difference_scheme(L):
    shape = (5, 7, 9)  # odd: no Nyquist frequencies
    rng = np.random.default_rng(4)
    u = rng.standard_normal((3,) + shape)
    F = rotated_fd_gradient(u, L)
    # adjoint check of the two stencils
    P = rng.standard_normal((3, 3) + shape)
    lhs = np.sum(F * P)
    rhs = np.sum(u * rotated_fd_divergence_adjoint(P, L))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    # discrete gradients are kept by G^'
    GF = sp.G(F, L, sp.KIND_DISCRETE)
    assert np.abs(GF - F).max() <= 1e-12 * np.abs(F).max()
    # the equilibrated part (I - G^') P has zero discrete divergence
    R = P - sp.G(P, L, sp.KIND_DISCRETE) - P.reshape(9, -1).mean(axis=1).reshape(3, 3)[:, :, None, None, None]
    div = rotated_fd_divergence_adjoint(R, L)
    assert np.abs(div).max() <= 1e-11 * np.abs(rotated_fd_divergence_adjoint(P, L)).max()
    # the continuous operator does not keep discrete gradients
    assert np.abs(sp.G(F, L, sp.KIND_CONTINUOUS) - F).max() > 1e-3 * np.abs(F).max()


@pytest.mark.parametrize("kind", [sp.KIND_CONTINUOUS, sp.KIND_DISCRETE])
def test_projection_on_grid_invariants(kind):
    shape = (6, 8, 10)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3) + shape)
    B = rng.standard_normal((3, 3) + shape)
    GA = sp.G(A, kind=kind)
    # real result, idempotent, self-adjoint, zero mean
    Ah = sp.project_hat(sp.fft3(A), shape, kind=kind)
    assert np.abs(np.imag(sp.ifft3(Ah))).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(sp.G(GA, kind=kind) - GA).max() <= 1e-13 * np.abs(GA).max()
    assert abs(np.sum(B * GA) - np.sum(sp.G(B, kind=kind) * A)) <= 1e-12 * np.sqrt(np.sum(A * A) * np.sum(B * B))
    assert np.abs(GA.reshape(9, -1).mean(axis=1)).max() <= 1e-14
    # no content at any Nyquist index
    h = sp.fft3(GA)
    assert np.abs(h[..., 3, :, :]).max() < 1e-12
    assert np.abs(h[..., :, 4, :]).max() < 1e-12
    assert np.abs(h[..., :, :, 5]).max() < 1e-12


def test_mixed_control_mask_acts_on_the_average():
    shape = (4, 4, 4)
    rng = np.random.default_rng(6)
    mask = np.array([0, 1, 1, 1, 1, 1, 1, 1, 0], dtype=np.float64)
    Abar = rng.standard_normal(9)
    A = np.broadcast_to(Abar.reshape(3, 3)[:, :, None, None, None], (3, 3) + shape).copy()
    out = sp.G(A, mask9=mask)
    assert np.allclose(out, (mask * Abar).reshape(3, 3)[:, :, None, None, None], atol=1e-15)
    fluct = rng.standard_normal((3, 3) + shape)
    fluct -= fluct.reshape(9, -1).mean(axis=1).reshape(3, 3)[:, :, None, None, None]
    assert np.allclose(sp.G(A + fluct, mask9=mask) - sp.G(fluct), out, atol=1e-13)
