"""Projection operators and the discrete equilibrium operator (Sect. 2.1-2.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Fields are numpy arrays of shape (3, 3, nz, ny, nx): tensor indices first,
then voxels with x fastest.  The discrete Fourier transform is numpy's
unnormalised forward fftn and 1/N inverse ifftn over the three voxel axes.

Readings of the paper used here:
  * frequencies (Eq. xis) are taken in FFT order: index k maps to
    q = 2 pi kappa / n with kappa = k for k < n/2 and k - n otherwise, which
    is the paper's set; for even n the index k = n/2 is the Nyquist
    frequency (kappa = -n/2, q = -pi).
  * the garbled length scaling of Eq. G is read as the physical wavenumber
    q~_j = q_j n_j / L_j (the derivative of Eq. 1Ddif on a voxel grid of
    spacing h_j = L_j / n_j); the discrete operator uses
    q~'_j = tan(q_j / 2) n_j / L_j.  The common complex factor of the
    rotated-difference wave vector cancels in G^', so G^' is real.
  * "null and Nyquist frequencies": the operator is zero where q = 0 or
    where any axis index sits at its Nyquist frequency.
  * mixed macroscopic control: at q = 0 the operator is replaced by the
    diagonal projector M onto the stress-controlled components (mask9[c] = 1),
    so that the zero frequency carries the average-stress condition.
"""

import numpy as np

KIND_CONTINUOUS = 0
KIND_DISCRETE = 1

_DELTA = np.eye(3)


def axis_frequencies(n):
    """q for each FFT index k of an axis with n voxels (Eq. xis, FFT order),
    and a flag marking the Nyquist index."""
    k = np.arange(n)
    kappa = np.where(k < n / 2.0, k, k - n)
    q = 2.0 * np.pi * kappa / n
    nyq = (n % 2 == 0) & (k == n // 2)
    return q, nyq


def wavevectors(shape, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS):
    """Scaled wave vector q~ (Eq. G) or q~' (discrete operator, Sect. 2.2)
    on the full grid, plus the masks of the zero frequency and of the
    frequencies where the operator vanishes (zero or any Nyquist index).

    shape = (nz, ny, nx); L = (Lx, Ly, Lz).  Returns qt of shape
    (3, nz, ny, nx) with qt[0] along x."""
    nz, ny, nx = shape
    out = []
    nyqs = []
    for n, Lj in ((nx, L[0]), (ny, L[1]), (nz, L[2])):
        q, nyq = axis_frequencies(n)
        if kind == KIND_CONTINUOUS:
            qt = q * n / Lj
        else:
            with np.errstate(divide="ignore", invalid="ignore"):
                qt = np.tan(q / 2.0) * n / Lj
            qt = np.where(nyq, 0.0, qt)  # value unused: the operator is zero there
        out.append(qt)
        nyqs.append(nyq)
    qz, qy, qx = np.meshgrid(out[2], out[1], out[0], indexing="ij")
    bz, by, bx = np.meshgrid(nyqs[2], nyqs[1], nyqs[0], indexing="ij")
    zero = np.zeros(shape, dtype=bool)
    zero[0, 0, 0] = True
    vanish = bx | by | bz | zero
    return np.stack([qx, qy, qz]), zero, vanish


def gamma_hat_tensor(qt):
    """Fourth-order projection at one non-null frequency:
    G_ijkl = delta_ik q_j q_l / (q . q)  (Eq. G with q -> q~, or Sect. 2.2's
    G^' with q -> q~')."""
    qt = np.asarray(qt, dtype=np.float64)
    return np.einsum("ik,j,l->ijkl", _DELTA, qt, qt) / (qt @ qt)


def project_hat(xh, shape, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """y^ = G^ : x^ at every frequency of a (3, 3, nz, ny, nx) spectrum."""
    qt, zero, vanish = wavevectors(shape, L, kind)
    qq = np.einsum("m...,m...->...", qt, qt)
    with np.errstate(divide="ignore", invalid="ignore"):
        nvec = np.where(vanish[None], 0.0, qt / np.sqrt(np.where(vanish, 1.0, qq))[None])
    yh = np.einsum("ik,j...,l...,kl...->ij...", _DELTA, nvec, nvec, xh)
    if mask9 is not None:
        m = np.asarray(mask9, dtype=np.float64).reshape(3, 3)
        yh[:, :, 0, 0, 0] = m * xh[:, :, 0, 0, 0]
    return yh


def fft3(A):
    """Forward DFT (unnormalised, exp(-2 pi i k.x / n)) over the voxel axes."""
    return np.fft.fftn(A, axes=(-3, -2, -1))


def ifft3(Ah):
    """Inverse DFT (scaled by 1/N) over the voxel axes."""
    return np.fft.ifftn(Ah, axes=(-3, -2, -1))


def G(A, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """Discrete equilibrium operator G(A) = F^-1{ G^ : F(A) } (Eq.
    eql_discrete3) of a real tensor field A (3, 3, nz, ny, nx)."""
    shape = A.shape[2:]
    return np.real(ifft3(project_hat(fft3(A), shape, L, kind, mask9)))


def ddot42(K, A):
    """(K : A)_ij = K_ijkl A_kl per voxel; K has shape (3,3,3,3,nz,ny,nx)."""
    return np.einsum("ijkl...,kl...->ij...", K, A)


def GK(K, A, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """Tangent operator G_K(A) = G(K : A) (Eq. newlinop)."""
    return G(ddot42(K, A), L, kind, mask9)


# --------------------------------------------------------------------------- small-strain variant
def project_hat_sym(xh, shape, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """Orthogonal projection onto compatible symmetric (small) strains,
    sym(q (x) u), at every frequency: with n the unit scaled wave vector and
    a = sym(x^) n,  y^ = n (x) a + a (x) n - (n . a) n (x) n.  Zero where the
    finite-strain operator is zero; the zero frequency takes the mask."""
    qt, zero, vanish = wavevectors(shape, L, kind)
    qq = np.einsum("m...,m...->...", qt, qt)
    with np.errstate(divide="ignore", invalid="ignore"):
        n = np.where(vanish[None], 0.0, qt / np.sqrt(np.where(vanish, 1.0, qq))[None])
    xs = 0.5 * (xh + np.swapaxes(xh, 0, 1))
    a = np.einsum("jk...,k...->j...", xs, n)
    na = np.einsum("j...,j...->...", n, a)
    yh = np.einsum("i...,j...->ij...", n, a) + np.einsum("i...,j...->ij...", a, n) - na * np.einsum(
        "i...,j...->ij...", n, n)
    if mask9 is not None:
        m = np.asarray(mask9, dtype=np.float64).reshape(3, 3)
        yh[:, :, 0, 0, 0] = m * xh[:, :, 0, 0, 0]
    return yh


def G_sym(A, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """Small-strain equilibrium operator F^-1{ G^s : F(A) } of a real field A (3, 3, nz, ny, nx)."""
    shape = A.shape[2:]
    return np.real(ifft3(project_hat_sym(fft3(A), shape, L, kind, mask9)))


def GK_sym(K, A, L=(1.0, 1.0, 1.0), kind=KIND_CONTINUOUS, mask9=None):
    """Small-strain tangent operator G^s(K : A)."""
    return G_sym(ddot42(K, A), L, kind, mask9)
