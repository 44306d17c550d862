"""Pins of the oracle's Appendix-A conversion of a umat's outputs (Cauchy
stress and the Jaumann-rate tangent C^ab of Eq. ABAtang) into the first
Piola-Kirchhoff stress and the tangent K = dP/dF the FFT solver needs.

The checks use a compressible neo-Hookean solid, whose P(F) has a closed
form independent of the conversion:
  * P from the conversion equals mu (F - F^-T) + lam ln(J) F^-T;
  * K from the conversion equals central differences of that closed form;
  * the neo-Hookean C^ab used as input equals central differences of the
    definition of Eq. ABAtang (Jaumann rate of the Kirchhoff stress along
    pure stretching rates d);
  * at F = I and zero stress, K = C^ab (the small-strain limit).
"""

import numpy as np

from oracle import materials as mat

LAM, MU = 111.1e9, 166.7e9


def _P_closed(F):
    Fit = np.linalg.inv(F).transpose(0, 2, 1)
    J = np.linalg.det(F)
    return MU * (F - Fit) + LAM * np.log(J)[:, None, None] * Fit


def _tau_closed(F):
    b = F @ F.transpose(0, 2, 1)
    return MU * (b - np.eye(3)) + LAM * np.log(np.linalg.det(F))[:, None, None] * np.eye(3)


def _random_F(n, scale, seed):
    rng = np.random.default_rng(seed)
    return np.eye(3)[None] + scale * rng.standard_normal((n, 3, 3))


def test_stress_is_the_closed_form_piola_stress():
    F = _random_F(20, 0.05, 1)
    sig, C = mat.neo_hookean_umat(F, LAM, MU)
    P, _ = mat.umat_to_PK(F, sig, C)
    assert np.allclose(P, _P_closed(F), rtol=0, atol=1e-12 * np.abs(_P_closed(F)).max())


def test_tangent_matches_finite_differences_of_P():
    F = _random_F(12, 0.08, 2)
    sig, C = mat.neo_hookean_umat(F, LAM, MU)
    _, K = mat.umat_to_PK(F, sig, C)
    h = 1e-6
    Kfd = np.empty_like(K)
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = h
            Kfd[:, :, :, k, l] = (_P_closed(F + E) - _P_closed(F - E)) / (2 * h)
    assert np.abs(K - Kfd).max() <= 1e-6 * np.abs(K).max()


def test_neo_hookean_Cab_is_the_jaumann_rate_tangent():
    """tau(F + eps d F) - tau(F) = eps J C^ab : d (+ O(eps^2)) for symmetric d (no spin)."""
    F = _random_F(6, 0.1, 3)
    sig, C = mat.neo_hookean_umat(F, LAM, MU)
    J = np.linalg.det(F)
    eps = 1e-6
    for k in range(3):
        for l in range(k, 3):
            d = np.zeros((3, 3))
            d[k, l] = d[l, k] = 0.5 if k != l else 1.0
            dF = d @ F  # velocity gradient L = d (pure stretching)
            rate = (_tau_closed(F + eps * dF) - _tau_closed(F - eps * dF)) / (2 * eps)
            want = J[:, None, None] * np.einsum("vijkl,kl->vij", C, d)
            assert np.abs(rate - want).max() <= 1e-6 * np.abs(want).max()


def test_small_strain_limit_returns_Cab():
    F = np.broadcast_to(np.eye(3), (3, 3, 3)).copy()
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 3, 3, 3, 3))
    Cab = 0.5 * (A + A.transpose(0, 1, 2, 4, 3))  # minor symmetry in kl
    Cab = 0.5 * (Cab + Cab.transpose(0, 2, 1, 3, 4))  # and in ij
    P, K = mat.umat_to_PK(F, np.zeros((3, 3, 3)), Cab)
    assert np.abs(P).max() == 0.0
    assert np.allclose(K, Cab, rtol=0, atol=1e-15)
