"""Pins of the oracle's constitutive laws (Sect. 3.2 and its reading).

Closed forms of rotations and cubic symmetry, energy/finite-difference
derivatives, and convergence of the implicit return map to an independent
explicit integration of the same rate equations."""

import numpy as np
import pytest

from oracle import materials as mat

C11, C12, C44 = 168.4e9, 121.4e9, 75.4e9


def test_quaternion_rotation_about_z():
    th = 0.7
    R = mat.quat_to_rot(np.array([np.cos(th / 2), 0, 0, np.sin(th / 2)]))
    assert np.allclose(R @ [1, 0, 0], [np.cos(th), np.sin(th), 0], atol=1e-15)
    assert np.allclose(R @ [0, 0, 1], [0, 0, 1], atol=1e-15)
    rng = np.random.default_rng(0)
    q = rng.standard_normal((20, 4))
    Rs = mat.quat_to_rot(q)
    assert np.allclose(np.einsum("vki,vkj->vij", Rs, Rs), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(Rs), 1.0, atol=1e-14)
    # q and -q are the same rotation
    assert np.allclose(mat.quat_to_rot(-q), Rs, atol=1e-15)


def test_cubic_stiffness_voigt_entries_and_symmetry():
    C = mat.cubic_stiffness(C11, C12, C44)
    assert C[0, 0, 0, 0] == C11 and C[1, 1, 2, 2] == C12 and C[1, 2, 1, 2] == C44
    assert C[0, 0, 0, 1] == 0.0
    # 90 degree rotation about [001] maps the cubic crystal onto itself
    R90 = mat.quat_to_rot([np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)])
    assert np.allclose(mat.rotate4(C, R90), C, atol=1e-6 * C11)
    # 45 degrees about [001]: C'_1111 = (C11 + C12 + 2 C44)/2, C'_1122 = (C11 + C12 - 2 C44)/2
    R45 = mat.quat_to_rot([np.cos(np.pi / 8), 0, 0, np.sin(np.pi / 8)])
    Cr = mat.rotate4(C, R45)
    assert abs(Cr[0, 0, 0, 0] - (C11 + C12 + 2 * C44) / 2) < 1e-6 * C11
    assert abs(Cr[0, 0, 1, 1] - (C11 + C12 - 2 * C44) / 2) < 1e-6 * C11
    assert abs(Cr[0, 1, 0, 1] - (C11 - C12) / 2) < 1e-6 * C11


def test_isotropic_stiffness_uniaxial_stress_gives_E_and_nu():
    E, nu = 400e9, 0.2
    C = mat.isotropic_stiffness(E, nu)
    # uniaxial strain state for unit uniaxial stress: eps = diag(1/E, -nu/E, -nu/E)
    eps = np.diag([1 / E, -nu / E, -nu / E])
    sig = np.einsum("ijkl,kl->ij", C, eps)
    assert np.allclose(sig, np.diag([1.0, 0, 0]), atol=1e-12)


def test_slip_systems_are_the_12_octahedral_systems():
    s, m = mat.fcc_slip_systems()
    assert s.shape == (12, 3) and m.shape == (12, 3)
    assert np.allclose(np.einsum("ai,ai->a", s, m), 0, atol=1e-15)
    assert np.allclose(np.linalg.norm(s, axis=1), 1) and np.allclose(np.linalg.norm(m, axis=1), 1)
    # all distinct systems, 4 planes x 3 directions, <110> directions and {111} normals
    assert len({tuple(np.round(np.r_[s[a], m[a]], 6)) for a in range(12)}) == 12
    assert np.allclose(np.sort(np.abs(s * np.sqrt(2)), axis=1), [[0, 1, 1]] * 12)
    assert np.allclose(np.abs(m * np.sqrt(3)), 1)


def _rand_F(rng, V, amp=0.05):
    return np.eye(3)[None] + amp * rng.standard_normal((V, 3, 3))


def test_svk_stress_is_energy_derivative_and_tangent_is_stress_derivative():
    rng = np.random.default_rng(1)
    C = mat.rotate4(mat.cubic_stiffness(C11, C12, C44), mat.quat_to_rot(rng.standard_normal(4)))
    F = _rand_F(rng, 4)
    P, K = mat.svk(F, C)

    def energy(F):
        E = 0.5 * (np.einsum("vki,vkj->vij", F, F) - np.eye(3))
        return 0.5 * np.einsum("vij,ijkl,vkl->v", E, C, E)

    h = 1e-6
    Pfd = np.zeros_like(P)
    Kfd = np.zeros_like(K)
    for k in range(3):
        for l in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[:, k, l] += h
            Fm[:, k, l] -= h
            Pfd[:, k, l] = (energy(Fp) - energy(Fm)) / (2 * h)
            Kfd[:, :, :, k, l] = (mat.svk(Fp, C)[0] - mat.svk(Fm, C)[0]) / (2 * h)
    assert np.abs(P - Pfd).max() <= 1e-7 * np.abs(P).max()
    assert np.abs(K - Kfd).max() <= 1e-7 * np.abs(K).max()
    # small-strain limit: linear elasticity with the same C
    e = 1e-7 * rng.standard_normal((1, 3, 3))
    P0, K0 = mat.svk(np.eye(3)[None] + e, C)
    lin = np.einsum("ijkl,vkl->vij", C, 0.5 * (e + np.swapaxes(e, 1, 2)))
    assert np.abs(P0 - lin).max() <= 1e-6 * np.abs(lin).max()
    assert np.abs(mat.svk(np.eye(3)[None], C)[1][0] - C).max() <= 1e-12 * C11


def _grain(seed):
    R = mat.quat_to_rot(np.random.default_rng(seed).standard_normal(4))
    return mat.rotate4(mat.cubic_stiffness(C11, C12, C44), R), mat.schmid_tensors(R)


def test_cp_tangent_matches_finite_differences():
    C, S0 = _grain(2)
    prm = mat.CPParams()
    rng = np.random.default_rng(3)
    F = np.eye(3)[None] + np.diag([3e-3, -1.5e-3, -1.5e-3])[None] + 2e-4 * rng.standard_normal((3, 3, 3))
    Fpi = np.eye(3)[None] + 1e-4 * rng.standard_normal((3, 3, 3))
    chi = 20e6 * rng.standard_normal((3, 12))
    out = mat.cp_return_map(F, Fpi, chi, 0.05, S0, C, prm)
    assert out["conv"].all()
    assert np.abs(out["dg"]).max() > 1e-5  # plastic flow is active
    h = 1e-7
    Kfd = np.zeros_like(out["K"])
    for k in range(3):
        for l in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[:, k, l] += h
            Fm[:, k, l] -= h
            Kfd[:, :, :, k, l] = (mat.cp_return_map(Fp, Fpi, chi, 0.05, S0, C, prm)["P"]
                                  - mat.cp_return_map(Fm, Fpi, chi, 0.05, S0, C, prm)["P"]) / (2 * h)
    assert np.abs(out["K"] - Kfd).max() <= 1e-6 * np.abs(out["K"]).max()


def test_cp_elastic_limit_is_svk():
    C, S0 = _grain(4)
    prm = mat.CPParams()
    F = np.eye(3)[None] + np.diag([2e-4, -1e-4, -1e-4])[None]
    out = mat.cp_return_map(F, np.eye(3)[None], np.zeros((1, 12)), 0.05, S0, C, prm)
    P, K = mat.svk(F, C)
    assert np.abs(out["dg"]).max() < 1e-15
    assert np.abs(out["P"] - P).max() <= 1e-12 * np.abs(P).max()
    assert np.abs(out["K"] - K).max() <= 1e-9 * np.abs(K).max()


def _explicit_cp(F_of_t, t_end, nsub, S0, C, prm):
    """Independent explicit RK4 integration of the rate equations the return
    map discretises: gdot_a = gdot0 h((tau_a - chi_a)/tau0),
    chi_dot = c gdot - d |gdot| chi, d(Fp^-1)/dt = -Fp^-1 sum_a gdot_a S0_a."""
    def rates(t, y):
        Fpi = y[:9].reshape(3, 3)
        chi = y[9:]
        F = F_of_t(t)
        Fe = F @ Fpi
        Ce = Fe.T @ Fe
        S = np.einsum("ijkl,kl->ij", C, 0.5 * (Ce - np.eye(3)))
        tau = np.einsum("ij,aij->a", Ce @ S, S0)
        x = (tau - chi) / prm.tau0
        gd = prm.gdot0 * np.sign(x) * np.abs(x) ** prm.p
        dFpi = -Fpi @ np.einsum("a,aij->ij", gd, S0)
        dchi = prm.c_af * gd - prm.d_af * np.abs(gd) * chi
        return np.r_[dFpi.ravel(), dchi]

    y = np.r_[np.eye(3).ravel(), np.zeros(12)]
    dt = t_end / nsub
    t = 0.0
    for _ in range(nsub):
        k1 = rates(t, y)
        k2 = rates(t + dt / 2, y + dt / 2 * k1)
        k3 = rates(t + dt / 2, y + dt / 2 * k2)
        k4 = rates(t + dt, y + dt * k3)
        y = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    Fpi = y[:9].reshape(3, 3)
    F = F_of_t(t_end)
    Fe = F @ Fpi
    S = np.einsum("ijkl,kl->ij", C, 0.5 * (Fe.T @ Fe - np.eye(3)))
    return Fe @ S @ Fpi.T, y[9:]


@pytest.mark.slow
def test_cp_return_map_converges_to_the_rate_equations():
    C, S0 = _grain(5)
    prm = mat.CPParams()
    t_end, eps = 1.0, 4e-3

    def F_of_t(t):
        f = 1 + eps * t / t_end
        return np.diag([f, f ** -0.5, f ** -0.5])

    Pref, chiref = _explicit_cp(F_of_t, t_end, 40000, S0, C, prm)
    errs = []
    for n in (20, 40, 80):
        Fpi, chi = np.eye(3)[None], np.zeros((1, 12))
        for k in range(n):
            out = mat.cp_return_map(F_of_t((k + 1) * t_end / n)[None], Fpi, chi, t_end / n, S0, C, prm)
            assert out["conv"].all()
            Fpi, chi = out["Fpi"], out["chi"]
        errs.append(np.abs(out["P"][0] - Pref).max() / np.abs(Pref).max())
    assert np.abs(chiref).max() > 10e6  # backstress really evolved
    # first-order (backward Euler) convergence to the same solution
    assert errs[2] < 2e-3
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6
