"""Constitutive laws of the oracle: St.Venant-Kirchhoff and FCC crystal
plasticity with Armstrong-Frederick backstress (Sect. 3.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Tensors are (..., 3, 3) / (..., 3, 3, 3, 3) numpy arrays with the batch
(voxel) axis first.  Units: Pa, s.

Crystal-plasticity reading (the paper cites its model, Cruzado et al. 2017,
without stating its equations; Eq. gamma_dot gives the flow rule):
  F = Fe Fp, Fp^-1 updated implicitly as Fp^-1_{n+1} = Fp^-1_n (I - sum_a dg_a S0_a)
  S0_a = s_a (x) m_a rotated to the sample frame, Ee = (Fe^T Fe - I)/2,
  S = C : Ee (second Piola-Kirchhoff in the intermediate frame),
  tau_a = (Ce S) : S0_a  (resolved Mandel stress),
  chi_a backward-Euler Armstrong-Frederick: chi_{n+1} = (chi_n + c dg)/(1 + d|dg|),
  dg_a = dt gdot0 |(tau_a - chi_a)/g|^p sign(tau_a - chi_a), g = tau0 constant
  (Eq. gamma_dot with g_c + g_s = tau0 and exponent 1/m = p),
  P = Fe S Fp^-T.
The local residual r_a = dg_a - dt gdot0 h((tau_a - chi_a)/g) is solved by a
plain Newton iteration from dg = 0 and K = dP/dF follows by implicit
differentiation of r = 0.
"""

import numpy as np

_I3 = np.eye(3)


# --------------------------------------------------------------------------- rotations, stiffness
def quat_to_rot(q):
    """Rotation matrix (crystal -> sample) of unit quaternions (w, x, y, z)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def cubic_stiffness(C11, C12, C44):
    """Cubic elasticity tensor in the crystal frame."""
    d = _I3
    C = (
        C12 * np.einsum("ij,kl->ijkl", d, d)
        + C44 * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    )
    for a in range(3):
        C[a, a, a, a] += C11 - C12 - 2 * C44
    return C


def isotropic_stiffness(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    d = _I3
    return lam * np.einsum("ij,kl->ijkl", d, d) + mu * (
        np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)
    )


def rotate4(C, R):
    """C'_ijkl = R_ia R_jb R_kc R_ld C_abcd."""
    return np.einsum("...ia,...jb,...kc,...ld,abcd->...ijkl", R, R, R, R, C)


def fcc_slip_systems():
    """The 12 octahedral {111}<110> systems: unit slip directions s and
    plane normals m (crystal frame).  Normals (111), (-111), (1-11), (11-1);
    for each, the three <110> directions orthogonal to it taken in the
    lexicographic order of the six <110> vectors whose first non-zero entry
    is positive."""
    normals = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.float64)
    dirs = sorted(
        [(0, 1, -1), (0, 1, 1), (1, -1, 0), (1, 0, -1), (1, 0, 1), (1, 1, 0)]
    )
    s, m = [], []
    for n in normals:
        for d in dirs:
            d = np.array(d, dtype=np.float64)
            if abs(d @ n) < 1e-12:
                s.append(d / np.linalg.norm(d))
                m.append(n / np.linalg.norm(n))
    return np.array(s), np.array(m)


def schmid_tensors(R):
    """S0_a = (R s_a) (x) (R m_a) for a rotation R (3,3)."""
    s, m = fcc_slip_systems()
    sr = s @ R.T
    mr = m @ R.T
    return np.einsum("ai,aj->aij", sr, mr)


# --------------------------------------------------------------------------- St.Venant-Kirchhoff
def svk(F, C):
    """St.Venant-Kirchhoff: E = (F^T F - I)/2, S = C : E, P = F S and the
    tangent K_ijkl = dP_ij/dF_kl = delta_ik S_lj + F_ip C_pjln F_kn.
    F (V,3,3); C (3,3,3,3) or (V,3,3,3,3)."""
    E = 0.5 * (np.einsum("vki,vkj->vij", F, F) - _I3)
    if C.ndim == 4:
        S = np.einsum("ijkl,vkl->vij", C, E)
        K = np.einsum("ik,vlj->vijkl", _I3, S) + np.einsum("vip,pjln,vkn->vijkl", F, C, F)
    else:
        S = np.einsum("vijkl,vkl->vij", C, E)
        K = np.einsum("ik,vlj->vijkl", _I3, S) + np.einsum("vip,vpjln,vkn->vijkl", F, C, F)
    P = np.einsum("vik,vkj->vij", F, S)
    return P, K


# --------------------------------------------------------------------------- crystal plasticity
class CPParams:
    """Flow-rule and backstress constants (SI units)."""

    def __init__(self, gdot0=1e-3, p=20, tau0=50e6, c_af=20e9, d_af=200.0):
        self.gdot0 = gdot0
        self.p = p
        self.tau0 = tau0
        self.c_af = c_af
        self.d_af = d_af


def _flow(x, p):
    """h(x) = |x|^p sign(x) and h'(x) = p |x|^(p-1)."""
    ax = np.abs(x)
    return np.sign(x) * ax**p, p * ax ** (p - 1)


def _elastic_state(F, A, dg, S0, C):
    """Fp^-1, Fe, Ce, S and resolved stresses for slip increments dg."""
    Fpi = np.einsum("vik,vkj->vij", A, _I3 - np.einsum("va,aij->vij", dg, S0))
    Fe = np.einsum("vik,vkj->vij", F, Fpi)
    Ce = np.einsum("vki,vkj->vij", Fe, Fe)
    S = np.einsum("ijkl,vkl->vij", C, 0.5 * (Ce - _I3))
    tau = np.einsum("vik,vkj,aij->va", Ce, S, S0)
    return Fpi, Fe, Ce, S, tau


def cp_return_map(F, Fpi_n, chi_n, dt, S0, C, prm, tol=1e-14, maxit=100):
    """Implicit return map of one increment for a batch of voxels sharing the
    Schmid tensors S0 (12,3,3) and stiffness C (3,3,3,3) of one grain.

    Returns dict with P, K (V,3,3,3,3), Fpi, chi, dg, tau and a per-voxel
    convergence flag."""
    V = F.shape[0]
    A = Fpi_n
    dg = np.zeros((V, 12))
    g = prm.tau0
    coef = dt * prm.gdot0
    conv = np.zeros(V, dtype=bool)

    def residual_and_jac(dg):
        Fpi, Fe, Ce, S, tau = _elastic_state(F, A, dg, S0, C)
        den = 1.0 + prm.d_af * np.abs(dg)
        chi = (chi_n + prm.c_af * dg) / den
        x = (tau - chi) / g
        h, dh = _flow(x, prm.p)
        r = dg - coef * h
        # d tau_a / d dg_b
        dFpi = -np.einsum("vik,bkj->vbij", A, S0)  # (V,12,3,3)
        dFe = np.einsum("vik,vbkj->vbij", F, dFpi)
        dCe = np.einsum("vbki,vkj->vbij", dFe, Fe) + np.einsum("vki,vbkj->vbij", Fe, dFe)
        dS = np.einsum("ijkl,vbkl->vbij", C, 0.5 * dCe)
        dM = np.einsum("vbik,vkj->vbij", dCe, S) + np.einsum("vik,vbkj->vbij", Ce, dS)
        dtau = np.einsum("vbij,aij->vab", dM, S0)
        dchi = (prm.c_af - prm.d_af * np.sign(dg) * chi) / den
        J = np.eye(12)[None] - (coef / g) * dh[:, :, None] * (dtau - dchi[:, :, None] * np.eye(12)[None])
        return r, J, (Fpi, Fe, Ce, S, tau, chi, dh)

    for _ in range(maxit):
        r, J, st = residual_and_jac(dg)
        conv = np.max(np.abs(r), axis=1) <= tol
        if conv.all():
            break
        dg = dg - np.linalg.solve(J, r[..., None])[..., 0]
    else:
        r, J, st = residual_and_jac(dg)
        conv = np.max(np.abs(r), axis=1) <= tol

    Fpi, Fe, Ce, S, tau, chi, dh = st
    P = np.einsum("vik,vkl,vjl->vij", Fe, S, Fpi)

    # ---- consistent tangent by implicit differentiation
    K = np.empty((V, 3, 3, 3, 3))
    Jinv = np.linalg.inv(J)
    dFpi_b = -np.einsum("vik,bkj->vbij", A, S0)
    dFe_b = np.einsum("vik,vbkj->vbij", F, dFpi_b)
    dCe_b = np.einsum("vbki,vkj->vbij", dFe_b, Fe) + np.einsum("vki,vbkj->vbij", Fe, dFe_b)
    dS_b = np.einsum("ijkl,vbkl->vbij", C, 0.5 * dCe_b)
    dP_b = (
        np.einsum("vbik,vkl,vjl->vbij", dFe_b, S, Fpi)
        + np.einsum("vik,vbkl,vjl->vbij", Fe, dS_b, Fpi)
        + np.einsum("vik,vkl,vbjl->vbij", Fe, S, dFpi_b)
    )
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = 1.0
            dFe = np.einsum("ik,vkj->vij", E, Fpi)
            dCe = np.einsum("vki,vkj->vij", dFe, Fe) + np.einsum("vki,vkj->vij", Fe, dFe)
            dS = np.einsum("ijkl,vkl->vij", C, 0.5 * dCe)
            dP = np.einsum("vik,vkl,vjl->vij", dFe, S, Fpi) + np.einsum("vik,vkl,vjl->vij", Fe, dS, Fpi)
            dM = np.einsum("vik,vkj->vij", dCe, S) + np.einsum("vik,vkj->vij", Ce, dS)
            dtau = np.einsum("vij,aij->va", dM, S0)
            dr = -(coef / g) * dh * dtau
            ddg = -np.einsum("vab,vb->va", Jinv, dr)
            K[:, :, :, k, l] = dP + np.einsum("vbij,vb->vij", dP_b, ddg)
    return {"P": P, "K": K, "Fpi": Fpi, "chi": chi, "dg": dg, "tau": tau, "conv": conv}
