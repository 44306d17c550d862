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
plain Newton iteration from dg = 0, voxel by voxel, and K = dP/dF follows by implicit
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


def _T(A):
    """Transpose of the last two axes (3x3 tensors of a batch)."""
    return np.swapaxes(A, -1, -2)


def _ddot_C(C, E):
    """S_ij = C_ijkl E_kl for a batch of tensors E (..., 3, 3)."""
    return (E.reshape(E.shape[:-2] + (9,)) @ C.reshape(9, 9).T).reshape(E.shape)


def _resolve(M, S0):
    """M : S0_a for a batch of tensors M (..., 3, 3) -> (..., 12)."""
    return M.reshape(M.shape[:-2] + (9,)) @ S0.reshape(12, 9).T


def _elastic_state(F, A, dg, S0, C):
    """Fp^-1, Fe, Ce, S and resolved stresses for slip increments dg.
    (Batched 3x3 products are written with @; index form in the comments.)"""
    Fpi = A @ (_I3 - (dg @ S0.reshape(12, 9)).reshape(-1, 3, 3))  # A_ik (delta_kj - dg_a S0_a,kj)
    Fe = F @ Fpi
    Ce = _T(Fe) @ Fe                                              # Fe_ki Fe_kj
    S = _ddot_C(C, 0.5 * (Ce - _I3))
    tau = _resolve(Ce @ S, S0)                                    # (Ce S)_ij S0_a,ij
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

    def residual_and_jac(dg, sel=slice(None)):
        """Local residual r(dg) and Jacobian dr/ddg of the voxels `sel`."""
        Fs, As, chis = F[sel], A[sel], chi_n[sel]
        Fpi, Fe, Ce, S, tau = _elastic_state(Fs, As, dg, S0, C)
        den = 1.0 + prm.d_af * np.abs(dg)
        chi = (chis + prm.c_af * dg) / den
        x = (tau - chi) / g
        h, dh = _flow(x, prm.p)
        r = dg - coef * h
        # d tau_a / d dg_b (derivatives along axis b = 1 of the (V,12,3,3) arrays)
        dFpi = -(As[:, None] @ S0)                                 # -A_ik S0_b,kj
        dFe = Fs[:, None] @ dFpi
        dCe = _T(dFe) @ Fe[:, None] + _T(Fe)[:, None] @ dFe
        dS = _ddot_C(C, 0.5 * dCe)
        dM = dCe @ S[:, None] + Ce[:, None] @ dS
        dtau = _T(_resolve(dM, S0))                                # [v, a, b] = dM_b : S0_a
        dchi = (prm.c_af - prm.d_af * np.sign(dg) * chi) / den
        J = np.eye(12)[None] - (coef / g) * dh[:, :, None] * (dtau - dchi[:, :, None] * np.eye(12)[None])
        return r, J, (Fpi, Fe, Ce, S, tau, chi, dh)

    # Each voxel's Newton iteration is independent: a voxel stops at its first
    # iterate with max|r| <= tol, the others go on (up to maxit iterations).
    active = np.arange(V)
    for _ in range(maxit):
        r, J, _st = residual_and_jac(dg[active], active)
        todo = np.max(np.abs(r), axis=1) > tol
        if not todo.any():
            break
        active = active[todo]
        dg[active] = dg[active] - np.linalg.solve(J[todo], r[todo][..., None])[..., 0]
    r, J, st = residual_and_jac(dg)
    conv = np.max(np.abs(r), axis=1) <= tol

    Fpi, Fe, Ce, S, tau, chi, dh = st
    P = Fe @ S @ _T(Fpi)                                           # Fe_ik S_kl Fpi_jl

    # ---- consistent tangent by implicit differentiation
    K = np.empty((V, 3, 3, 3, 3))
    Jinv = np.linalg.inv(J)
    # dP / d dg_b at fixed F, (V,12,3,3)
    dFpi_b = -(A[:, None] @ S0)
    dFe_b = F[:, None] @ dFpi_b
    dCe_b = _T(dFe_b) @ Fe[:, None] + _T(Fe)[:, None] @ dFe_b
    dS_b = _ddot_C(C, 0.5 * dCe_b)
    dP_b = (
        dFe_b @ (S @ _T(Fpi))[:, None]
        + Fe[:, None] @ dS_b @ _T(Fpi)[:, None]
        + (Fe @ S)[:, None] @ _T(dFpi_b)
    )
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = 1.0
            # dP / dF_kl at fixed dg, and d dg / dF_kl from J d dg = -dr
            dFe = E @ Fpi
            dCe = _T(dFe) @ Fe + _T(Fe) @ dFe
            dS = _ddot_C(C, 0.5 * dCe)
            dP = dFe @ S @ _T(Fpi) + Fe @ dS @ _T(Fpi)
            dM = dCe @ S + Ce @ dS
            dtau = _resolve(dM, S0)
            dr = -(coef / g) * dh * dtau
            ddg = -(Jinv @ dr[..., None])[..., 0]
            K[:, :, :, k, l] = dP + (ddg[:, None] @ dP_b.reshape(V, 12, 9)).reshape(V, 3, 3)
    return {"P": P, "K": K, "Fpi": Fpi, "chi": chi, "dg": dg, "tau": tau, "conv": conv}


# --------------------------------------------------------------------------- Appendix A: umat-style tangents
def umat_to_PK(F, sigma, Cab):
    """First Piola-Kirchhoff stress and tangent K = dP/dF from what an Abaqus
    umat returns (Appendix A): the Cauchy stress sigma and the tangent C^ab of
    the Jaumann rate of the Kirchhoff stress (Eq. ABAtang), at the deformation
    gradient F.  All arrays batched over voxels: F, sigma (V,3,3), Cab
    (V,3,3,3,3) with minor symmetries.

      P = J sigma F^-T                                            (Eq. fPK)
      d tau_ip / d F_kl = J C_ipkm Fi_lm + 1/2 delta_ik Fi_lm tau_mp
                          - 1/2 Fi_li tau_kp + 1/2 delta_pk Fi_lm tau_im
                          - 1/2 Fi_lp tau_ik                      (Eq. tau_F_function_Cab)
      K_ijkl = d tau_ip / d F_kl Fi_jp - tau_ip Fi_lp Fi_jk      (Eqs. indexx, derivativeinv)
    with tau = J sigma and Fi = F^-1."""
    J = np.linalg.det(F)
    Fi = np.linalg.inv(F)
    tau = J[:, None, None] * sigma
    d = _I3
    dtau = (
        J[:, None, None, None, None] * np.einsum("vipkm,vlm->vipkl", Cab, Fi)
        + 0.5 * np.einsum("ik,vlm,vmp->vipkl", d, Fi, tau)
        - 0.5 * np.einsum("vli,vkp->vipkl", Fi, tau)
        + 0.5 * np.einsum("pk,vlm,vim->vipkl", d, Fi, tau)
        - 0.5 * np.einsum("vlp,vik->vipkl", Fi, tau)
    )
    K = np.einsum("vipkl,vjp->vijkl", dtau, Fi) - np.einsum("vip,vlp,vjk->vijkl", tau, Fi, Fi)
    P = np.einsum("vip,vjp->vij", tau, Fi)
    return P, K


def neo_hookean_umat(F, lam, mu):
    """Compressible neo-Hookean solid in umat form: Kirchhoff stress
    tau = mu (b - I) + lam ln(J) I (b = F F^T), returned as the Cauchy stress
    sigma = tau / J and the Jaumann-rate tangent of Eq. ABAtang, for which
    J C^ab : d = mu (d b + b d) + lam tr(d) I, i.e.
    J C^ab_ijkl = mu/2 (delta_ik b_jl + delta_il b_jk + b_ik delta_jl + b_il delta_jk) + lam delta_ij delta_kl."""
    J = np.linalg.det(F)
    b = F @ _T(F)
    tau = mu * (b - _I3) + lam * np.log(J)[:, None, None] * _I3
    d = _I3
    JC = 0.5 * mu * (np.einsum("ik,vjl->vijkl", d, b) + np.einsum("il,vjk->vijkl", d, b)
                     + np.einsum("vik,jl->vijkl", b, d) + np.einsum("vil,jk->vijkl", b, d)) \
        + lam * np.einsum("ij,kl->ijkl", d, d)[None]
    return tau / J[:, None, None], JC / J[:, None, None, None, None]
