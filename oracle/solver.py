"""Newton-Raphson / conjugate-gradient solution of the discrete equilibrium
equations, increment by increment (Sect. 2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

One increment k (Eqs. F_dif, P_dif, linequil, linequil2, newlinop):
  F^0 = F_{k-1} + dFbar, dFbar_c = Fbar_c - <F_{k-1}>_c on strain-controlled
        components c and 0 on stress-controlled ones (the initial guess is
        not stated in the paper: the zero-fluctuation start is used);
  Newton iteration i:
     P, K = law(F^{i-1}, internal variables of t_{k-1}, dt)
     b = -G_M(P) + M : Pbar          (G_M: projection with G^(0) := M)
     stop when ||b||_2 / ||P||_2 <= newton_tol  (the paper's "sufficiently small")
     solve G_M(K : dF) = b by conjugate gradients from dF = 0,
           stopping when ||r||_2 <= max(cg_tol ||b||_2, 0.1 newton_tol ||P||_2)
           (the paper does not state the linear tolerance; the floor keeps
           the solve from chasing the rounding of G(P), which lies outside
           the range of G and cannot be reduced once ||b|| << ||P||)
     F^i = F^{i-1} + dF
  then the internal variables are committed (Sect. 2.1, last paragraph).
"""

import numpy as np

from . import spectral as sp
from . import materials as mat
from . import fips

SVK_CUBIC = 0
SVK_ISO = 1
CP_FCC = 2
NEO_HOOKE = 3  # compressible neo-Hookean, evaluated through the umat conversion of Appendix A


class Material:
    def __init__(self, kind, C11=168.4e9, C12=121.4e9, C44=75.4e9, E=400e9, nu=0.2,
                 gdot0=1e-3, p=20, tau0=50e6, c_af=20e9, d_af=200.0):
        self.kind = kind
        self.C11, self.C12, self.C44, self.E, self.nu = C11, C12, C44, E, nu
        self.cp = mat.CPParams(gdot0, p, tau0, c_af, d_af)


class Options:
    def __init__(self, projection=sp.KIND_CONTINUOUS, newton_tol=1e-8, cg_tol=1e-8,
                 newton_max=30, cg_max=2000, fs_k=0.5, fs_sigma_y=153e6, small_strain=False):
        self.projection = projection
        # small-strain variant (Sect. 2.3): the field is the strain eps, linear
        # elastic phases sigma = C : eps, symmetric projection G^s
        self.small_strain = small_strain
        self.newton_tol = newton_tol
        self.cg_tol = cg_tol
        self.newton_max = newton_max
        self.cg_max = cg_max
        self.fs_k = fs_k
        self.fs_sigma_y = fs_sigma_y


def field_to_voxels(A):
    """(3,3,nz,ny,nx) -> (V,3,3)"""
    return A.reshape(3, 3, -1).transpose(2, 0, 1)


def voxels_to_field(Av, shape):
    return Av.transpose(1, 2, 0).reshape((3, 3) + tuple(shape))


def cg(apply, b, tol, maxit, abs_floor=0.0):
    """Plain conjugate gradients from x = 0 (the Krylov solver of Sect. 2.1),
    stopped when ||r|| <= max(tol ||b||, abs_floor).
    Returns x, iterations, final ||r||."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.vdot(r, r))
    nb = np.sqrt(rr)
    it = 0
    stop = max(tol * nb, abs_floor)
    while it < maxit and np.sqrt(rr) > stop:
        Ap = apply(p)
        alpha = rr / float(np.vdot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr)


class OracleRVE:
    """State of one RVE: committed F field and internal variables."""

    def __init__(self, ms, materials, options=None):
        self.shape = (ms.nz, ms.ny, ms.nx)
        self.L = ms.L
        self.V = ms.n_voxels
        self.gid = ms.grain_id.reshape(-1).astype(np.int64)
        self.ngrains = ms.ngrains
        self.phase = np.asarray(ms.phase)
        self.materials = materials
        self.opt = options or Options()
        R = mat.quat_to_rot(ms.quat)
        self.grains = []
        s, m = mat.fcc_slip_systems()
        for g in range(self.ngrains):
            M = materials[int(self.phase[g])]
            if M.kind in (SVK_ISO, NEO_HOOKE):
                C = mat.isotropic_stiffness(M.E, M.nu)
            else:
                C = mat.rotate4(mat.cubic_stiffness(M.C11, M.C12, M.C44), R[g])
            self.grains.append(
                {
                    "idx": np.nonzero(self.gid == g)[0],
                    "C": C,
                    "S0": mat.schmid_tensors(R[g]),
                    "normals": m @ R[g].T,
                    "mat": M,
                }
            )
        F0 = np.zeros((3, 3)) if self.opt.small_strain else np.eye(3)
        self.F = voxels_to_field(np.broadcast_to(F0, (self.V, 3, 3)).copy(), self.shape)
        self.Fpi = np.broadcast_to(np.eye(3), (self.V, 3, 3)).copy()
        self.chi = np.zeros((self.V, 12))
        self.acc = fips.new_accumulators(self.V)
        self.P = np.zeros_like(self.F)
        self.K = None

    # ------------------------------------------------------------------ constitutive update
    def constitutive(self, F, dt):
        Fv = field_to_voxels(F)
        P = np.empty((self.V, 3, 3))
        K = np.empty((self.V, 3, 3, 3, 3))
        trial = {"Fpi": self.Fpi.copy(), "chi": self.chi.copy(),
                 "dg": np.zeros((self.V, 12)), "tau": np.zeros((self.V, 12)), "ok": True}
        for g in self.grains:
            idx = g["idx"]
            if idx.size == 0:
                continue
            M = g["mat"]
            if self.opt.small_strain:
                if M.kind not in (SVK_CUBIC, SVK_ISO):
                    raise ValueError("the small-strain variant takes linear elastic phases only")
                P[idx] = np.einsum("ijkl,vkl->vij", g["C"], Fv[idx])  # Cauchy stress C : eps
                K[idx] = g["C"][None]
            elif M.kind == CP_FCC:
                out = mat.cp_return_map(Fv[idx], self.Fpi[idx], self.chi[idx], dt, g["S0"], g["C"], M.cp)
                P[idx], K[idx] = out["P"], out["K"]
                trial["Fpi"][idx] = out["Fpi"]
                trial["chi"][idx] = out["chi"]
                trial["dg"][idx] = out["dg"]
                trial["tau"][idx] = out["tau"]
                trial["ok"] = trial["ok"] and bool(out["conv"].all())
            elif M.kind == NEO_HOOKE:
                lam = M.E * M.nu / ((1 + M.nu) * (1 - 2 * M.nu))
                mu = M.E / (2 * (1 + M.nu))
                sig, Cab = mat.neo_hookean_umat(Fv[idx], lam, mu)
                P[idx], K[idx] = mat.umat_to_PK(Fv[idx], sig, Cab)
            else:
                P[idx], K[idx] = mat.svk(Fv[idx], g["C"])
        Pf = voxels_to_field(P, self.shape)
        Kf = K.transpose(1, 2, 3, 4, 0).reshape((3, 3, 3, 3) + self.shape)
        return Pf, Kf, trial

    # ------------------------------------------------------------------ operators
    def G_M(self, A, mask9):
        if self.opt.small_strain:
            return sp.G_sym(A, self.L, self.opt.projection, mask9)
        return sp.G(A, self.L, self.opt.projection, mask9)

    def residual(self, P, mask9, Pbar):
        b = -self.G_M(P, mask9)
        b += (np.asarray(mask9, dtype=np.float64) * np.asarray(Pbar, dtype=np.float64)).reshape(3, 3)[:, :, None, None, None]
        return b

    # ------------------------------------------------------------------ one increment
    def step(self, dt, Fbar, mask, Pbar):
        mask9 = np.asarray(mask, dtype=np.float64).reshape(9)
        Fbar = np.asarray(Fbar, dtype=np.float64).reshape(9)
        Fmean = self.F.reshape(9, -1).mean(axis=1)
        dF = np.where(mask9 > 0, 0.0, Fbar - Fmean).reshape(3, 3)
        F = self.F + dF[:, :, None, None, None]
        rep = {"newton": 0, "cg": [], "res": [], "converged": False}
        for it in range(self.opt.newton_max + 1):
            P, K, trial = self.constitutive(F, dt)
            if not trial["ok"]:
                raise RuntimeError("crystal-plasticity return map did not converge")
            b = self.residual(P, mask9, Pbar)
            nP = np.linalg.norm(P)
            res = np.linalg.norm(b) / nP if nP > 0 else np.linalg.norm(b)
            rep["res"].append(res)
            if res <= self.opt.newton_tol:
                rep["converged"] = True
                break
            if it == self.opt.newton_max:
                break

            def apply(x):
                return self.G_M(sp.ddot42(K, x), mask9)

            dFx, ncg, _ = cg(apply, b, self.opt.cg_tol, self.opt.cg_max, 0.1 * self.opt.newton_tol * nP)
            rep["cg"].append(ncg)
            F = F + dFx
            rep["newton"] += 1
        if not rep["converged"]:
            raise RuntimeError("Newton did not converge: residuals %s" % rep["res"])
        # commit
        self.F = F
        self.P = P
        self.K = K
        self.Fpi = trial["Fpi"]
        self.chi = trial["chi"]
        Fv, Pv = field_to_voxels(F), field_to_voxels(P)
        for g in self.grains:
            if g["mat"].kind == CP_FCC and g["idx"].size:
                idx = g["idx"]
                fips.accumulate(self.acc, idx, trial["dg"][idx], trial["tau"][idx], g["S0"], g["normals"], Pv[idx], Fv[idx])
        rep["Pmacro"] = P.reshape(9, -1).mean(axis=1)
        rep["Fmacro"] = F.reshape(9, -1).mean(axis=1)
        return rep

    def run(self, hist, on_step=None):
        out = []
        for k in range(hist.nsteps):
            if hist.cycle_start[k]:
                fips.reset(self.acc)
            rep = self.step(hist.dt[k], hist.Fbar[k], hist.mask[k], hist.Pbar[k])
            out.append(rep)
            if on_step:
                on_step(k, rep)
        return out

    def band_fips(self, width):
        """Band-averaged W_cyc per grain (Eq. Wmax), bands of `width` along each slip plane."""
        cp = np.array([self.materials[int(self.phase[g])].kind == CP_FCC for g in range(self.ngrains)])
        normals = np.stack([g["normals"][0::3] for g in self.grains])
        return fips.band_fips(self.acc["w"], self.gid.reshape(self.shape), normals, cp, self.L, width)

    def grain_fips(self):
        cp = np.array([self.materials[int(self.phase[g])].kind == CP_FCC for g in range(self.ngrains)])
        return fips.grain_fips(self.acc, self.gid, self.ngrains, cp, self.opt.fs_k, self.opt.fs_sigma_y)
