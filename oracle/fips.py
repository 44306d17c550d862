"""Fatigue indicator parameters (Sect. 3.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per voxel and increment (backward-Euler increments dg_a of the return map):
  P_cyc += sqrt(2/3 dDp : dDp),  dDp = sum_a dg_a sym(S0_a)
      (Eq. eqplas read as the accumulated effective plastic strain: the
      printed integrand L_p : L_p has units of 1/s^2 x s, so the rate form
      sqrt(2/3 D_p : D_p) dt of the same quantity is used)
  W_a   += tau_a dg_a                                   (Eq. strainenergy)
  gamma_a += dg_a, with its running minimum and maximum over the cycle
  sn_a = max over the cycle of m_a . sigma . m_a, sigma = P F^T / det F
      (Eq. fPK inverted; m_a the sample-frame slip-plane normal)
Per grain at the end of a cycle:
  P_cyc^g = mean over the grain (Eq. Pmax before the max over grains)
  W_a^g   = mean over the grain of W_a
  FS^g    = max_a  (mean(gamma_max - gamma_min)/2) (1 + k mean(sn_a) / sigma_y)
      (Fatemi-Socie parameter; not in the paper)
Accumulators restart at the first increment of every cycle.
"""

import numpy as np

N_ACC = 1 + 12 + 12 + 12 + 12 + 12  # pcyc, W, gamma, gmin, gmax, sn


def new_accumulators(V):
    acc = {
        "pcyc": np.zeros(V),
        "w": np.zeros((V, 12)),
        "gamma": np.zeros((V, 12)),
        "gmin": np.zeros((V, 12)),
        "gmax": np.zeros((V, 12)),
        "sn": np.full((V, 12), -np.inf),
    }
    return acc


def reset(acc):
    acc["pcyc"][:] = 0.0
    acc["w"][:] = 0.0
    acc["gmin"][:] = acc["gamma"]
    acc["gmax"][:] = acc["gamma"]
    acc["sn"][:] = -np.inf


def accumulate(acc, idx, dg, tau, S0, normals, P, F):
    """Add one converged increment for voxels `idx` of one grain.
    dg, tau (v,12); S0 (12,3,3); normals (12,3) sample frame; P, F (v,3,3)."""
    symS0 = 0.5 * (S0 + np.swapaxes(S0, 1, 2))
    dDp = np.einsum("va,aij->vij", dg, symS0)
    acc["pcyc"][idx] += np.sqrt(2.0 / 3.0 * np.einsum("vij,vij->v", dDp, dDp))
    acc["w"][idx] += tau * dg
    g = acc["gamma"][idx] + dg
    acc["gamma"][idx] = g
    acc["gmin"][idx] = np.minimum(acc["gmin"][idx], g)
    acc["gmax"][idx] = np.maximum(acc["gmax"][idx], g)
    J = np.linalg.det(F)
    sigma = np.einsum("vik,vjk->vij", P, F) / J[:, None, None]
    sn = np.einsum("ai,vij,aj->va", normals, sigma, normals)
    acc["sn"][idx] = np.maximum(acc["sn"][idx], sn)


def grain_fips(acc, grain_id_flat, ngrains, cp_grain, fs_k=0.5, fs_sigma_y=153e6):
    """Per-grain P_cyc, W_a and Fatemi-Socie values.  Grains that are not
    crystal-plastic (cp_grain False) report zeros."""
    pc = np.zeros(ngrains)
    w = np.zeros((ngrains, 12))
    fs = np.zeros(ngrains)
    for gi in range(ngrains):
        if not cp_grain[gi]:
            continue
        sel = grain_id_flat == gi
        if not sel.any():
            continue
        pc[gi] = acc["pcyc"][sel].mean()
        w[gi] = acc["w"][sel].mean(axis=0)
        dgam = (acc["gmax"][sel] - acc["gmin"][sel]).mean(axis=0)
        sn = acc["sn"][sel].mean(axis=0)
        fs[gi] = np.max(0.5 * dgam * (1.0 + fs_k * sn / fs_sigma_y))
    return pc, w, fs


def band_coordinates(grain_id, L):
    """Minimum-image voxel offsets of every voxel from its grain's reference
    voxel (the grain's voxel with the lowest flat index), in voxel units per
    axis (x, y, z), each in [-n/2, n/2), and the voxel spacings h (x, y, z).
    grain_id (nz, ny, nx)."""
    nz, ny, nx = grain_id.shape
    g = grain_id.reshape(-1)
    order = np.argsort(g, kind="stable")
    first = np.full(int(g.max()) + 1, -1)
    gs = g[order]
    starts = np.r_[0, np.nonzero(np.diff(gs))[0] + 1]
    first[gs[starts]] = order[starts]
    ref = first[g]
    iz, iy, ix = np.unravel_index(np.arange(g.size), (nz, ny, nx))
    rz, ry, rx = np.unravel_index(ref, (nz, ny, nx))
    d = []
    for i, r, n in ((ix, rx, nx), (iy, ry, ny), (iz, rz, nz)):
        di = np.mod(i - r, n)
        d.append(np.where(di >= n / 2.0, di - n, di))
    h = np.array([L[0] / nx, L[1] / ny, L[2] / nz])
    return np.stack(d, axis=1).astype(np.float64), h


def band_fips(w_acc, grain_id, plane_normals, cp_grain, L, width):
    """Band-averaged dissipated energy W_cyc^b of Eq. Wmax per grain.

    Bands of width `width` (a length) parallel to each of a grain's four
    {111} slip planes cut the grain: the band index of a voxel for plane p is
    floor(s / width + 1/2), s = (x - x_ref) . m_p (the reference voxel sits in
    the middle of band 0), with x - x_ref the minimum-image
    offset of the voxel centre from the grain's reference voxel and m_p the
    sample-frame unit normal of the plane.  For each band, W_cyc^beta is
    averaged over the band's voxels for the three systems beta on that plane
    (systems 3p, 3p+1, 3p+2); the grain's value is the largest such average
    over its bands, planes and systems (Eq. Wmax before the max over grains).

    w_acc (V, 12) per-voxel W_cyc; grain_id (nz, ny, nx); plane_normals
    (ngrains, 4, 3); cp_grain (ngrains,) bool.  Returns (ngrains,) with 0 for
    grains that are not crystal-plastic or empty."""
    ngrains = plane_normals.shape[0]
    d, h = band_coordinates(grain_id, L)
    off = d * h[None, :]
    g = grain_id.reshape(-1)
    out = np.zeros(ngrains)
    for gi in range(ngrains):
        sel = np.nonzero(g == gi)[0]
        if not cp_grain[gi] or sel.size == 0:
            continue
        best = -np.inf
        for p in range(4):
            s = off[sel] @ plane_normals[gi, p]
            band = np.floor(s / width + 0.5).astype(np.int64)
            for j in np.unique(band):
                in_band = sel[band == j]
                best = max(best, w_acc[in_band][:, 3 * p:3 * p + 3].mean(axis=0).max())
        out[gi] = best
    return out
