"""Pins of the oracle's band-averaged dissipated energy W_cyc^b (Sect. 3.3,
Eq. Wmax) -- checked without the GPU against facts that do not depend on how
the bands are coded:

  * one band per plane (width beyond the box diagonal) is the whole grain, so
    W_cyc^b equals the largest grain average of W_cyc^alpha;
  * every band average is an average over part of the grain, and the grain
    average is the voxel-weighted mean of one plane's band averages, so
    W_cyc^b is never below the largest grain average;
  * a hand-counted case: one grain filling a 4^3 box in the cube orientation,
    bands one voxel step of x + y + z wide along the (111) plane, one voxel
    carrying W: the band holding it has as many voxels as there are ways to
    write its offset sum with three digits in {-2, -1, 0, 1}, read off the
    polynomial (z^-2 + z^-1 + 1 + z)^3.
"""

import numpy as np

from oracle import fips
from oracle import materials as mat
from rve_inputs import polycrystal, uniform01


def _normals(quats):
    R = mat.quat_to_rot(quats)
    _, m = mat.fcc_slip_systems()
    return np.stack([(m @ R[g].T)[0::3] for g in range(len(quats))])  # (ngrains, 4, 3)


def _grain_mean_max(w, gid, ngrains):
    return np.array([w[gid.reshape(-1) == g].mean(axis=0).max() for g in range(ngrains)])


def test_one_band_per_plane_is_the_grain_average():
    ms = polycrystal(8, 4, 3)
    V = ms.n_voxels
    w = uniform01(11, 12 * V).reshape(V, 12)
    wb = fips.band_fips(w, ms.grain_id, _normals(ms.quat), np.ones(4, bool), ms.L, width=10.0)
    assert np.allclose(wb, _grain_mean_max(w, ms.grain_id, 4), rtol=1e-14, atol=0)


def test_band_averages_never_fall_below_the_grain_average():
    ms = polycrystal((6, 10, 8), 5, 4)
    V = ms.n_voxels
    w = uniform01(12, 12 * V).reshape(V, 12) ** 3
    gmax = _grain_mean_max(w, ms.grain_id, 5)
    for width in (0.05, 0.13, 0.3):
        wb = fips.band_fips(w, ms.grain_id, _normals(ms.quat), np.ones(5, bool), ms.L, width)
        assert (wb >= gmax * (1 - 1e-14)).all()
    # narrower bands than the grain resolve more: some grain exceeds its average
    assert (fips.band_fips(w, ms.grain_id, _normals(ms.quat), np.ones(5, bool), ms.L, 0.05) > gmax * 1.01).any()


def test_hand_counted_band_in_a_single_crystal():
    n = 4
    gid = np.zeros((n, n, n), dtype=np.int32)
    normals = _normals(np.array([[1.0, 0.0, 0.0, 0.0]]))
    assert np.allclose(normals[0, 0], np.ones(3) / np.sqrt(3.0))
    h = 1.0 / n
    # s / width + 1/2 = (dx + dy + dz) / (1 + 1e-4) + 1/2 for integer offsets in [-2, 1]: band = the offset sum
    width = h / np.sqrt(3.0) * (1 + 1e-4)
    counts = np.array([1.0])
    for _ in range(3):
        counts = np.convolve(counts, np.ones(4))  # coefficients of (z^-2 + z^-1 + 1 + z)^k, lowest power -2k
    for (dx, dy, dz) in [(1, 1, -2), (1, 1, 1), (-2, -2, -2), (0, -1, 0)]:
        w = np.zeros((n ** 3, 12))
        ix, iy, iz = dx % n, dy % n, dz % n  # the reference voxel is (0, 0, 0)
        w[(iz * n + iy) * n + ix, 0] = 1.0  # system 0 lies on plane 0, the (111) plane
        wb = fips.band_fips(w, gid, normals, np.ones(1, bool), (1.0, 1.0, 1.0), width)
        t = dx + dy + dz
        assert abs(wb[0] - 1.0 / counts[t + 6]) < 1e-15, (dx, dy, dz, wb[0], counts)


def test_non_plastic_grains_report_zero():
    ms = polycrystal(8, 3, 5)
    w = uniform01(13, 12 * ms.n_voxels).reshape(ms.n_voxels, 12)
    wb = fips.band_fips(w, ms.grain_id, _normals(ms.quat), np.array([True, False, True]), ms.L, 0.2)
    assert wb[1] == 0.0 and wb[0] > 0 and wb[2] > 0
