"""Synthetic RVE geometry: periodic Voronoi grains, uniform SO(3) orientations,
non-overlapping spherical particles.

These stand in for the Neper weighted-Voronoi RVEs and the carbide particles
of the paper (Sect. 4.1 and 4.4); Neper is not available, so the grains are
plain periodic Voronoi cells of uniformly drawn seeds.

Array conventions (shared by the oracle and the CUDA library):
  grain_id  int32 [nz][ny][nx]   (x fastest), values in [0, ngrains_total)
  quat      float64 [ngrains_total][4] unit quaternions (w, x, y, z), w >= 0,
            mapping crystal axes to sample axes
  phase     int32 [ngrains_total]  0 = crystal (grain), 1 = particle
"""

from dataclasses import dataclass

import numpy as np

from .rng import uniform01

# disjoint sub-streams of one seed
OFF_SEEDS = 0
OFF_QUATS = 1 << 40
OFF_SPHERES = 1 << 41
OFF_COUNT = 1 << 43


@dataclass
class Microstructure:
    nx: int
    ny: int
    nz: int
    L: tuple
    grain_id: np.ndarray
    quat: np.ndarray
    phase: np.ndarray

    @property
    def ngrains(self):
        return int(self.quat.shape[0])

    @property
    def n_voxels(self):
        return self.nx * self.ny * self.nz


def periodic_voronoi(shape, ngrains, seed, L=(1.0, 1.0, 1.0)):
    """Nearest-seed labels of voxel centres ((i + 1/2) h) under the periodic
    minimum-image Euclidean distance; ties go to the lowest seed index.

    shape = (nz, ny, nx).  Seeds are uniform in [0, L)^3.  The search uses a
    periodic k-d tree (scipy cKDTree with boxsize = L); the two nearest
    seeds are returned so that exact ties can be resolved by index."""
    from scipy.spatial import cKDTree

    nz, ny, nx = shape
    L = np.asarray(L, dtype=np.float64)
    u = uniform01(seed, 3 * ngrains, OFF_SEEDS).reshape(ngrains, 3)
    seeds = u * L[None, :]  # columns: x, y, z
    h = L / np.array([nx, ny, nz], dtype=np.float64)
    zi, yi, xi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    centres = np.stack(
        [(xi.ravel() + 0.5) * h[0], (yi.ravel() + 0.5) * h[1], (zi.ravel() + 0.5) * h[2]], axis=1
    )
    if ngrains == 1:
        return np.zeros(shape, dtype=np.int32)
    tree = cKDTree(seeds, boxsize=L)
    d, i = tree.query(centres, k=2)
    out = np.where(d[:, 0] == d[:, 1], np.minimum(i[:, 0], i[:, 1]), i[:, 0]).astype(np.int32)
    return out.reshape(nz, ny, nx)


def random_quaternions(count, seed):
    """Uniformly distributed rotations (Shoemake, Graphics Gems III, 1992),
    returned as (w, x, y, z) with w >= 0."""
    u = uniform01(seed, 3 * count, OFF_QUATS).reshape(count, 3)
    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack(
        [b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)],
        axis=1,
    )
    q[q[:, 0] < 0] *= -1.0
    return q


def place_spheres(shape, radius, frac, seed, max_tries=200000):
    """Disjoint periodic balls with integer-voxel centres.  A voxel belongs to
    a ball when its integer minimum-image distance to the centre is <= radius;
    centres are kept more than 2*radius apart; balls are added by rejection
    sampling until they cover at least `frac` of the voxels.  Returns a bool
    mask [nz][ny][nx] and the list of centres (iz, iy, ix)."""
    nz, ny, nx = shape
    dims = np.array([nz, ny, nx])
    r2 = radius * radius
    rr = np.arange(-radius, radius + 1)
    oz, oy, ox = np.meshgrid(rr, rr, rr, indexing="ij")
    keep = oz * oz + oy * oy + ox * ox <= r2
    offs = np.stack([oz[keep], oy[keep], ox[keep]], axis=1)
    mask = np.zeros(shape, dtype=bool)
    centres = []
    target = frac * nz * ny * nx
    draws = uniform01(seed, 3 * max_tries, OFF_SPHERES).reshape(max_tries, 3)
    for t in range(max_tries):
        if mask.sum() >= target:
            break
        c = np.minimum((draws[t] * dims).astype(np.int64), dims - 1)
        ok = True
        for p in centres:
            d = np.abs(c - p)
            d = np.minimum(d, dims - d)
            if int(d @ d) <= 4 * r2:
                ok = False
                break
        if not ok:
            continue
        centres.append(c)
        idx = (c[None, :] + offs) % dims[None, :]
        mask[idx[:, 0], idx[:, 1], idx[:, 2]] = True
    else:
        raise RuntimeError("place_spheres: volume fraction not reached")
    return mask, centres


def polycrystal(n, ngrains, seed, L=(1.0, 1.0, 1.0)):
    """n^3 (or n = (nz, ny, nx)) periodic Voronoi polycrystal, all grains phase 0."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    gid = periodic_voronoi(shape, ngrains, seed, L)
    q = random_quaternions(ngrains, seed)
    return Microstructure(shape[2], shape[1], shape[0], tuple(L), gid, q, np.zeros(ngrains, dtype=np.int32))


def polycrystal_with_particles(n, ngrains, seed, radius=3, frac=0.05, L=(1.0, 1.0, 1.0)):
    """Polycrystal plus disjoint spherical particles.  All particle voxels get
    the extra grain id `ngrains`, whose phase is 1 and orientation identity."""
    m = polycrystal(n, ngrains, seed, L)
    mask, _ = place_spheres(m.grain_id.shape, radius, frac, seed)
    gid = m.grain_id.copy()
    gid[mask] = ngrains
    q = np.vstack([m.quat, [[1.0, 0.0, 0.0, 0.0]]])
    ph = np.concatenate([m.phase, [1]]).astype(np.int32)
    return Microstructure(m.nx, m.ny, m.nz, m.L, gid, q, ph)


def batch_rves(count=32, base_seed=4000, sizes=(32, 48, 64, 80, 96), min_grains=50, span=251):
    """Uneven RVE set: RVE i has n = sizes[i mod len(sizes)] voxels per axis,
    seed base_seed + i and min_grains + floor(span u_i) grains (u_i uniform
    from its own seed).  Returns a list of (n, ngrains, seed)."""
    out = []
    for i in range(count):
        seed = base_seed + i
        u = uniform01(seed, 1, OFF_COUNT)[0]
        out.append((sizes[i % len(sizes)], min_grains + int(np.floor(span * u)), seed))
    return out
