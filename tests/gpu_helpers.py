"""Shared helpers of the GPU parity tests (CUDA path via the C ABI vs the
CPU oracle on the same seeded inputs)."""

import numpy as np

from oracle import materials as omat
from oracle.solver import Material as OMaterial, SVK_CUBIC, SVK_ISO, CP_FCC, NEO_HOOKE

C11, C12, C44 = 168.4e9, 121.4e9, 75.4e9


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def gff():
    from paper_1806_10599_gb300 import gff as g

    return g


def gpu_materials(kinds):
    g = gff()
    out = {}
    for ph, kind in kinds.items():
        out[ph] = g.make_material({SVK_CUBIC: g.GFF_MAT_SVK_CUBIC, SVK_ISO: g.GFF_MAT_SVK_ISO,
                                   CP_FCC: g.GFF_MAT_CP_FCC, NEO_HOOKE: g.GFF_MAT_NEOHOOKE}[kind])
    return out


def oracle_materials(kinds, **kw):
    return {ph: OMaterial(kind, **kw) for ph, kind in kinds.items()}


def voxel_K_oracle(ms, F):
    """Oracle tangent field (3,3,3,3,nz,ny,nx) of St.Venant-Kirchhoff grains
    at the field F (3,3,nz,ny,nx)."""
    R = omat.quat_to_rot(ms.quat)
    Cc = omat.cubic_stiffness(C11, C12, C44)
    V = ms.n_voxels
    Fv = F.reshape(3, 3, V).transpose(2, 0, 1)
    gid = ms.grain_id.reshape(-1)
    K = np.empty((V, 3, 3, 3, 3))
    P = np.empty((V, 3, 3))
    for g in range(ms.ngrains):
        idx = np.nonzero(gid == g)[0]
        if idx.size:
            P[idx], K[idx] = omat.svk(Fv[idx], omat.rotate4(Cc, R[g]))
    shape = (ms.nz, ms.ny, ms.nx)
    return P.transpose(1, 2, 0).reshape((3, 3) + shape), K.transpose(1, 2, 3, 4, 0).reshape((3, 3, 3, 3) + shape)
