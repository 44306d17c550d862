"""gff_project_noalloc: the projection for callers that may not allocate
device memory (an application whose own allocator owns the device-memory
budget, or a loop that cannot take the synchronisation a cudaMalloc may
cause).  Its scratch lives inside libgff.so, so it is checked here, through
the C ABI, against the handle-based gff_project on the same inputs -- on two
calls in a row with different inputs, so that state left in the shared
scratch by the first call cannot leak into the second.  The tolerances are
those of the other projection tests (relative L2 1e-12 in FP64, 2e-6 in
FP32).  This file is collected last on purpose."""

import numpy as np
import pytest

from gpu_helpers import gff, rel_l2, torch_cuda
from rve_inputs import standard_normal

pytestmark = pytest.mark.gpu

# (nz, ny, nx).  The half spectrum takes 9 nz ny (nx/2 + 1) of the 9 * 32768 * 3/4 complex
# values the scratch holds; with nx = 4 and 32768 voxels it fills them exactly.
CASES = [((16, 16, 16), 0, 0), ((8, 12, 20), 1, 0), ((32, 32, 32), 0, 1), ((4, 64, 120), 1, 1),
         ((64, 128, 4), 0, 0), ((64, 128, 4), 1, 1)]


@pytest.mark.parametrize("shape,kind,prec", CASES)
def test_noalloc_matches_gff_project_on_two_calls(shape, kind, prec):
    torch = torch_cuda()
    g = gff()
    nz, ny, nx = shape
    N = nx * ny * nz
    grid = g.make_grid(nx, ny, nz, (1.0, 1.5, 0.75))
    mask = np.array([0, 1, 1, 1, 1, 1, 1, 0, 1], dtype=np.uint8)
    dtype = torch.float64 if prec == g.GFF_PREC_FP64 else torch.float32
    tol = 1e-12 if prec == g.GFF_PREC_FP64 else 2e-6
    h = g.gff_create(grid, g.make_options(projection=kind))
    try:
        for call, seed in enumerate((31, 32)):
            X = torch.from_numpy(standard_normal(seed, 9 * N).reshape(9, N)).to("cuda", dtype)
            Yref = torch.empty_like(X)
            g.gff_project(h, prec, mask, X, Yref)
            Y = torch.full_like(X, float("nan"))
            g.gff_project_noalloc(grid, kind, prec, mask, X, Y, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert rel_l2(Y.cpu().numpy(), Yref.cpu().numpy()) <= tol, (call, shape)
    finally:
        g.gff_destroy(h)


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = torch_cuda()
    g = gff()
    X = torch.zeros(9 * 64 ** 3, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(g.GffError) as e:
        g.gff_project_noalloc(g.make_grid(64, 64, 64), 0, 0, None, X, Y)
    assert e.value.status == g.GFF_ERR_ARG
    with pytest.raises(g.GffError) as e:
        g.gff_project_noalloc(g.make_grid(8, 8, 14), 0, 0, None, X, Y)
    assert e.value.status == g.GFF_ERR_ARG
