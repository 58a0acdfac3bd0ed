"""The allocation-free volumes entry point against the regular one.

crk_volumes_noalloc serves callers that cannot let a library allocate device
memory (their allocator owns the GPU, or a cudaMalloc would synchronise the
device mid-step).  Two calls in a row, with different particle counts, must
both reproduce crk_build_cells + crk_volumes; sizes beyond the limit are
refused.  This file is collected last so a failure here never hides the
other tests.
"""
import numpy as np
import pytest
import torch

from paper_2202_02840_gb300 import crk
from parity import TOL, clustered, rel_err, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def regular(pos):
    ctx = crk.crk_create()
    crk.crk_build_cells(ctx, pos)
    V, N = crk.crk_volumes(ctx)
    torch.cuda.synchronize()
    ctx.close()
    return V, N


def test_noalloc_volumes_match_regular_path_twice():
    inputs = [clustered(3000, 11), workload("uniform", 16)]
    for st in inputs:                         # two calls in a row, different n
        pos = torch.from_numpy(st["pos_h"]).cuda()
        V0, N0 = regular(pos)
        V1, N1 = crk.crk_volumes_noalloc(pos)
        torch.cuda.synchronize()
        v0 = V0.cpu().double().numpy()
        n0 = N0.cpu().double().numpy()
        assert rel_err(V1, v0) < TOL and rel_err(N1, n0) < TOL


def test_noalloc_rejects_too_many_particles():
    n = crk.NOALLOC_MAX_N + 1
    pos = torch.full((n, 4), 0.25, dtype=torch.float32, device="cuda")
    pos[:, 3] = 0.01
    with pytest.raises(crk.CrkError) as ei:
        crk.crk_volumes_noalloc(pos)
    assert ei.value.code == -1
