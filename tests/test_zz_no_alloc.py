"""The allocation-free volumes entry point against the regular one and the oracle.

crk_volumes_noalloc serves callers that cannot let a library allocate device
memory (their allocator owns the GPU, or a cudaMalloc would synchronise the
device mid-step).  Two calls in a row, with different particle counts, must
both reproduce crk_build_cells + crk_volumes; the largest accepted n, n = 0
and a null Nngb are exercised, and the volumes are checked against the FP64
oracle as well; sizes beyond the limit are refused.  This file is collected
last so a failure here never hides the other tests.
"""
import numpy as np
import pytest
import torch

from oracle import crk as O
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


def test_noalloc_at_its_largest_n_matches_regular_path_and_oracle():
    """n = NOALLOC_MAX_N exactly (512 tiles, every per-tile sub-buffer full),
    clustered so that tiles neighbour many tiles; then a call without Nngb."""
    st = clustered(crk.NOALLOC_MAX_N, 5)
    pos = torch.from_numpy(st["pos_h"]).cuda()
    V0, N0 = regular(pos)
    V1, N1 = crk.crk_volumes_noalloc(pos)
    torch.cuda.synchronize()
    o = O.volumes(st["pos_h"])
    e = {"V_regular": rel_err(V1, V0.cpu().double().numpy()), "N_regular": rel_err(N1, N0.cpu().double().numpy()),
         "V_oracle": rel_err(V1, o["V"]), "N_oracle": rel_err(N1, o["N"])}
    print(e)
    assert max(e.values()) < TOL, e
    V2, N2 = crk.crk_volumes_noalloc(pos, with_N=False)
    torch.cuda.synchronize()
    assert N2 is None and torch.equal(V2, V1)


def test_noalloc_empty_and_repeated_calls_leave_device_memory_alone():
    """n = 0 is a no-op; repeated calls change neither their results nor the
    device's free memory (the calls allocate nothing)."""
    V, N = crk.crk_volumes_noalloc(torch.zeros((0, 4), dtype=torch.float32, device="cuda"))
    assert V.numel() == 0 and N.numel() == 0
    st = workload("uniform", 16)
    pos = torch.from_numpy(st["pos_h"]).cuda()
    Va, Na = crk.crk_volumes_noalloc(pos)
    outV = torch.empty_like(Va)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        Vb, _ = crk.crk_volumes_noalloc(pos, with_N=False)
        outV.copy_(Vb)
        del Vb
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.equal(outV, Va)
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_too_many_particles():
    n = crk.NOALLOC_MAX_N + 1
    pos = torch.full((n, 4), 0.25, dtype=torch.float32, device="cuda")
    pos[:, 3] = 0.01
    with pytest.raises(crk.CrkError) as ei:
        crk.crk_volumes_noalloc(pos)
    assert ei.value.code == -1
