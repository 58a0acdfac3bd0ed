"""Tile orders on the GPU (crk_params.tile_order: Morton, Hilbert, recursive
coordinate bisection) against oracle/order.py: the sorted order is index work,
compared bit-exact; the passes and a KDK step in every order against the FP64
oracle (the order changes only the summation order within the lists)."""
import numpy as np
import pytest
import torch

from oracle import crk as O
from oracle import order as R
from paper_2202_02840_gb300 import crk, inputs
from parity import TOL, rel_err, as_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def clustered(n, seed=11):
    rng = np.random.default_rng(seed)
    c = rng.random((6, 3))
    x = (c[rng.integers(0, 6, n)] + 0.05 * rng.standard_normal((n, 3))) % 1.0
    pos = np.empty((n, 4), np.float32)
    pos[:, :3] = O._wrap_f32(x)
    pos[:, 3] = (0.02 + 0.06 * rng.random(n)).astype(np.float32)
    return pos


CASES = {
    "tiny1": lambda: clustered(1),
    "tiny33": lambda: clustered(33),
    "ragged100": lambda: clustered(100),
    "clustered3000": lambda: clustered(3000),
    "zeldovich32": lambda: inputs.zeldovich(32)["pos_h"],
    "sedov16": lambda: inputs.sedov(16)["pos_h"],
}
ORACLE = {0: lambda p: O.cells(p)[1], 1: R.hilbert_order, 2: R.bisection_order,
          "2-128": lambda p: R.bisection_order(p, leaf=128), "2-256": lambda p: R.bisection_order(p, leaf=256)}
ORDER_PARAMS = {0: dict(tile_order=0), 1: dict(tile_order=1), 2: dict(tile_order=2),
                "2-128": dict(tile_order=2, rcb_leaf=128), "2-256": dict(tile_order=2, rcb_leaf=256)}


@pytest.mark.parametrize("order", [0, 1, 2, "2-128", "2-256"])
@pytest.mark.parametrize("case", list(CASES))
def test_order_bit_exact(case, order):
    pos = CASES[case]()
    ctx = crk.crk_create(**ORDER_PARAMS[order])
    crk.crk_build_cells(ctx, dev(pos))
    got = crk.crk_order(ctx).cpu().numpy()
    want = ORACLE[order](pos)
    assert np.array_equal(got, want), (case, order, np.nonzero(got != want)[0][:8])


@pytest.mark.parametrize("order", [1, 2])
def test_forces_in_every_order(order):
    st = inputs.uniform(16)
    ev = O.evaluate(st)
    f = lambda a: dev(np.asarray(a, np.float64).astype(np.float32))
    ctx = crk.crk_create(tile_order=order)
    crk.crk_build_cells(ctx, dev(st["pos_h"]))
    acc, dudt, vsig, qmax, pairs = crk.crk_forces(
        ctx, dev(st["mass"]), dev(st["vel_u"]), f(ev["V"]), f(ev["A"]), f(ev["B"]), f(ev["gA"]), f(ev["gB"]),
        f(ev["gv"]), with_pairs=True)
    assert pairs == ev["pairs_union"]
    e = {"acc": rel_err(acc, ev["acc"], floor=ev["fscale"]), "dudt": rel_err(dudt, ev["dudt"]),
         "vsig": rel_err(vsig, ev["vsig"])}
    print(order, e)
    assert max(e.values()) < TOL, e


@pytest.mark.parametrize("order", [1, 2, "2-128"])
@pytest.mark.parametrize("case", ["uniform16", "zeldovich16"])
def test_one_step_in_every_order(case, order):
    st = inputs.uniform(16) if case == "uniform16" else inputs.zeldovich(16)
    ev = O.evaluate(st)
    dt = 0.5 * float(np.min(O.cfl_dt(ev)))
    ost, _, _ = O.kdk_step(st, ev=ev, dt=dt)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    ctx = crk.crk_create(**ORDER_PARAMS[order])
    crk.crk_step(ctx, pos, vel, mass, dt)
    gp, gv = as_np(pos), as_np(vel)
    dx = gp[:, :3] - ost["pos_h"][:, :3]
    dx -= np.round(dx)
    e = {"x": float(np.max(np.abs(dx))), "h": rel_err(gp[:, 3], ost["pos_h"][:, 3]),
         "v": rel_err(gv[:, :3], ost["vel_u"][:, :3]), "u": rel_err(gv[:, 3], ost["vel_u"][:, 3])}
    print(case, order, e)
    assert e["x"] < 1e-6 and max(e["h"], e["v"], e["u"]) < TOL, e


def test_bisection_order_is_refused_for_batches():
    bx = inputs.sedov_boxes(3, 16, 20)
    ctx = crk.crk_create(tile_order=2)
    with pytest.raises(crk.CrkError):
        crk.crk_build_cells_batched(ctx, dev(bx["pos_h"]), bx["box_start"])
