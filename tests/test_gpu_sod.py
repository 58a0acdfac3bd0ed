"""Sod shock tube (the paper's Sec. 4 test, inputs.sod): CRKSPH on the GPU
against the exact Riemann solution (oracle/riemann.py), and one KDK step of
the tube's two-lattice start against the FP64 oracle.

* L1 norms of density, velocity, pressure and specific energy over the
  isolated half at t = 0.075 (the paper's t = 0.15) fall with resolution at
  close to first order (doubling n_hi at least a factor 1.35 on every
  quantity; measured 1.6-1.9);
* the flow stays one-dimensional (transverse velocities < 1e-3);
* the shock sits where the exact solution puts it, within two high-side
  spacings.
"""
import numpy as np
import pytest
import torch

from oracle import crk as O
from oracle import riemann as R
from paper_2202_02840_gb300 import crk, inputs
from parity import TOL, as_np, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_sod(n):
    st = inputs.sod(n)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    d = crk.crk_step(crk.crk_create(), pos.clone(), vel.clone(), mass, 0.0, diag=True)
    ctx = crk.crk_create()
    t, dt_next = 0.0, d["dt"]
    while t < st["t_end"] - 1e-12:
        d = crk.crk_step(ctx, pos, vel, mass, min(dt_next, st["t_end"] - t), diag=True)
        t += d["dt"]
        dt_next = d["dt_next"]
    probe = crk.crk_create()
    crk.crk_build_cells(probe, pos)
    V, _ = crk.crk_volumes(probe)
    p, v = as_np(pos), as_np(vel)
    rho = st["mass"].astype(np.float64) / as_np(V)
    P = (st["gamma"] - 1.0) * rho * v[:, 3]
    sel = p[:, 0] < 0.5
    xi = (p[sel, 0] - st["x0"]) / t
    re, ue, pe = R.sample(xi, st["left"], st["right"], st["gamma"])
    ee = pe / ((st["gamma"] - 1.0) * re)
    L1 = {"rho": np.mean(np.abs(rho[sel] - re)), "v": np.mean(np.abs(v[sel, 0] - ue)),
          "P": np.mean(np.abs(P[sel] - pe)), "u": np.mean(np.abs(v[sel, 3] - ee))}
    return st, t, p, v, L1


def test_sod_converges_to_the_exact_solution():
    res = {n: run_sod(n) for n in (64, 128)}
    for q in ("rho", "v", "P", "u"):
        a, b = res[64][4][q], res[128][4][q]
        print(q, "L1", a, b, "ratio", a / b)
        assert a / b > 1.35, (q, a, b)
    st, t, p, v, L1 = res[128]
    assert L1["rho"] < 0.02 and L1["v"] < 0.035 and L1["P"] < 0.025 and L1["u"] < 0.035, L1
    assert np.max(np.abs(v[:, 1:3])) < 1e-3
    # the shock: where v_x falls below half the star velocity, right of the contact
    ps, us = R.star(st["left"], st["right"], st["gamma"])
    xs = np.linspace(0.25, 0.5, 2001)
    _, ue, _ = R.sample((xs - st["x0"]) / t, st["left"], st["right"], st["gamma"])
    x_exact = xs[np.nonzero(ue < 0.5 * us)[0][0]]
    sel = (p[:, 0] > st["x0"] + us * t) & (p[:, 0] < 0.5)
    order = np.argsort(p[sel, 0])
    x_sim = p[sel, 0][order][np.nonzero(v[sel, 0][order] < 0.5 * us)[0][0]]
    print("shock", x_sim, x_exact)
    assert abs(x_sim - x_exact) < 2.0 / 128


def test_sod_step_matches_the_oracle():
    st = inputs.sod(32)
    ev = O.evaluate(st)
    dt = 0.5 * float(np.min(O.cfl_dt(ev)))
    ost, _, _ = O.kdk_step(st, ev=ev, dt=dt)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    crk.crk_step(crk.crk_create(), pos, vel, mass, dt)
    gp, gv = as_np(pos), as_np(vel)
    dx = gp[:, :3] - ost["pos_h"][:, :3]
    dx -= np.round(dx)
    e = {"x": float(np.max(np.abs(dx))), "h": rel_err(gp[:, 3], ost["pos_h"][:, 3]),
         "v": rel_err(gv[:, :3], ost["vel_u"][:, :3]), "u": rel_err(gv[:, 3], ost["vel_u"][:, 3])}
    print("sod step", e)
    assert e["x"] < 1e-6 and max(e["h"], e["v"], e["u"]) < TOL, e
