"""Comoving variables on the GPU (crk_params.a, adot; crk_set_expansion)
against the FP64 oracle with the same scale factor and rate: grad v of the
peculiar velocity, forces and energy rates (eq:mom a^2, eq:eng, viscosity
with the Hubble flow, signal velocity), the compatible energy (1/(2a^4)), a
KDK step (drift p/a^2, expansion cooling), and graph replays across a change
of the scale factor."""
import numpy as np
import pytest
import torch

from oracle import crk as O
from paper_2202_02840_gb300 import crk, inputs
from parity import TOL, as_np, rel_err

pytestmark = pytest.mark.gpu

EXPANSIONS = [(0.6, 0.25), (1.7, -0.3)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f32(a):
    return dev(np.asarray(a, np.float64).astype(np.float32))


def flowing(case):
    st = inputs.uniform(16) if case == "uniform16" else inputs.zeldovich(16)
    st["vel_u"][:, :3] *= 10.0       # viscosity and signal speeds on
    return st


@pytest.mark.parametrize("a,adot", EXPANSIONS)
@pytest.mark.parametrize("case", ["uniform16", "zeldovich16"])
def test_passes_in_comoving_variables(case, a, adot):
    st = flowing(case)
    prm = O.params(a=a, adot=adot)
    ev = O.evaluate(st, prm)
    ctx = crk.crk_create(a=a, adot=adot)
    crk.crk_build_cells(ctx, dev(st["pos_h"]))
    out = crk.crk_corrections(ctx, f32(ev["V"]), dev(st["vel_u"]))
    gv = out[4]
    e = {"gv": rel_err(gv, ev["gv"])}
    acc, dudt, vsig, qmax, pairs = crk.crk_forces(
        ctx, dev(st["mass"]), dev(st["vel_u"]), f32(ev["V"]), f32(ev["A"]), f32(ev["B"]), f32(ev["gA"]),
        f32(ev["gB"]), f32(ev["gv"]), with_pairs=True)
    e.update({"acc": rel_err(acc, ev["acc"], floor=ev["fscale"]), "dudt": rel_err(dudt, ev["dudt"]),
              "vsig": rel_err(vsig, ev["vsig"]), "qmax": rel_err(qmax, ev["qmax"])})
    vel = st["vel_u"][:, :3].astype(np.float64)
    va = vel + 1e-3 * ev["acc"]
    du_o = O.compatible(ev["pos_h"], ev["vel"], ev["u"], ev["mass"], ev["V"], ev["A"], ev["B"], ev["gA"],
                        ev["gB"], ev["gv"], vel, va, prm)
    du_g = crk.crk_compatible(ctx, dev(st["mass"]), dev(st["vel_u"]), f32(ev["V"]), f32(ev["A"]), f32(ev["B"]),
                              f32(ev["gA"]), f32(ev["gB"]), f32(ev["gv"]), f32(vel), f32(va))
    e["du"] = rel_err(du_g, du_o)
    print(case, a, adot, e)
    assert max(e.values()) < TOL, e


@pytest.mark.parametrize("a,adot", EXPANSIONS)
def test_one_comoving_step_matches_the_oracle(a, adot):
    st = flowing("uniform16")
    prm = O.params(a=a, adot=adot)
    ev = O.evaluate(st, prm)
    dt = 0.5 * float(np.min(O.cfl_dt(ev, prm)))
    ost, _, _ = O.kdk_step(st, ev=ev, dt=dt, prm=prm)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    ctx = crk.crk_create(a=a, adot=adot)
    d = crk.crk_step(ctx, pos, vel, mass, dt, diag=True)
    gp, gv = as_np(pos), as_np(vel)
    dx = gp[:, :3] - ost["pos_h"][:, :3]
    dx -= np.round(dx)
    e = {"x": float(np.max(np.abs(dx))), "h": rel_err(gp[:, 3], ost["pos_h"][:, 3]),
         "v": rel_err(gv[:, :3], ost["vel_u"][:, :3]), "u": rel_err(gv[:, 3], ost["vel_u"][:, 3]),
         "dt_next": abs(d["dt_next"] / float(np.min(O.cfl_dt(O.evaluate(ost, prm), prm))) - 1.0)}
    print(a, adot, e)
    assert e["x"] < 1e-6 and max(e["h"], e["v"], e["u"]) < TOL, e


def test_graph_replays_follow_a_changing_scale_factor():
    st = flowing("uniform16")
    runs = []
    for use_graph in (True, False):
        pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
        ctx = crk.crk_create(a=0.8, adot=0.1)
        crk.crk_steps(ctx, pos, vel, mass, 4, 1e-4, use_graph=use_graph)
        crk.crk_set_expansion(ctx, 0.85, 0.12)
        crk.crk_steps(ctx, pos, vel, mass, 4, 1e-4, use_graph=use_graph)
        runs.append((as_np(pos), as_np(vel)))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("case", ["uniform16", "zeldovich16"])
def test_rk_density_forces_and_step(case):
    """crk_params.density = 1: the RK-corrected density feeds P, c_s, the
    viscosity, the forces and the compatible energy (and with a comoving box)."""
    st = flowing(case)
    prm = O.params(density=1.0, a=0.8, adot=0.1)
    ev = O.evaluate(st, prm)
    ctx = crk.crk_create(density=1, a=0.8, adot=0.1)
    crk.crk_build_cells(ctx, dev(st["pos_h"]))
    acc, dudt, vsig, qmax, pairs = crk.crk_forces(
        ctx, dev(st["mass"]), dev(st["vel_u"]), f32(ev["V"]), f32(ev["A"]), f32(ev["B"]), f32(ev["gA"]),
        f32(ev["gB"]), f32(ev["gv"]), with_pairs=True)
    e = {"acc": rel_err(acc, ev["acc"], floor=ev["fscale"]), "dudt": rel_err(dudt, ev["dudt"]),
         "vsig": rel_err(vsig, ev["vsig"]), "qmax": rel_err(qmax, ev["qmax"])}
    dt = 0.5 * float(np.min(O.cfl_dt(ev, prm)))
    ost, _, _ = O.kdk_step(st, ev=ev, dt=dt, prm=prm)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    crk.crk_step(crk.crk_create(density=1, a=0.8, adot=0.1), pos, vel, mass, dt)
    gp, gv = as_np(pos), as_np(vel)
    dx = gp[:, :3] - ost["pos_h"][:, :3]
    dx -= np.round(dx)
    e.update({"x": float(np.max(np.abs(dx))), "v": rel_err(gv[:, :3], ost["vel_u"][:, :3]),
              "u": rel_err(gv[:, 3], ost["vel_u"][:, 3]), "h": rel_err(gp[:, 3], ost["pos_h"][:, 3])})
    print(case, e)
    assert e["x"] < 1e-6 and max(v for k, v in e.items() if k != "x") < TOL, e
