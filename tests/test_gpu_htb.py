"""Hierarchical time bins on the GPU (crk_cycle, crk_htb_levels) against the
FP64 oracle of oracle/htb.py (CRK-HACC Sec. 2.1).

* Level assignment (sort into leaves, leaf boxes as periodic arcs, tile
  interaction lists, particle levels, the limiter's least fixed point) is
  integer work decided in FP64 on both sides from the same FP32 time steps:
  bit-exact, including a ragged last leaf and single-leaf inputs.
* A cycle with L = 0 is bitwise the KDK step crk_step(dt = Delta).
* A cycle from the same FP32 state as the oracle's: the same ticks, the same
  active and woken leaves, and states within FP32 tolerance, for a blast with
  wake-ups and for a bulk flow that carries leaves across the periodic
  boundary (leaf boxes that wrap).
* Chained cycles conserve momentum and nearly conserve energy, and track global
  stepping at the finest tick.
"""
import numpy as np
import pytest
import torch

from oracle import crk as O
from oracle import htb as H
from paper_2202_02840_gb300 import crk, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_levels(pos, dt, D, L, f):
    perm = H.leaf_order(pos)
    tt = H.tile_of(perm)
    nt = (len(perm) + 31) // 32
    adj = H.tile_adjacency(*H.tile_boxes(pos, perm))
    plev, unres = H.particle_levels(dt, D, L)
    lev = H.limit_levels(H.tile_max(plev, tt, nt), adj, f)
    return lev[tt], int(unres.sum())


def _clustered(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.random((6, 3))
    x = (c[rng.integers(0, 6, n)] + 0.05 * rng.standard_normal((n, 3))) % 1.0
    pos = np.empty((n, 4), np.float32)
    pos[:, :3] = O._wrap_f32(x)
    pos[:, 3] = (0.02 + 0.06 * rng.random(n)).astype(np.float32)
    return pos


@pytest.mark.parametrize("case", ["sedov16", "clustered3000", "tiny1", "tiny33"])
def test_levels_match_oracle_bitwise(case):
    rng = np.random.default_rng(7)
    if case == "sedov16":
        st = inputs.sedov(16)
        ev = O.evaluate(st)
        pos = st["pos_h"]
        dt = O.cfl_dt(ev).astype(np.float32)
        cases = [(16.0 * float(dt.min()), 6, f) for f in (0, 1, 2, 3)] + [(float(dt.min()), 2, 1)]
    elif case == "clustered3000":
        pos = _clustered(3000, 11)
        d = pos[:, :3].astype(np.float64) - pos[0, :3]
        d -= np.round(d)
        # spatially smooth steps (short near one particle, long far away) with noise
        dt = (1e-4 * (1.0 + 4000.0 * (d * d).sum(1)) * np.exp(0.3 * rng.standard_normal(len(pos)))).astype(np.float32)
        cases = [(0.5, 10, 1), (0.5, 10, 2), (0.5, 4, 2), (2.0 ** -3, 9, 3)]
    else:
        n = int(case[4:])
        pos = _clustered(n, 3)
        dt = np.exp(rng.uniform(np.log(1e-3), 0.0, n)).astype(np.float32)
        cases = [(0.25, 0, 2), (0.25, 5, 1), (0.25, 12, 0)]
    ctx = crk.crk_create()
    p = dev(pos)
    for D, L, f in cases:
        lev, unres = crk.crk_htb_levels(ctx, p, dev(dt), D, L, f)
        want, wu = oracle_levels(pos, dt.astype(np.float64), D, L, f)
        got = lev.cpu().numpy()
        assert np.array_equal(got, want), (case, D, L, f, np.nonzero(got != want)[0][:10])
        assert unres == wu
        if f > 0 and L > 2 and case != "tiny1":
            assert len(np.unique(want)) >= 2


def _run_cycle(st, D, L, f, **params):
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    ctx = crk.crk_create(**params)
    info = crk.crk_cycle(ctx, pos, vel, mass, D, L, f)
    return pos.cpu().numpy(), vel.cpu().numpy(), info, ctx


@pytest.mark.parametrize("pair_form", [0, 1])
def test_cycle_with_one_level_is_bitwise_the_kdk_step(pair_form):
    """With every leaf at level 0 a cycle is one KDK step, bitwise, in either
    form of P4 and P5 (the pair-once P5 of the opening kick reads the tile
    lists its P4 ran with, though the cycle has refitted them)."""
    for st in (inputs.sedov(16), inputs.uniform(16)):
        ev = O.evaluate(st)
        D = 2.0 * float(O.cfl_dt(ev).min())
        p1, v1, info, _ = _run_cycle(st, D, 0, 2, pair_form=pair_form)
        pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
        crk.crk_step(crk.crk_create(pair_form=pair_form), pos, vel, mass, D)
        assert info["ticks"] == 1 and info["evaluations"] == len(p1)
        np.testing.assert_array_equal(p1, pos.cpu().numpy())
        np.testing.assert_array_equal(v1, vel.cpu().numpy())


def level_margin(dt, D, L):
    """Smallest relative distance of any dt to a level boundary D / 2^l."""
    b = np.ldexp(D, -np.arange(L + 1))
    return float(np.min(np.abs(dt[:, None] / b[None, :] - 1.0)))


def pick_delta(dt, base, L, tries=40):
    best, bD = -1.0, base
    for k in range(tries):
        D = base * (1.0 + 0.0125 * k)
        m = level_margin(dt, D, L)
        if m > best:
            best, bD = m, D
    return bD, best


def compare_cycle(st, L, f, mult, min_wakeups=0, **params):
    ev = O.evaluate(st)
    dt = O.cfl_dt(ev)
    D, margin = pick_delta(dt, mult * float(dt.min()), L)
    assert margin > 1e-4
    out, ev1, info = H.cycle(st, ev, Delta=D, L=L, f_l=f)
    p, v, g, _ = _run_cycle(st, D, L, f, **params)
    n = len(p)
    lev0 = np.bincount(info["levels_start"], minlength=32)
    assert g["level_count"] == lev0.tolist()
    assert g["ticks"] == len(info["ticks"])
    assert g["evaluations"] == info["evaluations"]
    assert g["wakeups"] == info["wakeups"] >= min_wakeups
    assert g["unresolved"] == info["unresolved"]
    dx = np.abs(p[:, :3].astype(np.float64) - out["pos_h"][:, :3])
    dx = np.minimum(dx, 1.0 - dx)
    vs = np.max(np.abs(out["vel_u"][:, :3]))
    us = np.max(np.abs(out["vel_u"][:, 3]))
    ex = np.max(dx)
    ev_ = np.max(np.abs(v[:, :3].astype(np.float64) - out["vel_u"][:, :3])) / vs
    eu = np.max(np.abs(v[:, 3].astype(np.float64) - out["vel_u"][:, 3])) / us
    eh = np.max(np.abs(p[:, 3].astype(np.float64) - out["pos_h"][:, 3]) / out["pos_h"][:, 3])
    print("cycle vs oracle: x %.2e  v %.2e  u %.2e  h %.2e  (ticks %d, evals %d, wakeups %d)"
          % (ex, ev_, eu, eh, g["ticks"], g["evaluations"], g["wakeups"]))
    assert ex < 2e-6 and ev_ < 1e-4 and eu < 1e-4 and eh < 1e-5
    return info


@pytest.mark.parametrize("pair_form", [0, 1])
def test_cycle_matches_oracle_blast_with_wakeups(pair_form):
    """Also in the pair-once form, whose full evaluations (the cycle's ends)
    alternate with directed evaluations of the active tiles, each P5 taking
    the form of the P4 that stored its forces."""
    st, ev = inputs.sedov(16, u0=0.05, jitter=0.1), None
    for _ in range(8):
        st, ev, _ = O.kdk_step(st, ev=ev)
    info = compare_cycle(st, 4, 2, 12.0, min_wakeups=1, pair_form=pair_form)
    assert len(np.unique(info["levels_start"])) >= 3


def test_cycle_matches_oracle_bulk_flow_across_the_boundary():
    st = inputs.sedov(16, u0=0.05, jitter=0.1)
    st["vel_u"][:, 0] += np.float32(3.0)      # leaves drift ~1 spacing per cycle, across x = 1
    compare_cycle(st, 3, 1, 24.0)


def test_chained_cycles_conserve_and_track_global_stepping():
    st = inputs.sedov(32, u0=0.05)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    m = st["mass"].astype(np.float64)

    def EP(v):
        v = v.cpu().numpy().astype(np.float64)
        return float((0.5 * m * (v[:, :3] ** 2).sum(1) + m * v[:, 3]).sum()), (m[:, None] * v[:, :3]).sum(0)

    E0, _ = EP(vel)
    ctx = crk.crk_create()
    d = crk.crk_step(ctx, pos.clone(), vel.clone(), mass, 0.0, diag=True)   # CFL step at the start
    L = 4
    D = 16.0 * d["dt"]
    gpos, gvel = pos.clone(), vel.clone()
    ctx = crk.crk_create()
    evals = 0
    for k in range(3):
        info = crk.crk_cycle(ctx, pos, vel, mass, D, L, 2)
        evals += info["evaluations"]
    E, P = EP(vel)
    assert abs(E / E0 - 1) < 1e-3, E / E0 - 1
    assert np.max(np.abs(P)) < 1e-4 * np.sqrt(2 * E0)
    n = pos.shape[0]
    assert evals < 0.5 * 3 * n * (1 << L)
    gctx = crk.crk_create()
    for k in range(3 * (1 << L)):
        crk.crk_step(gctx, gpos, gvel, mass, D / (1 << L))
    def r(p):
        d = p[:, :3].cpu().numpy().astype(np.float64) - 0.5
        d -= np.round(d)
        return np.linalg.norm(d, axis=1)

    edges = np.linspace(0.0, 0.45, 19)

    def prof(p, q):
        i = np.digitize(r(p), edges) - 1
        ok = (i >= 0) & (i < len(edges) - 1)
        return np.bincount(i[ok], q[ok], len(edges) - 1) / np.maximum(np.bincount(i[ok], None, len(edges) - 1), 1)

    for col in (3,):
        a = prof(pos, vel[:, col].cpu().numpy().astype(np.float64))
        b = prof(gpos, gvel[:, col].cpu().numpy().astype(np.float64))
        err = np.max(np.abs(a - b)) / np.max(np.abs(b))
        print("u profile, time bins vs global stepping:", err)
        assert err < 0.02
