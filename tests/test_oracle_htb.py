"""Pins of the hierarchical time-bin oracle (oracle/htb.py; CRK-HACC Sec. 2.1)
against what the mathematics fixes:

* periodic arc gaps: closed forms, including arcs that straddle the origin;
* leaf boxes cover every pair of the pair set and are translation-equivariant
  (a uniform shift moves the arcs and keeps their extents);
* particle levels at the exact power-of-two boundaries;
* the limiter's least fixed point: a closed form on a chain of leaves, and
  the invariants (|l_I - l_J| <= f_l for interacting leaves, l >= lreq,
  minimality) on a Sedov state;
* streaming: the piecewise drift composes to the parabola of a constant
  acceleration, ends at x0 + len p_1/2, and a wake-up leaves it unchanged;
* a cycle with one level (L = 0) is the KDK step of eq:verletOP with dt = Delta,
  and a cycle whose leaves all share one level (f_l = 0) is the chain of KDK
  steps at the visited ticks;
* a cycle with mixed levels stays close to global stepping at the finest tick.
"""
import numpy as np
import pytest

from oracle import crk as O
from oracle import htb as H
from paper_2202_02840_gb300 import inputs

U = np.uint64


def test_arc_gap_closed_forms():
    C = 1 << 32
    g = lambda a0, a1, b0, b1: int(H.arc_gap(U(a0 % C), U(a1 % C), U(b0 % C), U(b1 % C)))
    assert g(10, 20, 15, 30) == 0                       # overlap
    assert g(10, 20, 20, 30) == 0                       # touching ends
    assert g(10, 20, 25, 30) == 5                       # b after a
    assert g(25, 30, 10, 20) == 5                       # symmetric
    assert g(0, 10, C - 20, C - 5) == 5                 # the short way crosses the origin
    assert g(C - 10, 5, 3, 8) == 0                      # a straddles the origin and holds b0
    assert g(C - 10, 5, 20, 30) == 15                   # straddling a, b after it
    assert g(C - 10, 5, C - 40, C - 30) == 20           # straddling a, b before it
    assert g(0, C - 1, 12345, 12346) == 0               # the full circle meets everything
    # the gap of disjoint arcs never exceeds half the circle
    rng = np.random.default_rng(0)
    a0, b0 = rng.integers(0, C, 1000, dtype=np.uint64), rng.integers(0, C, 1000, dtype=np.uint64)
    ea, eb = rng.integers(0, 1 << 20, 1000, dtype=np.uint64), rng.integers(0, 1 << 20, 1000, dtype=np.uint64)
    gg = H.arc_gap(a0, (a0 + ea) & H.MASK32, b0, (b0 + eb) & H.MASK32)
    assert np.all(gg <= U(C // 2))


def _clustered(n=2048, seed=5):
    rng = np.random.default_rng(seed)
    c = rng.random((8, 3))
    x = (c[rng.integers(0, 8, n)] + 0.06 * rng.standard_normal((n, 3))) % 1.0
    pos = np.empty((n, 4), np.float32)
    pos[:, :3] = O._wrap_f32(x)
    pos[:, 3] = (0.03 + 0.05 * rng.random(n)).astype(np.float32)
    return pos


def test_leaf_boxes_cover_the_pair_set_and_move_with_a_shift():
    pos = _clustered()
    perm = H.leaf_order(pos)
    tt = H.tile_of(perm)
    lo, hi, Hm = H.tile_boxes(pos, perm)
    adj = H.tile_adjacency(lo, hi, Hm)
    assert np.array_equal(adj, adj.T) and adj.diagonal().all()
    cnt, lists = O.neighbours(pos, mode=1)
    i = np.repeat(np.arange(len(pos)), cnt)
    assert adj[tt[i], tt[lists]].all()
    # shift every particle by 0.37 without re-sorting: tiles now straddle the
    # origin; the arcs keep their extents (to the rounding of the shifted
    # coordinates) and still cover every pair
    sh = pos.copy()
    sh[:, :3] = O._wrap_f32(pos[:, :3].astype(np.float64) + 0.37)
    lo2, hi2, Hm2 = H.tile_boxes(sh, perm)
    ext = (hi - lo) & H.MASK32
    ext2 = (hi2 - lo2) & H.MASK32
    assert np.max(np.abs(ext.astype(np.int64) - ext2.astype(np.int64))) <= 600   # < 2^-22 box
    adj2 = H.tile_adjacency(lo2, hi2, Hm2)
    cnt2, lists2 = O.neighbours(sh, mode=1)
    i2 = np.repeat(np.arange(len(sh)), cnt2)
    assert adj2[tt[i2], tt[lists2]].all()
    # tight: the shifted adjacency is the unshifted one up to the rounding margin
    assert abs(int(adj2.sum()) - int(adj.sum())) <= 0.02 * adj.sum()


def test_particle_levels_at_the_power_of_two_boundaries():
    D = 0.1
    dt = np.array([np.inf, 0.2, D, np.nextafter(D, 1.0), D / 2, np.nextafter(D / 2, 1.0), D / 8, D / 9, 1e-9])
    lev, unres = H.particle_levels(dt, D, 3)
    assert lev.tolist() == [0, 0, 1, 0, 2, 1, 3, 3, 3]
    assert unres.tolist() == [False] * 6 + [True, True, True]


def test_limiter_closed_form_on_a_chain():
    n = 12
    adj = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
    lreq = np.zeros(n, np.int64)
    lreq[5] = 7
    lreq[11] = 1
    for f in (0, 1, 2, 3):
        lev = H.limit_levels(lreq, adj, f)
        want = np.maximum(lreq, 7 - f * np.abs(np.arange(n) - 5))
        if f == 0:
            want[:] = 7
        assert lev.tolist() == want.tolist(), (f, lev)
    # fixed tiles keep their level and block nothing but themselves
    fixed = np.zeros(n, bool)
    fixed[7] = True
    lev = H.limit_levels(lreq, adj, 1, fixed=fixed)
    assert lev[7] == 0 and lev[6] == 6 and lev[8] == 0 and lev[4] == 6


def test_limiter_fixed_point_on_a_sedov_state():
    st = inputs.sedov(16)
    ev = O.evaluate(st)
    perm = H.leaf_order(st["pos_h"])
    tt = H.tile_of(perm)
    nt = len(perm) // 32
    adj = H.tile_adjacency(*H.tile_boxes(st["pos_h"], perm))
    dt = O.cfl_dt(ev)
    plev, _ = H.particle_levels(dt, 16 * dt.min(), 6)
    lreq = H.tile_max(plev, tt, nt)
    for f in (1, 2):
        lev = H.limit_levels(lreq, adj, f)
        I, J = np.nonzero(adj)
        assert np.all(np.abs(lev[I] - lev[J]) <= f)
        assert np.all(lev >= lreq)
        nb = np.where(adj, lev[None, :], H.NONE).max(axis=1) - f
        assert np.array_equal(lev, np.maximum(lreq, nb))
        assert lev.max() == lreq.max() and len(np.unique(lev)) > 2


def test_streaming_is_the_constant_acceleration_parabola():
    rng = np.random.default_rng(3)
    m = 64
    x0 = rng.random((m, 3))
    p0 = rng.standard_normal((m, 3))
    a = rng.standard_normal((m, 3))
    tick = 1e-3
    t0 = rng.integers(0, 8, m).astype(np.float64)
    ln = (2 ** rng.integers(0, 4, m)).astype(np.float64)
    p_half = p0 + 0.5 * a * (ln * tick)[:, None]
    par = lambda t: x0 + p0 * ((t - t0) * tick)[:, None] + 0.5 * a * (((t - t0) * tick) ** 2)[:, None]
    # pieces over an uneven partition of the step compose to the parabola
    x = x0.copy()
    t = t0.copy()
    for frac in (0.25, 0.5, 0.625, 1.0):
        tb = t0 + frac * ln
        x = H.stream(x, p_half, a, t, tb, t0, ln, tick)
        assert np.allclose(x, par(tb), rtol=0, atol=1e-13)
        t = tb
    # the step end is the drift of eq:verletOP: x0 + len p_1/2
    assert np.allclose(x, x0 + p_half * (ln * tick)[:, None], rtol=0, atol=1e-13)
    # a wake-up: shorter step len', p_1/2 shortened by a (len - len') tick / 2;
    # the trajectory is the same parabola
    ln2 = np.maximum(ln / 2, 1.0)
    ph2 = p_half - 0.5 * a * ((ln - ln2) * tick)[:, None]
    for frac in (0.3, 0.7, 1.0):
        tb = t0 + frac * ln2
        assert np.allclose(H.stream(x0, ph2, a, t0, tb, t0, ln2, tick), par(tb), rtol=0, atol=1e-13)


def _E(st):
    m = st["mass"].astype(np.float64)
    v = st["vel_u"].astype(np.float64)
    return float((0.5 * m * (v[:, :3] ** 2).sum(1) + m * v[:, 3]).sum())


def test_cycle_with_one_level_is_the_kdk_step():
    st = inputs.sedov(16)
    ev = O.evaluate(st)
    D = 2.0 * float(O.cfl_dt(ev).min())
    out, ev1, info = H.cycle(st, ev, Delta=D, L=0, f_l=2)
    ref, evr, dt = O.kdk_step(st, ev=ev, dt=D)
    assert info["ticks"] == [1] and info["unresolved"] > 0
    for key in ("pos_h", "vel_u"):
        np.testing.assert_array_equal(out[key], ref[key])
    np.testing.assert_array_equal(ev1["acc"], evr["acc"])


def test_cycle_with_one_shared_level_is_a_chain_of_kdk_steps():
    st = inputs.uniform(16)
    ev = O.evaluate(st)
    dtm = float(O.cfl_dt(ev).min())
    D = 3.0 * dtm
    out, ev1, info = H.cycle(st, ev, Delta=D, L=3, f_l=0)
    assert len(np.unique(info["levels_start"])) == 1 and info["wakeups"] == 0
    ticks = [0] + info["ticks"]
    assert len(ticks) > 2
    tick = D / 8
    ref, evr = st, ev
    for a, b in zip(ticks[:-1], ticks[1:]):
        ref, evr, _ = O.kdk_step(ref, ev=evr, dt=(b - a) * tick)
    # the chain stores FP32 velocities between its steps, the cycle keeps FP64
    dv = np.abs(out["vel_u"].astype(np.float64) - ref["vel_u"].astype(np.float64))
    assert np.max(dv[:, :3]) < 1e-7 and np.max(dv[:, 3]) < 1e-6
    dx = np.abs(out["pos_h"].astype(np.float64) - ref["pos_h"].astype(np.float64))
    assert np.max(np.minimum(dx[:, :3], 1 - dx[:, :3])) < 1e-7 and np.max(dx[:, 3]) < 1e-7
    assert abs(_E(out) / _E(st) - 1) < 1e-6


def test_cycle_with_mixed_levels_and_wakeups_tracks_global_stepping():
    """A blast in a warm, jittered background after 8 KDK steps: the shock
    moves into leaves stepping 8x longer, which the limiter wakes up
    mid-cycle; the background's pressure noise gives the woken leaves an
    acceleration, so their shortened half kick matters."""
    st, ev = inputs.sedov(16, u0=0.05, jitter=0.1), None
    for _ in range(8):
        st, ev, _ = O.kdk_step(st, ev=ev)
    dtm = float(O.cfl_dt(ev).min())
    L = 4
    D = 12.0 * dtm
    out, ev1, info = H.cycle(st, ev, Delta=D, L=L, f_l=2)
    assert info["unresolved"] == 0 and info["wakeups"] > 0
    assert len(np.unique(info["levels_start"])) >= 3
    n = st["pos_h"].shape[0]
    assert info["evaluations"] < 0.4 * n * (1 << L)       # most leaves step long
    ref, evr = st, ev
    for _ in range(1 << L):
        ref, evr, _ = O.kdk_step(ref, ev=evr, dt=D / (1 << L))
    E0 = _E(st)
    assert abs(_E(out) / E0 - 1) < 2e-4
    m = st["mass"].astype(np.float64)
    P = (m[:, None] * out["vel_u"][:, :3].astype(np.float64)).sum(0)
    assert np.max(np.abs(P)) < 1e-5 * np.sqrt(2 * E0)
    # velocities, energies and positions agree with global stepping at the finest tick
    dv = np.linalg.norm(out["vel_u"][:, :3].astype(np.float64) - ref["vel_u"][:, :3], axis=1)
    vs = np.max(np.linalg.norm(ref["vel_u"][:, :3].astype(np.float64), axis=1))
    assert np.max(dv) < 0.02 * vs, np.max(dv) / vs
    du = np.abs(out["vel_u"][:, 3].astype(np.float64) - ref["vel_u"][:, 3])
    assert np.max(du) < 1e-3 * np.max(ref["vel_u"][:, 3])
    dx = np.abs(out["pos_h"][:, :3].astype(np.float64) - ref["pos_h"][:, :3])
    assert np.max(np.minimum(dx, 1 - dx)) < 0.01 / 16
    # the woken leaves follow global stepping closely (their half kick shortened
    # to the new step; left at the old length they are off by ~2e-5 vs)
    w = np.array(sorted(info["woken"]))
    assert len(w) > 0 and np.max(dv[w]) < 1e-5 * vs, np.max(dv[w]) / vs
