"""FP64 oracle of the hierarchical power-of-two time bins of CRK-HACC (Sec. 2.1:
the hydro subcycles of eq:Usubsub, the per-particle criteria Delta y_hyd and
Delta y_acc, leaf-level bins, the f_l limiter and parabolic streaming of
passive leaves).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product path).
Shares no code with the CUDA library; the pair passes are the FP64 passes of
oracle.crk, evaluated for the particles of the active leaves only.

Readings (the paper states the scheme in words; these fix what it leaves open):
  * A cycle is one base step Delta of 2^L ticks (tick = Delta / 2^L); a leaf at
    level l steps 2^(L-l) ticks.  The leaves are the 32-particle tiles of the
    Morton order at the cycle start, kept for the whole cycle (the paper builds
    its tree once per long step and keeps the leaves through the hydro
    subcycles).
  * Particle level: the smallest l >= 0 with Delta / 2^l < dt_i (dt_i of the
    CFL and acceleration criteria); leaf level = the deepest of its particles;
    a particle needing l > L is held at L and counted as unresolved.
  * Interacting leaves: the leaf interaction list, i.e. tiles I, J whose
    fixed-point bounding boxes are closer than max(Hmax_I, Hmax_J).  A tile's
    box is the smallest periodic arc per axis containing its particles,
    measured from the tile's first particle.
  * Limiter (f_l): at the cycle start all levels are raised to the least fixed
    point of l_I = max(lreq_I, max_{J ~ I} l_J - f_l).  Mid-cycle, the leaves
    ending a step take max(lreq, l - 1 if the tick is aligned to the doubled
    step, else l), then the same fixed point over the active leaves with the
    passive levels held, and every passive neighbour of an active leaf is
    raised to at least (active level - f_l).
  * Raising a passive leaf (a wake-up) ends its current step at the first
    tick after now that is a multiple of its new step; its half kick is
    shortened to match, p_1/2 -= a (len_old - len_new) tick / 2 (and u alike),
    which leaves its trajectory unchanged.
  * Leaves move to shallower levels one level at a time, and only at a tick
    aligned with the doubled step ("every other time step").
  * Passive leaves are streamed: x(t) follows x0 + p0 (t - t0) + a (t - t0)^2 / 2,
    i.e. v(t) = p_1/2 + a (t - t_mid); u alike with the opening-kick energy rate.
    Active leaves see passive neighbours through their streamed x, v, u and
    their last evaluated V, A, B, grad A, grad B, grad v (the passive leaves
    evaluate no derivatives).
  * An active leaf closes its step with the predictor of eq:verletOP
    (v = p_1/2 + a len tick / 2), evaluates P1..P4, closes the kick with the
    compatible energy (passive neighbours contribute v_j + v'_j = 2 v_j(t)),
    advances h by one eq:thacker update and opens its next step.
  * At the end of the cycle every leaf ends its step; the full evaluation there
    is the one the next cycle opens with.
"""
import numpy as np

from . import crk as O

TWO32 = np.uint64(1 << 32)
MASK32 = np.uint64(0xFFFFFFFF)
TILE = 32
NONE = -(1 << 40)   # 'no level' sentinel (far below any level minus f_l)


def leaf_order(pos_h):
    """Sorted slot -> particle: stable sort by 30-bit Morton key of the top 10
    fixed-point bits per axis (the chaining-mesh order of Sec. 2.3)."""
    _, perm, _, _ = O.cells(pos_h)
    return perm.astype(np.int64)


def tile_of(perm, tile=TILE):
    t = np.empty(len(perm), np.int64)
    t[perm] = np.arange(len(perm)) // tile
    return t


def tile_boxes(pos_h, perm, tile=TILE):
    """Per tile: (lo, hi) fixed-point arcs per axis (uint64 values < 2^32) and
    Hmax.  The arc is measured from the tile's first particle: lo = q_ref +
    min_k d_k, hi = q_ref + max_k d_k (mod 2^32), d_k = signed (q_k - q_ref)."""
    q, H = O.fixed_point(pos_h)
    n = len(perm)
    nt = (n + tile - 1) // tile
    lo = np.zeros((nt, 3), np.uint64)
    hi = np.zeros((nt, 3), np.uint64)
    Hm = np.zeros(nt, np.uint64)
    q = q.astype(np.int64)
    for T in range(nt):
        m = perm[T * tile:(T + 1) * tile]
        ref = q[m[0]]
        d = (q[m] - ref) % (1 << 32)
        d = np.where(d >= (1 << 31), d - (1 << 32), d)
        lo[T] = ((ref + d.min(axis=0)) % (1 << 32)).astype(np.uint64)
        hi[T] = ((ref + d.max(axis=0)) % (1 << 32)).astype(np.uint64)
        Hm[T] = np.uint64(H[m].max())
    return lo, hi, Hm


def arc_gap(a0, a1, b0, b1):
    """Periodic gap between the arcs [a0, a1] and [b0, b1] of a circle of 2^32
    (uint64 arrays): 0 when they overlap, else the shorter way round."""
    with np.errstate(over="ignore"):   # unsigned wrap-around is the modular difference
        ea = (a1 - a0) & MASK32
        eb = (b1 - b0) & MASK32
        overlap = (((b0 - a0) & MASK32) <= ea) | (((a0 - b0) & MASK32) <= eb)
        g = np.minimum((b0 - a1) & MASK32, (a0 - b1) & MASK32)
    return np.where(overlap, np.uint64(0), g)


def tile_adjacency(lo, hi, Hm):
    """adj[I, J]: the tiles' boxes are closer than max(Hmax_I, Hmax_J)
    (squared fixed-point gap, exact in uint64)."""
    g2 = np.zeros((len(Hm), len(Hm)), np.uint64)
    for a in range(3):
        g = arc_gap(lo[:, None, a], hi[:, None, a], lo[None, :, a], hi[None, :, a])
        g2 += g * g
    R = np.maximum(Hm[:, None], Hm[None, :])
    return g2 < R * R


def particle_levels(dt, Delta, L):
    """Smallest l in [0, L] with Delta / 2^l < dt_i (exact power-of-two
    scaling, compared in FP64); unresolved where even l = L is too coarse."""
    dt = np.asarray(dt, np.float64)
    lev = np.full(dt.shape, -1, np.int64)
    for l in range(L, -1, -1):
        lev = np.where(np.ldexp(Delta, -l) < dt, l, lev)
    unresolved = lev < 0
    return np.where(unresolved, L, lev), unresolved


def tile_max(values, tiles, nt):
    out = np.full(nt, NONE, np.int64)
    np.maximum.at(out, tiles, values)
    return out


def limit_levels(lreq, adj, f_l, fixed=None, max_iter=100000):
    """Least fixed point of l_I = max(lreq_I, max_{J ~ I} l_J - f_l) over the
    tiles where `fixed` is False; fixed tiles keep lreq."""
    lev = lreq.copy()
    free = np.ones(len(lev), bool) if fixed is None else ~fixed
    for _ in range(max_iter):
        nb = np.where(adj, lev[None, :], NONE).max(axis=1) - f_l
        new = np.where(free, np.maximum(lreq, nb), lev)
        if np.array_equal(new, lev):
            return lev
        lev = new
    raise RuntimeError("level limiter did not converge")


def stream(x, p_half, acc, t_a, t_b, t0, ln, tick):
    """Streamed position at tick t_b from tick t_a (FP64, unwrapped): the exact
    integral of v(t) = p_1/2 + a (t - t_mid), t_mid = t0 + ln / 2, i.e. the
    parabola x0 + p0 (t - t0) + a (t - t0)^2 / 2 of a constant acceleration."""
    tmid = np.asarray(t0 + 0.5 * ln, np.float64)
    vmean = p_half + acc * (tick * (0.5 * (t_a + t_b) - tmid))[..., None]
    w = np.asarray((t_b - t_a) * tick, np.float64)
    return x + (w[..., None] if w.ndim else w) * vmean


def _merge(old, new, act):
    out = np.array(old, np.float64, copy=True)
    out[act] = np.asarray(new, np.float64)[act]
    return out


def _evaluate_active(pos, vpred, upred, mass, cache, act_idx, prm, k):
    """P1..P4 for the particles act_idx; everyone else keeps the cached V,
    A, B, grad A, grad B, grad v, acc, dudt, vsig, qmax."""
    c = dict(cache)
    tg = act_idx.astype(np.int32)
    p1 = O.volumes(pos, k, targets=tg)
    c["V"] = _merge(c["V"], p1["V"], act_idx)
    c["N"] = _merge(c["N"], p1["N"], act_idx)
    p2 = O.corrections(pos, c["V"], k, targets=tg)
    for key in ("A", "B", "gA", "gB"):
        c[key] = _merge(c[key], p2[key], act_idx)
    gv = O.gradv(pos, c["V"], vpred, c["A"], c["B"], c["gA"], c["gB"], k, targets=tg)
    c["gv"] = _merge(c["gv"], gv, act_idx)
    p4 = O.forces(pos, vpred, upred, mass, c["V"], c["A"], c["B"], c["gA"], c["gB"], c["gv"], prm, k,
                  targets=tg)
    for key in ("acc", "dudt", "vsig", "qmax"):
        c[key] = _merge(c[key], p4[key], act_idx)
    c["rho"], c["P"], c["cs"], c["s"] = O.thermo(c["V"], mass, upred, prm)
    c["pos_h"], c["vel"], c["u"], c["mass"] = pos.copy(), vpred, upred, mass
    return c


def _dt(c, prm):
    return O.cfl_dt(c, prm)


def cycle(state, ev=None, Delta=1e-3, L=4, f_l=2, prm=None, k=None, h_min=1e-6, h_max=0.3):
    """Advance the synchronized state by one base step Delta with hierarchical
    bins.  `ev` is the evaluation at the state (O.evaluate, or the one a
    previous cycle returned).  Returns (state', ev', info)."""
    prm = O.params() if prm is None else prm
    if prm[O.IA] != 1.0 or prm[O.IADOT] != 0.0 or prm[O.IDENS] != 0.0:
        raise ValueError("time bins are defined here for a static box (a = 1, adot = 0) and rho = m / V")
    if ev is None:
        ev = O.evaluate(state, prm, k)
    n = state["pos_h"].shape[0]
    T = 1 << L
    tick = Delta / T
    pos = np.array(state["pos_h"], np.float32, copy=True)
    mass = np.asarray(state["mass"], np.float64)
    vu = np.asarray(state["vel_u"], np.float64)
    p_sync, u_sync = vu[:, :3].copy(), vu[:, 3].copy()

    perm = leaf_order(pos)
    tt = tile_of(perm)
    nt = (n + TILE - 1) // TILE
    lo, hi, Hm = tile_boxes(pos, perm)
    adj = tile_adjacency(lo, hi, Hm)
    plev, unres = particle_levels(_dt(ev, prm), Delta, L)
    lev = limit_levels(tile_max(plev, tt, nt), adj, f_l)
    info = {"levels_start": lev.copy(), "unresolved": int(unres.sum()), "ticks": [], "active": [],
            "wakeups": 0, "evaluations": 0}
    t0 = np.zeros(nt, np.int64)
    ln = (1 << (L - lev)).astype(np.int64)

    cache = {key: np.array(ev[key], np.float64, copy=True)
             for key in ("V", "N", "A", "B", "gA", "gB", "gv", "acc", "dudt", "vsig", "qmax")}
    acc = cache["acc"]
    # opening kicks of every leaf, compatible energy of eq:compEng
    half = 0.5 * ln[tt] * tick
    p_half = p_sync + half[:, None] * acc
    du_open = O.compatible(ev["pos_h"], ev["vel"], ev["u"], mass, ev["V"], ev["A"], ev["B"], ev["gA"],
                           ev["gB"], ev["gv"], p_sync, p_half, prm, k)
    u_half = u_sync + half * du_open

    t = 0
    while True:
        t_end = t0 + ln
        t_next = int(t_end.min())
        tmid = (t0 + 0.5 * ln)[tt]
        # parabolic streaming of every particle from t to t_next
        pos[:, :3] = O._wrap_f32(stream(pos[:, :3].astype(np.float64), p_half, acc, t, t_next, t0[tt], ln[tt],
                                        tick))
        t = t_next
        vpred = p_half + acc * (tick * (t - tmid))[:, None]
        upred = u_half + du_open * (tick * (t - tmid))
        act_t = t_end == t
        act = act_t[tt]
        info["ticks"].append(t)
        info["active"].append(int(act.sum()))
        if t == T:
            break
        act_idx = np.nonzero(act)[0]
        # leaf boxes and interaction list at the drifted positions (h before the update)
        lo, hi, Hm = tile_boxes(pos, perm)
        adj = tile_adjacency(lo, hi, Hm)
        cache = _evaluate_active(pos, vpred, upred, mass, cache, act_idx, prm, k)
        info["evaluations"] += len(act_idx)
        acc = cache["acc"]
        # closing kick of the active leaves
        hc = 0.5 * ln[tt] * tick
        p1 = p_half + hc[:, None] * acc
        vb = np.where(act[:, None], p_half, vpred)
        va = np.where(act[:, None], p1, vpred)
        pos_ev = pos.copy()      # both kicks use the pair forces of this evaluation (h before the update)
        du_c = O.compatible(pos_ev, vpred, upred, mass, cache["V"], cache["A"], cache["B"], cache["gA"],
                            cache["gB"], cache["gv"], vb, va, prm, k, targets=act_idx.astype(np.int32))
        u1 = u_half + hc * np.where(act, du_c, 0.0)
        hnew = np.clip(O.thacker(pos[:, 3].astype(np.float64), cache["N"], prm), h_min, h_max)
        pos[:, 3] = np.where(act, hnew, pos[:, 3]).astype(np.float32)
        # new levels of the active leaves, limiter, wake-ups
        plev, unres = particle_levels(_dt(cache, prm), Delta, L)
        info["unresolved"] += int((unres & act).sum())
        lreq = tile_max(np.where(act, plev, -1), tt, nt)
        aligned = (t % (2 << (L - lev))) == 0      # tick aligned to the doubled step of the level
        base = np.where((lev > 0) & aligned, lev - 1, lev)
        tent = np.where(act_t, np.maximum(lreq, base), lev)
        new = limit_levels(tent, adj, f_l, fixed=~act_t)
        wake = np.where(adj[:, act_t], new[None, act_t], NONE).max(axis=1) - f_l
        raise_ = (~act_t) & (wake > lev)
        info["wakeups"] += int(raise_.sum())
        info.setdefault("woken", set()).update(np.nonzero(raise_[tt])[0].tolist())
        # woken leaves: shorter current step, half kick shortened to match
        for J in np.nonzero(raise_)[0]:
            Sn = 1 << (L - int(wake[J]))
            te = (t // Sn + 1) * Sn
            d_len = ln[J] - (te - t0[J])
            mJ = tt == J
            p_half[mJ] -= 0.5 * d_len * tick * acc[mJ]
            u_half[mJ] -= 0.5 * d_len * tick * du_open[mJ]
            ln[J] = te - t0[J]
            new[J] = wake[J]
        # opening kick of the active leaves
        lev = new
        for T_ in np.nonzero(act_t)[0]:
            t0[T_] = t
            ln[T_] = 1 << (L - int(lev[T_]))
        ho = 0.5 * ln[tt] * tick
        p_open = p1 + ho[:, None] * acc
        vb = np.where(act[:, None], p1, vpred)
        va = np.where(act[:, None], p_open, vpred)
        du_o = O.compatible(pos_ev, vpred, upred, mass, cache["V"], cache["A"], cache["B"], cache["gA"],
                            cache["gB"], cache["gv"], vb, va, prm, k, targets=act_idx.astype(np.int32))
        p_half = np.where(act[:, None], p_open, p_half)
        du_open = np.where(act, du_o, du_open)
        u_half = np.where(act, u1 + ho * du_o, u_half)

    # end of the cycle: every leaf ends its step; full evaluation, closing kicks
    st = {"pos_h": pos.copy(), "vel_u": np.empty((n, 4), np.float32),
          "mass": np.asarray(state["mass"], np.float32)}
    st["vel_u"][:, :3] = vpred
    st["vel_u"][:, 3] = upred
    ev1 = O.evaluate(st, prm, k)
    info["evaluations"] += n
    hc = 0.5 * ln[tt] * tick
    p1 = p_half + hc[:, None] * ev1["acc"]
    du_c = O.compatible(ev1["pos_h"], ev1["vel"], ev1["u"], mass, ev1["V"], ev1["A"], ev1["B"], ev1["gA"],
                        ev1["gB"], ev1["gv"], p_half, p1, prm, k)
    u1 = u_half + hc * du_c
    out = {"pos_h": pos.copy(), "vel_u": np.empty((n, 4), np.float32), "mass": st["mass"]}
    out["pos_h"][:, 3] = np.clip(O.thacker(pos[:, 3].astype(np.float64), ev1["N"], prm), h_min, h_max)
    out["vel_u"][:, :3] = p1
    out["vel_u"][:, 3] = u1
    info["levels_end"] = lev
    return out, ev1, info
