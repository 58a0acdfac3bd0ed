"""Batched boxes: independent periodic boxes in one particle set.

Each box is its own problem, so the oracle checks each box on its own: the
neighbour sets of a batched build must equal each box's brute-force sets
bit for bit (a particle never sees another box), every pass must match the
oracle box by box, and a batched step must advance each box as a step of
that box alone would (with its own CFL time step)."""
import numpy as np
import pytest
import torch

from oracle import crk as O
from paper_2202_02840_gb300 import crk, inputs
from parity import TOL, as_np, rel_err, set_hash, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def boxes():
    """Three boxes of uneven size and structure (uniform, clumped, blast)."""
    return [workload("uniform", 16), workload("clustered", 1500, 5), workload("sedov", 14)]


def concat(sts):
    start = np.cumsum([0] + [s["pos_h"].shape[0] for s in sts])
    cat = {k: np.concatenate([s[k] for s in sts]) for k in ("pos_h", "vel_u", "mass")}
    return cat, [int(x) for x in start]


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_neighbour_sets_are_per_box(mode):
    sts = boxes()
    cat, start = concat(sts)
    ctx = crk.crk_create()
    crk.crk_build_cells_batched(ctx, dev(cat["pos_h"]), start)
    cnt, hsh = crk.crk_neighbours(ctx, mode)
    cnt, hsh = cnt.cpu().numpy(), hsh.cpu().numpy().view(np.uint32)
    for b, st in enumerate(sts):
        oc, ol = O.neighbours(st["pos_h"], mode=mode)
        sl = slice(start[b], start[b + 1])
        assert np.array_equal(cnt[sl], oc), b
        assert np.array_equal(hsh[sl], set_hash(oc, ol + start[b])), b


def test_batched_passes_match_each_box():
    sts = boxes()
    cat, start = concat(sts)
    ctx = crk.crk_create()
    crk.crk_build_cells_batched(ctx, dev(cat["pos_h"]), start)
    V, N, pairs = crk.crk_volumes(ctx, with_pairs=True)
    vel = dev(cat["vel_u"])
    A, B, gA, gB, gv = crk.crk_corrections(ctx, V, vel)
    acc, dudt, vsig, qmax = crk.crk_forces(ctx, dev(cat["mass"]), vel, V, A, B, gA, gB, gv)
    tot_pairs = 0
    for b, st in enumerate(sts):
        sl = slice(start[b], start[b + 1])
        ev = O.evaluate(st)
        tot_pairs += ev["pairs"]
        e = {k: rel_err(as_np(g)[sl], ev[k]) for k, g in (("V", V), ("A", A), ("gv", gv), ("dudt", dudt),
                                                          ("vsig", vsig))}
        e.update({k: rel_err(as_np(g)[sl], ev[k], floor=ev["s" + k]) for k, g in (("B", B), ("gA", gA),
                                                                                  ("gB", gB))})
        e["acc"] = rel_err(as_np(acc)[sl], ev["acc"], floor=ev["fscale"])
        print("box", b, e)
        assert max(e.values()) < TOL, (b, e)
    assert pairs == tot_pairs


@pytest.mark.parametrize("pair_form", [0, 1])
def test_batched_step_matches_single_box_steps(pair_form):
    """Three KDK steps of all boxes at once against each box stepped alone, in
    either form of P4 and P5 (the pair-once form over boxes: the tile-pair
    lists, and with them the reverse index, stay within each box)."""
    sts = boxes()
    cat, start = concat(sts)
    pos, vel, mass = dev(cat["pos_h"]), dev(cat["vel_u"]), dev(cat["mass"])
    ctx = crk.crk_create(pair_form=pair_form)
    single = []
    for st in sts:
        single.append((dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"]), crk.crk_create(pair_form=pair_form)))
    for step in range(3):
        d = crk.crk_step_batched(ctx, pos, vel, mass, start, diag=True)
        for b, (p, v, m, c) in enumerate(single):
            ds = crk.crk_step(c, p, v, m, 0.0, diag=True)
            assert abs(d[b]["dt"] - ds["dt"]) <= 1e-5 * ds["dt"], (step, b, d[b]["dt"], ds["dt"])
            E, Es = d[b]["E_kin"] + d[b]["E_int"], ds["E_kin"] + ds["E_int"]
            assert abs(E - Es) <= 1e-6 * abs(Es), (step, b)
    gp, gv = pos.cpu().numpy(), vel.cpu().numpy()
    for b, (p, v, m, c) in enumerate(single):
        sl = slice(start[b], start[b + 1])
        sp, sv = p.cpu().numpy(), v.cpu().numpy()
        dx = np.abs(gp[sl, :3] - sp[:, :3])
        dx = np.minimum(dx, 1.0 - dx)
        e = {"x": float(dx.max()), "h": rel_err(gp[sl, 3], sp[:, 3]), "v": rel_err(gv[sl, :3], sv[:, :3]),
             "u": rel_err(gv[sl, 3], sv[:, 3])}
        print("box", b, e)
        assert e["x"] < 1e-6 and max(e["h"], e["v"], e["u"]) < TOL, (b, e)


def test_batched_fixed_steps_and_single_box_table():
    """Per-box fixed dt is honoured; a one-box table is the plain step."""
    sts = boxes()[:2]
    cat, start = concat(sts)
    ctx = crk.crk_create()
    pos, vel, mass = dev(cat["pos_h"]), dev(cat["vel_u"]), dev(cat["mass"])
    d = crk.crk_step_batched(ctx, pos, vel, mass, start, dt=[1e-4, 2e-4], diag=True)
    assert d[0]["dt"] == 1e-4 and d[1]["dt"] == 2e-4
    st = sts[0]
    p1, v1, m1 = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    p2, v2 = p1.clone(), v1.clone()
    c1, c2 = crk.crk_create(), crk.crk_create()
    crk.crk_step_batched(c1, p1, v1, m1, [0, p1.shape[0]])
    crk.crk_step(c2, p2, v2, m1, 0.0)
    assert torch.equal(p1, p2) and torch.equal(v1, v2)


@pytest.mark.parametrize("table", [[0, 100, 50, 4096], [0, 100, 4000], [1, 4096], []])
def test_bad_box_tables_are_rejected(table):
    st = workload("uniform", 16)
    ctx = crk.crk_create()
    with pytest.raises(crk.CrkError) as ei:
        crk.crk_build_cells_batched(ctx, dev(st["pos_h"]), table)
    assert ei.value.code == -1


# ---------------------------------------------------------------- autotuner

def test_autotuned_passes_give_identical_results():
    """Every variant visits each list in the same order: results do not depend
    on which one the tuner keeps (bitwise), and a choice is made per pass.
    P4 and P5 are tuned in their directed form (pair_form 0); the pair-once
    form has one loop form, so a pair-once context tunes P1-P3 only."""
    st = workload("clustered", 3000, 11)
    outs = []
    for tune in (False, True):
        ctx = crk.crk_create(pair_form=0)
        if tune:
            crk.crk_autotune(ctx, True)
        pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
        crk.crk_build_cells(ctx, pos)
        V, N = crk.crk_volumes(ctx)
        A, B, gA, gB, gv = crk.crk_corrections(ctx, V, vel)
        acc, dudt, vsig, qmax = crk.crk_forces(ctx, mass, vel, V, A, B, gA, gB, gv)
        du = crk.crk_compatible(ctx, mass, vel, V, A, B, gA, gB, gv, vel[:, :3].contiguous(),
                                (vel[:, :3] * 1.01).contiguous())
        for _ in range(2):
            crk.crk_step(ctx, pos, vel, mass, 0.0)
        outs.append([V, A, B, gA, gB, gv, acc, dudt, vsig, du, pos, vel])
        if tune:
            t = crk.crk_tuning(ctx)
            print(t)
            assert set(t) >= {"P1 volumes", "P2 corrections", "P3 grad v", "P4 forces", "P5 compatible energy"}
            assert all(0 <= v < crk.CRK_TUNE_NVARIANT and ms > 0 for v, ms in t.values())
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    ctx = crk.crk_create(pair_form=1)
    crk.crk_autotune(ctx, True)
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    for _ in range(2):
        crk.crk_step(ctx, pos, vel, mass, 0.0)
    t = crk.crk_tuning(ctx)
    assert set(t) >= {"P1 volumes", "P2 corrections", "P3 grad v"} and "P4 forces" not in t, t


def test_every_pass_variant_gives_identical_results():
    """Each list-pass variant, pinned with crk_tune_set, reproduces the default
    run bit for bit (same lists walked in the same order), including two KDK
    steps; a variant that a pass lacks is refused with CRK_EINVAL."""
    st = workload("clustered", 3000, 11)
    names = ("P1 volumes", "P2 corrections", "P3 grad v", "P4 forces", "P5 compatible energy")

    def run(v):
        ctx = crk.crk_create(pair_form=0)   # the directed P4 and P5 have the variants
        for name in names:
            crk.crk_tune_set(ctx, name, v)
        ran = set(names)

        def call(fn):
            # a pass pinned to a variant it lacks refuses it (CRK_EINVAL, naming
            # itself): unpin that pass and call again
            for _ in range(len(names) + 1):
                try:
                    return fn()
                except crk.CrkError as e:
                    assert e.code == crk.CRK_EINVAL and "has no variant" in str(e), str(e)
                    name = next(k for k in names if str(e).split(": ", 1)[1].startswith(k))
                    ran.discard(name)
                    crk.crk_tune_set(ctx, name, -1)
            raise AssertionError("variant %d refused repeatedly" % v)

        pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
        crk.crk_build_cells(ctx, pos)
        V, N = call(lambda: crk.crk_volumes(ctx))
        A, B, gA, gB, gv = call(lambda: crk.crk_corrections(ctx, V, vel))
        acc, dudt, vsig, qmax = call(lambda: crk.crk_forces(ctx, mass, vel, V, A, B, gA, gB, gv))
        du = call(lambda: crk.crk_compatible(ctx, mass, vel, V, A, B, gA, gB, gv, vel[:, :3].contiguous(),
                                             (vel[:, :3] * 1.01).contiguous()))
        for _ in range(2):   # every pass lacking v is unpinned by now
            crk.crk_step(ctx, pos, vel, mass, 0.0)
        return [V, N, A, B, gA, gB, gv, acc, dudt, vsig, qmax, du, pos, vel], ran

    ref, _ = run(-1)
    has = {name: set() for name in names}
    for v in range(crk.CRK_TUNE_NVARIANT):
        out, ran = run(v)
        for name in ran:
            has[name].add(v)
        for a, b in zip(ref, out):
            assert torch.equal(a, b), v
    every = set(range(crk.CRK_TUNE_NVARIANT)) - {21}   # 21: records by TMA gathers, P4 only
    assert has["P1 volumes"] == has["P2 corrections"] == has["P3 grad v"] == has["P5 compatible energy"] == every
    assert has["P4 forces"] == {0, 4, 8, 9, 10, 11, 12, 21}


# ---------------------------------------------------------------- CUDA graphs

@pytest.mark.parametrize("pair_form", [0, 1])
@pytest.mark.parametrize("case", ["uniform16", "sedov16"])
def test_graph_steps_equal_eager_steps(case, pair_form):
    """Captured-and-replayed steps are the eager steps, bit for bit (inputs
    whose neighbour counts stay within the list headroom), in either form of
    P4 and P5 (the pair-once arrays follow the tile lists' headroom)."""
    st = {"uniform16": lambda: workload("uniform", 16), "clustered3000": lambda: workload("clustered", 3000, 11),
          "sedov16": lambda: workload("sedov", 16)}[case]()
    res = []
    for mode in ("graph", "eager", "step"):
        ctx = crk.crk_create(pair_form=pair_form)
        pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
        if mode == "step":
            for _ in range(6):
                crk.crk_step(ctx, pos, vel, mass, 0.0)
            d = crk.crk_step(ctx, pos, vel, mass, 0.0, diag=True)
        else:
            crk.crk_steps(ctx, pos, vel, mass, 4, use_graph=(mode == "graph"))
            d = crk.crk_steps(ctx, pos, vel, mass, 3, use_graph=(mode == "graph"), diag=True)
        if mode == "graph":
            caps, reps, recs = crk.crk_graph_stats(ctx)
            print(case, "captures", caps, "replays", reps, "recoveries", recs)
            # replayed steps after the first (one more eager step when the list columns needed headroom)
            assert caps >= 2 and reps >= 5 and recs == 0, (caps, reps, recs)
        res.append((pos, vel, d))
    for p, v, d in res[1:]:
        assert torch.equal(p, res[0][0]) and torch.equal(v, res[0][1])
        assert d["E_kin"] == res[0][2]["E_kin"] and d["dt"] == res[0][2]["dt"]


@pytest.mark.parametrize("case", ["converging16", "clustered3000"])
def test_graph_steps_recover_from_list_overflow(case):
    """Neighbour counts that outgrow even the list headroom (a converging flow;
    clumps whose h grows towards N_res): the replays detect it, and the call
    restores the state its replays started from and redoes their steps
    eagerly, evaluating the rates afresh there.  The reference does the same
    with eager steps and a reset of the rates at that point."""
    if case == "converging16":
        st = dict(workload("uniform", 16))
        v = st["vel_u"].copy()
        v[:, :3] = -3.0 * (st["pos_h"][:, :3].astype(np.float64) - 0.5).astype(np.float32)
        st["vel_u"] = v
        dt = 0.04
    else:
        st = workload("clustered", 3000, 11)
        dt = 0.0
    ctx = crk.crk_create()
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    crk.crk_steps(ctx, pos, vel, mass, 6, dt=dt, use_graph=True)
    caps, reps, recs = crk.crk_graph_stats(ctx)
    print(case, "captures", caps, "replays", reps, "recoveries", recs)
    assert torch.isfinite(pos).all() and torch.isfinite(vel).all()
    ref = crk.crk_create()
    rp, rv = dev(st["pos_h"]), dev(st["vel_u"])
    if recs == 0:
        crk.crk_steps(ref, rp, rv, mass, 6, dt=dt, use_graph=False)
    else:
        # eager steps before the replays (the first, plus one if the columns were widened), then a reset
        eager = 6 - reps
        crk.crk_steps(ref, rp, rv, mass, eager, dt=dt, use_graph=False)
        crk.crk_reset_rates(ref)
        crk.crk_steps(ref, rp, rv, mass, 6 - eager, dt=dt, use_graph=False)
    assert torch.equal(pos, rp) and torch.equal(vel, rv)


def test_batched_graph_steps_equal_eager_steps():
    sts = [workload("uniform", 16), workload("sedov", 14), workload("sedov", 16)]
    cat, start = concat(sts)
    res = []
    for use_graph in (True, False):
        ctx = crk.crk_create()
        pos, vel, mass = dev(cat["pos_h"]), dev(cat["vel_u"]), dev(cat["mass"])
        crk.crk_steps_batched(ctx, pos, vel, mass, start, 5, use_graph=use_graph)
        if use_graph:
            caps, reps, recs = crk.crk_graph_stats(ctx)
            print("batched captures", caps, "replays", reps, "recoveries", recs)
            assert caps >= 2 and recs == 0
        res.append((pos, vel))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
