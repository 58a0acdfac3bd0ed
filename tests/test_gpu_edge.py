"""GPU parity on the degenerate neighbourhoods of the method.

Ill-conditioned moment matrices: particles on a thin sheet or a closed filament
(thickness 2e-5 of the box against h = 0.05-0.08), tilted against the axes,
make m2 = sum V x x W (Sec. 1.2 moment conditions) nearly singular along a
direction no axis shares, cond(m2) ~ 1e6-1e8; this is why the 3x3 systems of
eq:RK / eq:gRK are solved in FP64.  Coincident distinct
particles (r_ij = 0, i != j) exercise eq:gRK at x = 0 (where the corrected
gradient is (grad A + A B) W(0), not zero), eq:mu and eq:phiad at r = 0 and
the signal velocity's zero-separation case.  Each pass is checked in
isolation against the FP64 oracle at TOL (1e-5 of the field's RMS, or of the
per-particle force scale sum_j |F_ij| / m_i for the accelerations).
"""
import numpy as np
import pytest
import torch

from oracle import crk as O
from paper_2202_02840_gb300 import crk, inputs
from parity import TOL, rel_err, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))


def _frame(direction):
    """A unit vector along `direction` and two unit vectors normal to it."""
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    a = np.cross(d, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    return d, a, np.cross(d, a)


def sheet(side=24, spacing=1 / 48, delta=2e-5, seed=31):
    """A jittered square patch of particles in the plane through the box centre
    with normal (1, 2, 3), thickness delta: m2 is nearly singular along a
    direction no axis shares (axis-aligned ill-conditioning the adjugate
    inverse handles exactly; this kind it does not)."""
    r = inputs.rng(seed)
    nrm, a, b = _frame((1.0, 2.0, 3.0))
    g = (np.arange(side) - (side - 1) / 2) * spacing
    U, W = np.meshgrid(g, g, indexing="ij")
    n = side * side
    u = U.ravel() + r.uniform(-0.1, 0.1, n) * spacing
    w = W.ravel() + r.uniform(-0.1, 0.1, n) * spacing
    pos = 0.5 + u[:, None] * a + w[:, None] * b + (delta * r.normal(0, 1, n))[:, None] * nrm
    return inputs.pack(pos, 4 * spacing, r.normal(0, 0.05, (n, 3)), 1.0 + 0.2 * r.uniform(0, 1, n), 1.0 / n)


def filament(n=141, delta=2e-5, seed=32):
    """A closed row of particles along (1, 1, 0), which winds once round the
    periodic box (length sqrt 2, spacing ~0.01: no ends, whose one-sided
    neighbourhoods would reach cond ~1e8), thickness delta across it."""
    r = inputs.rng(seed)
    d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    a = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    b = np.array([0.0, 0.0, 1.0])
    t = (np.arange(n) + r.uniform(-0.1, 0.1, n)) / n          # fraction of the loop
    spacing = np.sqrt(2.0) / n
    pos = (np.array([0.2, 0.3, 0.5]) + t[:, None] * np.sqrt(2.0) * d + (delta * r.normal(0, 1, n))[:, None] * a
           + (delta * r.normal(0, 1, n))[:, None] * b)
    return inputs.pack(np.mod(pos, 1.0), 5 * spacing, r.normal(0, 0.05, (n, 3)), 1.0 + 0.2 * r.uniform(0, 1, n),
                       1.0 / n)


def coincident(copies=(5, 100, 2000, 4095), seed=33):
    """The 16^3 jittered lattice plus exact copies of a few particles (same
    position and h, their own velocity and u): n = 4100, a ragged last tile."""
    st = workload("uniform", 16)
    r = inputs.rng(seed)
    c = np.asarray(copies)
    pos = np.concatenate([st["pos_h"], st["pos_h"][c]], 0)
    vel = np.concatenate([st["vel_u"], st["vel_u"][c]], 0)
    vel[-len(c):, :3] += r.normal(0, 0.05, (len(c), 3)).astype(np.float32)
    vel[-len(c):, 3] *= np.float32(1.5)
    mass = np.concatenate([st["mass"], st["mass"][c]], 0)
    return {"pos_h": np.ascontiguousarray(pos), "vel_u": np.ascontiguousarray(vel), "mass": mass}


CASES = {"sheet": sheet, "filament": filament, "coincident": coincident}


def oracle_chain(st):
    pos = st["pos_h"]
    vel = st["vel_u"][:, :3].astype(np.float64)
    u = st["vel_u"][:, 3].astype(np.float64)
    m = st["mass"].astype(np.float64)
    p1 = O.volumes(pos)
    V = f32(p1["V"]).astype(np.float64)
    p2 = O.corrections(pos, V)
    r = {k: f32(p2[k]).astype(np.float64) for k in ("A", "B", "gA", "gB")}
    gv_o = O.gradv(pos, V, vel, r["A"], r["B"], r["gA"], r["gB"])
    gv = f32(gv_o).astype(np.float64)
    p4 = O.forces(pos, vel, u, m, V, r["A"], r["B"], r["gA"], r["gB"], gv)
    return dict(p1=p1, V=V, p2=p2, r=r, gv=gv, p4=p4, vel=vel, u=u, m=m)


def test_degenerate_inputs_are_what_they_claim():
    for name in ("sheet", "filament"):
        st = CASES[name]()
        V = f32(O.volumes(st["pos_h"])["V"]).astype(np.float64)
        cond = O.corrections(st["pos_h"], V)["cond"]
        assert np.median(cond) > 1e6, (name, np.median(cond))
    st = coincident()
    q, _ = O.fixed_point(st["pos_h"])
    assert len(np.unique(q, axis=0)) == len(q) - 4   # four exact pairs at r = 0


# P3 and P4 evaluate each pair in FP32.  On the sheet and the filament the RK
# coefficients are huge (|B| ~ 1e4, grad B larger still), so the corrected
# kernel gradient of a single pair, dA (1 + B.x) W + A (dB.x + B) W +
# A (1 + B.x) dW, is a sum of terms that cancel to ~1e-3 of themselves: its
# FP32 rounding leaves up to ~1e-4 of the fields (measured); held to this
# stated bar there, to TOL everywhere else.
DEGENERATE_PAIR_TOL = 1e-3


@pytest.mark.parametrize("precision", [1, 3])
@pytest.mark.parametrize("case", list(CASES))
def test_degenerate_passes(case, precision):
    st = CASES[case]()
    oc = oracle_chain(st)
    ctx = crk.crk_create(precision=precision)
    crk.crk_build_cells(ctx, dev(st["pos_h"]))
    V, N = crk.crk_volumes(ctx)
    e1 = {"V": rel_err(V, oc["p1"]["V"]), "N": rel_err(N, oc["p1"]["N"])}
    A, B, gA, gB, gv = crk.crk_corrections(ctx, dev(f32(oc["V"])), dev(st["vel_u"]))
    p2 = oc["p2"]
    # the coincident set is a jittered lattice, whose moment sums cancel: there
    # precision 1 is held to the no-cancellation scales (its RMS-relative
    # error is the stated one of the lattice cases), precision 3 to the RMS
    lattice = case == "coincident" and precision < 3
    fl = {k: (p2["s" + k] if lattice else None) for k in ("B", "gA", "gB")}
    e2 = {"A": rel_err(A, p2["A"]), "B": rel_err(B, p2["B"], floor=fl["B"]),
          "gA": rel_err(gA, p2["gA"], floor=fl["gA"]), "gB": rel_err(gB, p2["gB"], floor=fl["gB"])}
    ogv = O.gradv(st["pos_h"], oc["V"], oc["vel"], p2["A"], p2["B"], p2["gA"], p2["gB"])
    e3 = {"gv": rel_err(gv, ogv)}
    r = oc["r"]
    acc, dudt, vsig, qmax = crk.crk_forces(
        ctx, dev(st["mass"]), dev(st["vel_u"]), dev(f32(oc["V"])), dev(f32(r["A"])), dev(f32(r["B"])),
        dev(f32(r["gA"])), dev(f32(r["gB"])), dev(f32(oc["gv"])))
    p4 = oc["p4"]
    e4 = {"acc": rel_err(acc, p4["acc"], floor=p4["fscale"]), "dudt": rel_err(dudt, p4["dudt"]),
          "vsig": rel_err(vsig, p4["vsig"]), "qmax": rel_err(qmax, p4["qmax"])}
    print(case, precision, e1, e2, e3, e4)
    assert max(e1.values()) < TOL, e1
    degenerate = case != "coincident"
    if precision == 3:
        # float-float moments reach the oracle however ill-conditioned m2 is;
        # with FP32 moments (precision 1) a tilted sheet's B is off by
        # cond(m2) x 1e-7 ~ 0.1 (the test below), and on the lattice of the
        # coincident set P2 and P3 carry precision 1's stated lattice error
        # (test_gpu_parity.test_corrections): neither is held here
        assert max(e2.values()) < TOL, e2
        assert e3["gv"] < (DEGENERATE_PAIR_TOL if degenerate else TOL), e3
    assert max(e4.values()) < (DEGENERATE_PAIR_TOL if degenerate else TOL), e4
    F = acc.cpu().double().numpy() * oc["m"][:, None]
    assert np.max(np.abs(F.sum(axis=0))) < 1e-6 * np.abs(F).sum()


def test_ill_conditioned_moments_need_float_float():
    """Why precision 3 exists, shown on the tilted sheet (cond(m2) ~ 1e6): FP32
    moment sums miss the oracle's B by ~cond x 1e-7 whether the 3x3 system is
    then solved in FP32 (precision 0) or FP64 (precision 1); only moments
    carried in float-float and solved in FP64 reach it."""
    st = sheet()
    oc = oracle_chain(st)
    errs = {}
    for precision in (0, 1, 3):
        ctx = crk.crk_create(precision=precision)
        crk.crk_build_cells(ctx, dev(st["pos_h"]))
        A, B, gA, gB, _ = crk.crk_corrections(ctx, dev(f32(oc["V"])), dev(st["vel_u"]))
        errs[precision] = rel_err(B, oc["p2"]["B"])
    print("B error on the tilted sheet by precision mode:", errs)
    assert errs[3] < TOL and min(errs[0], errs[1]) > 100 * errs[3]
