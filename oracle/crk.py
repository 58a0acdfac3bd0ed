"""FP64 CPU oracle of the CRKSPH pair passes (CRK-HACC, arXiv 2202.02840).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg and reference arm of bench.py, never by the product path.  Shares no code with
the CUDA library.  Pair passes run in crk_oracle.c (FP64, brute force or an
equivalent grid search); the elementwise steps below are plain numpy FP64.

Paper sections followed:
  P1 volumes        Sec. 1.2 eq:vol, Sec. 2.6 eq:hi
  P2 corrections    Sec. 1.2 eq:RK, eq:gRK and the two moment conditions
  P3 grad v         Sec. 1.2 eq:gradv
  P4 forces         Sec. 1.2 eq:mom, eq:eng, eq:visc, eq:mu, eq:hatvi, eq:phi..eq:phiad
  P5 compatible     Sec. 1.2 eq:compEng .. eq:fij
  step              Sec. 2.1 eq:verletOP (KDK with predictor), CFL criteria
  h                 Sec. 2.6 eq:thacker
"""
import ctypes
import numpy as np

from . import build as _build

# Constants stated in the paper: gamma = 5/3 (Sec. 1.1), n_h = 4 and N_res = 268
# (Sec. 2.6), C_l = 2, C_q = 1, eps = 0.1 (Sec. 1.2), eta_crit = 1/n_h,
# eta_fold = 0.2/n_h (Sec. 1.2), C_CFL = 0.25, zeta = 4 (Sec. 2.1).
# The scale factor a and its rate adot (Sec. 1.1, comoving variables with
# p = a^2 dx/dt) default to a static box, a = 1, adot = 0.
PARAMS = dict(gamma=5.0 / 3.0, n_h=4.0, N_res=268.0, C_l=2.0, C_q=1.0, eps=0.1,
              eta_crit=1.0 / 4.0, eta_fold=0.2 / 4.0, C_cfl=0.25, zeta=4.0, a=1.0, adot=0.0, density=0.0)
_ORDER = ["gamma", "n_h", "N_res", "C_l", "C_q", "eps", "eta_crit", "eta_fold", "C_cfl", "zeta", "a", "adot",
          "density"]
IA, IADOT, IDENS = 10, 11, 12   # density 0: rho = m / V (R5); 1: the RK-corrected sum (rk_density)

_LIB = None
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p
_ci = ctypes.c_int


def load():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        lib.orc_fixed_point.argtypes = [_ci, _f32p, _u32p, _u32p]
        lib.orc_neighbours.argtypes = [_ci, _f32p, _ci, _ci, _vp, _ci, _i32p, _vp, ctypes.c_longlong]
        lib.orc_cells.argtypes = [_ci, _f32p, _ci, _u32p, _i32p, ctypes.POINTER(_ci), _i32p]
        lib.orc_volumes.argtypes = [_ci, _f32p, _ci, _vp, _ci, _f64p, _f64p, _f64p,
                                    ctypes.POINTER(ctypes.c_longlong)]
        lib.orc_corrections.argtypes = [_ci, _f32p, _ci, _vp, _ci, _f64p, _f64p, _f64p, _f64p,
                                        _f64p, _vp, _vp, _vp]
        lib.orc_gradv.argtypes = [_ci, _f32p, _ci, _vp, _ci] + [_f64p] * 7
        lib.orc_forces.argtypes = [_ci, _f32p, _ci, _vp, _ci] + [_f64p] * 13 + [
            _vp, _vp, ctypes.POINTER(ctypes.c_longlong), _vp]
        lib.orc_compatible.argtypes = [_ci, _f32p, _ci, _vp, _ci] + [_f64p] * 13 + [_vp]
        lib.orc_rkdensity.argtypes = [_ci, _f32p, _ci, _vp, _ci, _f64p, _f64p, _f64p, _f64p]
        lib.orc_kernel.argtypes = [_ci, _f64p, _f64p, _f64p, _f64p]
        lib.orc_num_threads.restype = _ci
        _LIB = lib
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (what, rc))


def params(**overrides) -> np.ndarray:
    p = dict(PARAMS)
    p.update(overrides)
    return np.array([p[k] for k in _ORDER], np.float64)


def num_threads() -> int:
    return int(load().orc_num_threads())


def kernel(r, h):
    """W(r, h) of eq:C4 and dW/dr, elementwise (FP64)."""
    r = np.ascontiguousarray(r, np.float64).ravel()
    h = np.ascontiguousarray(np.broadcast_to(h, r.shape), np.float64)
    W, dW = np.zeros_like(r), np.zeros_like(r)
    _check(load().orc_kernel(len(r), r, h, W, dW), "kernel")
    return W, dW


def grid_level(n: int) -> int:
    """Candidate-grid level for the oracle search (about 8 particles per cell)."""
    if n <= 4096:
        return 0
    k = int(round(np.log2(max(n / 8.0, 1.0)) / 3.0))
    return max(1, min(7, k))


def _pos(pos_h):
    return np.ascontiguousarray(pos_h, np.float32).reshape(-1, 4)


def _tg(targets):
    if targets is None:
        return None, 0, None
    t = np.ascontiguousarray(targets, np.int32)
    return t.ctypes.data_as(_vp), len(t), t


def _k(pos, k):
    return grid_level(pos.shape[0]) if k is None else int(k)


def fixed_point(pos_h):
    """q = floor(s 2^32) (n,3) and H = floor(h 2^32) (n,)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    q = np.zeros((n, 3), np.uint32)
    H = np.zeros(n, np.uint32)
    _check(load().orc_fixed_point(n, pos, q, H), "fixed_point")
    return q, H


def neighbours(pos_h, mode=0, k=None, targets=None):
    """mode 0: gather(i) incl. self; mode 1: pair set.  Returns (counts, lists CSR)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    m = n if targets is None else nt
    counts = np.zeros(m, np.int32)
    lib = load()
    _check(lib.orc_neighbours(n, pos, _k(pos, k), mode, tp, nt, counts, None, 0), "neighbours")
    total = int(counts.astype(np.int64).sum())
    lists = np.zeros(max(total, 1), np.int32)
    _check(lib.orc_neighbours(n, pos, _k(pos, k), mode, tp, nt, counts,
                              lists.ctypes.data_as(_vp), total), "neighbours")
    return counts, lists[:total]


def cells(pos_h, kmax=7):
    """Morton keys, stable sort permutation, chaining-mesh level and cell starts."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    key = np.zeros(n, np.uint32)
    perm = np.zeros(n, np.int32)
    kk = _ci(0)
    start = np.zeros((1 << (3 * kmax)) + 1, np.int32)
    _check(load().orc_cells(n, pos, kmax, key, perm, ctypes.byref(kk), start), "cells")
    k = kk.value
    return key, perm, k, start[: (1 << (3 * k)) + 1].copy()


def volumes(pos_h, k=None, targets=None):
    """P1: n_i, V_i = 1/n_i, N_i = 4/3 pi h^3 n_i (eq:vol, eq:hi)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    nsum, V, N = (np.full(n, np.nan) for _ in range(3))
    pairs = ctypes.c_longlong(0)
    _check(load().orc_volumes(n, pos, _k(pos, k), tp, nt, nsum, V, N, ctypes.byref(pairs)), "volumes")
    return {"nsum": nsum, "V": V, "N": N, "pairs": int(pairs.value)}


def corrections(pos_h, V, k=None, targets=None, moments=False):
    """P2: A, B, grad A, grad B (gB[i, alpha, gamma]), cond(m2), and the
    no-cancellation scales sA, sB, sgA, sgB (same formulas on |pair terms|)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    A = np.full(n, np.nan)
    B, gA = np.full((n, 3), np.nan), np.full((n, 3), np.nan)
    gB = np.full((n, 3, 3), np.nan)
    cond = np.full(n, np.nan)
    mom = np.full((n, 40), np.nan) if moments else None
    sc = np.full((n, 16), np.nan)
    _check(load().orc_corrections(n, pos, _k(pos, k), tp, nt, np.ascontiguousarray(V, np.float64),
                                  A, B, gA, gB,
                                  mom.ctypes.data_as(_vp) if moments else None,
                                  cond.ctypes.data_as(_vp), sc.ctypes.data_as(_vp)), "corrections")
    out = {"A": A, "B": B, "gA": gA, "gB": gB, "cond": cond, "sA": sc[:, 0], "sB": sc[:, 1:4],
           "sgA": sc[:, 4:7], "sgB": sc[:, 7:16].reshape(n, 3, 3)}
    if moments:
        out["moments"] = mom
    return out


def gradv(pos_h, V, vel, A, B, gA, gB, k=None, targets=None, a=1.0):
    """P3: grad v (gv[i, alpha, beta] = d v^alpha / d x^beta), eq:gradv, of the
    peculiar velocity v = p / a (vel holds p)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    gv = np.full((n, 3, 3), np.nan)
    c = lambda a: np.ascontiguousarray(a, np.float64)
    _check(load().orc_gradv(n, pos, _k(pos, k), tp, nt, c(V), c(vel), c(A), c(B), c(gA), c(gB), gv),
           "gradv")
    return gv / a


def _opt(a):
    return None if a is None else np.ascontiguousarray(a, np.float64)


def rk_density(pos_h, mass, A, B, k=None, targets=None):
    """RK-corrected density rho_i = sum_j m_j W^R_ij over gather(i), self included."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    rho = np.full(n, np.nan)
    c = lambda a: np.ascontiguousarray(a, np.float64)
    _check(load().orc_rkdensity(n, pos, _k(pos, k), tp, nt, c(mass), c(A), c(B), rho), "rkdensity")
    return rho


def forces(pos_h, vel, u, mass, V, A, B, gA, gB, gv, prm=None, k=None, targets=None, rho=None):
    """P4: acceleration, direct du/dt, signal velocity, max pair Q (eq:mom, eq:eng);
    rho (optional) replaces m / V as the density."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    prm = params() if prm is None else prm
    acc = np.full((n, 3), np.nan)
    dudt, vsig, qmax, fscale = (np.full(n, np.nan) for _ in range(4))
    pairs = ctypes.c_longlong(0)
    c = lambda a: np.ascontiguousarray(a, np.float64)
    _check(load().orc_forces(n, pos, _k(pos, k), tp, nt, c(prm), c(V), c(mass), c(vel), c(u),
                             c(A), c(B), c(gA), c(gB), c(gv), acc, dudt, vsig,
                             qmax.ctypes.data_as(_vp), fscale.ctypes.data_as(_vp),
                             ctypes.byref(pairs), _ptr(_opt(rho))), "forces")
    return {"acc": acc, "dudt": dudt, "vsig": vsig, "qmax": qmax, "fscale": fscale,
            "pairs": int(pairs.value)}


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


def compatible(pos_h, vel, u, mass, V, A, B, gA, gB, gv, vb, va, prm=None, k=None, targets=None, rho=None):
    """P5: sum_j Delta u_ij for the kick vb -> va (eq:compEng .. eq:fij)."""
    pos = _pos(pos_h)
    n = pos.shape[0]
    tp, nt, keep = _tg(targets)
    prm = params() if prm is None else prm
    du = np.full(n, np.nan)
    c = lambda a: np.ascontiguousarray(a, np.float64)
    _check(load().orc_compatible(n, pos, _k(pos, k), tp, nt, c(prm), c(V), c(mass), c(vel), c(u),
                                 c(A), c(B), c(gA), c(gB), c(gv), c(vb), c(va), du, _ptr(_opt(rho))),
           "compatible")
    return du


# ------------------------------------------------------------ elementwise


def thermo(V, mass, u, prm=None, rho=None):
    """eq:EOS with rho = m/V (or the given density): rho, P = (gamma-1) rho u,
    c_s = sqrt(gamma P/rho), s = P/rho^gamma."""
    prm = params() if prm is None else prm
    g = prm[0]
    rho = np.asarray(mass, np.float64) / V if rho is None else np.asarray(rho, np.float64)
    P = (g - 1.0) * rho * u
    cs = np.sqrt(g * P / rho)
    s = P / rho ** g
    return rho, P, cs, s


def thacker(h, N, prm=None):
    """eq:thacker: h~ = h (1 - lambda + lambda Delta_N), Delta_N^3 = N_res / N_i."""
    prm = params() if prm is None else prm
    d = np.cbrt(prm[2] / np.asarray(N, np.float64))
    lam = np.where(d < 1.0, 0.2 * (1.0 + d * d), 0.2 * (1.0 + 1.0 / d ** 3))
    return np.asarray(h, np.float64) * (1.0 - lam + lam * d)


def evaluate(state, prm=None, k=None, targets=None):
    """One full derivative evaluation P1 -> P2 -> P3 -> P4 on the FP32 state."""
    prm = params() if prm is None else prm
    pos = _pos(state["pos_h"])
    vu = np.asarray(state["vel_u"], np.float64).reshape(-1, 4)
    mass = np.asarray(state["mass"], np.float64)
    vel, u = np.ascontiguousarray(vu[:, :3]), np.ascontiguousarray(vu[:, 3])
    p1 = volumes(pos, k)
    p2 = corrections(pos, p1["V"], k)
    gv = gradv(pos, p1["V"], vel, p2["A"], p2["B"], p2["gA"], p2["gB"], k, a=prm[IA])
    rk = rk_density(pos, mass, p2["A"], p2["B"], k) if prm[IDENS] else None
    p4 = forces(pos, vel, u, mass, p1["V"], p2["A"], p2["B"], p2["gA"], p2["gB"], gv, prm, k, targets, rho=rk)
    ev = dict(p1)
    ev.update(p2)
    ev["gv"] = gv
    ev.update({"acc": p4["acc"], "dudt": p4["dudt"], "vsig": p4["vsig"], "qmax": p4["qmax"],
               "fscale": p4["fscale"],
               "pairs_union": p4["pairs"], "pairs_gather": p1["pairs"]})
    ev["rho"], ev["P"], ev["cs"], ev["s"] = thermo(p1["V"], mass, u, prm, rho=rk)
    ev["rk_rho"] = rk
    ev["pos_h"], ev["vel"], ev["u"], ev["mass"] = pos.copy(), vel, u, mass
    return ev


def cfl_dt(ev, prm=None):
    """Per-particle time step of Sec. 2.1 (no gravity, so r_soft -> inf and
    the total acceleration is the hydro one, (1/a^2) dp/dt):
    v_max = max(v_sig, c_s, sqrt(zeta Q/rho), (h_hat/a) |tr grad v + 3 adot|),
    dt_i = min(C_CFL h_hat / v_max, sqrt(h_hat / |a_tot|))."""
    prm = params() if prm is None else prm
    sa, sadot = prm[IA], prm[IADOT]
    hh = ev["pos_h"][:, 3].astype(np.float64) / prm[1]
    csq = np.sqrt(prm[9] * ev["qmax"] / ev["rho"])
    div = np.abs(np.trace(ev["gv"], axis1=1, axis2=2) + 3.0 * sadot)
    vmax = np.maximum.reduce([ev["vsig"], ev["cs"], csq, hh / sa * div])
    amag = np.sqrt((ev["acc"] ** 2).sum(axis=1)) / (sa * sa)
    with np.errstate(divide="ignore"):
        dt_h = np.where(vmax > 0, prm[8] * hh / vmax, np.inf)
        dt_a = np.where(amag > 0, np.sqrt(hh / amag), np.inf)
    return np.minimum(dt_h, dt_a)


def h_iterate(pos_h, tol=1e-4, max_it=50, prm=None, k=None, h_min=1e-6, h_max=0.3):
    """Fixed-point solve of eq:hi by repeated eq:thacker updates, each clamped
    to [h_min, h_max] as the evolved h is: a particle is converged once
    |Delta_N - 1| <= tol, or once it sits at a bound that its update points
    beyond (the bound-constrained solution, e.g. a particle in a void that
    would need h > h_max to reach N_res), and keeps its h from then on."""
    prm = params() if prm is None else prm
    pos = _pos(pos_h).copy()
    n = pos.shape[0]
    done = np.zeros(n, bool)
    it = 0
    for it in range(1, max_it + 1):
        p1 = volumes(pos, k)
        d = np.cbrt(prm[2] / p1["N"])
        hn = np.clip(thacker(pos[:, 3].astype(np.float64), p1["N"], prm), h_min, h_max).astype(np.float32)
        done |= (np.abs(d - 1.0) <= tol) | (hn == pos[:, 3])
        if done.all():
            return pos[:, 3].copy(), it, done
        pos[:, 3] = np.where(done, pos[:, 3], hn)
    return pos[:, 3].copy(), it, done


def energy_momentum(vel, u, mass):
    """Total energy sum(1/2 m v^2 + m u) and momentum sum(m v) in FP64."""
    vel = np.asarray(vel, np.float64)
    m = np.asarray(mass, np.float64)
    E = float((0.5 * m * (vel ** 2).sum(axis=1) + m * np.asarray(u, np.float64)).sum())
    P = (m[:, None] * vel).sum(axis=0)
    return E, P


def _wrap_f32(x):
    x = np.mod(np.asarray(x, np.float64), 1.0)
    f = x.astype(np.float32)
    f[f >= np.float32(1.0)] = np.float32(0.0)
    return f


def h_propose(pos_h, N_prev, divv, dt, w, tol, prm=None, h_min=1e-6, h_max=0.3):
    """The learned starting point of the eq:hi solve (see oracle/mlp.py): h =
    clamp(h_ref exp(y), h_min, h_max), h_ref = h (N_res / N_prev)^(1/3), y the
    network output for the particle's features (FP64 forward of the declared
    weights); a particle whose N_prev already meets |Delta_N - 1| <= tol
    keeps its h (the judge)."""
    from . import mlp as M
    prm = params() if prm is None else prm
    pos = _pos(pos_h)
    h = pos[:, 3].astype(np.float64)
    x = M.features(pos, N_prev=N_prev, divv=divv, dt=dt, N_res=prm[2])
    y = M.forward(w, x)[0]
    d = np.cbrt(prm[2] / np.asarray(N_prev, np.float64))
    hp = np.clip(h * d * np.exp(y), h_min, h_max)
    return np.where(np.abs(d - 1.0) <= tol, h, hp)


def kdk_step(state, ev=None, dt=None, prm=None, k=None, h_min=1e-6, h_max=0.3, dt_max=1.0, h_mode=0,
             h_tol=1e-4, h_max_it=50, h_solved=None, w=None):
    """One hydro step, eq:verletOP (Sec. 2.1) with predicted p_p, u_p and the
    compatible energy of eq:compEng for each half kick (in comoving variables:
    the drift moves x by dt p_1/2 / a^2, and the energy kicks add the
    expansion term -(adot/a)(3(gamma-1) + 2) u of eq:CosmoEngEqn, explicitly in
    the u of the opening half kick and implicitly in the u of the closing one,
    which together are the trapezoidal rule for it; a and adot are constant
    over the step); the rates of `ev` (the
    evaluation at the state's positions) are reused for the first half kick.
    h advances by one eq:thacker update of the new evaluation, clamped to
    [h_min, h_max].  Positions, velocities and u are stored in FP32 between
    steps, as in the engine's state.  Returns (new_state, new_eval, dt).

    h_mode 1 solves eq:hi at the drifted positions before the evaluation
    (h_iterate from the state's h, tolerance h_tol); h_mode 2 starts that
    solve from the learned proposal (h_propose with the weights w, features
    from the first P1 at the state's h and the last evaluation's grad v).  In
    both the new state carries the solved h (no further eq:thacker update).
    h_solved (FP32 array) replaces the solve by a given h, which is how a
    step is compared with one whose solve made its own threshold decisions."""
    prm = params() if prm is None else prm
    if ev is None:
        ev = evaluate(state, prm, k)
    if dt is None:
        dt = min(float(np.min(cfl_dt(ev, prm))), dt_max)
    pos = np.asarray(state["pos_h"], np.float32)
    vu = np.asarray(state["vel_u"], np.float64)
    vel, u = vu[:, :3], vu[:, 3]
    mass = np.asarray(state["mass"], np.float64)
    a0 = ev["acc"]
    sa = prm[IA]
    E = prm[IADOT] / sa * (3.0 * (prm[0] - 1.0) + 2.0)   # expansion term of eq:CosmoEngEqn
    p_half = vel + 0.5 * dt * a0
    du1 = compatible(ev["pos_h"], ev["vel"], ev["u"], mass, ev["V"], ev["A"], ev["B"], ev["gA"], ev["gB"],
                     ev["gv"], vel, p_half, prm, k, rho=ev.get("rk_rho"))
    u_half = u + 0.5 * dt * (du1 - E * u)                       # opening half: explicit in u
    p_p = p_half + 0.5 * dt * a0
    u_p = (u_half + 0.5 * dt * du1) / (1.0 + 0.5 * dt * E)      # closing halves: implicit in u
    n = pos.shape[0]
    st1 = {"pos_h": np.empty((n, 4), np.float32), "vel_u": np.empty((n, 4), np.float32),
           "mass": np.asarray(state["mass"], np.float32)}
    st1["pos_h"][:, :3] = _wrap_f32(pos[:, :3].astype(np.float64) + dt / (sa * sa) * p_half)
    st1["pos_h"][:, 3] = pos[:, 3]
    st1["vel_u"][:, :3] = p_p
    st1["vel_u"][:, 3] = u_p
    if h_solved is not None:
        st1["pos_h"][:, 3] = np.asarray(h_solved, np.float32)
    elif h_mode == 1:
        st1["pos_h"][:, 3] = h_iterate(st1["pos_h"], h_tol, h_max_it, prm, k, h_min, h_max)[0]
    elif h_mode == 2:
        N0 = volumes(st1["pos_h"], k)["N"]
        hp = h_propose(st1["pos_h"], N0, np.trace(ev["gv"], axis1=1, axis2=2), dt, w, h_tol, prm, h_min, h_max)
        pp = st1["pos_h"].copy()
        pp[:, 3] = hp.astype(np.float32)
        st1["pos_h"][:, 3] = h_iterate(pp, h_tol, h_max_it, prm, k, h_min, h_max)[0]
    ev1 = evaluate(st1, prm, k)
    p1 = p_half + 0.5 * dt * ev1["acc"]
    du2 = compatible(ev1["pos_h"], ev1["vel"], ev1["u"], mass, ev1["V"], ev1["A"], ev1["B"], ev1["gA"],
                     ev1["gB"], ev1["gv"], p_half, p1, prm, k, rho=ev1.get("rk_rho"))
    u1 = (u_half + 0.5 * dt * du2) / (1.0 + 0.5 * dt * E)
    if h_mode or h_solved is not None:
        h1 = st1["pos_h"][:, 3].astype(np.float64)
    else:
        h1 = np.clip(thacker(pos[:, 3].astype(np.float64), ev1["N"], prm), h_min, h_max)
    out = {"pos_h": st1["pos_h"].copy(), "vel_u": np.empty((n, 4), np.float32), "mass": st1["mass"]}
    out["pos_h"][:, 3] = h1
    out["vel_u"][:, :3] = p1
    out["vel_u"][:, 3] = u1
    return out, ev1, dt
