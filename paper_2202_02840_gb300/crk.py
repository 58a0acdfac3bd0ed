"""Python binding of the C ABI declared in include/crk.h.

Argument marshalling only: every function checks its torch tensors (CUDA,
float32, contiguous, shape), passes raw device pointers and the current CUDA
stream to libcrk.so and turns a non-zero status into CrkError.  Every step of
the computation runs in the library's kernels.  The library must have been
built (build.build()); there is no fallback.
"""
import ctypes
import os

import torch

from . import build as _build

CRK_OK = 0
CRK_ENONCONV = -5
CRK_EINVAL = -1
_CODES = {-1: "CRK_EINVAL", -2: "CRK_ENOMEM", -3: "CRK_ECUDA", -4: "CRK_ETIMEOUT",
          -5: "CRK_ENONCONV", -6: "CRK_ECAPACITY", -7: "CRK_ESTATE"}


class CrkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_CODES.get(code, "?"), code, msg))
        self.code = code


class crk_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("gamma", "n_h", "N_res", "C_l", "C_q", "eps", "eta_crit", "eta_fold", "C_cfl", "zeta",
                 "h_min", "h_max", "dt_max", "a", "adot")] + [
        ("precision", ctypes.c_int), ("kmax", ctypes.c_int), ("tile_order", ctypes.c_int),
        ("density", ctypes.c_int), ("h_mode", ctypes.c_int), ("h_max_it", ctypes.c_int),
        ("h_tol", ctypes.c_float), ("rcb_leaf", ctypes.c_int), ("pair_form", ctypes.c_int)]


class crk_diag(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dt_next", ctypes.c_double), ("E_kin", ctypes.c_double),
                ("E_int", ctypes.c_double), ("P", ctypes.c_double * 3),
                ("pairs_gather", ctypes.c_longlong), ("pairs_union", ctypes.c_longlong),
                ("h_iterations", ctypes.c_longlong), ("h_unconverged", ctypes.c_longlong)]


class crk_htb_stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int), ("evaluations", ctypes.c_longlong), ("wakeups", ctypes.c_longlong),
                ("unresolved", ctypes.c_longlong), ("leaves", ctypes.c_int), ("level_count", ctypes.c_int * 32)]


_LIB = None
_vp = ctypes.c_void_p
_ci = ctypes.c_int


def lib():
    """Load libcrk.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libcrk.so is not built (%s); run paper_2202_02840_gb300.build.build()"
                               % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        L.crk_default_params.argtypes = [ctypes.POINTER(crk_params)]
        L.crk_create.argtypes = [ctypes.POINTER(crk_params), ctypes.POINTER(_vp)]
        L.crk_destroy.argtypes = [_vp]
        L.crk_last_error.argtypes = [_vp]
        L.crk_last_error.restype = ctypes.c_char_p
        L.crk_sync.argtypes = [_vp, _vp]
        L.crk_build_cells.argtypes = [_vp, _ci, _vp, _vp]
        L.crk_cells.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(_ci), _vp]
        L.crk_build_stats.argtypes = [_vp, ctypes.POINTER(_ci), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong), _vp]
        L.crk_walk_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong), _vp]
        L.crk_neighbours.argtypes = [_vp, _ci, _vp, _vp, _vp]
        L.crk_neighbour_lists.argtypes = [_vp, _ci, _vp, _vp, _vp]
        L.crk_volumes.argtypes = [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong), _vp]
        L.crk_corrections.argtypes = [_vp] + [_vp] * 7 + [_vp]
        L.crk_forces.argtypes = [_vp] + [_vp] * 12 + [ctypes.POINTER(ctypes.c_longlong), _vp]
        L.crk_compatible.argtypes = [_vp] + [_vp] * 11 + [_vp]
        L.crk_step.argtypes = [_vp, _ci, _vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(crk_diag), _vp]
        L.crk_reset_rates.argtypes = [_vp]
        L.crk_set_expansion.argtypes = [_vp, ctypes.c_double, ctypes.c_double]
        L.crk_order.argtypes = [_vp, _vp, _vp]
        L.crk_cycle.argtypes = [_vp, _ci, _vp, _vp, _vp, ctypes.c_double, _ci, _ci, ctypes.POINTER(crk_htb_stats),
                                _vp]
        L.crk_htb_levels.argtypes = [_vp, _ci, _vp, _vp, ctypes.c_double, _ci, _ci, _vp,
                                     ctypes.POINTER(ctypes.c_longlong), _vp]
        L.crk_h_iterate.argtypes = [_vp, _ci, _vp, ctypes.c_float, _ci, ctypes.POINTER(_ci), _vp]
        L.crk_volumes_noalloc.argtypes = [_ci, _vp, _vp, _vp, _vp]
        L.crk_mlp_set_weights.argtypes = [_vp, _vp, _vp]
        L.crk_mlp_get_weights.argtypes = [_vp, _vp, _vp]
        L.crk_h_features.argtypes = [_vp, _ci, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _vp]
        L.crk_mlp_forward.argtypes = [_vp, _ci, _vp, _vp, _vp]
        L.crk_h_propose.argtypes = [_vp, _ci, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp]
        L.crk_mlp_train_step.argtypes = [_vp, _ci, _vp, _vp, ctypes.c_float, _vp, _vp, _vp]
        L.crk_mlp_train.argtypes = [_vp, _ci, _vp, _vp, _vp, _ci, _ci, _ci, ctypes.c_float, ctypes.c_ulonglong,
                                    _vp, _vp]
        L.crk_h_select.argtypes = [_vp, _ci, _vp, ctypes.c_float, _ci, _vp, ctypes.POINTER(_ci), _vp]
        L.crk_build_cells_batched.argtypes = [_vp, _ci, _ci, _vp, _vp, _vp]
        L.crk_step_batched.argtypes = [_vp, _ci, _ci, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.crk_steps.argtypes = [_vp, _ci, _vp, _vp, _vp, _ci, ctypes.c_double, _ci, ctypes.POINTER(crk_diag), _vp]
        L.crk_graph_stats.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_longlong)] * 3
        L.crk_steps_batched.argtypes = [_vp, _ci, _ci, _vp, _vp, _vp, _vp, _ci, ctypes.c_double, _ci, _vp]
        L.crk_autotune.argtypes = [_vp, _ci]
        L.crk_tuning.argtypes = [_vp, _vp, _vp]
        L.crk_tune_set.argtypes = [_vp, _ci, _ci]
        L.crk_profile.argtypes = [_vp, _ci]
        L.crk_profile_read.argtypes = [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong)]
        _LIB = L
    return _LIB


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _t(x, shape, name, dtype=torch.float32):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if x.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(x.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(x.shape), tuple(shape)))
    return _vp(x.data_ptr())


class Context:
    """Owns one crk_ctx (freed on close / garbage collection)."""

    def __init__(self, handle):
        self.handle = handle
        self.n = 0

    def close(self):
        if self.handle:
            lib().crk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != CRK_OK:
            raise CrkError(rc, lib().crk_last_error(self.handle).decode())
        return rc


def crk_default_params(**overrides) -> crk_params:
    p = crk_params()
    lib().crk_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def crk_create(params=None, **overrides) -> Context:
    p = params if params is not None else crk_default_params(**overrides)
    h = _vp()
    rc = lib().crk_create(ctypes.byref(p), ctypes.byref(h))
    if rc != CRK_OK:
        raise CrkError(rc, "crk_create failed")
    return Context(h)


def crk_sync(ctx, stream=None):
    ctx.check(lib().crk_sync(ctx.handle, _stream(stream)))


def crk_build_cells(ctx, pos_h, stream=None):
    n = pos_h.shape[0]
    p = _t(pos_h, (n, 4), "pos_h")
    ctx.check(lib().crk_build_cells(ctx.handle, n, p, _stream(stream)))
    ctx.n = n


def crk_cells(ctx, kmax=7, stream=None):
    """(keys int32 (bit pattern of the uint32 keys), perm int32, cell_start int32, k)."""
    dev = torch.device("cuda")
    keys = torch.empty(ctx.n, dtype=torch.int32, device=dev)
    perm = torch.empty(ctx.n, dtype=torch.int32, device=dev)
    cs = torch.empty((1 << (3 * kmax)) + 1, dtype=torch.int32, device=dev)
    k = _ci(0)
    ctx.check(lib().crk_cells(ctx.handle, _vp(keys.data_ptr()), _vp(perm.data_ptr()), _vp(cs.data_ptr()),
                              ctypes.byref(k), _stream(stream)))
    return keys, perm, cs[: (1 << (3 * k.value)) + 1], k.value


def crk_order(ctx, stream=None):
    """Sorted order of the last build: perm[s] = caller row in slot s (int32)."""
    perm = torch.empty(ctx.n, dtype=torch.int32, device=torch.device("cuda"))
    ctx.check(lib().crk_order(ctx.handle, _vp(perm.data_ptr()), _stream(stream)))
    return perm


def crk_build_stats(ctx, stream=None):
    nt, g, u = _ci(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
    ctx.check(lib().crk_build_stats(ctx.handle, ctypes.byref(nt), ctypes.byref(g), ctypes.byref(u),
                                    _stream(stream)))
    return nt.value, g.value, u.value


def crk_walk_stats(ctx, stream=None):
    """Lane tests of the exact predicate in the last neighbour-list walk."""
    t = ctypes.c_longlong(0)
    ctx.check(lib().crk_walk_stats(ctx.handle, ctypes.byref(t), _stream(stream)))
    return t.value


def crk_neighbours(ctx, mode=0, stream=None):
    """Per particle: neighbour count and order-independent hash of the neighbour set."""
    dev = torch.device("cuda")
    cnt = torch.empty(ctx.n, dtype=torch.int32, device=dev)
    hsh = torch.empty(ctx.n, dtype=torch.int32, device=dev)
    ctx.check(lib().crk_neighbours(ctx.handle, int(mode), _vp(cnt.data_ptr()), _vp(hsh.data_ptr()),
                                   _stream(stream)))
    return cnt, hsh


def crk_neighbour_lists(ctx, mode=0, stream=None):
    """The neighbour lists the passes walk, in caller order: (offsets[n+1], lists)
    as int64 / int32 CUDA tensors (mode 0 entries carry bit 31 = i in gather(j))."""
    cnt, _ = crk_neighbours(ctx, mode, stream)
    dev = cnt.device
    off = torch.zeros(ctx.n + 1, dtype=torch.int64, device=dev)
    if ctx.n:
        off[1:] = torch.cumsum(cnt.to(torch.int64), 0)
    total = int(off[-1].item()) if ctx.n else 0
    lists = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    ctx.check(lib().crk_neighbour_lists(ctx.handle, int(mode), _vp(off.data_ptr()), _vp(lists.data_ptr()),
                                        _stream(stream)))
    return off, lists[:total]


def crk_volumes(ctx, with_pairs=False, stream=None):
    n = ctx.n
    dev = torch.device("cuda")
    V = torch.empty(n, dtype=torch.float32, device=dev)
    N = torch.empty(n, dtype=torch.float32, device=dev)
    pairs = ctypes.c_longlong(0)
    ctx.check(lib().crk_volumes(ctx.handle, _vp(V.data_ptr()), _vp(N.data_ptr()),
                                ctypes.byref(pairs) if with_pairs else None, _stream(stream)))
    return (V, N, pairs.value) if with_pairs else (V, N)


def crk_corrections(ctx, V, vel_u=None, gradv=True, stream=None):
    n = ctx.n
    dev = torch.device("cuda")
    A = torch.empty(n, dtype=torch.float32, device=dev)
    B = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gA = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gB = torch.empty((n, 3, 3), dtype=torch.float32, device=dev)
    gv = torch.empty((n, 3, 3), dtype=torch.float32, device=dev) if gradv else None
    pv = _t(V, (n,), "V")
    pu = _t(vel_u, (n, 4), "vel_u") if vel_u is not None else None
    if gradv and vel_u is None:
        raise ValueError("vel_u is needed for grad v")
    ctx.check(lib().crk_corrections(ctx.handle, pv, pu, _vp(A.data_ptr()), _vp(B.data_ptr()),
                                    _vp(gA.data_ptr()), _vp(gB.data_ptr()),
                                    _vp(gv.data_ptr()) if gradv else None, _stream(stream)))
    return A, B, gA, gB, gv


def _force_inputs(ctx, mass, vel_u, V, A, B, gA, gB, gv):
    n = ctx.n
    return [_t(mass, (n,), "mass"), _t(vel_u, (n, 4), "vel_u"), _t(V, (n,), "V"), _t(A, (n,), "A"),
            _t(B, (n, 3), "B"), _t(gA, (n, 3), "gradA"), _t(gB, (n, 3, 3), "gradB"),
            _t(gv, (n, 3, 3), "gradv")]


def crk_forces(ctx, mass, vel_u, V, A, B, gA, gB, gv, with_pairs=False, stream=None):
    n = ctx.n
    dev = torch.device("cuda")
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    dudt = torch.empty(n, dtype=torch.float32, device=dev)
    vsig = torch.empty(n, dtype=torch.float32, device=dev)
    qmax = torch.empty(n, dtype=torch.float32, device=dev)
    pairs = ctypes.c_longlong(0)
    args = _force_inputs(ctx, mass, vel_u, V, A, B, gA, gB, gv)
    ctx.check(lib().crk_forces(ctx.handle, *args, _vp(acc.data_ptr()), _vp(dudt.data_ptr()),
                               _vp(vsig.data_ptr()), _vp(qmax.data_ptr()),
                               ctypes.byref(pairs) if with_pairs else None, _stream(stream)))
    out = (acc, dudt, vsig, qmax)
    return out + (pairs.value,) if with_pairs else out


def crk_compatible(ctx, mass, vel_u, V, A, B, gA, gB, gv, vel_before, vel_after, stream=None):
    n = ctx.n
    du = torch.empty(n, dtype=torch.float32, device=torch.device("cuda"))
    args = _force_inputs(ctx, mass, vel_u, V, A, B, gA, gB, gv)
    ctx.check(lib().crk_compatible(ctx.handle, *args, _t(vel_before, (n, 3), "vel_before"),
                                   _t(vel_after, (n, 3), "vel_after"), _vp(du.data_ptr()), _stream(stream)))
    return du


def crk_step(ctx, pos_h, vel_u, mass, dt=0.0, diag=False, stream=None):
    """One KDK step in place on pos_h, vel_u; returns a dict of FP64 diagnostics if diag."""
    n = pos_h.shape[0]
    d = crk_diag()
    ctx.check(lib().crk_step(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _t(vel_u, (n, 4), "vel_u"),
                             _t(mass, (n,), "mass"), float(dt), ctypes.byref(d) if diag else None,
                             _stream(stream)))
    ctx.n = n
    if not diag:
        return None
    return {"dt": d.dt, "dt_next": d.dt_next, "E_kin": d.E_kin, "E_int": d.E_int, "P": list(d.P),
            "pairs_gather": d.pairs_gather, "pairs_union": d.pairs_union, "h_iterations": d.h_iterations,
            "h_unconverged": d.h_unconverged}


def crk_cycle(ctx, pos_h, vel_u, mass, Delta, L, f_l=2, stream=None):
    """One cycle of hierarchical time bins (base step Delta, 2^L ticks, limiter
    f_l) in place on pos_h, vel_u; returns the cycle's statistics."""
    n = pos_h.shape[0]
    st = crk_htb_stats()
    ctx.check(lib().crk_cycle(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _t(vel_u, (n, 4), "vel_u"),
                              _t(mass, (n,), "mass"), float(Delta), int(L), int(f_l), ctypes.byref(st),
                              _stream(stream)))
    ctx.n = n
    return {"ticks": st.ticks, "evaluations": st.evaluations, "wakeups": st.wakeups, "unresolved": st.unresolved,
            "leaves": st.leaves, "level_count": list(st.level_count)}


def crk_htb_levels(ctx, pos_h, dt, Delta, L, f_l=2, stream=None):
    """Leaf level of every particle (int32, caller order) after the limiter,
    from the per-particle time steps dt; returns (level, unresolved)."""
    n = pos_h.shape[0]
    level = torch.empty(n, dtype=torch.int32, device=pos_h.device)
    unres = ctypes.c_longlong(0)
    ctx.check(lib().crk_htb_levels(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _t(dt, (n,), "dt"), float(Delta),
                                   int(L), int(f_l), _t(level, (n,), "level", torch.int32), ctypes.byref(unres),
                                   _stream(stream)))
    ctx.n = n
    return level, int(unres.value)


def crk_set_expansion(ctx, a, adot):
    """Scale factor and its rate for the following calls (comoving variables)."""
    ctx.check(lib().crk_set_expansion(ctx.handle, float(a), float(adot)))


def crk_reset_rates(ctx):
    ctx.check(lib().crk_reset_rates(ctx.handle))


def crk_h_iterate(ctx, pos_h, tol=1e-4, max_it=50, stream=None):
    """Fixed-point h solve in place; returns (iterations, converged)."""
    n = pos_h.shape[0]
    it = _ci(0)
    rc = lib().crk_h_iterate(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), float(tol), int(max_it),
                             ctypes.byref(it), _stream(stream))
    ctx.n = n
    if rc == CRK_ENONCONV:
        return it.value, False
    ctx.check(rc)
    return it.value, True


PASS_NAMES = ["P1 volumes", "neighbour sets", "P2 corrections", "P3 grad v", "P4 forces",
              "P5 compatible energy", "cell build", "neighbour lists", "h proposal", "mlp train step",
              "RK density"]
NPASS = len(PASS_NAMES)


def crk_profile(ctx, enable=True):
    ctx.check(lib().crk_profile(ctx.handle, 1 if enable else 0))


def crk_profile_read(ctx):
    """({pass: total ms}, {pass: records}, total kernel launches since creation)."""
    ms = (ctypes.c_double * NPASS)()
    cnt = (ctypes.c_longlong * NPASS)()
    tot = ctypes.c_longlong(0)
    ctx.check(lib().crk_profile_read(ctx.handle, ms, cnt, ctypes.byref(tot)))
    return ({PASS_NAMES[k]: ms[k] for k in range(NPASS)}, {PASS_NAMES[k]: cnt[k] for k in range(NPASS)},
            tot.value)


def crk_launches(ctx):
    """Kernels launched by ctx since it was created."""
    tot = ctypes.c_longlong(0)
    ctx.check(lib().crk_profile_read(ctx.handle, None, None, ctypes.byref(tot)))
    return tot.value


NOALLOC_MAX_N = 16384


def crk_volumes_noalloc(pos_h, stream=None, with_N=True):
    """Volumes without any device allocation by the library (n <= NOALLOC_MAX_N).
    Returns (V, Nngb), Nngb None with with_N=False (the library is then given a
    null Nngb); the output tensors are the caller's (allocated here by torch)."""
    n = pos_h.shape[0]
    dev = pos_h.device
    V = torch.empty(n, dtype=torch.float32, device=dev)
    N = torch.empty(n, dtype=torch.float32, device=dev) if with_N else None
    rc = lib().crk_volumes_noalloc(n, _t(pos_h, (n, 4), "pos_h"), _vp(V.data_ptr()),
                                   _vp(N.data_ptr()) if with_N else None, _stream(stream))
    if rc != CRK_OK:
        raise CrkError(rc, "crk_volumes_noalloc failed")
    return V, N


# ---------------------------------------------------------------- learned h proposal

MLP_NPARAM = 4801
MLP_NFEAT = 8


def _opt(x, shape, name):
    return _vp(None) if x is None else _t(x, shape, name)


def crk_mlp_set_weights(ctx, w, stream=None):
    """Load the FP32 parameters (CUDA tensor of MLP_NPARAM) and reset Adam."""
    ctx.check(lib().crk_mlp_set_weights(ctx.handle, _t(w, (MLP_NPARAM,), "w"), _stream(stream)))


def crk_mlp_get_weights(ctx, stream=None):
    w = torch.empty(MLP_NPARAM, dtype=torch.float32, device=torch.device("cuda"))
    ctx.check(lib().crk_mlp_get_weights(ctx.handle, _vp(w.data_ptr()), _stream(stream)))
    return w


def crk_h_features(ctx, pos_h, gradv=None, Nngb=None, pos_conv=None, dt=0.0, stream=None):
    """Features (n, 8); with pos_conv also the targets log(h_conv / h_prev) -> (feat, target)."""
    n = pos_h.shape[0]
    dev = pos_h.device
    feat = torch.empty((n, MLP_NFEAT), dtype=torch.float32, device=dev)
    target = torch.empty(n, dtype=torch.float32, device=dev) if pos_conv is not None else None
    ctx.check(lib().crk_h_features(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _opt(gradv, (n, 3, 3), "gradv"),
                                   _opt(Nngb, (n,), "Nngb"), float(dt), _opt(pos_conv, (n, 4), "pos_conv"),
                                   _vp(feat.data_ptr()), _vp(None if target is None else target.data_ptr()),
                                   _stream(stream)))
    return (feat, target) if pos_conv is not None else feat


def crk_mlp_forward(ctx, feat, stream=None):
    n = feat.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=feat.device)
    ctx.check(lib().crk_mlp_forward(ctx.handle, n, _t(feat, (n, MLP_NFEAT), "feat"), _vp(y.data_ptr()),
                                    _stream(stream)))
    return y


def crk_h_propose(ctx, pos_h, gradv=None, Nngb=None, dt=0.0, tol=1e-4, stream=None):
    """Write the proposed h into pos_h[:, 3] in place."""
    n = pos_h.shape[0]
    ctx.check(lib().crk_h_propose(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _opt(gradv, (n, 3, 3), "gradv"),
                                  _opt(Nngb, (n,), "Nngb"), float(dt), float(tol), _stream(stream)))


def crk_mlp_train_step(ctx, feat, target, lr=0.0, stream=None):
    """One full-batch step; returns (grad, loss) as CUDA tensors."""
    n = feat.shape[0]
    dev = feat.device
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    ctx.check(lib().crk_mlp_train_step(ctx.handle, n, _t(feat, (n, MLP_NFEAT), "feat"), _t(target, (n,), "target"),
                                       float(lr), _vp(grad.data_ptr()), _vp(loss.data_ptr()), _stream(stream)))
    return grad, loss


def crk_h_select(ctx, Nngb, tol=1e-4, base=0, stream=None):
    """Indices (int32 CUDA tensor, base-offset) of the rows the judge hands to the proposal."""
    n = Nngb.shape[0]
    rows = torch.empty(max(n, 1), dtype=torch.int32, device=Nngb.device)
    cnt = _ci(0)
    ctx.check(lib().crk_h_select(ctx.handle, n, _t(Nngb, (n,), "Nngb"), float(tol), int(base),
                                 _vp(rows.data_ptr()), ctypes.byref(cnt), _stream(stream)))
    return rows[:cnt.value]


def crk_mlp_train(ctx, feat, target, rows=None, batch=4096, steps=1000, lr=1e-3, seed=1, stream=None):
    """`steps` Adam steps on batches sampled from all rows (rows None) or from the
    listed rows; returns the per-step losses (list of floats)."""
    n = feat.shape[0]
    hist = (ctypes.c_float * max(int(steps), 1))()
    nr = 0 if rows is None else rows.shape[0]
    ctx.check(lib().crk_mlp_train(ctx.handle, n, _t(feat, (n, MLP_NFEAT), "feat"), _t(target, (n,), "target"),
                                  _vp(None) if rows is None else _t(rows, (nr,), "rows", torch.int32), nr,
                                  int(batch), int(steps), float(lr), int(seed), hist, _stream(stream)))
    return [hist[k] for k in range(int(steps))]


# ---------------------------------------------------------------- batched boxes

def _box_table(box_start, n):
    b = [int(x) for x in box_start]
    arr = (ctypes.c_int32 * len(b))(*b)
    return arr, len(b) - 1


def crk_build_cells_batched(ctx, pos_h, box_start, stream=None):
    """Bin independent boxes; box b owns rows box_start[b]:box_start[b+1] of pos_h."""
    n = pos_h.shape[0]
    arr, nbox = _box_table(box_start, n)
    ctx.check(lib().crk_build_cells_batched(ctx.handle, n, nbox, arr, _t(pos_h, (n, 4), "pos_h"), _stream(stream)))
    ctx.n = n


def crk_step_batched(ctx, pos_h, vel_u, mass, box_start, dt=None, diag=False, stream=None):
    """One KDK step of every box in place; dt (per box, None = CFL); per-box diagnostics if diag."""
    n = pos_h.shape[0]
    arr, nbox = _box_table(box_start, n)
    dta = None if dt is None else (ctypes.c_double * nbox)(*[float(x) for x in dt])
    d = (crk_diag * nbox)() if diag else None
    ctx.check(lib().crk_step_batched(ctx.handle, n, nbox, arr, _t(pos_h, (n, 4), "pos_h"),
                                     _t(vel_u, (n, 4), "vel_u"), _t(mass, (n,), "mass"), dta, d, _stream(stream)))
    ctx.n = n
    if not diag:
        return None
    return [{"dt": x.dt, "dt_next": x.dt_next, "E_kin": x.E_kin, "E_int": x.E_int, "P": list(x.P),
             "pairs_gather": x.pairs_gather, "pairs_union": x.pairs_union} for x in d]


# ---------------------------------------------------------------- autotuner

def crk_autotune(ctx, enable=True):
    ctx.check(lib().crk_autotune(ctx.handle, 1 if enable else 0))


def crk_tuning(ctx):
    """{pass name: (variant, ms)} for the tuned passes."""
    v = (ctypes.c_int * NPASS)()
    ms = (ctypes.c_float * NPASS)()
    ctx.check(lib().crk_tuning(ctx.handle, v, ms))
    return {PASS_NAMES[k]: (v[k], ms[k]) for k in range(NPASS) if v[k] >= 0}


CRK_TUNE_NVARIANT = 23


def crk_tune_set(ctx, pass_name, variant):
    """Pin one list pass (a name of PASS_NAMES) to a variant (-1: its default)."""
    ctx.check(lib().crk_tune_set(ctx.handle, PASS_NAMES.index(pass_name), int(variant)))


# ---------------------------------------------------------------- multi-step, CUDA graphs

def crk_steps(ctx, pos_h, vel_u, mass, nsteps, dt=0.0, use_graph=True, diag=False, stream=None):
    """nsteps KDK steps in place (captured once into CUDA graphs and replayed with use_graph)."""
    n = pos_h.shape[0]
    d = crk_diag()
    ctx.check(lib().crk_steps(ctx.handle, n, _t(pos_h, (n, 4), "pos_h"), _t(vel_u, (n, 4), "vel_u"),
                              _t(mass, (n,), "mass"), int(nsteps), float(dt), 1 if use_graph else 0,
                              ctypes.byref(d) if diag else None, _stream(stream)))
    ctx.n = n
    if not diag:
        return None
    return {"dt": d.dt, "dt_next": d.dt_next, "E_kin": d.E_kin, "E_int": d.E_int, "P": list(d.P),
            "pairs_gather": d.pairs_gather, "pairs_union": d.pairs_union, "h_iterations": d.h_iterations,
            "h_unconverged": d.h_unconverged}


def crk_graph_stats(ctx):
    """(graphs captured, graph launches, replay runs redone eagerly) since the context was created."""
    c, r, v = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
    ctx.check(lib().crk_graph_stats(ctx.handle, ctypes.byref(c), ctypes.byref(r), ctypes.byref(v)))
    return c.value, r.value, v.value


def crk_steps_batched(ctx, pos_h, vel_u, mass, box_start, nsteps, dt=0.0, use_graph=True, stream=None):
    """nsteps KDK steps of every box in place (CUDA graphs with use_graph)."""
    n = pos_h.shape[0]
    arr, nbox = _box_table(box_start, n)
    ctx.check(lib().crk_steps_batched(ctx.handle, n, nbox, arr, _t(pos_h, (n, 4), "pos_h"),
                                      _t(vel_u, (n, 4), "vel_u"), _t(mass, (n,), "mass"), int(nsteps), float(dt),
                                      1 if use_graph else 0, _stream(stream)))
    ctx.n = n
