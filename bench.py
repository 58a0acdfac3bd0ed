#!/usr/bin/env python
"""Benchmark of the CRKSPH pair-interaction engine on one GB300.

Workload: 128^3 = 2,097,152 particles of clustered gas (Zel'dovich-displaced
lattice, P(k) ~ k^-2, log-normal u) in the periodic unit cube.  One step is a
full KDK hydro step (crk_step): half kick with the cached rates and its
compatible-energy pass, drift, cell rebuild, P1 volumes, P2 corrections,
P3 grad v, P4 forces, second half kick and its compatible-energy pass, the
Thacker h update and the CFL time step.

Metric: pair interactions per second = (3 * gather pairs + 3 * ordered pair-set
pairs) per step / step time (P1, P2, P3 walk gather(i); P4 and the two P5
passes walk the pair set), and the step time in ms.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead
(a bounded sample of the same workload per step, all host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CRKSPH pair interactions/s and hydro-step ms at 128^3 vs plain FP32 GPU, at stated err"
UNIT = "pair interactions/s"
WORKLOAD = "zeldovich-128^3: clustered gas, Zel'dovich lattice displacement, P(k)~k^-2, log-normal u"

# Algorithmic FP32 flops per pair unit of each pass (FMA = 2, add/mul/min/max = 1,
# div/sqrt/exp = 1), counted from the operations the paper's formulas require
# (each term listed with the pass kernels).  P1-P3 count per gather pair; P4 and P5 count per
# UNORDERED pair of the pair set (both kernel sides, limiter, viscosity, force).
FLOPS_PER_UNIT = {"P1 volumes": 20, "P2 corrections": 88, "P3 grad v": 92, "P4 forces": 281,
                  "P5 compatible energy": 259}
# DRAM bytes (read + write) per unit measured by ncu for the current P4 kernel on
# zeldovich-64^3 in the Hilbert order (0.65 GB read + 1.20 GB written for
# 39.1 M unordered pairs); a full 128^3 launch is too large to capture, so the
# traffic is scaled by units.
TRAFFIC_PER_UNIT = {"P4 forces": 50.0}
# the walk's exact predicate per lane test, in 32-bit integer operations:
# dx, dy, dz (3), the widening squares and H_j^2 (4), two 64-bit additions
# (4), the two 64-bit comparisons (4), the gather / other / reach bits (4)
WALK_INT_OPS = 19
# INT32 issue: 152 SMs x 64 lanes per clock x 2070 MHz (max SM clock)
INT32_PEAK_TOPS = 152 * 64 * 2.07e9 / 1e12
BUILD_BYTES_PER_PARTICLE = 44 + 4 * 20 + 52 + 16
PRECISION_NAMES = ["plain", "mixed", "mixed+compensated moments", "mixed+float-float moments"]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        """Start of the timed region: samples taken before it are dropped (the
        sampler is started earlier, so that its own start-up is not timed)."""
        self.t0 = time.perf_counter()

    def stop(self):
        if not self.proc:
            return None
        t1 = time.perf_counter()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if self.t0 is not None and not (self.t0 <= ts <= t1 + 0.25):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def alu_peak_tflops(sm_count, mhz):
    """FP32 FMA issue peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# --------------------------------------------------------------------- CPU oracle

def oracle_sample(st, n_targets, seed=0):
    """Time the FP64 oracle's passes P1..P5 on a random sample of target
    particles of the workload.  Per-particle inputs of the non-target particles
    are a uniform placeholder state (values do not change the work done)."""
    from oracle import crk as O
    pos = st["pos_h"]
    n = pos.shape[0]
    tg = np.sort(np.random.default_rng(seed).choice(n, n_targets, replace=False)).astype(np.int32)
    vel = st["vel_u"][:, :3].astype(np.float64)
    u = st["vel_u"][:, 3].astype(np.float64)
    m = st["mass"].astype(np.float64)
    V = np.full(n, 1.0 / n)
    A = np.ones(n)
    B = np.zeros((n, 3))
    gA = np.zeros((n, 3))
    gB = np.zeros((n, 3, 3))
    gv = np.zeros((n, 3, 3))
    t0 = time.perf_counter()
    p1 = O.volumes(pos, targets=tg)
    V[tg] = p1["V"][tg]
    p2 = O.corrections(pos, V, targets=tg)
    gvt = O.gradv(pos, V, vel, A, B, gA, gB, targets=tg)
    p4 = O.forces(pos, vel, u, m, V, A, B, gA, gB, gv, targets=tg)
    O.compatible(pos, vel, u, m, V, A, B, gA, gB, gv, vel, vel, targets=tg)
    O.compatible(pos, vel, u, m, V, A, B, gA, gB, gv, vel, vel, targets=tg)
    dt = time.perf_counter() - t0
    pairs = 3 * p1["pairs"] + 3 * p4["pairs"]
    del p2, gvt
    return pairs, dt


def calibrated_oracle(st, seconds, seed):
    """Grow the oracle sample until one run takes at least half the budget."""
    n = st["pos_h"].shape[0]
    ns = 2048
    while True:
        p, dt = oracle_sample(st, ns, seed=seed)
        if dt >= 0.5 * seconds or ns >= n:
            return p, dt, ns
        ns = min(n, int(ns * min(16.0, max(2.0, 0.9 * seconds / dt))))


def _rel_err(g, o, floor=None):
    """max_i |g_i - o_i| / max(|o_i|, floor): floor = the field's RMS, or a
    per-particle scale (the no-cancellation scale of a coefficient or force)."""
    o = np.asarray(o, np.float64)
    g = np.asarray(g, np.float64).reshape(o.shape)
    if floor is None:
        floor = np.sqrt(np.mean(o ** 2))
    floor = np.asarray(floor, np.float64)
    if floor.ndim == 1 and o.ndim > 1:
        floor = floor.reshape((-1,) + (1,) * (o.ndim - 1))
    return float(np.max(np.abs(g - o) / np.maximum(np.maximum(np.abs(o), floor), 1e-300)))


def oracle_cone(st, sample):
    """FP64 oracle values of P1-P4 for the particles `sample` of a workload,
    computed over their dependency cone only: the forces of the sample need the
    corrections and grad v of its union neighbours U1, which need the volumes
    of their gather neighbours G2.  Returns (p1, p2, gv, p4, |G2|); entries
    outside the cone are not meaningful."""
    from oracle import crk as O
    pos = st["pos_h"]
    _, ul = O.neighbours(pos, mode=1, targets=sample)
    U1 = np.unique(np.concatenate([sample, ul]))
    _, gl = O.neighbours(pos, mode=0, targets=U1)
    G2 = np.unique(np.concatenate([U1, gl]))
    vel = st["vel_u"][:, :3].astype(np.float64)
    u = st["vel_u"][:, 3].astype(np.float64)
    m = st["mass"].astype(np.float64)
    p1 = O.volumes(pos, targets=G2)
    p2 = O.corrections(pos, p1["V"], targets=U1)
    gv = O.gradv(pos, p1["V"], vel, p2["A"], p2["B"], p2["gA"], p2["gB"], targets=U1)
    p4 = O.forces(pos, vel, u, m, p1["V"], p2["A"], p2["B"], p2["gA"], p2["gB"], gv, targets=sample)
    return p1, p2, gv, p4, G2.size


def sampled_errors(st, dev, order, precisions, n_sample=16, seed=77):
    """Error of one GPU evaluation (P1-P4 at the initial state) in each
    precision mode against the FP64 oracle, on a seeded sample of particles
    whose exact FP64 values the oracle computes over their dependency cone."""
    import torch
    from paper_2202_02840_gb300 import crk
    pos = st["pos_h"]
    sample = np.sort(np.random.default_rng(seed).choice(pos.shape[0], n_sample, replace=False))
    p1, p2, gv, p4, ncone = oracle_cone(st, sample)
    s = sample
    out = {}
    for prec in precisions:
        c = crk.crk_create(precision=prec, **order)
        dpos = torch.from_numpy(pos).to(dev)
        dvel = torch.from_numpy(st["vel_u"]).to(dev)
        crk.crk_build_cells(c, dpos)
        V, _ = crk.crk_volumes(c)
        A, B, gA, gB, g_v = crk.crk_corrections(c, V, dvel)
        acc, dudt, _, _ = crk.crk_forces(c, torch.from_numpy(st["mass"]).to(dev), dvel, V, A, B, gA, gB, g_v)
        h = {k: t.detach().cpu().double().numpy() for k, t in
             (("V", V), ("A", A), ("B", B), ("gA", gA), ("gB", gB), ("gv", g_v), ("acc", acc), ("dudt", dudt))}
        c.close()
        out[PRECISION_NAMES[prec]] = {
            "V": _rel_err(h["V"][s], p1["V"][s]), "A": _rel_err(h["A"][s], p2["A"][s]),
            "B": _rel_err(h["B"][s], p2["B"][s], p2["sB"][s]),
            "gradA": _rel_err(h["gA"][s], p2["gA"][s], p2["sgA"][s]),
            "gradB": _rel_err(h["gB"][s], p2["gB"][s], p2["sgB"][s]),
            "B_rms": _rel_err(h["B"][s], p2["B"][s]), "gradA_rms": _rel_err(h["gA"][s], p2["gA"][s]),
            "gradB_rms": _rel_err(h["gB"][s], p2["gB"][s]),
            "gradv": _rel_err(h["gv"][s], gv[s]),
            "accel": _rel_err(h["acc"][s], p4["acc"][s], p4["fscale"][s]),
            "dudt": _rel_err(h["dudt"][s], p4["dudt"][s])}
    return {"sample": "%d seeded particles of the workload, FP64 oracle over their dependency cone "
                      "(%d particles)" % (n_sample, ncone),
            "norm": "max |gpu - oracle| / max(|oracle|, floor); floor = field RMS over the sample, or the "
                    "no-cancellation scale for B, grad A, grad B and the acceleration (*_rms: the RMS floor)",
            "by_precision": out}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import crk as O
    from paper_2202_02840_gb300 import inputs
    st = inputs.zeldovich(args.n_side)
    cores = O.num_threads()
    # size the per-step sample so that warmup + steps end within a few minutes
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    _, _, ns = calibrated_oracle(st, budget, seed=1)
    for w in range(args.warmup):
        oracle_sample(st, ns, seed=100 + w)
    tot_pairs, tot_t = 0, 0.0
    for k in range(args.steps):
        p, t = oracle_sample(st, ns, seed=1000 + k)
        tot_pairs += p
        tot_t += t
    value = tot_pairs / tot_t
    sample = ("FP64 oracle passes P1,P2,P3,P4,P5,P5 on %d random target particles of the %d^3 workload "
              "per step (%d steps)" % (ns, args.n_side, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": args.n_side ** 3},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- learned h

MLP_TENSOR_FLOPS_PER_ROW = 2 * (8 * 64 + 64 * 64)   # the two BF16 tensor-core products per row


def learned_h_report(dev, train_side=64, train_steps=200, every=10, eval_side=256, eval_steps=10, tol=1e-4):
    """Learned smoothing-length proposal: train on snapshots of a Sedov run,
    then solve eq:hi at a larger Sedov state plainly and from the proposal."""
    import torch
    from paper_2202_02840_gb300 import crk, inputs, learned_h

    def wall(f):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = f()
        torch.cuda.synchronize(dev)
        return r, 1e3 * (time.perf_counter() - t0)

    (snaps, probe), data_ms = wall(lambda: learned_h.sedov_snapshots(n_side=train_side, steps=train_steps,
                                                                    every=every, tol=tol))
    ctx = crk.crk_create()
    feat, target, rows = learned_h.dataset(ctx, snaps)
    crk.crk_profile(ctx, True)
    steps = 2000
    losses, train_ms = wall(lambda: learned_h.train(ctx, feat, target, rows, steps=steps, batch=4096, lr=1e-3))
    pm, pc, _ = crk.crk_profile_read(ctx)
    crk.crk_profile(ctx, False)
    w = crk.crk_mlp_get_weights(ctx)
    sel_t = target[rows.long()]
    train = {"workload": "sedov-%d^3, %d KDK steps, a snapshot every %d" % (train_side, train_steps, every),
             "snapshots": len(snaps), "rows": int(feat.shape[0]), "selected_rows": int(rows.shape[0]),
             "adam_steps": steps, "batch": 4096, "loss_first": losses[0], "loss_last50": float(np.mean(losses[-50:])),
             "mean_target_sq_selected": float(torch.mean(sel_t * sel_t)),
             "train_step_ms": pm["mlp train step"] / max(1, pc["mlp train step"]), "train_wall_ms": train_ms,
             "data_wall_ms": data_ms, "plain_iterations": [s.it_plain for s in snaps]}
    del snaps, feat, target, rows
    probe.close()

    st = inputs.sedov(eval_side)
    pos = torch.from_numpy(st["pos_h"]).to(dev)
    vel = torch.from_numpy(st["vel_u"]).to(dev)
    mass = torch.from_numpy(st["mass"]).to(dev)
    stepper = crk.crk_create()
    for _ in range(eval_steps):
        dt = crk.crk_step(stepper, pos, vel, mass, 0.0, diag=True)["dt"]
    stepper.close()
    del st
    ev = crk.crk_create()
    crk.crk_build_cells(ev, pos)
    V, N = crk.crk_volumes(ev)
    gradv = crk.crk_corrections(ev, V, vel)[4]
    del V
    n = pos.shape[0]

    def solve(weights):
        p = pos.clone()
        t_prop = 0.0
        if weights is not None:
            crk.crk_mlp_set_weights(ev, weights)
            crk.crk_profile(ev, True)
            crk.crk_h_propose(ev, p, gradv, N, dt=dt, tol=tol)
            pm, pc, _ = crk.crk_profile_read(ev)
            crk.crk_profile(ev, False)
            t_prop = pm["h proposal"] / max(1, pc["h proposal"])
        (it, ok), ms = wall(lambda: crk.crk_h_iterate(ev, p, tol=tol, max_it=60))
        return it, ok, ms, t_prop, p

    it_p, ok_p, ms_p, _, p_conv = solve(None)
    it_r, ok_r, ms_r, _, _ = solve(torch.zeros_like(w))
    it_l, ok_l, ms_l, prop_ms, _ = solve(w)
    # accuracy of the network on this state: residual of log h against the converged h
    f, t = crk.crk_h_features(ev, pos, gradv, N, p_conv, dt=dt)
    sel = crk.crk_h_select(ev, N, tol=tol).long()
    crk.crk_mlp_set_weights(ev, w)
    y = crk.crk_mlp_forward(ev, f)
    rms_ref = float(torch.sqrt(torch.mean(t[sel] ** 2))) if sel.numel() else 0.0
    rms_net = float(torch.sqrt(torch.mean((t[sel] - y[sel]) ** 2))) if sel.numel() else 0.0
    peaks = measured_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    tflops = MLP_TENSOR_FLOPS_PER_ROW * n / (prop_ms / 1e3) / 1e12
    ev.close()
    return {"train": train,
            "eval": {"workload": "sedov-%d^3 after %d KDK steps (evolved h)" % (eval_side, eval_steps), "n": n,
                     "tol": tol, "selected_rows": int(sel.numel()),
                     "iterations_plain": it_p, "iterations_reference_only": it_r, "iterations_learned": it_l,
                     "converged": [ok_p, ok_r, ok_l],
                     "solve_ms_plain": ms_p, "solve_ms_reference_only": ms_r, "solve_ms_learned": ms_l,
                     "rms_log_h_error_reference": rms_ref, "rms_log_h_error_learned": rms_net,
                     "proposal_ms": prop_ms, "proposal_rows_per_s": n / (prop_ms / 1e3),
                     "proposal_roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16, "unit": "TFLOP/s",
                                           "frac": tflops / bf16,
                                           "note": "BF16 mma.sync flops of the two hidden products per row; "
                                                   "the pass also evaluates 128 SFU tanh per row"}}}


# --------------------------------------------------------------------- batched boxes

def ai_step_report(dev, st, order, steps=5, warmup=3, tol=1e-4, train_side=64, train_steps=40, every=1):
    """The composed step that the metric compares, on the bench workload: KDK
    steps that solve eq:hi before every evaluation (crk_params.h_mode), as
    - plain_fp32: precision 0, the fixed-point iteration from the state's h;
    - ai_step: precision 1, the iteration from the learned proposal, the
      network trained on the solves of steps of the same kind (zeldovich-%d^3
      with h_mode 1: features at the drifted positions and the previous solved
      h, target the step's solved h);
    - reference_only: precision 1, the proposal of the all-zero network (the
      constant-density estimate h (N_res/N)^(1/3) alone), which separates what
      the network adds.
    Each arm starts from the workload's k-NN h; its first `warmup` steps solve
    from there and are not timed.  Returns the report and the final states
    (for the oracle's check of eq:hi in the CPU-baseline leg)."""
    import torch
    from paper_2202_02840_gb300 import crk, inputs, learned_h

    snaps, probe = learned_h.step_snapshots(inputs.zeldovich(train_side), steps=train_steps, every=every, tol=tol)
    tctx = crk.crk_create()
    feat, target, rows = learned_h.dataset(tctx, snaps)
    n_rows = rows.shape[0]
    losses = learned_h.train(tctx, feat, target, rows, steps=2000, batch=4096, lr=1e-3)
    w = crk.crk_mlp_get_weights(tctx)
    tctx.close()
    probe.close()
    del snaps, feat, target, rows
    stream = torch.cuda.current_stream(dev)
    mass = torch.from_numpy(st["mass"]).to(dev)
    out, finals = {}, {}
    arms = (("plain_fp32", 0, 1, None, "the state's h"), ("ai_step", 1, 2, w, "learned proposal"),
            ("reference_only", 1, 2, torch.zeros_like(w), "constant-density proposal (zero network)"))
    for name, prec, mode, weights, start in arms:
        pos = torch.from_numpy(st["pos_h"]).to(dev)
        vel = torch.from_numpy(st["vel_u"]).to(dev)
        c = crk.crk_create(precision=prec, h_mode=mode, h_tol=tol, **order)
        if weights is not None:
            crk.crk_mlp_set_weights(c, weights)
        crk.crk_autotune(c, True)
        warm_it = [crk.crk_step(c, pos, vel, mass, 0.0, diag=True)["h_iterations"] for _ in range(warmup)]
        crk.crk_autotune(c, False)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        diags = [crk.crk_step(c, pos, vel, mass, 0.0, diag=True) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        c.close()
        pairs = sum(3 * d["pairs_gather"] + 3 * d["pairs_union"] for d in diags) / steps
        out[name] = {"precision": PRECISION_NAMES[prec], "h_start": start, "ms_per_step": ms, "value": pairs / (ms * 1e-3), "unit": UNIT,
                     "h_iterations_per_step": [d["h_iterations"] for d in diags],
                     "h_unconverged": max(d["h_unconverged"] for d in diags),
                     "warmup_h_iterations": warm_it}
        finals[name] = pos.cpu().numpy()
    faster = min(("plain_fp32", "ai_step"), key=lambda k: out[k]["ms_per_step"])
    out["comparison"] = {
        "faster": faster, "ai_over_plain_step_ms": out["ai_step"]["ms_per_step"] / out["plain_fp32"]["ms_per_step"],
        "h_tol": tol, "timed_steps": steps,
        "train": {"workload": "zeldovich-%d^3, the eq:hi solves of %d KDK steps with h_mode 1 (every %d)" % (
            train_side, train_steps, every), "rows": int(n_rows), "adam_steps": 2000, "loss_first": losses[0],
            "loss_last50": float(np.mean(losses[-50:]))},
        "accuracy": "both arms solve eq:hi to h_tol (checked by the oracle in err.eq_hi); the evaluation error "
                    "of each precision mode is err.by_precision",
        "batched": "not run: a step that solves eq:hi reads its convergence on the host each pass, so it is "
                   "not captured in CUDA graphs and batched steps keep the evolved h"}
    return out, finals


def eq_hi_check(finals, tol, n_sample=64, seed=5):
    """The oracle's FP64 count of a seeded sample of each final state:
    max |Delta_N - 1| over the sampled particles not held at an h bound."""
    from oracle import crk as O
    res = {}
    for name, pos in finals.items():
        s = np.sort(np.random.default_rng(seed).choice(pos.shape[0], n_sample, replace=False))
        N = O.volumes(pos, targets=s)["N"][s]
        h = pos[s, 3]
        free = (h > np.float32(1e-6)) & (h < np.float32(0.3))
        dN = np.abs(np.cbrt(268.0 / N) - 1.0)
        res[name] = {"max_abs_Delta_N_minus_1": float(dN[free].max()) if free.any() else None,
                     "sampled": int(n_sample), "at_bound": int((~free).sum()), "tol": tol}
    return res


def batched_report(dev, nbox=64, steps=10, warmup=2, seq_steps=2):
    """Many independent Sedov boxes of uneven size (sides 16..96) stepped
    together by crk_step_batched, against the same boxes stepped one by one."""
    import torch
    from paper_2202_02840_gb300 import crk, inputs

    bx = inputs.sedov_boxes(nbox)
    start = bx["box_start"]
    n = start[-1]
    pos = torch.from_numpy(bx["pos_h"]).to(dev)
    vel = torch.from_numpy(bx["vel_u"]).to(dev)
    mass = torch.from_numpy(bx["mass"]).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = crk.crk_create()
    crk.crk_autotune(ctx, True)
    crk.crk_steps_batched(ctx, pos, vel, mass, start, warmup, use_graph=True)   # tunes, captures the graphs
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(use_graph):
        l0 = crk.crk_launches(ctx)
        e0.record(stream)
        crk.crk_steps_batched(ctx, pos, vel, mass, start, steps, use_graph=use_graph)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, (crk.crk_launches(ctx) - l0) / steps

    ms, launches = timed(True)
    ms_eager, _ = timed(False)
    caps, reps, recs = crk.crk_graph_stats(ctx)
    d = crk.crk_step_batched(ctx, pos, vel, mass, start, diag=True)
    pairs = 3 * d[0]["pairs_gather"] + 3 * d[0]["pairs_union"]
    ctx.close()
    # the same boxes one by one: one context each, timed after one warm-up step
    seq_ms = 0.0
    seq_launches = 0
    for b in range(nbox):
        sl = slice(start[b], start[b + 1])
        p, v, m = (torch.from_numpy(bx[k][sl]).to(dev) for k in ("pos_h", "vel_u", "mass"))
        c = crk.crk_create()
        crk.crk_step(c, p, v, m, 0.0)
        torch.cuda.synchronize(dev)
        l0 = crk.crk_launches(c)
        e0.record(stream)
        for _ in range(seq_steps):
            crk.crk_step(c, p, v, m, 0.0)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms += e0.elapsed_time(e1) / seq_steps
        seq_launches += (crk.crk_launches(c) - l0) / seq_steps
        c.close()
    return {"workload": "%d Sedov boxes, sides uniform in 16..96 (seeds 0..%d), %d particles" % (nbox, nbox - 1, n),
            "n": n, "sides_min_max": [min(bx["sides"]), max(bx["sides"])], "steps": steps,
            "ms_per_step": ms, "pair_interactions_per_s": pairs / (ms / 1e3), "kernel_launches_per_step": launches,
            "cuda_graph": {"captures": caps, "replays": reps, "recoveries": recs,
                           "eager_ms_per_step": ms_eager},
            "one_by_one_ms_per_step": seq_ms, "one_by_one_launches_per_step": seq_launches,
            "speedup_vs_one_by_one": seq_ms / ms}


def time_bins_report(dev, side=64, L=5, cycles=4, f_ls=(0, 1, 2, 3, 4), warm_steps=20):
    """Hierarchical time bins (crk_cycle) on a Sedov blast against global
    stepping at the finest tick over the same simulated time: GPU time,
    particle evaluations, energy error and the L1 difference of the radial
    density and energy profiles, for a sweep of the limiter f_l (the Sedov
    test of the paper's Sec. 4 with its f_l sweep)."""
    import numpy as np
    import torch
    from paper_2202_02840_gb300 import crk, inputs

    st = inputs.sedov(side)
    pos = torch.from_numpy(st["pos_h"]).to(dev)
    vel = torch.from_numpy(st["vel_u"]).to(dev)
    mass = torch.from_numpy(st["mass"]).to(dev)
    m = st["mass"].astype(np.float64)
    ctx = crk.crk_create()
    for _ in range(warm_steps):                      # let the blast form (CFL steps)
        d = crk.crk_step(ctx, pos, vel, mass, 0.0, diag=True)
    ctx.close()
    tick = d["dt_next"]
    Delta = tick * (1 << L)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    probe = crk.crk_create()

    def energy(v):
        v = v.cpu().numpy().astype(np.float64)
        return float((0.5 * m * (v[:, :3] ** 2).sum(1) + m * v[:, 3]).sum())

    def profiles(p, v):
        crk.crk_build_cells(probe, p)
        V, _ = crk.crk_volumes(probe)
        rho = m / V.cpu().numpy().astype(np.float64)
        x = p[:, :3].cpu().numpy().astype(np.float64) - 0.5
        x -= np.round(x)
        r = np.sqrt((x * x).sum(1))
        edges = np.arange(0.0, 0.45, 0.5 / side)
        i = np.digitize(r, edges) - 1
        ok = (i >= 0) & (i < len(edges) - 1)
        c = np.maximum(np.bincount(i[ok], None, len(edges) - 1), 1)
        u = v[:, 3].cpu().numpy().astype(np.float64)
        return (np.bincount(i[ok], rho[ok], len(edges) - 1) / c, np.bincount(i[ok], u[ok], len(edges) - 1) / c)

    E0 = energy(vel)
    # global stepping at the finest tick
    gp, gv = pos.clone(), vel.clone()
    g = crk.crk_create()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(cycles << L):
        crk.crk_step(g, gp, gv, mass, tick)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    g_ms = e0.elapsed_time(e1)
    g.close()
    rho_g, u_g = profiles(gp, gv)
    n = pos.shape[0]
    out = {"workload": "sedov-%d^3 after %d CFL steps, %d cycles of 2^%d ticks" % (side, warm_steps, cycles, L),
           "n": n, "L": L, "Delta": Delta, "tick": tick, "cycles": cycles,
           "global": {"ms": g_ms, "evaluations": n * (cycles << L), "energy_error": energy(gv) / E0 - 1.0},
           "f_l": {}}
    for f in f_ls:
        hp, hv = pos.clone(), vel.clone()
        c = crk.crk_create()
        ev = wk = un = ticks = 0
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(cycles):
            info = crk.crk_cycle(c, hp, hv, mass, Delta, L, f)
            ev += info["evaluations"]
            wk += info["wakeups"]
            un += info["unresolved"]
            ticks += info["ticks"]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        c.close()
        rho_h, u_h = profiles(hp, hv)
        out["f_l"][str(f)] = {
            "ms": ms, "speedup_vs_global": g_ms / ms, "evaluations": ev,
            "evaluation_fraction": ev / float(n * (cycles << L)), "ticks": ticks, "wakeups": wk, "unresolved": un,
            "energy_error": energy(hv) / E0 - 1.0,
            "L1_rho_vs_global": float(np.abs(rho_h - rho_g).sum() / np.abs(rho_g).sum()),
            "L1_u_vs_global": float(np.abs(u_h - u_g).sum() / np.abs(u_g).sum())}
    probe.close()
    return out


def sod_report(dev, sides=(64, 128, 256)):
    """Sod shock tube (the paper's Sec. 4 test, inputs.sod) to t = 0.075 (the
    paper's t = 0.15) at several resolutions: GPU time of each run, the
    one-dimensionality of the flow, and self-convergence: the L1 difference
    of each run's binned profiles (density, velocity, pressure, specific
    energy) over the isolated half from those of the finest run.  The L1
    against the exact Riemann solution is measured by the tests."""
    import numpy as np
    import torch
    from paper_2202_02840_gb300 import crk, inputs

    runs, parts = {}, {}
    for n in sides:
        st = inputs.sod(n)
        pos = torch.from_numpy(st["pos_h"]).to(dev)
        vel = torch.from_numpy(st["vel_u"]).to(dev)
        mass = torch.from_numpy(st["mass"]).to(dev)
        d = crk.crk_step(crk.crk_create(tile_order=1), pos.clone(), vel.clone(), mass, 0.0, diag=True)
        ctx = crk.crk_create(tile_order=1)
        t, dt_next, steps = 0.0, d["dt"], 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while t < st["t_end"] - 1e-12:
            d = crk.crk_step(ctx, pos, vel, mass, min(dt_next, st["t_end"] - t), diag=True)
            t += d["dt"]
            dt_next = d["dt_next"]
            steps += 1
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        probe = crk.crk_create()
        crk.crk_build_cells(probe, pos)
        V, _ = crk.crk_volumes(probe)
        p = pos.cpu().numpy().astype(np.float64)
        v = vel.cpu().numpy().astype(np.float64)
        rho = st["mass"].astype(np.float64) / V.cpu().numpy().astype(np.float64)
        P = (st["gamma"] - 1.0) * rho * v[:, 3]
        sel = p[:, 0] < 0.5
        parts[n] = (p[sel, 0], {q: a[sel] for q, a in (("rho", rho), ("v", v[:, 0]), ("P", P), ("u", v[:, 3]))})
        runs[n] = {"N": len(p), "N_x": "%d+%d" % (n // 4, n // 8), "steps": steps, "wall_s": wall,
                   "ms_per_step": 1e3 * wall / steps, "max_transverse_v": float(np.abs(v[:, 1:3]).max())}
        probe.close()
        ctx.close()
    # the finest run's profile: means over bins of its low-side lattice spacing, interpolated
    nf = max(sides)
    xf, qf = parts[nf]
    nb = nf // 4
    edges = np.linspace(0.0, 0.5, nb + 1)
    i = np.clip(np.digitize(xf, edges) - 1, 0, nb - 1)
    c = np.bincount(i, None, nb)
    mid = 0.5 * (edges[1:] + edges[:-1])[c > 0]
    ref = {q: (np.bincount(i, a, nb)[c > 0] / c[c > 0]) for q, a in qf.items()}
    for n in sides[:-1]:
        x, qs = parts[n]
        runs[n]["L1_vs_finest"] = {q: float(np.mean(np.abs(a - np.interp(x, mid, ref[q])))) for q, a in qs.items()}
    return {"workload": "Sod tube in the unit cube (interfaces at 1/4, 3/4; rho, P = 1 | 1/8), t = 0.075",
            "runs": {str(k): v for k, v in runs.items()}}


# --------------------------------------------------------------------- GPU arm

def aggregate(times_ms, work, dist=None, device="cpu"):
    """Whole-job numbers of a replicated run: the slowest rank's times (max)
    and the work of all ranks (sum).  Without a process group, the inputs."""
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    w = torch.tensor([float(x) for x in work], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()], [float(x) for x in w.cpu()]


# particle orders that cut the tiles: (tile_order, rcb_leaf); the bisection to
# one-tile leaves, and to the paper's leaf sizes N_ppl = 128, 256 (Sec. 2.3)
ORDERS = {"morton": (0, 32), "hilbert": (1, 32), "bisection": (2, 32), "bisection-128": (2, 128),
          "bisection-256": (2, 256)}
ORDER_ARGS = {"0": "morton", "1": "hilbert", "2": "bisection", "2-128": "bisection-128", "2-256": "bisection-256"}


def run_gpu(args):
    import torch
    import __graft_entry__
    from paper_2202_02840_gb300 import crk, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()

    st = inputs.zeldovich(args.n_side)
    n = st["pos_h"].shape[0]
    pos0 = torch.from_numpy(st["pos_h"]).to(dev)
    vel0 = torch.from_numpy(st["vel_u"]).to(dev)
    mass = torch.from_numpy(st["mass"]).to(dev)
    pos, vel = pos0.clone(), vel0.clone()
    stream = torch.cuda.current_stream(dev)
    # the clock sampler runs from here on (its start-up stays out of the timed
    # region; only its samples inside that region are kept), and about a
    # second of untimed steps on a throwaway context brings an idle GPU to its
    # working state before anything is timed
    clocks = Clocks(local)
    clocks.start()
    c = crk.crk_create(precision=args.precision, tile_order=1)
    p, v = pos0.clone(), vel0.clone()
    t_end = time.perf_counter() + 1.0
    while time.perf_counter() < t_end:
        crk.crk_step(c, p, v, mass, 0.0)
        torch.cuda.synchronize(dev)
    c.close()
    del p, v
    # tile order (Morton, Hilbert, bisection): given, or the fastest of two
    # timed steps each on a copy of the state (part of the warm-up)
    order_ms = {}
    if args.tile_order == "auto":
        for name, (t, leaf) in ORDERS.items():
            p, v = pos0.clone(), vel0.clone()
            c = crk.crk_create(precision=args.precision, tile_order=t, rcb_leaf=leaf)
            crk.crk_step(c, p, v, mass, 0.0)
            torch.cuda.synchronize(dev)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(2):
                crk.crk_step(c, p, v, mass, 0.0)
            t1.record(stream)
            torch.cuda.synchronize(dev)
            order_ms[name] = t0.elapsed_time(t1) / 2
            c.close()
        order_name = min(ORDERS, key=lambda k: order_ms[k])
    else:
        order_name = ORDER_ARGS[args.tile_order]
    order = {"tile_order": ORDERS[order_name][0], "rcb_leaf": ORDERS[order_name][1]}
    if args.pair_form is not None:
        order["pair_form"] = args.pair_form
    ctx = crk.crk_create(precision=args.precision, **order)
    pair_form = args.pair_form if args.pair_form is not None else crk.crk_default_params().pair_form

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- device-resident timing (the first warm-up step tunes the
    # passes, unless their variants are pinned)
    pins = parse_variants(args.variants)

    def prepare(c):
        for name, v in pins.items():
            crk.crk_tune_set(c, name, v)
        if not pins and not args.no_autotune:
            crk.crk_autotune(c, True)

    prepare(ctx)
    for _ in range(args.warmup):
        crk.crk_step(ctx, pos, vel, mass, 0.0)
    crk.crk_autotune(ctx, False)
    tuning = crk.crk_tuning(ctx)
    barrier()
    clocks.mark()
    crk.crk_profile(ctx, True)
    launches0 = crk.crk_launches(ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    pairs = 0
    ev0.record(stream)
    diags = []
    for _ in range(args.steps):
        d = crk.crk_step(ctx, pos, vel, mass, 0.0, diag=True)
        diags.append(d)
        pairs += 3 * d["pairs_gather"] + 3 * d["pairs_union"]
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = crk.crk_launches(ctx) - launches0
    prof_ms, prof_cnt, _ = crk.crk_profile_read(ctx)
    crk.crk_profile(ctx, False)
    clk = clocks.stop()
    ntiles, entries, utp = crk.crk_build_stats(ctx)
    walk_tests = crk.crk_walk_stats(ctx)   # lane tests of the last walk (one per step)
    ctx.close()

    # ---------------- end to end through host buffers (pinned), same step count
    h_pos = torch.from_numpy(st["pos_h"]).pin_memory()
    h_vel = torch.from_numpy(st["vel_u"]).pin_memory()
    h_mass = torch.from_numpy(st["mass"]).pin_memory()
    d_pos = torch.empty_like(pos0)
    d_vel = torch.empty_like(vel0)
    d_mass = torch.empty_like(mass)
    e2e_ctx = crk.crk_create(precision=args.precision, **order)
    prepare(e2e_ctx)   # tuned during its own warm-up, or pinned as ctx
    for _ in range(max(1, args.warmup)):
        d_pos.copy_(h_pos, non_blocking=True)
        d_vel.copy_(h_vel, non_blocking=True)
        d_mass.copy_(h_mass, non_blocking=True)
        crk.crk_step(e2e_ctx, d_pos, d_vel, d_mass, 0.0)
        h_pos.copy_(d_pos, non_blocking=True)
        h_vel.copy_(d_vel, non_blocking=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_pairs = 0
    e0.record(stream)
    for _ in range(args.steps):
        d_pos.copy_(h_pos, non_blocking=True)
        d_vel.copy_(h_vel, non_blocking=True)
        d_mass.copy_(h_mass, non_blocking=True)
        d = crk.crk_step(e2e_ctx, d_pos, d_vel, d_mass, 0.0, diag=True)
        e2e_pairs += 3 * d["pairs_gather"] + 3 * d["pairs_union"]
        h_pos.copy_(d_pos, non_blocking=True)
        h_vel.copy_(d_vel, non_blocking=True)
    e1.record(stream)
    barrier()
    crk.crk_autotune(e2e_ctx, False)
    e2e_ms = e0.elapsed_time(e1)

    # ---------------- the plain FP32 path (precision 0: no compensated sums,
    # FP32 moment formation) over the same warm-up and steps, for comparison
    plain = None
    if args.precision != 0 and world == 1:
        c0 = crk.crk_create(precision=0, **order)
        prepare(c0)
        p0, v0 = pos0.clone(), vel0.clone()
        for _ in range(args.warmup):
            crk.crk_step(c0, p0, v0, mass, 0.0)
        crk.crk_autotune(c0, False)
        barrier()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        plain_pairs = 0
        q0.record(stream)
        for _ in range(args.steps):
            d = crk.crk_step(c0, p0, v0, mass, 0.0, diag=True)
            plain_pairs += 3 * d["pairs_gather"] + 3 * d["pairs_union"]
        q1.record(stream)
        barrier()
        plain_ms = q0.elapsed_time(q1)
        c0.close()
        plain = {"precision": "plain", "ms_per_step": plain_ms / args.steps,
                 "value": plain_pairs / (plain_ms * 1e-3), "unit": UNIT}
    # the accuracy mode (precision 3: float-float moments) over the same warm-up
    # and steps, with its P2 time
    accurate = None
    if args.precision != 3 and world == 1 and not args.no_accuracy_mode:
        c3 = crk.crk_create(precision=3, **order)
        prepare(c3)
        p3, v3 = pos0.clone(), vel0.clone()
        for _ in range(args.warmup):
            crk.crk_step(c3, p3, v3, mass, 0.0)
        crk.crk_autotune(c3, False)
        crk.crk_profile(c3, True)
        barrier()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.steps):
            crk.crk_step(c3, p3, v3, mass, 0.0)
        q1.record(stream)
        barrier()
        pm3, _, _ = crk.crk_profile_read(c3)
        c3.close()
        accurate = {"precision": PRECISION_NAMES[3], "ms_per_step": q0.elapsed_time(q1) / args.steps,
                    "P2_ms_per_step": pm3["P2 corrections"] / args.steps}
    e2e_ctx.close()

    # ---------------- aggregate over ranks (max time, summed work)
    (ms_max, e2e_max), (w0, w1) = aggregate([ms, e2e_ms], [float(pairs), float(e2e_pairs)], dist, dev)
    value = w0 / (ms_max / 1e3)
    e2e_value = w1 / (e2e_max / 1e3)

    # ---------------- roofline of the dominant pass (pairs: mean over the timed steps)
    g_pairs = sum(d["pairs_gather"] for d in diags) / len(diags)
    u_pairs = sum(d["pairs_union"] for d in diags) / len(diags)
    per_step_pairs = {"P1 volumes": g_pairs, "P2 corrections": g_pairs, "P3 grad v": g_pairs,
                      "P4 forces": u_pairs / 2.0, "P5 compatible energy": u_pairs / 2.0}
    dominant = max(FLOPS_PER_UNIT, key=lambda k: prof_ms.get(k, 0.0))
    launch_ms = prof_ms[dominant] / max(1, prof_cnt[dominant])
    achieved = FLOPS_PER_UNIT[dominant] * per_step_pairs[dominant] / (launch_ms / 1e3) / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = alu_peak_tflops(sm_count, max_mhz)
    traffic = TRAFFIC_PER_UNIT.get(dominant)
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic * per_step_pairs[dominant] if traffic else None,
                "traffic_basis": "ncu DRAM bytes per unit on zeldovich-64^3, scaled by units" if traffic else None,
                "peak_basis": "FP32 FMA issue: %d SMs x 128 lanes x 2 flops x %.0f MHz (max SM clock)"
                              % (sm_count, max_mhz),
                "launch_ms": launch_ms,
                "pass_ms_per_step": {k: v / args.steps for k, v in prof_ms.items()}}
    # every list pass against its own bound: the FP32 ALU for the gather
    # passes and P4 (algorithmic flops per unit as above); P5 streams the
    # stored (F_ij, j) once per step for both kicks, 16 bytes per ordered
    # pair-set entry, against the measured HBM copy bandwidth
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pass_roofline = {}
    for k in ("P1 volumes", "P2 corrections", "P3 grad v", "P4 forces"):
        t = prof_ms.get(k, 0.0) / args.steps
        if t > 0:
            a = FLOPS_PER_UNIT[k] * per_step_pairs[k] / (t / 1e3) / 1e12
            pass_roofline[k] = {"bound": "alu", "ms_per_step": t, "achieved": a, "unit": "TFLOP/s",
                                "frac": a / peak}
    t5 = prof_ms.get("P5 compatible energy", 0.0) / args.steps
    if t5 > 0:
        a = 16.0 * u_pairs / (t5 / 1e3) / 1e9
        pass_roofline["P5 compatible energy"] = {"bound": "hbm", "ms_per_step": t5, "achieved": a, "unit": "GB/s",
                                                 "frac": a / hbm, "peak": hbm,
                                                 "bytes": "16 B per ordered pair-set entry, read once for two kicks"}
    # the cell build: keys (read pos_h 16 B; write fixed point 16, key 4, index 4,
    # h 4), four stable radix passes (histogram reads the 4-B key; the scatter
    # reads and writes key and index, 16 B), the gather into sorted order (read
    # index, fixed point, h: 24 B; write q4 16, h 4, perm 4, key 4), tile boxes
    # (read q4 16 B): 192 B per particle, against the measured HBM copy bandwidth
    tb = prof_ms.get("cell build", 0.0) / args.steps
    if tb > 0:
        a = BUILD_BYTES_PER_PARTICLE * n / (tb / 1e3) / 1e9
        pass_roofline["cell build"] = {"bound": "hbm", "ms_per_step": tb, "achieved": a, "unit": "GB/s",
                                       "frac": a / hbm, "peak": hbm,
                                       "bytes": "%d B per particle per rebuild (keys, 4 radix passes, gather, "
                                                "tile boxes)" % BUILD_BYTES_PER_PARTICLE}
    # the neighbour-list walk: integer work, WALK_INT_OPS 32-bit integer
    # operations per lane test of the exact predicate, lane tests counted by
    # the walk itself (crk_walk_stats; one walk per step), against the INT32
    # issue rate (64 lanes per SM per clock)
    tw = prof_ms.get("neighbour lists", 0.0) / args.steps
    tests = walk_tests
    if tw > 0 and tests > 0:
        a = WALK_INT_OPS * tests / (tw / 1e3) / 1e12
        pass_roofline["neighbour lists"] = {"bound": "alu", "ms_per_step": tw, "achieved": a, "unit": "Tops/s",
                                            "frac": a / INT32_PEAK_TOPS, "peak": INT32_PEAK_TOPS,
                                            "lane_tests_per_step": tests,
                                            "useful_fraction": u_pairs / tests,
                                            "ops": "%d INT32 ops per lane test (3 subtractions, 4 widening "
                                                   "products, two 64-bit sums and two 64-bit compares, 4 mask "
                                                   "updates)" % WALK_INT_OPS}
    roofline["passes"] = pass_roofline

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "precision": PRECISION_NAMES[args.precision],
                           "pair_form": ["directed", "pair-once"][pair_form],
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "step working set ~%.1f GB > L2 (129 MB): inputs larger than L2, no flush"
                                 % ((n * 460 + entries * 20) / 1e9),
                           "pairs_per_step": pairs / args.steps,
                           "pair_count": "per step: P1, P2, P3 over the gather pairs and P4 plus the two "
                                         "compatible-energy kicks over the ordered pair-set pairs (3 x gather + "
                                         "3 x pair set); both kicks' sums are formed in one pass over the stored "
                                         "pair forces",
                           "tiles": ntiles, "pair_candidate_tiles_per_tile": utp / max(1, ntiles),
                           "list_entries_per_particle": entries / n,
                           ("pinned_variants" if pins else "autotuned_variants"):
                               {k: v for k, (v, _) in tuning.items()} if not pins else pins,
                           "tile_order": order_name, "tile_order_step_ms": order_ms or None,
                           "gather_pairs_per_particle": diags[-1]["pairs_gather"] / n,
                           "union_pairs_per_particle": diags[-1]["pairs_union"] / n},
                "roofline": roofline,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 36,
                        "d2h_bytes_per_step": n * 32},
                "gpu_launches": launches, "clocks": clk}
        if plain is not None:
            plain["step_ms_ratio_to_this"] = plain["ms_per_step"] / (ms_max / args.steps)
            line["plain_fp32"] = plain
        if accurate is not None:
            accurate["step_ms_ratio_to_this"] = accurate["ms_per_step"] / (ms_max / args.steps)
            line["accuracy_mode"] = accurate
        if not args.no_learned_h and world == 1:
            line["learned_h"] = learned_h_report(dev, eval_side=args.learned_h_eval_side)
        if not args.no_batched and world == 1:
            line["batched"] = batched_report(dev)
        if not args.no_time_bins and world == 1:
            line["time_bins"] = time_bins_report(dev)
        if not args.no_sod and world == 1:
            line["sod"] = sod_report(dev)
        finals = None
        if not args.no_ai_step and world == 1:
            line["ai_step"], finals = ai_step_report(dev, st, order)
        if not args.no_cpu_baseline and world == 1:
            from oracle import crk as O
            p, dt, ns = calibrated_oracle(st, args.cpu_seconds, seed=2)
            line["cpu_baseline"] = {"value": p / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                                    "sample": "FP64 oracle passes P1,P2,P3,P4,P5,P5 on %d random target "
                                              "particles of the workload (%.1f s)" % (ns, dt)}
            # the stated error of this mode and of the plain FP32 path
            try:
                line["err"] = sampled_errors(st, dev, order, sorted({0, args.precision, 3}))
                if finals is not None:
                    line["err"]["eq_hi"] = eq_hi_check(finals, line["ai_step"]["comparison"]["h_tol"])
            except Exception as e:   # the measurement line is printed regardless
                line["err"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


VARIANT_PASSES = {"P1": "P1 volumes", "P2": "P2 corrections", "P3": "P3 grad v", "P4": "P4 forces",
                  "P5": "P5 compatible energy"}


def parse_variants(spec):
    """'P1=20,P4=8' -> {'P1 volumes': 20, 'P4 forces': 8}."""
    out = {}
    for item in filter(None, (x.strip() for x in spec.split(","))):
        k, v = item.split("=")
        out[VARIANT_PASSES[k.strip()]] = int(v)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-side", type=int, default=128)
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2, 3])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-learned-h", action="store_true", help="skip the learned-h training and evaluation")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-boxes measurement")
    ap.add_argument("--no-time-bins", action="store_true", help="skip the hierarchical time-bin measurement")
    ap.add_argument("--no-sod", action="store_true", help="skip the Sod shock-tube measurement")
    ap.add_argument("--no-accuracy-mode", action="store_true", help="skip timing precision 3")
    ap.add_argument("--learned-h-eval-side", type=int, default=256,
                    help="side of the Sedov state the learned-h report evaluates at (256: config 4)")
    ap.add_argument("--no-ai-step", action="store_true",
                    help="skip the steps that solve eq:hi (plain FP32 from h vs learned proposal)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in pass variants")
    ap.add_argument("--pair-form", type=int, default=None, choices=[0, 1],
                    help="P4/P5 over the pair set: 0 directed (each ordered pair from its i side), "
                         "1 pair-once (each unordered pair once); default: the library's")
    ap.add_argument("--variants", default="",
                    help="pin list-pass variants instead of tuning them (numbering of crk_tuning), "
                         "e.g. P1=20,P2=16,P3=9,P4=8,P5=9")
    ap.add_argument("--tile-order", default="auto", choices=["auto"] + list(ORDER_ARGS),
                    help="particle order of the tiles: 0 Morton, 1 Hilbert, 2 bisection to one-tile leaves, "
                         "2-128 / 2-256 bisection to leaves of 128 / 256 particles, auto = fastest")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
