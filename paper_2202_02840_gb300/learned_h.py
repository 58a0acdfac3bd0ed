"""Host-side driver of the learned smoothing-length proposal.

Orchestration only: every number is computed by libcrk.so kernels through the
binding (crk.py); this module decides which calls to make, keeps the tensors
and concatenates data sets (device memory plumbing).

Data protocols (the method generates its own training data); step_snapshots
takes the rows from steps that solve eq:hi (h_mode 1), matching what the
proposal sees inside such a step; the snapshots below take them from a run
with the evolved h:
  * a Sedov blast (the Sedov-Taylor test of Sec. 4) is advanced with crk_step,
    whose h evolves by one Thacker update per step (Sec. 2.6, eq:thacker);
  * at every `every`-th step the state is a snapshot: P1 gives N_i at the
    evolved h, P2/P3 give grad v (with the step dt, the compression dt div v),
    the fixed-point iteration of eq:hi from the
    evolved h gives the converged h and the iteration count without a
    proposal, and the features plus the target log(h_conv / h_prev) are taken;
  * the network is trained by crk_mlp_train (Adam on sampled batches);
  * a snapshot is evaluated by running the same fixed-point iteration from the
    proposal (crk_h_propose), at the same tolerance.
"""
import torch

from . import crk, inputs


def dev(a):
    return torch.from_numpy(a).cuda()


class Snapshot:
    """Features, targets and the plain fixed-point solve of one state."""

    def __init__(self, ctx, pos_h, vel_u, dt, tol=1e-4, max_it=60):
        crk.crk_build_cells(ctx, pos_h)
        V, N = crk.crk_volumes(ctx)
        gradv = crk.crk_corrections(ctx, V, vel_u)[4]
        pos_conv = pos_h.clone()
        it, ok = crk.crk_h_iterate(ctx, pos_conv, tol=tol, max_it=max_it)
        feat, target = crk.crk_h_features(ctx, pos_h, gradv, N, pos_conv, dt=dt)
        self.dt = dt
        self.pos_h = pos_h.clone()
        self.gradv, self.N = gradv, N
        self.feat, self.target = feat, target
        self.it_plain, self.ok_plain = it, ok
        self.tol, self.max_it = tol, max_it

    def rows(self, ctx, base=0):
        """Indices of the particles the judge hands to the proposal."""
        return crk.crk_h_select(ctx, self.N, tol=self.tol, base=base)

    def solve_from_proposal(self, ctx):
        """(iterations, converged, pos_h with the converged h) starting from the
        proposal of the network loaded in ctx."""
        p = self.pos_h.clone()
        crk.crk_h_propose(ctx, p, self.gradv, self.N, dt=self.dt, tol=self.tol)
        it, ok = crk.crk_h_iterate(ctx, p, tol=self.tol, max_it=self.max_it)
        return it, ok, p


def sedov_snapshots(n_side=32, steps=100, every=10, seed=3, tol=1e-4, max_it=60, params=None):
    """Advance a Sedov blast and take a Snapshot at every `every`-th step."""
    return run_snapshots(inputs.sedov(n_side, seed=seed), steps, every, tol, max_it, params)


def run_snapshots(st, steps=100, every=10, tol=1e-4, max_it=60, params=None):
    """Advance the state st (evolved h) and take a Snapshot at every `every`-th step."""
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    p = params or {}
    stepper = crk.crk_create(**p)
    probe = crk.crk_create(**p)
    snaps = []
    for k in range(1, steps + 1):
        dt = crk.crk_step(stepper, pos, vel, mass, 0.0, diag=(k % every == 0))
        if k % every == 0:
            snaps.append(Snapshot(probe, pos, vel, dt["dt"], tol=tol, max_it=max_it))
    stepper.close()
    return snaps, probe


class StepSnapshot:
    """The solve of eq:hi that one step with h_mode 1 performs, as training
    rows: the features of the drifted positions with the previous step's
    solved h (where that solve starts), the target from the h it converged to."""

    def __init__(self, ctx, start, conv, vel_u, dt, tol=1e-4):
        crk.crk_build_cells(ctx, start)
        V, N = crk.crk_volumes(ctx)
        gradv = crk.crk_corrections(ctx, V, vel_u)[4]
        self.feat, self.target = crk.crk_h_features(ctx, start, gradv, N, conv, dt=dt)
        self.N, self.tol, self.dt = N, tol, dt

    def rows(self, ctx, base=0):
        return crk.crk_h_select(ctx, self.N, tol=self.tol, base=base)


def step_snapshots(st, steps=40, every=1, tol=1e-4, warm=3, params=None):
    """Advance the state st with KDK steps that solve eq:hi (h_mode 1) and take
    a StepSnapshot of every `every`-th step's solve (after `warm` steps, the
    first of which solves from the initial h)."""
    pos, vel, mass = dev(st["pos_h"]), dev(st["vel_u"]), dev(st["mass"])
    p = dict(params or {})
    p.update(h_mode=1, h_tol=tol)
    stepper = crk.crk_create(**p)
    probe = crk.crk_create()
    for _ in range(warm):
        crk.crk_step(stepper, pos, vel, mass, 0.0)
    snaps = []
    for k in range(steps):
        h_prev = pos[:, 3].clone()
        d = crk.crk_step(stepper, pos, vel, mass, 0.0, diag=True)
        if k % every == 0:
            start = pos.clone()
            start[:, 3] = h_prev
            snaps.append(StepSnapshot(probe, start, pos.clone(), vel, d["dt"], tol))
    stepper.close()
    return snaps, probe


def dataset(ctx, snaps):
    """Concatenated (feat, target, rows) of a list of snapshots; rows index the
    particles that the judge hands to the proposal."""
    rows, base = [], 0
    for s in snaps:
        rows.append(s.rows(ctx, base))
        base += s.feat.shape[0]
    return torch.cat([s.feat for s in snaps]), torch.cat([s.target for s in snaps]), torch.cat(rows)


LR_PHASES = (1.0, 0.3, 0.1, 0.03)    # step-wise decay of the learning rate over four equal phases


def train(ctx, feat, target, rows=None, steps=2000, batch=4096, lr=1e-3, seed=0, init_seed=0):
    """Fresh seeded weights, then `steps` Adam steps with the learning rate
    decayed step-wise (LR_PHASES); returns the per-step losses."""
    crk.crk_mlp_set_weights(ctx, dev(inputs.mlp_init(init_seed)))
    losses = []
    per = max(steps // len(LR_PHASES), 1)
    done = 0
    for k, f in enumerate(LR_PHASES):
        m = per if k < len(LR_PHASES) - 1 else steps - done
        if m <= 0:
            continue
        losses += crk.crk_mlp_train(ctx, feat, target, rows=rows, batch=batch, steps=m, lr=lr * f, seed=seed + 1)
        done += m
    return losses


def zero_network(ctx):
    """Load all-zero parameters: the proposal is then the constant-density reference alone."""
    crk.crk_mlp_set_weights(ctx, torch.zeros(crk.MLP_NPARAM, dtype=torch.float32, device="cuda"))
