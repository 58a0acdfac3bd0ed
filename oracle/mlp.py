"""FP64 oracle of the learned smoothing-length proposal (TEST INFRASTRUCTURE ONLY).

The paper evolves h with one Thacker update per step (Sec. 2.6, eq:thacker)
and notes that solving eq:hi iteratively is the alternative; the learned part
proposes a starting h for that fixed-point iteration.  Definitions (the same
readings as the CUDA path, written independently here):

features (8 per particle), cells of the grid level kf = the largest k in
[1, 7] with 2^-k >= 4 N^(-1/3) (64 * 8^k <= N), cell of a particle = top kf bits of each
fixed-point coordinate, counts over the periodic grid (an offset that wraps
onto the same cell counts again):
  f0 log1p(own cell)      f1 log1p(6 face cells)   f2 log1p(12 edge cells)
  f3 log1p(8 corner cells) f4 log1p(all 27)        f5 log(h_prev / N^(-1/3))
  f6 dt * div v            f7 log(N_prev / N_res)
(f6 is the compression h div v made dimensionless by the step, (dt / h) h div v:
h div v itself carries the flow's velocity scale, which grows with resolution
in the Sedov runs, and does not transfer from one resolution to another)
network: y = s_y (W3 . silu(W2 silu(W1 x + b1) + b2) + b3), silu(z) = z sigmoid(z),
s_y = 2^-6 a fixed output scale (log-h corrections are of order 1%, which
keeps the network's own outputs of order one), W1 64x8, W2 64x64, W3 64,
packed as [W1, b1, W2, b2, W3, b3] (4801 values); proposal h = h_ref exp(y),
h_ref = h_prev (N_res / N_prev)^(1/3) (the constant-density solution of
eq:hi; h_prev without N_prev); target log(h_conv / h_ref); loss mean (y - t)^2.
Declared arithmetic of the tensor-core path (forward/loss_and_grad with
rnd=bf16_round, round_weights(w), bf16_round(x)): BF16 weight matrices,
features and hidden activations, BF16 deltas into the weight-gradient
products, every sum in FP64 here (FP32 on the GPU), FP32 biases.
"""
import numpy as np

from . import crk as O

N_PARAM = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1
Y_SCALE = 2.0 ** -6


def grid_level(n):
    """Largest k in [1, 7] with 2^-k >= 4 n^(-1/3), i.e. 64 * 8^k <= n (exact in integers)."""
    k = 1
    while k < 7 and 64 * 8 ** (k + 1) <= int(n):
        k += 1
    return k


def unpack(w):
    w = np.asarray(w, np.float64)
    o = 0
    W1 = w[o:o + 512].reshape(64, 8); o += 512
    b1 = w[o:o + 64]; o += 64
    W2 = w[o:o + 4096].reshape(64, 64); o += 4096
    b2 = w[o:o + 64]; o += 64
    W3 = w[o:o + 64]; o += 64
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def features(pos_h, N_prev=None, divv=None, dt=0.0, kf=None, N_res=268.0):
    pos = np.asarray(pos_h, np.float32).reshape(-1, 4)
    n = pos.shape[0]
    kf = grid_level(n) if kf is None else kf
    q, _ = O.fixed_point(pos)
    c = (q >> np.uint32(32 - kf)).astype(np.int64)
    g = 1 << kf
    cid = (c[:, 2] * g + c[:, 1]) * g + c[:, 0]
    counts = np.bincount(cid, minlength=g ** 3).astype(np.float64)
    own = np.zeros(n); face = np.zeros(n); edge = np.zeros(n); corner = np.zeros(n)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                m = abs(dx) + abs(dy) + abs(dz)
                cc = ((c[:, 2] + dz) % g * g + (c[:, 1] + dy) % g) * g + (c[:, 0] + dx) % g
                v = counts[cc]
                if m == 0:
                    own += v
                elif m == 1:
                    face += v
                elif m == 2:
                    edge += v
                else:
                    corner += v
    h = pos[:, 3].astype(np.float64)
    f = np.empty((n, 8))
    f[:, 0] = np.log1p(own)
    f[:, 1] = np.log1p(face)
    f[:, 2] = np.log1p(edge)
    f[:, 3] = np.log1p(corner)
    f[:, 4] = np.log1p(own + face + edge + corner)
    f[:, 5] = np.log(h * float(n) ** (1.0 / 3.0))
    f[:, 6] = 0.0 if divv is None else float(dt) * np.asarray(divv, np.float64)
    f[:, 7] = 0.0 if N_prev is None else np.log(np.asarray(N_prev, np.float64) / N_res)
    return f


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _ident(a):
    return a


def forward(w, x, rnd=None):
    """FP64 forward: returns y and the intermediates (z1, a1, z2, a2).

    rnd (optional) rounds each hidden activation where the declared arithmetic
    stores it: bf16_round gives the BF16-activation network that the
    tensor-core path computes (with round_weights(w) and bf16_round(x))."""
    r = _ident if rnd is None else rnd
    W1, b1, W2, b2, W3, b3 = unpack(w)
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    a1 = np.asarray(r(silu(z1)), np.float64)
    z2 = a1 @ W2.T + b2
    a2 = np.asarray(r(silu(z2)), np.float64)
    y = Y_SCALE * (a2 @ W3 + b3)
    return y, (z1, a1, z2, a2)


def loss_and_grad(w, x, t, rnd=None):
    """Mean squared error and its gradient by hand-written backpropagation.

    With rnd, the activations of the forward pass and the two back-propagated
    deltas that enter matrix products (dL/dz2, dL/dz1) are rounded where the
    declared arithmetic stores them; bias gradients take the unrounded deltas."""
    r = _ident if rnd is None else rnd
    W1, b1, W2, b2, W3, b3 = unpack(w)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    y, (z1, a1, z2, a2) = forward(w, x, rnd)
    B = x.shape[0]
    res = y - t
    L = float(np.mean(res * res))
    dy = Y_SCALE * 2.0 * res / B
    gW3 = a2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * dsilu(z2)
    gb2 = dz2.sum(0)
    dz2 = np.asarray(r(dz2), np.float64)
    gW2 = dz2.T @ a1
    dz1 = (dz2 @ W2) * dsilu(z1)
    gb1 = dz1.sum(0)
    dz1 = np.asarray(r(dz1), np.float64)
    gW1 = dz1.T @ x
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return L, g


def round_weights(w):
    """The declared weight precision: W1, W2, W3 rounded to BF16, biases kept."""
    w = np.asarray(w, np.float64).copy()
    for a, b in ((0, 512), (576, 4672), (4736, 4800)):
        w[a:b] = bf16_round(w[a:b])
    return w


def bf16_round(a):
    """Round FP32 values to bfloat16 (nearest-even) and back, as the GPU stores them."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))
