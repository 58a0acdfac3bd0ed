"""Pins of the FP64 oracle of the learned smoothing-length proposal.

Each check rests on something other than the oracle's own formulas: finite
differences of the forward map for the hand-written backward pass, special
weight settings that reduce the network to a known scalar function (which fix
the packing order and every transpose), closed-form cell counts on a perfect
lattice, a pairwise brute-force count for the feature binning, and PyTorch's
bfloat16 conversion for the rounding helper.
"""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import crk as O
from paper_2202_02840_gb300 import inputs


def _rand_w(seed=3, scale=1.0):
    r = np.random.default_rng(seed)
    return r.normal(0, scale, M.N_PARAM) * np.concatenate([
        np.full(512, 1 / np.sqrt(8)), np.full(64, 0.3), np.full(4096, 1 / 8), np.full(64, 0.3),
        np.full(64, 1 / 8), [0.3]])


def test_parameter_count_and_packing():
    assert M.N_PARAM == 4801
    w = np.arange(M.N_PARAM, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = M.unpack(w)
    assert W1.shape == (64, 8) and W2.shape == (64, 64) and W3.shape == (64,)
    assert W1[0, 1] == 1 and b1[0] == 512 and W2[0, 0] == 576 and b2[0] == 4672
    assert W3[0] == 4736 and b3 == 4800


def test_silu_special_values():
    z = np.array([0.0, 40.0, -40.0, 1.0])
    s = M.silu(z)
    assert s[0] == 0.0
    assert abs(s[1] - 40.0) < 1e-12 and abs(s[2]) < 1e-15
    assert abs(s[3] - 1.0 / (1.0 + np.exp(-1.0))) < 1e-15
    # derivative: zero crossing of silu' near z = -1.2785 (the silu minimum)
    zs = -1.27846454276107
    assert abs(M.dsilu(np.array([zs]))[0]) < 1e-12


def test_single_path_network_is_double_silu():
    """Only W1[3,5], W2[7,3], W3[7] set: y = s_y (2 silu(silu(x5)) + b3)."""
    w = np.zeros(M.N_PARAM)
    W1, b1, W2, b2, W3, _ = M.unpack(w)   # views into w
    W1[3, 5] = 1.0
    W2[7, 3] = 1.0
    W3[7] = 2.0
    w[-1] = 0.25
    x = np.zeros((5, 8))
    x[:, 5] = [-3.0, -0.5, 0.0, 0.7, 4.0]
    x[:, 2] = 9.0     # other inputs do not reach the output
    y, _ = M.forward(w, x)
    sig = lambda v: 1.0 / (1.0 + np.exp(-v))
    a = x[:, 5] * sig(x[:, 5])
    expect = (2.0 * a * sig(a) + 0.25) / 64.0
    np.testing.assert_allclose(y, expect, rtol=1e-14, atol=1e-15)


def test_zero_first_layer_makes_output_input_independent():
    w = _rand_w()
    w[:512] = 0.0
    x = np.random.default_rng(0).normal(0, 2, (7, 8))
    y, _ = M.forward(w, x)
    assert np.ptp(y) < 1e-14


def test_backward_matches_central_differences():
    """Hand-written backpropagation against FP64 central differences of the loss."""
    w = _rand_w(seed=5)
    r = np.random.default_rng(6)
    x = r.normal(0, 1, (9, 8))
    t = r.normal(0, 0.5, 9)
    L, g = M.loss_and_grad(w, x, t)
    assert np.isfinite(L) and L > 0
    idx = np.concatenate([r.choice(512, 24, replace=False), 512 + np.arange(0, 64, 9),
                          576 + r.choice(4096, 40, replace=False), 4672 + np.arange(0, 64, 7),
                          4736 + np.arange(0, 64, 5), [4800]])
    d = 1e-6
    for k in idx:
        wp = w.copy(); wp[k] += d
        wm = w.copy(); wm[k] -= d
        Lp, _ = M.loss_and_grad(wp, x, t)
        Lm, _ = M.loss_and_grad(wm, x, t)
        fd = (Lp - Lm) / (2 * d)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_loss_is_zero_at_target_and_gradient_vanishes():
    w = _rand_w(seed=8)
    x = np.random.default_rng(9).normal(0, 1, (6, 8))
    y, _ = M.forward(w, x)
    L, g = M.loss_and_grad(w, x, y)
    assert L == 0.0 and not np.any(g)


def test_declared_precision_network():
    """rnd = identity is the FP64 network; rnd = bf16_round stays within the
    first-order bound of rounding every hidden activation by half a BF16 ulp."""
    w = M.round_weights(_rand_w(seed=4))
    x = M.bf16_round(np.random.default_rng(5).normal(0, 1.5, (200, 8)))
    y, (z1, a1, z2, a2) = M.forward(w, x)
    yi, _ = M.forward(w, x, rnd=lambda a: a)
    np.testing.assert_array_equal(y, yi)
    yb, _ = M.forward(w, x, rnd=M.bf16_round)
    W1, b1, W2, b2, W3, b3 = M.unpack(w)
    u = 2.0 ** -9
    bound = M.Y_SCALE * (u * np.abs(a2) + 1.1 * (u * np.abs(a1)) @ np.abs(W2).T) @ np.abs(W3)
    assert np.all(np.abs(yb - y) <= 1.01 * bound + 1e-15)
    assert np.any(yb != y)
    # weight rounding leaves the biases and rounds every matrix entry
    w0 = _rand_w(seed=4)
    assert np.array_equal(w[512:576], w0[512:576]) and w[4800] == w0[4800]
    assert np.array_equal(w[576:4672], M.bf16_round(w0[576:4672]))
    # the rounded-delta gradient differs from the FP64 one by BF16-level amounts only
    t = np.random.default_rng(6).normal(0, 0.3, 200)
    _, g = M.loss_and_grad(w, x, t)
    _, gb = M.loss_and_grad(w, x, t, rnd=M.bf16_round)
    assert 0 < np.linalg.norm(gb - g) <= 2e-2 * np.linalg.norm(g)


def test_grid_level():
    assert M.grid_level(16 ** 3) == 2
    assert M.grid_level(64 ** 3) == 4
    assert M.grid_level(128 ** 3) == 5
    assert M.grid_level(256 ** 3) == 6
    for n in (1000, 4096, 30000, 262144, 2097152):
        k = M.grid_level(n)
        assert 64 * 8 ** k <= n and (k == 7 or 64 * 8 ** (k + 1) > n)
        assert 2.0 ** -k >= 4 * n ** (-1 / 3) * (1 - 1e-12)


@pytest.mark.parametrize("side,kf", [(16, 2), (16, 1), (12, 2)])
def test_lattice_features_closed_form(side, kf):
    """m = (side / 2^kf)^3 particles per cell: counts 1, 6, 12, 8, 27 times m."""
    n = side ** 3
    pos = inputs.lattice(side)
    nh = 4.0 if side >= 16 else 3.0      # h < 1/3 of the box
    h = nh / side
    ph = np.concatenate([pos, np.full((n, 1), h)], 1).astype(np.float32)
    m = n / 8 ** kf
    divv = np.full(n, 0.5)
    f = M.features(ph, N_prev=np.full(n, 268.0), divv=divv, dt=0.125, kf=kf, N_res=268.0)
    np.testing.assert_allclose(f[:, 0], np.log1p(m))
    np.testing.assert_allclose(f[:, 1], np.log1p(6 * m))
    np.testing.assert_allclose(f[:, 2], np.log1p(12 * m))
    np.testing.assert_allclose(f[:, 3], np.log1p(8 * m))
    np.testing.assert_allclose(f[:, 4], np.log1p(27 * m))
    np.testing.assert_allclose(f[:, 5], np.log(nh), rtol=1e-6)
    np.testing.assert_allclose(f[:, 6], 0.5 * 0.125, rtol=1e-15)
    assert not np.any(f[:, 7])


def test_features_match_pairwise_cell_count():
    """Brute force: classify every ordered pair by the periodic cell offset."""
    r = np.random.default_rng(12)
    n = 300
    kf = 3
    g = 8
    pos = inputs._to_unit_f32(r.uniform(0, 1, (n, 3))).astype(np.float32)
    ph = np.concatenate([pos, np.full((n, 1), 0.05, np.float32)], 1)
    f = M.features(ph, kf=kf)
    q, _ = O.fixed_point(ph)
    cell = [tuple(int(v) >> (32 - kf) for v in q[i, :3]) for i in range(n)]
    for i in range(0, n, 7):
        cls = [0, 0, 0, 0]
        for j in range(n):
            d = [((cell[j][a] - cell[i][a] + 1) % g) - 1 for a in range(3)]
            if all(-1 <= v <= 1 for v in d):
                cls[sum(abs(v) for v in d)] += 1
        np.testing.assert_allclose(f[i, :4], np.log1p(cls), rtol=1e-14)
        np.testing.assert_allclose(f[i, 4], np.log1p(sum(cls)), rtol=1e-14)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.7182817, 3.0e-39, 65504.0, 1e30], np.float32)
    v = np.concatenate([v, np.random.default_rng(1).normal(0, 10, 1000).astype(np.float32)])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(M.bf16_round(v), ref)
    assert M.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert M.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
