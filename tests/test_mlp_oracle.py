"""Pins of the surrogate's CPU reference (features and network), CPU only.

The surrogate is this project's addition (the paper has no network); its
reference is pinned by: brute-force rounding to bfloat16, finite differences
of the float64 network, a hand-set network with a known output, the first
Adam step's closed form, and feature invariants tied to the pinned RBSM
oracle (the centre bit is the shadow test, the four neighbour bits give the
discontinuity directions).
"""
import numpy as np
import pytest

from oracle import mlp
from oracle import rbsm as orc
from rbsm_scenes import shapes


def test_bf16_round_is_nearest_even():
    rng = np.random.default_rng(0)
    f = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 20000),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 65504.0, 3.0e38], np.float32)])
    f = f.astype(np.float32)
    got = mlp.bf16_round(f)
    # independent: the two bfloat16 neighbours by truncation, pick the nearer,
    # ties to the one with an even last mantissa bit
    u = f.view(np.uint32)
    lo = (u & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi_bits = (u & np.uint32(0xFFFF0000)) + np.uint32(0x10000)
    hi = hi_bits.view(np.float32).astype(np.float64)
    x = f.astype(np.float64)
    dlo, dhi = np.abs(x - lo), np.abs(hi - x)
    lo_even = ((u >> 16) & 1) == 0
    want = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo_even, lo, hi)))
    assert np.array_equal(got, want)
    assert mlp.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6
    assert np.isinf(mlp.bf16_round(np.float32(np.inf)))


def _params(rng, scale=0.5):
    return {"W1": rng.standard_normal((32, 64)) * scale, "b1": rng.standard_normal(64) * 0.1,
            "W2": rng.standard_normal((64, 64)) * scale / 4, "b2": rng.standard_normal(64) * 0.1,
            "W3": rng.standard_normal((64, 2)) * scale / 4, "b3": rng.standard_normal(2) * 0.1}


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    P = _params(rng)
    X = rng.standard_normal((9, 32))
    t = rng.uniform(0, 1, 9)
    _, G = mlp.loss_and_grads(P, X, t, bf16=False)
    y0, _ = mlp.forward(P, X, bf16=False)
    e_target = np.abs(np.clip(y0[:, 0], 0, 1) - t)      # held constant, as in the loss

    def loss(Q):
        y, _ = mlp.forward(Q, X, bf16=False)
        return np.sum((y[:, 0] - t) ** 2) / 9 + np.sum((y[:, 1] - e_target) ** 2) / 9

    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            Q = {kk: vv.copy() for kk, vv in P.items()}
            Q[k].reshape(-1)[idx] += h
            up = loss(Q)
            Q[k].reshape(-1)[idx] -= 2 * h
            dn = loss(Q)
            fd = (up - dn) / (2 * h)
            an = G[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_hand_set_network_selects_fx():
    """W1 copies fx into hidden unit 0, W2 and W3 pass it on: y0 = fx."""
    P = {"W1": np.zeros((32, 64)), "b1": np.zeros(64), "W2": np.zeros((64, 64)), "b2": np.zeros(64),
         "W3": np.zeros((64, 2)), "b3": np.array([0.0, 0.25])}
    P["W1"][25, 0] = 1.0
    P["W2"][0, 0] = 1.0
    P["W3"][0, 0] = 1.0
    X = np.zeros((5, 32))
    X[:, 25] = [0.0, 0.125, 0.5, 0.75, 0.96875]
    for bf16 in (False, True):
        y, _ = mlp.forward(P, X, bf16=bf16)
        assert np.array_equal(y[:, 0], X[:, 25]) and np.all(y[:, 1] == 0.25)


def test_first_adam_step_moves_by_lr_sign():
    """After one step m_hat = g and v_hat = g^2, so each weight moves by
    lr * g / (|g| + eps): lr times the sign of its gradient."""
    rng = np.random.default_rng(2)
    P = _params(rng)
    P0 = {k: v.copy() for k, v in P.items()}
    G = {k: rng.standard_normal(v.shape) for k, v in P.items()}
    G = {k: np.where(np.abs(g) < 0.1, 0.1 * np.sign(g) + (g == 0) * 0.1, g) for k, g in G.items()}
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    mlp.adam_step(P, G, M, V, 1, 1e-3)
    for k in P:
        assert np.allclose(P[k], P0[k] - 1e-3 * np.sign(G[k]), rtol=0, atol=1e-9)


def test_encode_puts_each_feature_in_its_column():
    bits = np.array([1 << k for k in range(25)] + [0, (1 << 25) - 1], np.uint32)
    n = bits.size
    feat = {"bits": bits, "fx": np.full(n, 0.25, np.float32), "fy": np.full(n, 0.5, np.float32),
            "gap": np.full(n, -0.125, np.float32)}
    X = mlp.encode(feat)
    assert np.array_equal(X[:25, :25], np.eye(25))
    assert np.all(X[25, :25] == 0) and np.all(X[26, :25] == 1)
    assert np.all(X[:, 25] == 0.25) and np.all(X[:, 26] == 0.5) and np.all(X[:, 27] == -0.125)
    assert np.all(X[:, 28:] == 0)


def test_feature_pattern_invariants():
    """Centre bit = shadow test; neighbour bits give the discontinuity
    directions of the pinned oracle; an occluder texel clears exactly its bit;
    clamping repeats the edge texel; gap = depth - nearest blocker."""
    rng = np.random.default_rng(3)
    n = 24
    lv = np.array([0.25, 0.5, 1.0], np.float32)
    depth = lv[rng.integers(0, 3, (n, n))]
    X = rng.integers(0, n, 3000) + (rng.integers(0, 8, 3000) + 0.5) / 8
    Y = rng.integers(0, n, 3000) + (rng.integers(0, 8, 3000) + 0.5) / 8
    x, y = shapes.to_texcoords(X, Y, n, n)
    z = lv[rng.integers(0, 3, 3000)]
    f = orc.features(depth, x, y, z)
    r = orc.evaluate(depth, x, y, z, orc.MODE_FILTER)
    b = f["bits"]
    bit = lambda k: ((b >> k) & 1).astype(np.uint16)
    assert np.array_equal(1 - bit(12), (r["codes"] >> 4) & 1)
    d4 = (bit(11) != bit(12)) | ((bit(13) != bit(12)) << 1) | ((bit(17) != bit(12)) << 2) | ((bit(7) != bit(12)) << 3)
    assert np.array_equal(d4.astype(np.uint16), r["codes"] & 0xF)
    i, j = np.floor(X).astype(int), np.floor(Y).astype(int)
    win_min = np.array([depth[np.clip(jj + np.arange(-2, 3), 0, n - 1)][:, np.clip(ii + np.arange(-2, 3), 0, n - 1)].min()
                        for ii, jj in zip(i, j)], np.float32)
    assert np.array_equal(f["gap"], z - win_min)
    assert np.array_equal(f["fx"], (X - i).astype(np.float32)) and np.array_equal(f["fy"], (Y - j).astype(np.float32))
    # one occluder texel at (10 + dx, 10 + dy) clears exactly bit (dy+2)*5 + dx+2
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            d = np.ones((n, n), np.float32)
            d[10 + dy, 10 + dx] = 0.5
            xs, ys = shapes.to_texcoords(np.array([10.5]), np.array([10.5]), n, n)
            g = orc.features(d, xs, ys, np.ones(1, np.float32))
            assert g["bits"][0] == ((1 << 25) - 1) ^ (1 << ((dy + 2) * 5 + dx + 2))
            assert g["gap"][0] == np.float32(0.5)
    # at the corner texel, clamping repeats row 0 / column 0
    d = np.ones((n, n), np.float32)
    d[0, 0] = 0.5
    xs, ys = shapes.to_texcoords(np.array([0.5]), np.array([0.5]), n, n)
    g = orc.features(d, xs, ys, np.ones(1, np.float32))["bits"][0]
    cleared = [(dy + 2) * 5 + dx + 2 for dx in (-2, -1, 0) for dy in (-2, -1, 0)]
    assert g == ((1 << 25) - 1) ^ sum(1 << k for k in cleared)
