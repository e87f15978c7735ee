"""CPU checks of the element-wise bounds the surrogate's GPU tests use.

A float32 restatement of the tensor-core kernels' arithmetic (BF16 operands
and activations, FP32 sums in another order: numpy's float32 products, and
128-sample tiles added in sequence) must stay within the bounds of
tests/mlp_bounds.py, and the bounds must be tight enough that the slips a
tiled tensor-core kernel can make (a dropped K step of 16 samples, one 8 x 8
core matrix transposed, a tile's rows paired off by one sample, a ReLU mask
bit ignored) break them.  Nothing here needs a GPU.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from tests import mlp_bounds as mb

B = 4096
f32 = np.float32


@pytest.fixture(scope="module")
def case():
    import rbsm_scenes as sc
    rng = np.random.Generator(np.random.PCG64(77))
    feat = {
        "bits": rng.integers(0, 1 << 25, B, dtype=np.uint64).astype(np.uint32),
        "fx": rng.random(B, dtype=np.float32),
        "fy": rng.random(B, dtype=np.float32),
        "gap": (rng.random(B, dtype=np.float32) * 0.3).astype(np.float32),
    }
    labels = rng.random(B).astype(np.float32)
    P32 = sc.mlp_init(3)
    P = {k: v.astype(np.float64) for k, v in P32.items()}
    X = omlp.encode(feat)
    loss, loss_bound, G, bound = mb.gradient_bounds(P, X, labels)
    return P32, P, X, labels, loss, loss_bound, G, bound


def _bf(a):
    return omlp.bf16_round(a).astype(f32)


def gpu_like(P32, X, t, mistake=None):
    """The kernels' arithmetic in float32: every product of BF16 values,
    sums in numpy's float32 order, per-tile weight-gradient sums added tile
    by tile.  `mistake` plants one slip."""
    W1, W2, W3 = (_bf(P32[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (P32[k].astype(f32) for k in ("b1", "b2", "b3"))
    Xr = _bf(X)
    a1 = Xr @ W1 + b1
    h1 = _bf(np.maximum(a1, 0))
    a2 = h1 @ W2 + b2
    h2 = _bf(np.maximum(a2, 0))
    y = h2 @ W3 + b3
    t = t.astype(f32)
    v, e = y[:, 0], y[:, 1]
    rv = v - t
    et = np.abs(np.clip(v, f32(0), f32(1)) - t)
    re = e - et
    inv = f32(1.0 / B)
    dy = np.stack([f32(2) * rv * inv, f32(2) * re * inv], axis=1)
    dyr = _bf(dy)
    dh2 = dyr @ W3.T
    mask2 = a2 > 0
    if mistake == "mask":
        mask2 = mask2.copy()
        mask2[:, 5] = True
    da2 = dh2 * mask2
    da2r = _bf(da2)
    dh1 = da2r @ W2.T
    da1 = dh1 * (a1 > 0)
    da1r = _bf(da1)

    def tiled(a, b):
        out = np.zeros((a.shape[1], b.shape[1]), f32)
        for s in range(0, B, 128):
            aa, bb = a[s:s + 128], b[s:s + 128]
            if mistake == "shift" and s == 1024:
                bb = np.roll(bb, 1, axis=0)
            part = aa.T @ bb
            if mistake == "drop_k" and s == 2048:
                part = aa[16:].T @ bb[16:]
            out = out + part
        return out

    g = {"W3": tiled(h2, dyr), "W2": tiled(h1, da2r), "W1": tiled(Xr, da1r)}
    if mistake == "core_transpose":
        blk = g["W1"][8:16, 16:24].copy()
        g["W1"][8:16, 16:24] = blk.T
    g["b3"], g["b2"], g["b1"] = dy.sum(0), da2.sum(0), da1.sum(0)
    loss = float((rv * rv + re * re).sum()) / B
    return loss, g


def _worst(g, G, bound):
    """Largest |g - G| / bound (a difference where the bound is 0 counts as inf)."""
    out = 0.0
    for k in G:
        d = np.abs(g[k] - G[k])
        r = np.where(bound[k] > 0, d / np.where(bound[k] > 0, bound[k], 1.0), np.where(d > 0, np.inf, 0.0))
        out = max(out, float(np.max(r)))
    return out


def test_float32_restatement_is_within_the_bounds(case):
    P32, P, X, t, loss, loss_bound, G, bound = case
    lg, g = gpu_like(P32, X, t)
    assert abs(lg - loss) <= loss_bound
    for k in G:
        assert np.all(np.abs(g[k] - G[k]) <= bound[k]), k
    # the bound is a worst case (every addition losing a full ulp, every
    # interval near a rounding boundary flipping), far above the float32
    # restatement's actual deviation, yet a few per cent of the gradients'
    # scale at most; what it must catch, it catches (next test)
    assert _worst(g, G, bound) < 0.05
    for k in ("W1", "W2", "W3"):
        assert np.median(bound[k]) < 5e-2 * np.median(np.abs(G[k])), k


@pytest.mark.parametrize("mistake", ["drop_k", "core_transpose", "shift", "mask"])
def test_planted_kernel_slips_break_the_bounds(case, mistake):
    P32, P, X, t, loss, loss_bound, G, bound = case
    _, g = gpu_like(P32, X, t, mistake)
    assert _worst(g, G, bound) > 1.0, mistake


def test_forward_bound_covers_float32_and_catches_a_flipped_unit(case):
    P32, P, X, t, *_ = case
    c = mb.forward_intervals(P, X)
    W1, W2, W3 = (_bf(P32[k]) for k in ("W1", "W2", "W3"))
    h1 = _bf(np.maximum(_bf(X) @ W1 + P32["b1"].astype(f32), 0))
    h2 = _bf(np.maximum(h1 @ W2 + P32["b2"].astype(f32), 0))
    y = h2 @ W3 + P32["b3"].astype(f32)
    assert np.all(np.abs(y - c["y"]) <= c["d_y"])
    # a hidden unit of layer 2 dropped (one column of a B tile lost)
    h2_bad = h2.copy()
    h2_bad[:, 17] = 0
    y_bad = h2_bad @ W3 + P32["b3"].astype(f32)
    assert np.any(np.abs(y_bad - c["y"]) > c["d_y"])


def test_adam_bound_covers_a_float32_step(case):
    P32, P, X, t, loss, loss_bound, G, bound = case
    lr = 1e-3
    Pn, dev = mb.adam_first_step_bounds(P, G, bound, lr)
    _, g = gpu_like(P32, X, t)
    b1, b2, eps = f32(0.9), f32(0.999), f32(1e-8)
    bc1, bc2 = f32(1.0 - 0.9), f32(1.0 - 0.999)
    for k in P:
        gk = g[k].astype(f32)
        m = b1 * f32(0) + (f32(1) - b1) * gk
        v = b2 * f32(0) + (f32(1) - b2) * gk * gk
        val = P32[k] - f32(lr) * (m / bc1) / (np.sqrt(v / bc2) + eps)
        assert np.all(np.abs(val.astype(np.float64) - Pn[k]) <= dev[k]), k
