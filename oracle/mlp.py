"""Plain float64 reference of the learned penumbra surrogate (test infrastructure).

Not in the paper.  This project's surrogate estimates the Listing 5 (RSMSS)
visibility of an edge fragment from its 5x5 shadow-test pattern, in-texel
offsets and depth gap (``rbsm.features``), with a 2-layer perceptron:

    x (32: 25 pattern bits, fx, fy, gap, 4 zeros)
    h1 = relu(x W1 + b1)          W1: 32 x 64
    h2 = relu(h1 W2 + b2)         W2: 64 x 64
    y  = h2 W3 + b3               W3: 64 x 2
    y[0]: visibility estimate (clamped to [0, 1] when used)
    y[1]: estimate of its own absolute error (the guard reads it)

Loss per batch of B samples with RSMSS targets t:
    L = sum_b (y0 - t)^2 / B + sum_b (y1 - |clamp(y0, 0, 1) - t|)^2 / B
where the error target is a constant (no gradient flows through it).

Precision: the surrogate's arithmetic is BF16 with FP32 accumulation.  With
``bf16=True`` this reference rounds to BF16 (round to nearest, ties to even)
exactly where that arithmetic does: inputs and weights, the hidden
activations, and the gradients entering each backward matrix product; every
sum is then taken in float64.  With ``bf16=False`` it is the exact float64
network (used for the finite-difference pins).

Plain numpy matrix products serve as the matrix steps; nothing is blocked or
fused.
"""
import numpy as np

IN, HID, OUT = 32, 64, 2
N_BITS = 25


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as
    float64.  bfloat16 keeps the top 16 bits of a float32: the float32 bit
    pattern is rounded at bit 16 and the low half cleared."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep = ((u >> 16) & 1) + 0x7FFF
    r = ((u + keep) >> 16) << 16
    finite = np.isfinite(f)
    out = np.where(finite, r, u).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def encode(feat):
    """Input matrix (n, 32) from the feature dict of ``rbsm.features``."""
    bits = np.asarray(feat["bits"], dtype=np.uint64)
    n = bits.shape[0]
    x = np.zeros((n, IN), np.float64)
    for k in range(N_BITS):
        x[:, k] = ((bits >> np.uint64(k)) & np.uint64(1)).astype(np.float64)
    x[:, 25] = np.asarray(feat["fx"], np.float32)
    x[:, 26] = np.asarray(feat["fy"], np.float32)
    x[:, 27] = np.asarray(feat["gap"], np.float32)
    return x


def _r(a, on):
    return bf16_round(a) if on else np.asarray(a, np.float64)


def forward(P, X, bf16=True):
    """Outputs (n, 2) and the intermediates the backward pass needs."""
    Xr = _r(X, bf16)
    W1, W2, W3 = (_r(P[k], bf16) for k in ("W1", "W2", "W3"))
    a1 = Xr @ W1 + P["b1"]
    h1 = _r(np.maximum(a1, 0.0), bf16)
    a2 = h1 @ W2 + P["b2"]
    h2 = _r(np.maximum(a2, 0.0), bf16)
    y = h2 @ W3 + P["b3"]
    return y, {"X": Xr, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grads(P, X, t, bf16=True):
    """Loss (float) and gradients of every parameter (dict of float64)."""
    y, c = forward(P, X, bf16)
    B = X.shape[0]
    t = np.asarray(t, np.float64)
    v, e = y[:, 0], y[:, 1]
    e_target = np.abs(np.clip(v, 0.0, 1.0) - t)
    loss = float(np.sum((v - t) ** 2) / B + np.sum((e - e_target) ** 2) / B)
    dy = np.zeros_like(y)
    dy[:, 0] = 2.0 * (v - t) / B
    dy[:, 1] = 2.0 * (e - e_target) / B
    dyr = _r(dy, bf16)
    g = {"W3": c["h2"].T @ dyr, "b3": dy.sum(0)}
    dh2 = dyr @ c["W3"].T
    da2 = dh2 * (c["a2"] > 0)
    da2r = _r(da2, bf16)
    g["W2"] = c["h1"].T @ da2r
    g["b2"] = da2.sum(0)
    dh1 = da2r @ c["W2"].T
    da1 = dh1 * (c["a1"] > 0)
    da1r = _r(da1, bf16)
    g["W1"] = c["X"].T @ da1r
    g["b1"] = da1.sum(0)
    return loss, g


ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(P, G, M, V, step, lr):
    """One Adam update (Kingma and Ba, Algorithm 1) of every parameter, in
    place; `step` counts from 1."""
    for k in P:
        M[k] = ADAM_BETA1 * M[k] + (1.0 - ADAM_BETA1) * G[k]
        V[k] = ADAM_BETA2 * V[k] + (1.0 - ADAM_BETA2) * G[k] * G[k]
        mhat = M[k] / (1.0 - ADAM_BETA1 ** step)
        vhat = V[k] / (1.0 - ADAM_BETA2 ** step)
        P[k] = P[k] - lr * mhat / (np.sqrt(vhat) + ADAM_EPS)
