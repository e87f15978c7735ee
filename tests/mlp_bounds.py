"""Element-wise bounds between the surrogate's tensor-core arithmetic and the
float64 reference of oracle/mlp.py (``bf16=True``).

Test infrastructure.  Both sides round to BF16 at the same places (inputs,
weights, hidden activations, and the gradients entering each backward
product) and keep biases, bias gradients and the loss unrounded.  They
differ in two ways only:

* every sum is accumulated in FP32 on the GPU (tensor-core products of BF16
  values are exact; each addition may lose up to one FP32 ulp, 2^-23
  relative, of a partial sum no larger than the sum of |terms|), and in
  float64 in the reference;
* when a pre-rounding value differs by that much between the sides and lies
  that close to a BF16 rounding boundary, or to zero for a ReLU decision,
  the two sides round to neighbouring values (or mask differently), and the
  difference propagates through the rest of that sample's computation.

So every per-sample quantity carries its reference value and a bound on the
GPU's deviation from it.  A linear step adds the accumulation bound plus the
incoming deviations times the absolute weights.  A ReLU and a rounding to
BF16 are monotone, so the deviation after them is the larger distance from
the reference value to the image of either end of the interval.  A ReLU
mask whose pre-activation interval contains zero may be either value on
the GPU: the masked gradient may then be zero or the unmasked one.
Weight gradients sum products over the batch, so their bound is the FP32
bound of that sum plus every sample's deviation of the two factors.

The bounds hold for any order of the FP32 additions, so they do not depend on
how the kernels tile the batch beyond the number of additions in a chain,
which ``accumulation_depth`` states for the gradient kernel's decomposition:
per-CTA sums over 128-sample tiles, then the per-CTA rows added in CTA
order within 8 strided subsets and the subsets combined pairwise.
"""
import numpy as np

from oracle import mlp as omlp

U = 2.0 ** -23          # one FP32 addition, rounding or truncating


def accumulation_depth(batch, tile=128, max_ctas=256):
    """Longest chain of FP32 additions in a batch sum of the gradient kernel."""
    tiles = -(-batch // tile)
    ctas = min(tiles, max_ctas)
    per_cta = tile * -(-tiles // ctas)
    return per_cta + -(-ctas // 8) + 3 + 8


def _rn(a):
    return omlp.bf16_round(a)


def _spread(ref, *cands):
    """Largest |candidate - ref|."""
    return np.max(np.stack([np.abs(c - ref) for c in cands]), axis=0)


def _dot_err(a, w, bias=None, k=None):
    """FP32 accumulation bound of a @ w (+ bias) with K terms per sum."""
    k = a.shape[1] if k is None else k
    s = np.abs(a) @ np.abs(w)
    if bias is not None:
        s = s + np.abs(bias)[None, :]
    return (k + 2) * U * s


def forward_intervals(P, X):
    """Reference forward values and deviation bounds (dicts of arrays)."""
    y, c = omlp.forward(P, X, bf16=True)
    W1, W2, W3 = c["W1"], c["W2"], c["W3"]
    d_a1 = _dot_err(c["X"], W1, P["b1"])
    h1_lo, h1_hi = _rn(np.maximum(c["a1"] - d_a1, 0.0)), _rn(np.maximum(c["a1"] + d_a1, 0.0))
    d_h1 = _spread(c["h1"], h1_lo, h1_hi)
    d_a2 = _dot_err(c["h1"] + d_h1, W2, P["b2"]) + d_h1 @ np.abs(W2)
    h2_lo, h2_hi = _rn(np.maximum(c["a2"] - d_a2, 0.0)), _rn(np.maximum(c["a2"] + d_a2, 0.0))
    d_h2 = _spread(c["h2"], h2_lo, h2_hi)
    d_y = _dot_err(c["h2"] + d_h2, W3, P["b3"]) + d_h2 @ np.abs(W3)
    c.update(y=y, d_a1=d_a1, d_h1=d_h1, d_a2=d_a2, d_h2=d_h2, d_y=d_y)
    return c


def _masked(dh, d_dh, pre, d_pre):
    """Reference dh * (pre > 0), its rounded copy, and deviation bounds of both.
    Where |pre| <= d_pre the GPU's mask may differ: its value is then 0 or
    dh (within d_dh)."""
    on = pre > 0
    ref = dh * on
    ref_r = _rn(ref)
    amb = np.abs(pre) <= d_pre
    lo, hi = dh - d_dh, dh + d_dh
    # mask as the reference took it
    dev = np.where(on, d_dh, 0.0)
    dev_r = np.where(on, _spread(ref_r, _rn(lo), _rn(hi)), 0.0)
    # either mask
    dev_amb = _spread(ref, np.zeros_like(ref), lo, hi)
    dev_r_amb = _spread(ref_r, np.zeros_like(ref), _rn(lo), _rn(hi))
    return ref, ref_r, np.where(amb, dev_amb, dev), np.where(amb, dev_r_amb, dev_r)


def gradient_bounds(P, X, t):
    """Reference loss and gradients (oracle/mlp.py) with an element-wise bound
    on the GPU's deviation from each gradient entry."""
    B = X.shape[0]
    t = np.asarray(t, np.float64)
    c = forward_intervals(P, X)
    y, d_y = c["y"], c["d_y"]
    v, e, dv, de = y[:, 0], y[:, 1], d_y[:, 0], d_y[:, 1]
    # output gradient, FP32 on the GPU: rv = v - t, et = |clip(v) - t|, re = e - et, dy = 2 r / B
    rv = v - t
    vc = np.clip(v, 0.0, 1.0)
    et = np.abs(vc - t)
    re = e - et
    d_rv = dv + U * (np.abs(v) + np.abs(t))
    d_et = dv + U * (np.abs(vc) + np.abs(t))
    d_re = de + d_et + U * (np.abs(e) + np.abs(et))
    dy = np.stack([2.0 * rv / B, 2.0 * re / B], axis=1)
    d_dy = np.stack([2.0 * d_rv / B, 2.0 * d_re / B], axis=1) + 2 * U * np.abs(dy)
    dyr = _rn(dy)
    d_dyr = _spread(dyr, _rn(dy - d_dy), _rn(dy + d_dy))
    W1, W2, W3 = c["W1"], c["W2"], c["W3"]
    # backward-data products (K = 16 padded for dY, 64 for dA2)
    dh2 = dyr @ W3.T
    d_dh2 = _dot_err(dyr + d_dyr, W3.T, k=16) + d_dyr @ np.abs(W3).T
    da2, da2r, d_da2, d_da2r = _masked(dh2, d_dh2, c["a2"], c["d_a2"])
    dh1 = da2r @ W2.T
    d_dh1 = _dot_err(np.abs(da2r) + d_da2r, W2.T) + d_da2r @ np.abs(W2).T
    da1, da1r, d_da1, d_da1r = _masked(dh1, d_dh1, c["a1"], c["d_a1"])
    g_batch = accumulation_depth(B) * U

    def wgrad(a, d_a, b, d_b):
        ma, mb = np.abs(a) + d_a, np.abs(b) + d_b
        return a.T @ b, g_batch * (ma.T @ mb) + d_a.T @ mb + np.abs(a).T @ d_b

    def bgrad(a, d_a):
        return a.sum(0), g_batch * (np.abs(a) + d_a).sum(0) + d_a.sum(0)

    G, bound = {}, {}
    G["W3"], bound["W3"] = wgrad(c["h2"], c["d_h2"], dyr, d_dyr)
    G["W2"], bound["W2"] = wgrad(c["h1"], c["d_h1"], da2r, d_da2r)
    G["W1"], bound["W1"] = wgrad(c["X"], np.zeros_like(c["X"]), da1r, d_da1r)
    G["b3"], bound["b3"] = bgrad(dy, d_dy)
    G["b2"], bound["b2"] = bgrad(da2, d_da2)
    G["b1"], bound["b1"] = bgrad(da1, d_da1)
    loss_terms = rv ** 2 + re ** 2
    d_loss = (2 * np.abs(rv) * d_rv + d_rv ** 2 + 2 * np.abs(re) * d_re + d_re ** 2 + 4 * U * loss_terms).sum()
    loss = float(loss_terms.sum() / B)
    loss_bound = float(d_loss / B + g_batch * loss_terms.sum() / B)
    return loss, loss_bound, G, bound


def adam_first_step_bounds(P, G, bound, lr):
    """Parameters after one Adam step from zero moments (float64 reference,
    oracle/mlp.py) and the element-wise deviation the GPU may show: its
    update is lr * r(g) with r(g) = g / (|g| + eps), monotone in g, at a
    gradient within `bound` of the reference's, plus FP32 rounding of the
    update (a few ulps of lr) and of the stored parameter.  The GPU's decay
    rates are the FP32 values nearest 0.9 and 0.999: 1 - 0.999f is 1.3e-5
    below 0.001, so its first step is about 6.5e-6 lr longer (2^-16 lr
    allowed)."""
    Pn = {k: v.copy() for k, v in P.items()}
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    omlp.adam_step(Pn, G, M, V, 1, lr)
    eps = omlp.ADAM_EPS

    def r(g):
        return g / (np.abs(g) + eps)

    dev = {}
    for k in P:
        rr = r(G[k])
        dev[k] = (lr * _spread(rr, r(G[k] - bound[k]), r(G[k] + bound[k])) + 2.0 ** -16 * lr + 16 * U * lr
                  + U * (np.abs(P[k]) + lr))
    return Pn, dev
