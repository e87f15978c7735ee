"""Pins of the RPCF oracle (PCF over the RSMSS answer, §5.3; readings R18,
R19 in oracle/rbsm_oracle.c) against facts fixed outside it:

* k = 1 is RSMSS itself (the pinned Listing 5 oracle);
* on maps of power-of-two size, shifting the texel-space position by whole
  texels is the same as shifting the texture coordinate by a / W, so RPCF
  is the mean of the RSMSS oracle at the k x k shifted coordinates;
* beside a long straight edge every sample is an I shape, whose RSMSS
  answer is the plain shadow test, so RPCF is classic PCF there: the lit
  fraction of the k x k sample texels (closed form);
* inside fully lit / fully shadowed regions it is 1 / 0.
"""
import numpy as np
import pytest

from oracle import rbsm as orc
from rbsm_scenes import shapes


def test_k1_is_rsmss():
    import rbsm_scenes as sc
    rng = np.random.default_rng(3)
    cases = []
    f = sc.config1(2)
    cases.append((f.depth, f.x, f.y, f.z))
    for w, h in [(37, 23), (1, 9), (64, 48)]:
        d = np.where(rng.random((h, w)) < 0.4, np.float32(0.5), np.float32(1.0)).astype(np.float32)
        x = rng.uniform(-0.2, 1.2, 4000).astype(np.float32)
        y = rng.uniform(-0.2, 1.2, 4000).astype(np.float32)
        x[::37] = np.nan
        cases.append((d, x, y, np.ones_like(x)))
    for d, x, y, z in cases:
        for md in (1, 5, 16):
            got = orc.rpcf(d, x, y, z, k=1, max_dist=md)
            ref = orc.evaluate(d, x, y, z, orc.MODE_FILTER, max_dist=md)["vis"]
            both_nan = np.isnan(got) & np.isnan(ref)
            assert np.array_equal(got[~both_nan], ref[~both_nan])


@pytest.mark.parametrize("k", [3, 5])
def test_mean_of_shifted_rsmss_on_power_of_two_maps(k):
    import rbsm_scenes as sc
    f = sc.config1(1)                  # 256 x 256
    h, w = f.depth.shape
    sel = slice(0, 20000)
    x, y, z = f.x[sel], f.y[sel], f.z[sel]
    r = (k - 1) // 2
    acc = np.zeros(x.shape[0], np.float64)
    for b in range(-r, r + 1):
        for a in range(-r, r + 1):
            xs = (x + np.float32(a) / np.float32(w)).astype(np.float32)
            ys = (y + np.float32(b) / np.float32(h)).astype(np.float32)
            acc += orc.evaluate(f.depth, xs, ys, z, orc.MODE_FILTER)["vis"]
    got = orc.rpcf(f.depth, x, y, z, k=k)
    assert np.abs(got - acc / (k * k)).max() <= 1e-12
    assert np.any((got > 0) & (got < 1))


@pytest.mark.parametrize("k", [3, 5, 7])
@pytest.mark.parametrize("orient", ["id", "T"])
def test_classic_pcf_beside_a_long_straight_edge(k, orient):
    """Columns < 60 hold a blocker, the rest are lit; fragments in rows far
    from the map's ends (every walk along the edge runs out, so every
    sample is an I shape) near the edge."""
    n = 128
    mask = np.zeros((n, n), bool)
    mask[:, :60] = True
    depth = np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32)
    X, Y = shapes.fragment_grid(52, 68, 40, 88, [(0.5, 0.5), (0.1, 0.9), (0.9, 0.2)])
    if orient == "T":
        depth, X, Y = np.ascontiguousarray(depth.T), Y, X
    x, y = shapes.to_texcoords(X, Y, n, n)
    got = orc.rpcf(depth, x, y, np.ones_like(x), k=k)
    r = (k - 1) // 2
    col = np.floor(Y if orient == "T" else X).astype(int)
    lit = np.zeros_like(got)
    for a in range(-r, r + 1):
        lit += (col + a >= 60)
    assert np.array_equal(got, lit / k)


def test_flat_regions():
    depth = np.ones((64, 64), np.float32)
    depth[:, 32:] = 0.25
    x = np.array([0.1, 0.2, 0.8, 0.9], np.float32)
    y = np.full(4, 0.5, np.float32)
    got = orc.rpcf(depth, x, y, np.full(4, 0.5, np.float32), k=5)
    assert np.array_equal(got, [1.0, 1.0, 0.0, 0.0])


def test_bad_k_is_rejected():
    d = np.ones((4, 4), np.float32)
    x = np.zeros(1, np.float32)
    for k in (0, 2, 9, -1):
        with pytest.raises(ValueError):
            orc.rpcf(d, x, x, x, k=k)


def test_thirds_of_nine_by_multiplication():
    """The RPCF kernel takes the mean of a k = 3 fragment without edge
    samples as c * RN(1/9) for its c lit samples; that is RN(c / 9), the
    division's result, for every c in 0..9 (float32), and not for 25 or 49
    samples, which keep the division."""
    inv = np.float32(1.0) / np.float32(9.0)
    for c in range(10):
        assert np.float32(c) * inv == np.float32(c) / np.float32(9.0), c
    assert any(np.float32(c) * (np.float32(1) / np.float32(25)) != np.float32(c) / np.float32(25) for c in range(26))
