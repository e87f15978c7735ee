"""CPU pin of the surrogate's structural guard against the oracle.

For every fragment whose walks stop inside the 5x5 window (tests/window_rule.py),
re-drawing every texel outside that window must leave the oracle's Listing 5
answer unchanged bit for bit; for the fragments the rule rejects, the
answer must depend on texels outside the window for some of them (the rule
is not vacuous), and it must depend on them for none of those it accepts.
"""
import numpy as np

from oracle import rbsm as orc
from tests.window_rule import walks_inside_window

W = H = 48


def _binary_map(rng):
    """Occluder rectangles (depth 0.2) on the ground (depth 1.0): runs of
    every length from 1 to over 16 texels along both axes."""
    d = np.ones((H, W), np.float32)
    for _ in range(14):
        x0, y0 = rng.integers(0, W - 2), rng.integers(0, H - 2)
        w, h = rng.integers(1, 20), rng.integers(1, 20)
        d[y0:y0 + h, x0:x0 + w] = 0.2
    d[rng.random((H, W)) < 0.04] = 0.2
    return d


def _fragments(i, j, rng, k=6):
    fx, fy = rng.random(k), rng.random(k)
    x = ((i + fx) / W).astype(np.float32)
    y = ((j + fy) / H).astype(np.float32)
    return x, y, np.full(k, 0.5, np.float32)


def test_accepted_fragments_depend_on_their_window_only():
    rng = np.random.Generator(np.random.PCG64(21))
    accepted = rejected_dependent = rejected = 0
    for trial in range(3):
        d = _binary_map(rng)
        for j in range(4, H - 4):
            for i in range(4, W - 4):
                x, y, z = _fragments(i, j, rng)
                ref = orc.evaluate(d, x, y, z, orc.MODE_FILTER)
                edge = ((ref["codes"] >> 9) & 1) == 1
                if not edge.any():
                    continue
                f = orc.features(d, x, y, z)
                inside = walks_inside_window(f["bits"])
                assert np.all(inside == inside[0])              # one texel, one pattern
                changed = np.zeros(x.size, bool)
                for _ in range(4):
                    d2 = d.copy()
                    out = np.ones((H, W), bool)
                    out[j - 2:j + 3, i - 2:i + 3] = False
                    d2[out] = np.where(rng.random(out.sum()) < 0.5, 0.2, 1.0).astype(np.float32)
                    got = orc.evaluate(d2, x, y, z, orc.MODE_FILTER)
                    changed |= got["vis"] != ref["vis"]
                if inside[0]:
                    accepted += int(edge.sum())
                    assert not np.any(changed[edge]), (trial, i, j)
                else:
                    rejected += int(edge.sum())
                    rejected_dependent += int(np.sum(changed[edge]))
    assert accepted > 500 and rejected > 500
    assert rejected_dependent > 0.3 * rejected


def test_max_dist_two_or_less_keeps_every_walk_inside():
    bits = np.arange(0, 1 << 25, 9973, dtype=np.uint32)
    assert walks_inside_window(bits, 2).all() and walks_inside_window(bits, 1).all()
    # a long horizontal edge through the window: lit row above a shadowed row
    row = lambda dy, v: sum((v << ((dy + 2) * 5 + dx + 2)) for dx in range(-2, 3))
    edge = np.uint32(row(1, 1) | row(2, 1))                 # rows above lit, fragment's row and below shadowed
    assert not walks_inside_window(np.array([edge]), 16)[0]
