"""Pins of the CPU oracle to what the paper and geometry fix (CPU only).

Each test checks the oracle against something other than itself:
  - the worked example of Fig. 3 (four 3x3 shapes, expected result drawn at
    0.2-texel resolution), stored verbatim in tests/golden/fig3_shapes.txt;
  - closed forms on straight staircase edges: the revectorised silhouette of
    a point-sampled half-plane Y < X/L is that half-plane, and the filtered
    result is the one-texel ramp clamp(1 + Y - X/L, 0, 1), in all eight
    orientations of the square;
  - the shape outcomes §4.1-§4.2 state in words (I keeps plain shadow
    mapping, short/long O closes, U returns the distance to the edge);
  - invariants (range, plain shadow mapping off the edge, shadowed fragments
    stay shadowed under silhouette recovery);
  - exhaustive symmetry on every 4x4 binary map.
"""
import os

import numpy as np
import pytest

from oracle import rbsm as orc
from rbsm_scenes import shapes

SIL, FIL = orc.MODE_SILHOUETTE, orc.MODE_FILTER


def run(depth, X, Y, mode, z=None, max_dist=orc.MAXDIST, **kw):
    h, w = depth.shape
    x, y = shapes.to_texcoords(X, Y, w, h)
    if z is None:
        z = np.full(x.shape, shapes.RECEIVER, np.float32)
    return orc.evaluate(depth, x, y, z, mode, max_dist=max_dist, **kw)


# ----------------------------------------------------------------- Fig. 3 --

def _load_fig3(golden_dir):
    rects = {}
    with open(os.path.join(golden_dir, "fig3_shapes.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            shape, kind, *c = line.split()
            rects.setdefault(shape, {"in": [], "out": []})[kind].append(tuple(float(v) for v in c))
    return rects


def _inside(rs, X, Y):
    hit = np.zeros(np.shape(X), bool)
    for x0, y0, x1, y1 in rs:
        hit |= (X > x0) & (X < x1) & (Y > y0) & (Y < y1)
    return hit


@pytest.mark.parametrize("shape", ["a", "b", "c", "d"])
def test_fig3_worked_example(golden_dir, shape):
    """Fig. 3: I stays lit, U and O close, the L edge follows the drawn line.
    Fragments at the figure's 0.2-texel resolution (5 x 5 per texel)."""
    rects = _load_fig3(golden_dir)[shape]
    n, off = 32, 12
    ti, tj = np.meshgrid(np.arange(3), np.arange(3), indexing="xy")
    mask = _inside(rects["in"], ti + 0.5, tj + 0.5)
    depth = shapes.embed(mask, n, off)
    sub = [((a + 0.5) / 5, (b + 0.5) / 5) for a in range(5) for b in range(5)]
    X, Y = shapes.fragment_grid(0, 3, 0, 3, sub)
    expected = np.where(_inside(rects["out"], X, Y), 0.0, 1.0)
    got = run(depth, X + off, Y + off, SIL)["vis"]
    bad = np.nonzero(got != expected)[0]
    assert bad.size == 0, [(X[k], Y[k], got[k], expected[k]) for k in bad[:10]]
    # the figure must exercise its shape: (c) really needs the L branch
    if shape == "c":
        assert ((expected == 0) & (X > 2) & (Y > 1)).sum() > 0


# ------------------------------------------------------ staircase closed form --

OFFS4 = [((a + 0.5) / 4, (b + 0.5) / 4) for a in range(4) for b in range(4)]
OFFS16 = [((a + 0.5) / 16, (b + 0.5) / 16) for a in range(16) for b in range(16)]


def _staircase_case(run_len, orient, mode, max_dist=orc.MAXDIST, n=128, keep_ties=False):
    """Fragments on a 4 x 4 in-texel grid everywhere away from the border, and
    on a 16 x 16 grid in the texels within two texels of the true line (the
    first texel of each run is only reached by the fine grid)."""
    a0, b0 = 8, 40
    mask = shapes.staircase_mask(n, run_len, a0, b0)
    depth = np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32)
    Xc, Yc = shapes.fragment_grid(34, n - 34, 34, n - 34, [(0.5, 0.5)])
    near = np.abs((Yc - b0) - (Xc - a0) / run_len) < 2.0
    Xa, Ya = shapes.fragment_grid(34, n - 34, 34, n - 34, OFFS4)
    Xb = (np.floor(Xc[near])[:, None] + np.array([o[0] for o in OFFS16])[None, :]).ravel()
    Yb = (np.floor(Yc[near])[:, None] + np.array([o[1] for o in OFFS16])[None, :]).ravel()
    X, Y = np.concatenate([Xa, Xb]), np.concatenate([Ya, Yb])
    margin = (Y - b0) - (X - a0) / run_len          # > 0 above the true line
    if not keep_ties:
        keep = np.abs(margin) > 1e-6                  # ties are checked separately
        X, Y, margin = X[keep], Y[keep], margin[keep]
    Xt, Yt = shapes.d4_points(X, Y, n, orient)
    out = run(shapes.d4_map(depth, orient), Xt, Yt, mode, max_dist=max_dist)
    return out, margin


@pytest.mark.parametrize("orient", shapes.D4_NAMES)
@pytest.mark.parametrize("run_len", list(range(1, 17)))
def test_staircase_silhouette_is_the_true_line(run_len, orient):
    """§4.1 on straight edges at slopes 1/L (L <= MAXDIST) and their D4 images:
    the revectorised silhouette is exactly the half-plane Y >= X/L."""
    out, margin = _staircase_case(run_len, orient, SIL)
    expected = (margin > 0).astype(np.float64)
    assert np.array_equal(out["vis"], expected), np.count_nonzero(out["vis"] != expected)


@pytest.mark.parametrize("orient", shapes.D4_NAMES)
@pytest.mark.parametrize("run_len", list(range(1, 17)))
def test_staircase_filter_is_a_unit_ramp(run_len, orient):
    """§4.2 on the same edges: the fake penumbra is clamp(1 + Y - X/L, 0, 1)."""
    out, margin = _staircase_case(run_len, orient, FIL)
    expected = np.clip(1.0 + margin, 0.0, 1.0)
    assert np.max(np.abs(out["vis"] - expected)) < 1e-12


def test_staircase_beyond_maxdist_is_not_exact():
    """Runs longer than the traversal cap (§3.1.3) are not fully measured:
    with L = MAXDIST + 1 the closed form fails at the first texel of each run
    (its walk along the run gives up one texel short), with a larger cap it
    holds."""
    out, margin = _staircase_case(orc.MAXDIST + 1, "id", FIL)
    err = np.max(np.abs(out["vis"] - np.clip(1.0 + margin, 0.0, 1.0)))
    assert err > 1e-2
    out, margin = _staircase_case(orc.MAXDIST + 1, "id", FIL, max_dist=32)
    assert np.max(np.abs(out["vis"] - np.clip(1.0 + margin, 0.0, 1.0))) < 1e-12


@pytest.mark.parametrize("orient", ["id", "transpose", "rot180"])
@pytest.mark.parametrize("run_len", [1, 2, 4, 8, 16])
def test_staircase_points_on_the_line_stay_lit(run_len, orient):
    """Listing 4 uses step(1 - nrd.x, nrd.y), which is 1 when nrd.y equals the
    edge: a fragment exactly on the revectorisation line is lit.  With dyadic
    positions and power-of-two runs every quantity is exact in single
    precision, so the tie is a real tie."""
    n, a0, b0 = 128, 8, 40
    mask = shapes.staircase_mask(n, run_len, a0, b0)
    depth = np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32)
    X = 40 + np.arange(1, 48 * 16) / 16.0
    Y = b0 + (X - a0) / run_len                       # exactly on the line
    keep = (Y > 34) & (Y < n - 34) & (Y != np.floor(Y)) & (X != np.floor(X))
    Xt, Yt = shapes.d4_points(X[keep], Y[keep], n, orient)
    out = run(shapes.d4_map(depth, orient), Xt, Yt, SIL)
    assert keep.sum() > 20
    assert np.all(out["vis"] == 1.0)


# ------------------------------------------------------------ shape outcomes --

SUB4 = [((a + 0.5) / 4, (b + 0.5) / 4) for a in range(4) for b in range(4)]


def test_i_shape_reproduces_shadow_mapping():
    """§4.1/§4.2: on a long straight axis-aligned edge (I shape) both visibility
    functions return the plain shadow test, on both sides of the edge."""
    n = 96
    mask = np.zeros((n, n), bool)
    mask[:, :48] = True                       # vertical edge at X = 48
    for orient in shapes.D4_NAMES:
        depth = shapes.d4_map(np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32), orient)
        X, Y = shapes.fragment_grid(40, 56, 30, 66, SUB4)
        Xt, Yt = shapes.d4_points(X, Y, n, orient)
        plain = (X >= 48).astype(np.float64)
        for mode in (SIL, FIL):
            out = run(depth, Xt, Yt, mode, want_nrd=True)
            assert np.array_equal(out["vis"], plain)
        edge = (out["codes"] >> 9) & 1
        assert edge.sum() > 0   # the edge fragments did go through the I branch


def test_o_shapes_close():
    """§4.1/§4.2: an isolated lit texel (short O) or a 2 x 2 lit hole (long O)
    inside shadow is shadowed by both functions; a shadow island of the same
    shapes is closed to lit by filtering and stays shadowed in silhouette mode."""
    n = 48
    for k in (1, 2):
        hole = np.ones((n, n), bool)
        hole[20:20 + k, 20:20 + k] = False
        island = ~hole
        X, Y = shapes.fragment_grid(20, 20 + k, 20, 20 + k, SUB4)
        for mode in (SIL, FIL):
            assert np.all(run(shapes.embed(hole, n, 0), X, Y, mode)["vis"] == 0.0)
        assert np.all(run(shapes.embed(island, n, 0), X, Y, FIL)["vis"] == 1.0)
        assert np.all(run(shapes.embed(island, n, 0), X, Y, SIL)["vis"] == 0.0)


@pytest.mark.parametrize("orient", shapes.D4_NAMES)
@pytest.mark.parametrize("width", [3, 8, 15])
def test_u_cup_filter_is_distance_to_floor(width, orient):
    """§4.2 U shape: the lit bottom row of a cup (shadow floor below, shadow
    walls at both ends, within the traversal cap) gets its normalised distance
    to the floor edge, i.e. Y - floor(Y); silhouette recovery (§4.1, long U)
    puts that row in shadow."""
    n = 64
    mask = np.zeros((n, n), bool)
    mask[20:30, 24:24 + width + 2] = True        # block of shadow
    mask[25:30, 25:25 + width] = False           # carve the cup, floor at row 24
    depth = shapes.d4_map(np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32), orient)
    X, Y = shapes.fragment_grid(25, 25 + width, 25, 26, SUB4)   # bottom row of the cup
    inner = (X >= 26) & (X < 24 + width)                          # away from the walls
    Xt, Yt = shapes.d4_points(X, Y, n, orient)
    fil = run(depth, Xt, Yt, FIL)["vis"]
    assert np.max(np.abs(fil[inner] - (Y[inner] - 25))) < 1e-12
    sil = run(depth, Xt, Yt, SIL)["vis"]
    assert np.all(sil == 0.0)


# --------------------------------------------------------------- invariants --

def _random_scene(rng, n=32, m=4000):
    levels = np.array([0.25, 0.5, 0.75, 1.0], np.float32)
    depth = levels[rng.integers(0, 4, size=(n, n))]
    # smooth-ish blobs so that edges are long enough to traverse
    blob = rng.integers(0, 2, size=(n // 4, n // 4)).repeat(4, 0).repeat(4, 1).astype(bool)
    depth = np.where(blob, depth, np.float32(1.0)).astype(np.float32)
    X = rng.integers(0, n, m) + (rng.integers(0, 16, m) + 0.5) / 16
    Y = rng.integers(0, n, m) + (rng.integers(0, 16, m) + 0.5) / 16
    z = levels[rng.integers(0, 4, m)]
    return depth, X, Y, z


def test_invariants_on_random_maps():
    """Listing 1: off the edge (no discontinuity) both functions return the
    shadow test (Eq. 1); silhouette output is 0/1 and never lights a shadowed
    fragment; filtering output lies in [0, 1]."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        depth, X, Y, z = _random_scene(rng)
        n = depth.shape[0]
        i, j = np.floor(X).astype(int), np.floor(Y).astype(int)
        s0 = (z <= depth[j, i]).astype(np.float64)
        sil = run(depth, X, Y, SIL, z=z)
        fil = run(depth, X, Y, FIL, z=z)
        d4 = fil["codes"] & 0xF
        off_edge = d4 == 0
        assert np.array_equal(fil["vis"][off_edge], s0[off_edge])
        assert np.array_equal(sil["vis"][off_edge], s0[off_edge])
        assert set(np.unique(sil["vis"])) <= {0.0, 1.0}
        assert np.all(sil["vis"] <= s0)
        assert np.all((fil["vis"] >= 0) & (fil["vis"] <= 1))
        # code bit 4 is the failed shadow test; bit 9 marks traversed fragments
        assert np.array_equal((fil["codes"] >> 4) & 1, (1 - s0).astype(np.uint16))
        assert np.array_equal(((fil["codes"] >> 9) & 1) == 1, d4 != 0)
        assert np.array_equal(((sil["codes"] >> 9) & 1) == 1, (d4 != 0) & (s0 == 1))
        assert n == 32


@pytest.mark.parametrize("orient", ["flipx", "flipy", "transpose"])
def test_symmetry_on_random_maps(orient):
    """§4 builds the 9 cases on symmetry: mirroring or transposing the map and
    the fragments gives the same visibility, with the discontinuity codes
    permuted accordingly."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        depth, X, Y, z = _random_scene(rng)
        n = depth.shape[0]
        Xt, Yt = shapes.d4_points(X, Y, n, orient)
        dt = shapes.d4_map(depth, orient)
        for mode in (SIL, FIL):
            a = run(depth, X, Y, mode, z=z, want_nrd=True)
            b = run(dt, Xt, Yt, mode, z=z, want_nrd=True)
            if mode == SIL:
                nx, ny = a["nrd"][:, 0], a["nrd"][:, 1]
                near_tie = np.abs(nx + ny - 1.0) < 1e-6
                assert np.array_equal(a["vis"][~near_tie], b["vis"][~near_tie])
            else:
                assert np.max(np.abs(a["vis"] - b["vis"])) < 1e-12
            ca, cb = a["codes"].astype(np.uint16), b["codes"].astype(np.uint16)
            L, R, U, D = [(ca >> k) & 1 for k in range(4)]
            ex, ey = (ca >> 5) & 3, (ca >> 7) & 3
            if orient == "flipx":
                L, R = R, L
            elif orient == "flipy":
                U, D = D, U
            else:  # transpose: x <-> y, left <-> -y, right <-> +y
                L, R, U, D, ex, ey = D, U, R, L, ey, ex
            expect = (ca & 0x210) | L | (R << 1) | (U << 2) | (D << 3) | (ex << 5) | (ey << 7)
            assert np.array_equal(cb, expect.astype(np.uint16))


def test_exhaustive_4x4_symmetry():
    """Brute force over all 2^16 binary 4 x 4 maps (clamped borders): results
    agree between each map and its mirror images and transpose, at four
    in-texel positions per texel that the symmetries permute."""
    offs = [(5 / 16, 5 / 16), (5 / 16, 11 / 16), (11 / 16, 5 / 16), (11 / 16, 11 / 16)]
    X, Y = shapes.fragment_grid(0, 4, 0, 4, offs)
    npat = 1 << 16
    bits = ((np.arange(npat)[:, None] >> np.arange(16)[None, :]) & 1).astype(bool)
    res = {FIL: np.empty((npat, X.size)), SIL: np.empty((npat, X.size))}
    for p in range(npat):
        depth = np.where(bits[p].reshape(4, 4), shapes.BLOCKER, shapes.LIT).astype(np.float32)
        for mode in (SIL, FIL):
            res[mode][p] = run(depth, X, Y, mode)["vis"]
    assert np.all((res[FIL] >= 0) & (res[FIL] <= 1))
    key = {(a, b): k for k, (a, b) in enumerate(zip(X, Y))}
    weights = 1 << np.arange(16)
    for orient in ("flipx", "flipy", "transpose"):
        tb = np.stack([shapes.d4_map(b.reshape(4, 4), orient).ravel() for b in bits])
        pidx = (tb * weights).sum(1)
        Xt, Yt = shapes.d4_points(X, Y, 4, orient)
        fidx = np.array([key[(a, b)] for a, b in zip(Xt, Yt)])
        for mode in (SIL, FIL):
            mapped = res[mode][pidx][:, fidx]
            assert np.max(np.abs(mapped - res[mode])) < 1e-12, orient


def test_rejects_bad_arguments():
    depth = np.ones((4, 4), np.float32)
    x = np.zeros(3, np.float32)
    with pytest.raises(ValueError):
        orc.evaluate(depth, x, x, x, 3)
    with pytest.raises(ValueError):
        orc.evaluate(depth, x, x, x, SIL, max_dist=0)
    with pytest.raises(ValueError):
        orc.evaluate(depth, x, x[:2], x, SIL)
