"""The oracle's visibility functions, written from the shape definitions of
§4 (I, L, U, O told apart first, then each shape's answer), against the
branch order of Listings 4 and 5.

The oracle (oracle/rbsm_oracle.c) restates §4.1 and §4.2 shape by shape;
the kernels follow the listings' if-chains.  Here a plain transcription of
the listings' branches (Listing 5's I-shape test under reading R11, and as
printed) is compared with the oracle on every combination the traversal can
produce: per axis, discontinuity directions on both sides or not, and 0, 1
or 2 ends found (directions on both sides force an end at the first step on
both sides), the fragment's side of the edge, and normalised distances on a
grid that includes the values the normalisation gives without an end (1)
and points on the revectorisation line.  No GPU needed.
"""
import itertools

import numpy as np

from oracle import rbsm as orc

EQ5 = {2: 1, 1: 0, 0: -1}      # ends found -> nrd.z / nrd.w


def listing4(dxq, dyq, cx, cy, nx, ny):
    if dxq == 3 or dyq == 3:
        return 0.0
    if cx == 1 or cy == 1:
        return 0.0
    if cx == -1 or cy == -1:
        return 1.0
    return 0.0 if np.float32(ny) < np.float32(1.0) - np.float32(nx) else 1.0


def listing5(dxq, dyq, dz, cx, cy, nx, ny, printed=False):
    sign = -2.0 * dz + 1.0
    if dxq == 3 and dyq == 3:
        return float(dz)
    if cx == 1 and cy == 1:
        return float(dz)
    if cx == 1:
        return dz + sign * ny
    if cy == 1:
        return dz + sign * nx
    if cx == -1 or (cy == 1 if printed else cy == -1):
        return 1.0 - dz
    return min(max(dz + sign * ny + sign * nx, 0.0), 1.0)


def combos():
    grid = [0.0, 0.125, 0.25, 1.0 / 3.0, 0.5, 0.6, 2.0 / 3.0, 0.75, 0.875, 1.0]
    for ox, oy in itertools.product((0, 1), repeat=2):
        for ex, ey in itertools.product((0, 1, 2), repeat=2):
            if (ox and ex != 2) or (oy and ey != 2):
                continue                      # both-side directions end both walks at step 1
            for dz in (0, 1):
                for nx, ny in itertools.product(grid, repeat=2):
                    # no end along an axis: the normalised distance is 1
                    nxv = 1.0 if ex == 0 else nx
                    nyv = 1.0 if ey == 0 else ny
                    yield ox, oy, ex, ey, dz, nxv, nyv


def test_silhouette_shapes_equal_listing4():
    n = 0
    for ox, oy, ex, ey, dz, nx, ny in combos():
        if dz:
            continue                          # silhouette recovery answers lit fragments only
        got = orc.edge_visibility(orc.MODE_SILHOUETTE, ox, oy, ex, ey, dz, nx, ny)
        want = listing4(3 * ox, 3 * oy, EQ5[ex], EQ5[ey], nx, ny)
        assert got == want, (ox, oy, ex, ey, nx, ny)
        n += 1
    assert n > 500


def test_filter_shapes_equal_listing5_both_readings():
    n = 0
    for ox, oy, ex, ey, dz, nx, ny in combos():
        got = orc.edge_visibility(orc.MODE_FILTER, ox, oy, ex, ey, dz, nx, ny)
        want = listing5(3 * ox, 3 * oy, dz, EQ5[ex], EQ5[ey], nx, ny)
        printed = listing5(3 * ox, 3 * oy, dz, EQ5[ex], EQ5[ey], nx, ny, printed=True)
        assert got == want == printed, (ox, oy, ex, ey, dz, nx, ny)
        n += 1
    assert n > 1000


def test_each_shape_answers_as_section_4_describes():
    """One case per shape, answers stated from the text of §4.1-§4.2 and
    Fig. 2, not from the listings."""
    S, F = orc.MODE_SILHOUETTE, orc.MODE_FILTER
    # I: no end along an axis -- the shadow test stands (lit 1, shadowed 0)
    assert orc.edge_visibility(S, 0, 0, 0, 1, 0, 1.0, 0.3) == 1.0
    assert orc.edge_visibility(F, 0, 0, 1, 0, 0, 0.3, 1.0) == 1.0
    assert orc.edge_visibility(F, 0, 0, 1, 0, 1, 0.3, 1.0) == 0.0
    # U: ends on both sides of an axis -- silhouette recovery closes it,
    # filtering answers the normalised distance across the open axis
    assert orc.edge_visibility(S, 0, 0, 2, 1, 0, 0.4, 0.3) == 0.0
    assert orc.edge_visibility(F, 0, 0, 2, 1, 0, 0.4, 0.3) == 0.3
    assert orc.edge_visibility(F, 0, 0, 1, 2, 1, 0.4, 0.3) == 1.0 - 0.4
    # U by directions alone (short U): closed by silhouette recovery
    assert orc.edge_visibility(S, 1, 0, 2, 1, 0, 0.4, 0.3) == 0.0
    # O: closed on both axes -- the opposite of the shadow test
    assert orc.edge_visibility(F, 1, 1, 2, 2, 0, 0.5, 0.5) == 1.0 - 1.0
    assert orc.edge_visibility(F, 0, 0, 2, 2, 1, 0.5, 0.5) == 1.0
    assert orc.edge_visibility(S, 1, 1, 2, 2, 0, 0.5, 0.5) == 0.0
    # L: an end along each axis -- the revectorisation line ny = 1 - nx
    # (a point on it stays lit) and the clamped sum of the distances
    assert orc.edge_visibility(S, 0, 0, 1, 1, 0, 0.25, 0.5) == 0.0
    assert orc.edge_visibility(S, 0, 0, 1, 1, 0, 0.25, 0.75) == 1.0
    assert orc.edge_visibility(S, 0, 0, 1, 1, 0, 0.5, 0.75) == 1.0
    assert orc.edge_visibility(F, 0, 0, 1, 1, 0, 0.25, 0.5) == 0.75
    assert orc.edge_visibility(F, 0, 0, 1, 1, 1, 0.25, 0.5) == 0.25
    assert orc.edge_visibility(F, 0, 0, 1, 1, 0, 0.75, 0.5) == 1.0
