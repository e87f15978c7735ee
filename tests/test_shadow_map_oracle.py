"""Pins of the shadow-map oracle (analytic occluders point-sampled at texel
centres, smallest depth; oracle/shadow_map_oracle.c) against facts fixed
outside it:

* the input generator's rasteriser (rbsm_scenes, a separate span-based
  implementation that tests only the texels of each row's span) gives the
  same bytes on the generator's own scenes;
* an axis-aligned rectangle covers exactly the texels whose centres lie in
  it (integer counting), in both orientations of its axis;
* a disc centred on a texel centre covers the integer points of the Gauss
  circle problem (N(r) for r = 0..10, a published sequence) and its depth at
  the centre is centre - R / zscale;
* overlapping occluders keep the smaller depth; whole-texel translations
  move the map.
"""
import numpy as np
import pytest

from oracle import rbsm as orc

# Gauss circle problem, N(r) = #{(a, b) in Z^2 : a^2 + b^2 <= r^2}
GAUSS_N = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]


@pytest.mark.parametrize("which", ["c1", "c2", "c5"])
def test_equals_the_generator_rasteriser(which):
    import rbsm_scenes as sc
    if which == "c1":
        # rotated rectangles at 256^2, as C1 draws them
        rng = np.random.default_rng(1)
        rects = np.array([[rng.uniform(32, 224), rng.uniform(32, 224), np.cos(a), np.sin(a),
                           rng.uniform(4, 32), rng.uniform(4, 32)] for a in rng.uniform(0, np.pi, 8)])
        dep = rng.uniform(0.2, 0.8, 8).astype(np.float32)
        occ = sc.Occluders(rects, dep, np.zeros((0, 4)))
        w = h = 256
        zs = 256.0
    elif which == "c2":
        d = sc._Draw(sc._seed(2, 0))
        occ = sc._fence_scene(d, 2048, 40, 30, 1.0)
        w = h = 2048
        zs = 2048.0
    else:
        c5 = sc.Config5(0, size=1024, frames=4)
        occ = c5.occluders(3)
        w = h = 1024
        zs = 1024.0
    gen = sc.raster(occ, w, h, zs)
    ref = orc.shadow_map(w, h, occ.rects, occ.rect_depth, occ.spheres, zs)
    assert np.array_equal(gen.view(np.uint32), ref.view(np.uint32))
    assert np.mean(ref < 1.0) > 0.01


@pytest.mark.parametrize("axis", [(1.0, 0.0), (0.0, 1.0)])
def test_axis_aligned_rectangle_counts(axis):
    rng = np.random.default_rng(7)
    for _ in range(20):
        cx, cy = rng.uniform(10, 54), rng.uniform(10, 54)
        ha, hb = rng.uniform(0.5, 9), rng.uniform(0.5, 9)
        ux, uy = axis
        m = orc.shadow_map(64, 64, [[cx, cy, ux, uy, ha, hb]], [0.25], np.zeros((0, 4)), 64.0)
        ex, ey = (ha, hb) if axis == (1.0, 0.0) else (hb, ha)   # extents along x and y
        i = np.arange(64) + 0.5
        cols = np.abs(i - cx) <= ex
        rows = np.abs(i - cy) <= ey
        want = np.where(rows[:, None] & cols[None, :], np.float32(0.25), np.float32(1.0))
        assert np.array_equal(m, want)


def test_gauss_circle_counts_and_centre_depth():
    for r, n in enumerate(GAUSS_N):
        c = 20.5                                    # a texel centre
        m = orc.shadow_map(41, 41, np.zeros((0, 6)), np.zeros(0, np.float32), [[c, c, float(r), 0.75]], 64.0)
        assert int(np.sum(m < 1.0)) == n
        assert m[20, 20] == np.float32(0.75 - r / 64.0)


def test_min_of_overlaps_and_ground():
    rects = [[16, 16, 1, 0, 6, 6], [18, 16, 1, 0, 6, 6]]
    m = orc.shadow_map(32, 32, rects, np.array([0.6, 0.3], np.float32), np.zeros((0, 4)), 32.0, ground=0.9)
    assert m[16, 11] == np.float32(0.6)             # only the first
    assert m[16, 17] == np.float32(0.3)             # both: the smaller
    assert m[2, 2] == np.float32(0.9)               # neither: ground


def test_translation_by_whole_texels():
    rects = np.array([[20.3, 18.7, 0.6, 0.8, 7.1, 3.3]])
    sph = np.array([[40.2, 30.9, 6.5, 0.7]])
    a = orc.shadow_map(64, 64, rects, [0.4], sph, 64.0)
    rects2, sph2 = rects.copy(), sph.copy()
    rects2[:, :2] += [5, 7]
    sph2[:, :2] += [5, 7]
    b = orc.shadow_map(64, 64, rects2, [0.4], sph2, 64.0)
    assert np.array_equal(b[7:, 5:], a[:-7, :-5])


def test_edges_through_texel_centres_are_covered():
    """Dyadic rectangles whose edges pass exactly through texel centres: the
    centre on the edge is covered (|s| <= ha)."""
    m = orc.shadow_map(16, 16, [[8.0, 8.0, 1.0, 0.0, 2.5, 1.5]], [0.5], np.zeros((0, 4)), 16.0)
    cols = np.nonzero(m[8] < 1.0)[0]
    rows = np.nonzero(m[:, 8] < 1.0)[0]
    assert cols.tolist() == [5, 6, 7, 8, 9, 10] and rows.tolist() == [6, 7, 8, 9]


def test_bad_arguments():
    with pytest.raises(ValueError):
        orc.shadow_map(0, 4, np.zeros((0, 6)), np.zeros(0), np.zeros((0, 4)), 1.0)
    with pytest.raises(ValueError):
        orc.shadow_map(4, 4, np.zeros((0, 6)), np.zeros(0), np.zeros((0, 4)), 0.0)
