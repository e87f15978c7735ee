"""Pins of the depth-buffer projection oracle (reading R21: p = M (px + 0.5,
py + 0.5, d, 1) with the perspective divide, float32):

* identity and power-of-two scalings give the exact screen coordinates and
  depths;
* a matrix whose every product and sum is exact in float32 (dyadic
  entries, small integers) gives the closed form;
* the C5 camera in depth-buffer form reproduces the generator's own
  light-space fragments (computed separately, in double) to float32
  rounding;
* composed with the RBSM oracle it is the RBSM oracle on the projected
  planes.
"""
import numpy as np

from oracle import rbsm as orc


def test_identity_and_scalings():
    g = (np.arange(35, dtype=np.float32).reshape(5, 7) - 3.0) / 8.0
    x, y, z = orc.project(g, np.eye(4, dtype=np.float32))
    px, py = np.meshgrid(np.arange(7) + 0.5, np.arange(5) + 0.5)
    assert np.array_equal(x, px.ravel().astype(np.float32))
    assert np.array_equal(y, py.ravel().astype(np.float32))
    assert np.array_equal(z, g.ravel())
    m = np.diag([1 / 8, 1 / 4, 2.0, 1.0]).astype(np.float32)
    x, y, z = orc.project(g, m)
    assert np.array_equal(x, (px.ravel() / 8).astype(np.float32))
    assert np.array_equal(y, (py.ravel() / 4).astype(np.float32))
    assert np.array_equal(z, 2 * g.ravel())


def test_exact_perspective():
    """w = 2 + sx/2 (sx = px + 0.5 a half-integer, so w is exact); rows chosen
    so that X, Y, Z are small exact values and the divides are by powers
    of two on a subset of pixels."""
    m = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0.5, 0, 0, 2]], np.float32)
    g = np.full((2, 12), 3.0, np.float32)
    x, y, z = orc.project(g, m)
    sx = np.tile(np.arange(12) + 0.5, 2)
    sy = np.repeat(np.arange(2) + 0.5, 12)
    w = 2 + sx / 2
    assert np.array_equal(x, (sx / w).astype(np.float32))
    assert np.array_equal(y, (sy / w).astype(np.float32))
    assert np.array_equal(z, (3.0 / w).astype(np.float32))


def test_c5_camera_reproduces_the_generator_fragments():
    import rbsm_scenes as sc
    c5 = sc.Config5(0, size=1024, screen=(640, 360), frames=1)
    fr = c5.frame(0)
    d, m = c5.gbuffer(fr.z)
    x, y, z = orc.project(d, m)
    assert np.abs(x - fr.x).max() <= 4e-7
    assert np.abs(y - fr.y).max() <= 4e-7
    assert np.abs(z - fr.z).max() <= 4e-7


def test_composition_with_rbsm():
    import rbsm_scenes as sc
    c5 = sc.Config5(0, size=1024, screen=(320, 180), frames=1)
    fr = c5.frame(0)
    d, m = c5.gbuffer(fr.z)
    x, y, z = orc.project(d, m)
    a = orc.evaluate(fr.depth, x, y, z, orc.MODE_FILTER)
    b = orc.evaluate(fr.depth, fr.x, fr.y, fr.z, orc.MODE_FILTER)
    assert np.mean(a["codes"] == b["codes"]) > 0.999     # the same scene, up to rounding of p
