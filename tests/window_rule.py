"""When the exact answer of an edge fragment lies inside its 5x5 window
(test infrastructure).

The learned surrogate sees the 5x5 shadow-test pattern around the
fragment's texel (bit (dy+2)*5 + (dx+2) set when texel (i+dx, j+dy) is lit),
its in-texel offsets and a depth gap.  A Listing 3 walk along +x goes on past
step k while texel (k, 0) has the fragment's shadow test and shares a
discontinuity direction with the fragment's texel.  For such a texel the
directions along the walk are never discontinuous on both sides (its own
test equals the fragment's, and so do the texels between them), so sharing
means a +y (or -y) discontinuity at both (k, 0) and (0, 0).  Steps 1 and 2
read window texels only; a walk that goes on past step 2 reads step 3,
outside the window.  So the exact answer is a function of the window when no
walk goes on past step 2 (or max_dist <= 2).
"""
import numpy as np


def walks_inside_window(bits, max_dist=16):
    """Boolean array: the four walks of each fragment stop inside the window."""
    bits = np.asarray(bits, np.uint32)
    if max_dist <= 2:
        return np.ones(bits.shape, bool)

    def lit(dx, dy):
        return ((bits >> np.uint32((dy + 2) * 5 + (dx + 2))) & np.uint32(1)).astype(bool)

    s0 = lit(0, 0)

    def diff(dx, dy):
        return lit(dx, dy) != s0

    up, down, left, right = diff(0, 1), diff(0, -1), diff(-1, 0), diff(1, 0)

    def on_x(dx):
        return ~diff(dx, 0) & ((up & diff(dx, 1)) | (down & diff(dx, -1)))

    def on_y(dy):
        return ~diff(0, dy) & ((left & diff(-1, dy)) | (right & diff(1, dy)))

    past = (on_x(1) & on_x(2)) | (on_x(-1) & on_x(-2)) | (on_y(1) & on_y(2)) | (on_y(-1) & on_y(-2))
    return ~past
