"""Hand-built shadow maps and fragment grids: the pins' inputs and the bench's
staircase sweep.

Nothing here computes any step of the method: these helpers only place
occluder texels and fragment positions, and apply the eight symmetries of the
square (the dihedral group D4) to a map and to fragment positions.
"""
import numpy as np

LIT = 1.0       # receiver plane depth (nothing in front of it)
BLOCKER = 0.5   # depth stored where an occluder covers the texel
RECEIVER = 1.0  # fragment depth on the plane


def embed(mask, size, off):
    """A size x size map, lit everywhere except where the boolean mask
    (rows = y index) is True, with mask[0, 0] placed at texel (off, off)."""
    m = np.full((size, size), LIT, np.float32)
    h, w = mask.shape
    m[off:off + h, off:off + w] = np.where(mask, BLOCKER, LIT)
    return m


def fragment_grid(i0, i1, j0, j1, offsets):
    """Fragment positions in texel units: every texel (i, j) with i in
    [i0, i1), j in [j0, j1) and every (a, b) in offsets gives X = i + a,
    Y = j + b.  Returns float64 arrays X, Y."""
    ii, jj = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="xy")
    xs, ys = [], []
    for a, b in offsets:
        xs.append((ii + a).ravel())
        ys.append((jj + b).ravel())
    return np.concatenate(xs).astype(np.float64), np.concatenate(ys).astype(np.float64)


def to_texcoords(X, Y, width, height):
    """Texture coordinates of texel-space positions, in single precision."""
    return (np.asarray(X, np.float64) / width).astype(np.float32), \
        (np.asarray(Y, np.float64) / height).astype(np.float32)


# D4 acting on a square N x N map stored as m[y, x]; positions in texel units.
D4_NAMES = ["id", "flipx", "flipy", "rot180", "transpose", "antitranspose", "rot90", "rot270"]


def d4_map(m, name):
    if name == "id":
        return m.copy()
    if name == "flipx":
        return m[:, ::-1].copy()
    if name == "flipy":
        return m[::-1, :].copy()
    if name == "rot180":
        return m[::-1, ::-1].copy()
    if name == "transpose":
        return m.T.copy()
    if name == "antitranspose":
        return m[::-1, ::-1].T.copy()
    if name == "rot90":      # transpose then flip x
        return m.T[:, ::-1].copy()
    if name == "rot270":     # transpose then flip y
        return m.T[::-1, :].copy()
    raise ValueError(name)


def d4_points(X, Y, n, name):
    """Image of texel-space positions under the same map symmetry."""
    if name == "id":
        return X, Y
    if name == "flipx":
        return n - X, Y
    if name == "flipy":
        return X, n - Y
    if name == "rot180":
        return n - X, n - Y
    if name == "transpose":
        return Y, X
    if name == "antitranspose":
        return n - Y, n - X
    if name == "rot90":
        return n - Y, X
    if name == "rot270":
        return Y, n - X
    raise ValueError(name)


def staircase_mask(n, run, a, b):
    """Shadow iff (j - b) < floor((i - a) / run): the point-sampled half-plane
    below the line Y - b = (X - a) / run, with horizontal runs of `run` texels."""
    i = np.arange(n)[None, :]
    j = np.arange(n)[:, None]
    return (j - b) < np.floor_divide(i - a, run)
