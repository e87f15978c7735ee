"""ctypes front end of the plain C oracle (test infrastructure).

``evaluate`` follows Listing 1 of the paper with Listings 2-5 for every
fragment: shadow test (Eq. 1), four-neighbourhood discontinuity (Eqs. 2-4),
edge traversal (Listing 3), normalisation (Eq. 5) and the optimized
silhouette (Listing 4) or filtering (Listing 5) visibility.  The readings of
the paper's undefined helpers are documented in ``rbsm_oracle.c``.
"""
import ctypes
import numpy as np

from . import build as _build

MODE_SILHOUETTE = 1
MODE_FILTER = 2
MAXDIST = 16  # §3.1.3: the traversal cap the paper used

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_rbsm_eval.restype = ctypes.c_int
        lib.oracle_rbsm_eval.argtypes = [
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int32, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_project.restype = ctypes.c_int
        lib.oracle_project.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_rpcf.restype = ctypes.c_int
        lib.oracle_rpcf.argtypes = [
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        lib.oracle_shadow_map.restype = ctypes.c_int
        lib.oracle_shadow_map.argtypes = [
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
            ctypes.c_double, ctypes.c_float]
        lib.oracle_edge_visibility.restype = ctypes.c_double
        lib.oracle_edge_visibility.argtypes = [ctypes.c_int32] * 6 + [ctypes.c_double, ctypes.c_double]
        lib.oracle_features.restype = ctypes.c_int
        lib.oracle_features.argtypes = [
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def evaluate(depth, x, y, z, mode, max_dist=MAXDIST, want_rd=False, want_nrd=False):
    """Visibility (float64), codes (uint16) and optionally the four walks and
    the normalised vector for every fragment.

    depth: 2-D float32 array (height, width), row-major.
    x, y, z: 1-D float32 arrays of equal length.
    """
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    n = x.shape[0]
    if y.shape[0] != n or z.shape[0] != n:
        raise ValueError("x, y, z must have the same length")
    h, w = depth.shape
    vis = np.empty(n, np.float64)
    codes = np.empty(n, np.uint16)
    rd = np.empty((n, 4), np.int32) if want_rd else None
    nrd = np.empty((n, 4), np.float64) if want_nrd else None
    rc = lib.oracle_rbsm_eval(_ptr(depth), w, h, w, _ptr(x), _ptr(y), _ptr(z), n,
                              int(mode), int(max_dist), _ptr(vis), _ptr(codes), _ptr(rd), _ptr(nrd))
    if rc != 0:
        raise ValueError("oracle_rbsm_eval rejected its arguments (rc=%d)" % rc)
    out = {"vis": vis, "codes": codes}
    if want_rd:
        out["rd"] = rd
    if want_nrd:
        out["nrd"] = nrd
    return out


def project(gdepth, m):
    """Light-space planes (x, y, z float32, fragment f = py * width + px) of
    a depth buffer `gdepth` (height, width) through the 4 x 4 float32 matrix
    `m` (reading R21 in rbsm_oracle.c)."""
    lib = _load()
    gdepth = np.ascontiguousarray(gdepth, dtype=np.float32)
    m = np.ascontiguousarray(np.asarray(m, np.float32).reshape(4, 4))
    h, w = gdepth.shape
    out = [np.empty(h * w, np.float32) for _ in range(3)]
    rc = lib.oracle_project(_ptr(gdepth), w, h, w, _ptr(m), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
    if rc != 0:
        raise ValueError("oracle_project rejected its arguments (rc=%d)" % rc)
    return tuple(out)


def rpcf(depth, x, y, z, k=3, max_dist=MAXDIST):
    """RPCF visibility (float64) of every fragment: the mean RSMSS answer of
    the k x k samples shifted by whole texels around it (readings R18, R19
    in rbsm_oracle.c; k = 1 is RSMSS)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    n = x.shape[0]
    if y.shape[0] != n or z.shape[0] != n:
        raise ValueError("x, y, z must have the same length")
    h, w = depth.shape
    vis = np.empty(n, np.float64)
    rc = lib.oracle_rpcf(_ptr(depth), w, h, w, _ptr(x), _ptr(y), _ptr(z), n, int(k), int(max_dist), _ptr(vis))
    if rc != 0:
        raise ValueError("oracle_rpcf rejected its arguments (rc=%d)" % rc)
    return vis


def shadow_map(width, height, rects, rect_depth, spheres, zscale, ground=1.0):
    """Shadow map (float32, (height, width)) of analytic occluders by brute
    force (oracle/shadow_map_oracle.c): every texel centre against every
    occluder, smallest depth, `ground` where nothing covers it.
    rects: (n, 6) float64 cx cy ux uy ha hb; rect_depth: (n,) float32;
    spheres: (m, 4) float64 cx cy R centre-depth."""
    lib = _load()
    rects = np.ascontiguousarray(np.asarray(rects, np.float64).reshape(-1, 6))
    rect_depth = np.ascontiguousarray(np.asarray(rect_depth, np.float32).reshape(-1))
    spheres = np.ascontiguousarray(np.asarray(spheres, np.float64).reshape(-1, 4))
    if rect_depth.shape[0] != rects.shape[0]:
        raise ValueError("one depth per rectangle")
    depth = np.empty((height, width), np.float32)
    rc = lib.oracle_shadow_map(depth.ctypes.data, int(width), int(height), int(width),
                               _ptr(rects) if len(rects) else None, _ptr(rect_depth) if len(rects) else None,
                               len(rects), _ptr(spheres) if len(spheres) else None, len(spheres),
                               float(zscale), float(ground))
    if rc != 0:
        raise ValueError("oracle_shadow_map rejected its arguments (rc=%d)" % rc)
    return depth


def features(depth, x, y, z):
    """Surrogate features of every fragment: 25-bit 5x5 shadow-test pattern
    (uint32), in-texel offsets fx, fy and depth gap (float32)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    x, y, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
    n = x.shape[0]
    h, w = depth.shape
    bits = np.empty(n, np.uint32)
    fx, fy, gap = (np.empty(n, np.float32) for _ in range(3))
    rc = lib.oracle_features(_ptr(depth), w, h, w, _ptr(x), _ptr(y), _ptr(z), n,
                             _ptr(bits), _ptr(fx), _ptr(fy), _ptr(gap))
    if rc != 0:
        raise ValueError("oracle_features rejected its arguments (rc=%d)" % rc)
    return {"bits": bits, "fx": fx, "fy": fy, "gap": gap}


def edge_visibility(mode, opposite_x, opposite_y, ends_x, ends_y, dz, nx, ny):
    """The oracle's visibility of an edge fragment from its shape inputs
    (§4: discontinuity directions on both sides of each axis, ends found
    along each axis, dz = 1 - shadow test, normalised distances)."""
    return _load().oracle_edge_visibility(int(mode), int(opposite_x), int(opposite_y), int(ends_x), int(ends_y),
                                          int(dz), float(nx), float(ny))
