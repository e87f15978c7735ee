"""Seeded synthetic scenes: shadow maps and light-space fragments.

Input generation only.  This module draws occluder and camera parameters
from a seeded PCG64 stream and hands the per-texel / per-pixel loops to
``scenegen.c``.  It holds no step of the revectorisation method (no shadow
test, no discontinuity, no visibility), imports neither the CUDA library nor
the oracle, and serves both of them the same arrays.

Scenes stand in for the paper's Fence and QuadBot scenes (§5), which are not
available: an orthographic light over a ground plane at depth 1, occluders
(rotated rectangles, thin tilted "fence" bars, spheres) at depth 1 - height,
and a perspective camera looking at a window of the ground.  Fragments on the
ground have depth exactly 1.0; fragments on a sphere's light-facing cap have
the sphere's analytic depth raised by RECEIVER_OFFSET towards the light.

Workloads (the five named configurations):
  C1  256^2 map, plane + 8 rectangles, 320x240 fragments on the plane
  C2  2048^2 map, fence of 40 bars + 30 spheres, 1920x1080 fragments
  C3  16 maps (4 lights x cascades 4096^2..512^2), 8 views 720p..4K, each
      pixel against every light with its cascade picked by screen band
  C4  4096^2 map, C2 mix scaled by 2, 3840x2160 fragments
  C5  8192^2 maps, 200 mixed occluders, 32 frames of 3840x2160 fragments,
      light moving 0.5 degrees per frame
"""
import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libscenegen.so")
SRC = os.path.join(HERE, "scenegen.c")

PLANE_DEPTH = 1.0
RECEIVER_OFFSET = 1e-3

_lib = None


def build(force=False):
    """Compile scenegen.c (OpenMP when the compiler has it)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    base = [os.environ.get("CC", "gcc"), "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
    try:
        subprocess.run(base + ["-fopenmp", SRC, "-o", tmp, "-lm"], check=True,
                       stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.run(base + [SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64, f64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        lib.sg_fill.argtypes = [vp, i32, i32, i64, f32]
        lib.sg_raster_rects.argtypes = [vp, i32, i32, i64, i32, vp, vp]
        lib.sg_raster_spheres.argtypes = [vp, i32, i32, i64, i32, vp, f64]
        lib.sg_fragments.argtypes = [i32, i32, vp, i32, i32, i32, vp, f64, f64, f32, vp, vp, vp, vp]
        lib.sg_fragments.restype = i32
        lib.sg_threads.restype = i32
        _lib = lib
    return _lib


def threads():
    return _load().sg_threads()


# ------------------------------------------------------------- parameters --

class _Draw:
    """Uniform draws from numpy's PCG64 stream (raw doubles only)."""

    def __init__(self, seed):
        self.g = np.random.Generator(np.random.PCG64(seed))

    def u(self, a, b):
        return a + (b - a) * float(self.g.random())

    def axis(self):
        """Uniformly oriented unit vector (direction of a rectangle's axis)."""
        while True:
            x, y = self.u(-1, 1), self.u(-1, 1)
            r2 = x * x + y * y
            if 1e-4 < r2 <= 1.0:
                r = math.sqrt(r2)
                return x / r, y / r

    def tilted(self, max_deg):
        """Unit vector at angle U[-max_deg, max_deg] from the +y (v) axis."""
        a = math.radians(self.u(-max_deg, max_deg))
        return math.sin(a), math.cos(a)


@dataclass
class Occluders:
    rects: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))   # cx cy ux uy ha hb
    rect_depth: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # cx cy R centre-depth

    def shifted(self, du):
        """Light-space parallax: every occluder moves by du * height along u."""
        r = self.rects.copy()
        s = self.spheres.copy()
        if len(r):
            r[:, 0] += du * (1.0 - self.rect_depth.astype(np.float64))
        if len(s):
            s[:, 0] += du * (1.0 - s[:, 3])
        return Occluders(r, self.rect_depth.copy(), s)


def _rects(d, n, size, side_lo, side_hi, h_lo, h_hi, margin=0.0):
    rects, dep = [], []
    for _ in range(n):
        cx, cy = d.u(margin, size - margin), d.u(margin, size - margin)
        ux, uy = d.axis()
        a, b = d.u(side_lo, side_hi), d.u(side_lo, side_hi)
        rects.append((cx, cy, ux, uy, a / 2, b / 2))
        dep.append(1.0 - d.u(h_lo, h_hi))
    return np.array(rects, np.float64).reshape(-1, 6), np.array(dep, np.float32)


def _bars(d, n, size, w_lo, w_hi, l_lo, l_hi, depth_lo, depth_hi, tilt_deg=30.0):
    rects, dep = [], []
    for _ in range(n):
        cx, cy = d.u(0, size), d.u(0, size)
        ux, uy = d.tilted(tilt_deg)
        length, width = d.u(l_lo, l_hi), d.u(w_lo, w_hi)
        rects.append((cx, cy, ux, uy, length / 2, width / 2))
        dep.append(d.u(depth_lo, depth_hi))
    return np.array(rects, np.float64).reshape(-1, 6), np.array(dep, np.float32)


def _spheres(d, n, size, r_lo, r_hi, c_lo, c_hi):
    out = []
    for _ in range(n):
        r = d.u(r_lo, r_hi)
        out.append((d.u(r, size - r), d.u(r, size - r), r, d.u(c_lo, c_hi)))
    return np.array(out, np.float64).reshape(-1, 4)


def raster(occ, width, height, zscale, out=None):
    """The shadow map of an occluder set (smallest depth per texel centre).
    `out`, when given, is a C-contiguous (height, width) float32 array."""
    lib = _load()
    depth = np.empty((height, width), np.float32) if out is None else out
    if depth.shape != (height, width) or depth.dtype != np.float32 or not depth.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous (height, width) float32 array")
    lib.sg_fill(depth.ctypes.data, width, height, width, PLANE_DEPTH)
    if len(occ.rects):
        r = np.ascontiguousarray(occ.rects, np.float64)
        dp = np.ascontiguousarray(occ.rect_depth, np.float32)
        lib.sg_raster_rects(depth.ctypes.data, width, height, width, len(r), r.ctypes.data, dp.ctypes.data)
    if len(occ.spheres):
        s = np.ascontiguousarray(occ.spheres, np.float64)
        lib.sg_raster_spheres(depth.ctypes.data, width, height, width, len(s), s.ctypes.data, float(zscale))
    return depth


# ------------------------------------------------------------------ camera --

def homography(src, dst):
    """3x3 matrix taking the four 2-D points src to dst (projective)."""
    A, b = [], []
    for (u, v), (X, Y) in zip(src, dst):
        A.append([u, v, 1, 0, 0, 0, -u * X, -v * X]); b.append(X)
        A.append([0, 0, 0, u, v, 1, -u * Y, -v * Y]); b.append(Y)
    h = np.linalg.solve(np.array(A, np.float64), np.array(b, np.float64))
    return np.append(h, 1.0).reshape(3, 3)


def view_window(d, size, sw, sh, side_lo, side_hi, margin=24.0, depth_ratio=2.0):
    """A perspective camera over the ground: the screen maps to a trapezoid of
    the light's texel space whose far (top) edge is depth_ratio times wider
    than its near (bottom) edge, side texels long, randomly rotated, at least
    `margin` texels inside the map."""
    side = d.u(side_lo, side_hi)
    half = side / 2
    reach = half * math.sqrt(2.0)
    cx, cy = d.u(margin + reach, size - margin - reach), d.u(margin + reach, size - margin - reach)
    ux, uy = d.axis()
    vx, vy = -uy, ux
    corners_local = [(-half, -half), (half, -half), (half / depth_ratio, half), (-half / depth_ratio, half)]
    dst = [(cx + a * ux + b * vx, cy + a * uy + b * vy) for a, b in corners_local]
    src = [(0.0, 0.0), (float(sw), 0.0), (float(sw), float(sh)), (0.0, float(sh))]
    return homography(src, dst), side


def fragments(hom, sw, sh, width, height, receivers=None, zscale=1.0, want_kind=False, out=None):
    """Light-space fragments (x, y, z) of every pixel, row-major.  `out`, when
    given, is a tuple of three contiguous float32 arrays of sw * sh elements."""
    lib = _load()
    n = sw * sh
    if out is None:
        x, y, z = (np.empty(n, np.float32) for _ in range(3))
    else:
        x, y, z = out
        for a in out:
            if a.shape != (n,) or a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError("out planes must be contiguous float32 arrays of sw * sh elements")
    kind = np.empty(n, np.int32) if want_kind else None
    sph = np.ascontiguousarray(receivers if receivers is not None else np.zeros((0, 4)), np.float64)
    h = np.ascontiguousarray(hom, np.float64)
    rc = lib.sg_fragments(sw, sh, h.ctypes.data, width, height, len(sph), sph.ctypes.data if len(sph) else None,
                          float(zscale), RECEIVER_OFFSET, PLANE_DEPTH, x.ctypes.data, y.ctypes.data, z.ctypes.data,
                          kind.ctypes.data if want_kind else None)
    if rc != 0:
        raise MemoryError("sg_fragments could not allocate its lookup grid")
    return x, y, z, kind


# ------------------------------------------------------------------ scenes --

@dataclass
class Frame:
    """One shadow map and one view's fragments."""
    name: str
    depth: np.ndarray          # (height, width) float32
    x: np.ndarray              # (n,) float32 texture coordinates
    y: np.ndarray
    z: np.ndarray              # (n,) float32 light depth
    screen: tuple              # (sw, sh)
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.x.shape[0])


def _seed(config_id, seed):
    return config_id * 1000 + seed


def config1(seed=0):
    """C1: 256^2 map, ground plane + 8 rotated rectangles (centre U[32,224],
    sides U[8,64] texels, height U[0.2,0.8]); 320x240 fragments on the plane,
    view window side U[48,128] texels (about 2.5-7 fragments per texel)."""
    d = _Draw(_seed(1, seed))
    size, sw, sh = 256, 320, 240
    r, dep = _rects(d, 8, size, 8, 64, 0.2, 0.8, margin=32)
    occ = Occluders(r, dep)
    depth = raster(occ, size, size, size)
    hom, side = view_window(d, size, sw, sh, 48, 128)
    x, y, z, _ = fragments(hom, sw, sh, size, size)
    return Frame("C1", depth, x, y, z, (sw, sh), {"window_side": side, "occluders": occ})


def _fence_scene(d, size, n_bars, n_sph, scale):
    r, dep = _bars(d, n_bars, size, 1 * scale, 6 * scale, 256 * scale, 2048 * scale, 0.05, 0.2)
    s = _spheres(d, n_sph, size, 10 * scale, 120 * scale, 0.4, 0.8)
    return Occluders(r, dep, s)


def config2(seed=0, screen=(1920, 1080)):
    """C2: 2048^2 map of a fence (40 bars, width U[1,6], length U[256,2048],
    tilt U[-30,30] degrees, depth U[0.05,0.2]) and 30 spheres (radius U[10,120],
    centre depth U[0.4,0.8]); 1920x1080 fragments on the plane and on sphere
    caps; window side U[480,960] texels."""
    d = _Draw(_seed(2, seed))
    size = 2048
    sw, sh = screen
    occ = _fence_scene(d, size, 40, 30, 1)
    depth = raster(occ, size, size, size)
    hom, side = view_window(d, size, sw, sh, 480, 960)
    x, y, z, kind = fragments(hom, sw, sh, size, size, occ.spheres, size, want_kind=True)
    return Frame("C2", depth, x, y, z, (sw, sh),
                 {"window_side": side, "sphere_fraction": float(np.mean(kind > 0)), "occluders": occ})


def config4(seed=0, screen=(3840, 2160)):
    """C4: 4096^2 map with the C2 mix scaled by two (80 bars, 60 spheres);
    3840x2160 fragments, window side U[960,1920] texels."""
    d = _Draw(_seed(4, seed))
    size = 4096
    sw, sh = screen
    occ = _fence_scene(d, size, 80, 60, 2)
    depth = raster(occ, size, size, size)
    hom, side = view_window(d, size, sw, sh, 960, 1920)
    x, y, z, kind = fragments(hom, sw, sh, size, size, occ.spheres, size, want_kind=True)
    return Frame("C4", depth, x, y, z, (sw, sh),
                 {"window_side": side, "sphere_fraction": float(np.mean(kind > 0)), "occluders": occ})


C5_FRAMES = 32
C5_SIZE = 8192
C5_SCREEN = (3840, 2160)
C5_DEG_PER_FRAME = 0.5
C5_PARALLAX = 2048.0   # texels of light-space shift per unit height per unit tan(angle)


class Config5:
    """C5: 8192^2 maps with 200 mixed occluders (70 rectangles, 70 bars, 60
    spheres) and a static camera of 3840x2160 fragments; the light turns
    0.5 degrees per frame, which shifts each occluder along u by its height
    times tan(angle) (parallax) and gives every frame its own map."""

    def __init__(self, seed=0, size=C5_SIZE, screen=C5_SCREEN, frames=C5_FRAMES):
        d = _Draw(_seed(5, seed))
        self.size, self.screen, self.frames = size, screen, frames
        sc = size / 8192.0
        r1, d1 = _rects(d, 70, size, 64 * sc, 512 * sc, 0.2, 0.8)
        r2, d2 = _bars(d, 70, size, 2 * sc, 24 * sc, 1024 * sc, 8192 * sc, 0.05, 0.2)
        sph = _spheres(d, 60, size, 40 * sc, 480 * sc, 0.4, 0.8)
        self.base = Occluders(np.concatenate([r1, r2]), np.concatenate([d1, d2]), sph)
        sw, sh = screen
        self.hom, self.window_side = view_window(d, size, sw, sh, 1536 * sc, 3072 * sc, margin=300 * sc)
        self.parallax = C5_PARALLAX * sc

    def occluders(self, f):
        du = self.parallax * math.tan(math.radians(C5_DEG_PER_FRAME * f))
        return self.base.shifted(du)

    def gbuffer(self, z):
        """(d, M) of this camera for light depths z (see gbuffer_of)."""
        return gbuffer_of(self.hom, z, self.screen[0], self.screen[1], self.size, self.size)

    def frame(self, f, out_depth=None, out_xyz=None):
        occ = self.occluders(f)
        depth = raster(occ, self.size, self.size, self.size, out=out_depth)
        sw, sh = self.screen
        x, y, z, kind = fragments(self.hom, sw, sh, self.size, self.size, occ.spheres, self.size,
                                  want_kind=True, out=out_xyz)
        return Frame("C5[%d]" % f, depth, x, y, z, self.screen,
                     {"window_side": self.window_side, "sphere_fraction": float(np.mean(kind > 0))})


def gbuffer_of(hom, z, sw, sh, width, height):
    """Depth-buffer form of a frame whose fragments come from the homography
    `hom` (screen pixel centre -> texel units) with light depths `z`: the
    4 x 4 float32 matrix M taking (px + 0.5, py + 0.5, d, 1) to light clip
    space (rows x, y, z, w: the homography scaled to texture coordinates,
    d itself, the homography's w) and the buffer d = z * w (float32,
    (sh, sw)), so that (X / W, Y / W, Z / W) is the fragment again, up to
    single-precision rounding."""
    h = np.asarray(hom, np.float64)
    m = np.zeros((4, 4), np.float64)
    m[0, [0, 1, 3]] = h[0] / width
    m[1, [0, 1, 3]] = h[1] / height
    m[2, 2] = 1.0
    m[3, [0, 1, 3]] = h[2]
    m = m.astype(np.float32)
    # w as the projection forms it (float32, row summed left to right, the
    # d term 0), so that a fragment on the ground (z = 1) projects back to
    # exactly z = 1 and keeps its shadow-test ties
    u = np.arange(sw, dtype=np.float32) + np.float32(0.5)
    v = np.arange(sh, dtype=np.float32) + np.float32(0.5)
    w = (m[3, 0] * u[None, :] + m[3, 1] * v[:, None]) + np.float32(0.0)
    w = w + m[3, 3]
    d = np.asarray(z, np.float32).reshape(sh, sw) * w
    return d.astype(np.float32), m


C3_VIEWS = [(1280, 720), (1600, 900), (1920, 1080), (2560, 1080),
            (2560, 1440), (3440, 1440), (3200, 1800), (3840, 2160)]
C3_CASCADES = [4096, 2048, 1024, 512]
C3_LIGHTS = 4


@dataclass
class Job:
    """One (view, light, cascade) group of fragments against one map."""
    map_index: int
    view: int
    light: int
    cascade: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray


class Config3:
    """C3: 4 lights x 4 cascades = 16 maps of uneven size (4096^2 .. 512^2,
    fence bars + spheres as in C2 scaled to the cascade) and 8 views of
    uneven resolution (720p .. 4K).  Every pixel is evaluated against every
    light; the cascade is picked by the pixel's screen band (bottom = near =
    finest cascade).  One job per (view, light, cascade)."""

    def __init__(self, seed=0, views=C3_VIEWS, cascades=C3_CASCADES, lights=C3_LIGHTS):
        d = _Draw(_seed(3, seed))
        self.views, self.cascades, self.lights = list(views), list(cascades), lights
        self.maps = []
        for l in range(lights):
            for c, size in enumerate(cascades):
                sc = size / 2048.0
                occ = _fence_scene(d, size, 40, 30, sc)
                self.maps.append(raster(occ, size, size, size))
        self.jobs = []
        nc = len(cascades)
        for v, (sw, sh) in enumerate(self.views):
            for l in range(lights):
                for c, size in enumerate(cascades):
                    # band c (0 = bottom rows) of the screen, nc bands
                    r0 = sh - (c + 1) * sh // nc
                    r1 = sh - c * sh // nc
                    bh = r1 - r0
                    hom, _ = view_window(d, size, sw, bh, size * 0.25, size * 0.5)
                    x, y, z, _ = fragments(hom, sw, bh, size, size)
                    self.jobs.append(Job(l * nc + c, v, l, c, x, y, z))

    @property
    def n(self):
        return sum(j.x.shape[0] for j in self.jobs)


# ------------------------------------------------------ surrogate weights --

MLP_IN, MLP_HID, MLP_OUT = 32, 64, 2


def mlp_init(seed):
    """Seeded initial weights of the 32-64-64-2 surrogate network (He-normal
    weights, zero biases), float32; both the GPU trainer and the oracle start
    from these arrays."""
    g = np.random.Generator(np.random.PCG64(7000 + seed))

    def he(fan_in, shape):
        return (g.standard_normal(shape) * math.sqrt(2.0 / fan_in)).astype(np.float32)

    return {"W1": he(28, (MLP_IN, MLP_HID)), "b1": np.zeros(MLP_HID, np.float32),
            "W2": he(MLP_HID, (MLP_HID, MLP_HID)), "b2": np.zeros(MLP_HID, np.float32),
            "W3": he(MLP_HID, (MLP_HID, MLP_OUT)) * np.float32(0.1), "b3": np.array([0.5, 0.05], np.float32)}
