"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

The bar: discontinuity codes bit-exact; silhouette visibility (0/1, decided
in float32 on both sides) bit-exact; filtering visibility within 1e-5
absolute (the oracle computes it in float64, the kernel in float32: one
rounded add and divide per axis and two adds, all far below 1e-5).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402
from rbsm_scenes import shapes  # noqa: E402

FILTER_TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api as A
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gpu(api, depth, x, y, z, mode, max_dist=16, codes=True):
    d = depth if isinstance(depth, (torch.Tensor, api.MapTexture)) else dev(depth)
    fn = api.rbsm_visibility if mode == orc.MODE_SILHOUETTE else api.rsmss_filter
    xs, ys, zs = (t if isinstance(t, torch.Tensor) else dev(t) for t in (x, y, z))
    vis, cod = fn(d, xs, ys, zs, codes=codes, max_dist=max_dist)
    torch.cuda.synchronize()
    return vis.cpu().numpy(), (cod.cpu().numpy().view(np.uint16) if cod is not None else None)


def assert_parity(vis, codes, ref, mode, where=""):
    if codes is not None:
        bad = np.nonzero(codes != ref["codes"])[0]
        assert bad.size == 0, "%s: %d code mismatches, first %s gpu=%x cpu=%x" % (
            where, bad.size, bad[0], codes[bad[0]], ref["codes"][bad[0]])
    v = vis.astype(np.float64)
    if mode == orc.MODE_SILHOUETTE:
        bad = np.nonzero(~((v == ref["vis"]) | (np.isnan(v) & np.isnan(ref["vis"]))))[0]
        assert bad.size == 0, "%s: %d silhouette mismatches" % (where, bad.size)
    else:
        diff = np.abs(v - ref["vis"])
        both_nan = np.isnan(v) & np.isnan(ref["vis"])
        diff[both_nan] = 0.0
        assert not np.any(np.isnan(diff)), where
        assert diff.max(initial=0.0) <= FILTER_TOL, "%s: max |diff| %g" % (where, diff.max())


def check_both(api, depth, x, y, z, where, max_dist=16, texture=False):
    """Both visibility modes against the oracle; with texture=True through a
    texture view of the map as well (odd row pitches padded first)."""
    maps = [("loads", depth)]
    tex = None
    if texture:
        tex = _texture(api, dev(depth))
        maps.append(("texture", tex))
    for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
        ref = orc.evaluate(depth, x, y, z, mode, max_dist=max_dist)
        for name, d in maps:
            vis, cod = run_gpu(api, d, x, y, z, mode, max_dist=max_dist)
            assert_parity(vis, cod, ref, mode, "%s %s mode %d" % (where, name, mode))
    if tex is not None:
        tex.close()


# ------------------------------------------------------------- workloads --

def test_config1_full(api):
    import rbsm_scenes as sc
    for seed in range(3):
        f = sc.config1(seed)
        check_both(api, f.depth, f.x, f.y, f.z, "C1 seed %d" % seed)


def test_config2_full(api):
    import rbsm_scenes as sc
    f = sc.config2(0)
    check_both(api, f.depth, f.x, f.y, f.z, "C2")


def test_config4_full(api):
    import rbsm_scenes as sc
    f = sc.config4(0)
    check_both(api, f.depth, f.x, f.y, f.z, "C4")


def test_paper_shapes_on_gpu(api, golden_dir):
    """The Fig. 3 and staircase inputs of the oracle pins, on the GPU."""
    from tests.test_oracle_pins import _load_fig3, _inside
    rects = _load_fig3(golden_dir)
    for shape in "abcd":
        ti, tj = np.meshgrid(np.arange(3), np.arange(3), indexing="xy")
        depth = shapes.embed(_inside(rects[shape]["in"], ti + 0.5, tj + 0.5), 32, 12)
        X, Y = shapes.fragment_grid(12, 15, 12, 15, [((a + .5) / 5, (b + .5) / 5) for a in range(5) for b in range(5)])
        x, y = shapes.to_texcoords(X, Y, 32, 32)
        check_both(api, depth, x, y, np.ones_like(x), "fig3 %s" % shape, texture=True)
    for run_len in (1, 3, 7, 16):
        for orient in shapes.D4_NAMES:
            mask = shapes.staircase_mask(128, run_len, 8, 40)
            depth = shapes.d4_map(np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32), orient)
            X, Y = shapes.fragment_grid(20, 108, 20, 108, [((a + .5) / 4, (b + .5) / 4) for a in range(4) for b in range(4)])
            Xt, Yt = shapes.d4_points(X, Y, 128, orient)
            x, y = shapes.to_texcoords(Xt, Yt, 128, 128)
            check_both(api, depth, x, y, np.ones_like(x), "stair %d %s" % (run_len, orient), texture=True)


# ------------------------------------------------------------- edge cases --

def _random_case(rng, w, h, n, levels=(0.25, 0.5, 0.75, 1.0), spread=0.0):
    lv = np.array(levels, np.float32)
    depth = lv[rng.integers(0, len(lv), size=(h, w))]
    blob = rng.integers(0, 2, size=((h + 3) // 4, (w + 3) // 4)).repeat(4, 0).repeat(4, 1)[:h, :w].astype(bool)
    depth = np.where(blob, depth, np.float32(1.0)).astype(np.float32)
    x = rng.uniform(-spread, 1 + spread, n).astype(np.float32)
    y = rng.uniform(-spread, 1 + spread, n).astype(np.float32)
    z = lv[rng.integers(0, len(lv), n)]
    return depth, x, y, z


@pytest.mark.parametrize("n", [0, 1, 3, 1023, 1024, 1025, 4097, 100003])
def test_ragged_sizes(api, n):
    rng = np.random.default_rng(n)
    depth, x, y, z = _random_case(rng, 64, 48, n)
    if n == 0:
        vis, cod = run_gpu(api, depth, x, y, z, orc.MODE_FILTER)
        assert vis.shape == (0,)
        return
    check_both(api, depth, x, y, z, "n=%d" % n)


@pytest.mark.parametrize("w,h", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 700), (1000, 3), (257, 129)])
def test_degenerate_and_odd_maps(api, w, h):
    rng = np.random.default_rng(w * 1000 + h)
    depth, x, y, z = _random_case(rng, w, h, 5000)
    check_both(api, depth, x, y, z, "%dx%d" % (w, h), texture=True)


def test_out_of_range_and_nan_coordinates(api):
    """Clamp-to-edge addressing; a NaN coordinate maps to texel 0 on both sides."""
    rng = np.random.default_rng(5)
    depth, x, y, z = _random_case(rng, 40, 40, 20000, spread=0.3)
    x[::97] = np.nan
    y[::89] = -np.inf
    x[::83] = np.inf
    check_both(api, depth, x, y, z, "out-of-range")


def test_border_texels(api):
    """Fragments on every texel of the first and last rows and columns of
    random two-level maps, whose edges run along and across the borders: a
    walk there reads its side lines only towards neighbours inside the map
    (a clamped neighbour is the texel itself and shows no discontinuity), and
    the answers and codes match the oracle on plain loads and textures."""
    rng = np.random.default_rng(11)
    for w, h in ((64, 48), (7, 5), (2, 33)):
        depth = np.where(rng.random((h, w)) < 0.5, 0.3, 0.9).astype(np.float32)
        cols = np.concatenate([np.arange(w), np.arange(w), np.zeros(h, int), np.full(h, w - 1)])
        rows = np.concatenate([np.zeros(w, int), np.full(w, h - 1), np.arange(h), np.arange(h)])
        offs = [(0.25, 0.25), (0.75, 0.5), (0.5, 0.9)]
        x = np.concatenate([(cols + fx) / w for fx, _ in offs]).astype(np.float32)
        y = np.concatenate([(rows + fy) / h for _, fy in offs]).astype(np.float32)
        z = np.full(x.shape, 0.6, np.float32)
        for md in (2, 16):
            check_both(api, depth, x, y, z, "border %dx%d max_dist=%d" % (w, h, md), max_dist=md, texture=True)


@pytest.mark.parametrize("max_dist", [1, 2, 3, 5, 16, 17, 64, 255])
def test_max_dist(api, max_dist):
    """Every traversal cap, odd and even (the texture walk takes two steps
    per fetch), on plain loads and on a texture view."""
    import rbsm_scenes as sc
    f = sc.config1(1)
    check_both(api, f.depth, f.x, f.y, f.z, "max_dist=%d" % max_dist, max_dist=max_dist, texture=True)
    for run_len in (1, 2, 3, 16):
        mask = shapes.staircase_mask(96, run_len, 4, 30)
        depth = np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32)
        X, Y = shapes.fragment_grid(10, 86, 10, 86, [(0.25, 0.25), (0.75, 0.6)])
        x, y = shapes.to_texcoords(X, Y, 96, 96)
        for tr in (False, True):   # runs along x, then (transposed) along y
            d, u, v = (np.ascontiguousarray(depth.T), y, x) if tr else (depth, x, y)
            check_both(api, d, u, v, np.ones_like(x), "stair %d%s max_dist=%d" % (run_len, " T" if tr else "", max_dist),
                       max_dist=max_dist, texture=True)


def test_pitched_map_and_unaligned_planes(api):
    """A map whose rows are padded (pitch > width) and fragment planes that
    start 4 bytes past a 16-byte boundary (scalar path) give the same answers."""
    import rbsm_scenes as sc
    f = sc.config1(2)
    h, w = f.depth.shape
    big = torch.full((h, w + 13), 7.0, dtype=torch.float32, device="cuda")
    big[:, :w] = dev(f.depth)
    pitched = big[:, :w]
    assert pitched.stride(0) == w + 13
    n = f.n
    planes = []
    for a in (f.x, f.y, f.z):
        buf = torch.empty(n + 1, dtype=torch.float32, device="cuda")
        buf[1:] = dev(a)
        planes.append(buf[1:])
    assert planes[0].data_ptr() % 16 != 0
    for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
        ref = orc.evaluate(f.depth, f.x, f.y, f.z, mode)
        vis, cod = run_gpu(api, pitched, *planes, mode)
        assert_parity(vis, cod, ref, mode, "pitched/unaligned")
        vis2, _ = run_gpu(api, f.depth, f.x, f.y, f.z, mode, codes=False)
        assert np.array_equal(vis, vis2)


def test_equal_depth_ties(api):
    """Eq. 1 is strict: a fragment at exactly the stored depth is lit."""
    rng = np.random.default_rng(9)
    depth, x, y, z = _random_case(rng, 33, 31, 50000, levels=(0.5, 0.5000001, 1.0))
    check_both(api, depth, x, y, z, "ties")


def test_host_buffers_roundtrip(api):
    """CPU (host) tensors go through the same kernels and give the same answers."""
    import rbsm_scenes as sc
    f = sc.config1(0)
    args = [torch.from_numpy(a).pin_memory() for a in (f.depth, f.x, f.y, f.z)]
    vis_h, cod_h = api.rsmss_filter(*args, codes=True)
    ref = orc.evaluate(f.depth, f.x, f.y, f.z, orc.MODE_FILTER)
    assert_parity(vis_h.numpy(), cod_h.numpy().view(np.uint16), ref, orc.MODE_FILTER, "host")


TEX_PITCH_FLOATS = 128       # 512-byte rows: a multiple of any texture pitch alignment


def _texture(api, depth):
    """A texture view of the map (CUDA tensor).  A map whose rows are not a
    multiple of 512 bytes is first copied into a buffer of 512-byte rows
    (the view keeps its width), so every map size goes through the texture
    path; creation must succeed."""
    w = depth.shape[1]
    if (depth.stride(0) * 4) % 512 != 0:
        pitch = -(-w // TEX_PITCH_FLOATS) * TEX_PITCH_FLOATS
        padded = torch.full((depth.shape[0], pitch), float("nan"), dtype=torch.float32, device=depth.device)
        padded[:, :w] = depth
        depth = padded[:, :w]
    return api.MapTexture(depth)


@pytest.mark.parametrize("w,h", [(65536, 3), (3, 65536)])
def test_maximum_extent(api, w, h):
    """Maps at the largest extent a side may have (65536 texels): positions
    just below every power of two up to 2^16 and at the far border along the
    long side, both modes against the oracle, with plain loads and, where
    the device's texture limits take the map, texture gathers.  Only the
    tall map may be refused a texture (pitch-linear textures are limited in
    height)."""
    from paper_1711_07793_gb300 import _native as N
    rng = np.random.default_rng(w + 7 * h)
    depth, x, y, z = _random_case(rng, w, h, 30000, spread=0.05)
    long_side = max(w, h)
    pos = []
    for p in range(1, 17):
        b = 2.0 ** p
        for t in range(4):
            pos += [b - t * b * 2.0 ** -24, b - 1.0 - t * b * 2.0 ** -24, b + 0.5]
    pos += [long_side - 0.25, long_side - 1.0, long_side - 1.5]
    pos = np.array(pos, np.float64)
    pos = np.unique(pos[(pos >= 0) & (pos < long_side)].astype(np.float32))
    t_long = (np.repeat(pos.astype(np.float64), 40) / long_side).astype(np.float32)
    t_short = rng.uniform(0, 1, t_long.size).astype(np.float32)
    z_more = np.array([0.25, 0.5, 0.75, 1.0], np.float32)[rng.integers(0, 4, t_long.size)]
    if w > h:
        x, y = np.concatenate([x, t_long]), np.concatenate([y, t_short])
    else:
        x, y = np.concatenate([x, t_short]), np.concatenate([y, t_long])
    z = np.concatenate([z, z_more])
    check_both(api, depth, x, y, z, "%dx%d" % (w, h))
    d = dev(depth)
    try:
        tex = _texture(api, d)
    except N.RBSMError as e:
        assert e.code == N.RBSM_ERR_ARG and h > w
        return
    for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
        ref = orc.evaluate(depth, x, y, z, mode)
        vis, cod = run_gpu(api, tex, x, y, z, mode)
        assert_parity(vis, cod, ref, mode, "%dx%d texture mode %d" % (w, h, mode))
    tex.close()


def test_texture_refused_only_for_unaligned_rows(api):
    """rbsm_map_texture_create answers RBSM_ERR_ARG for rows that break the
    device's pitch alignment, and nothing else."""
    from paper_1711_07793_gb300 import _native as N
    buf = torch.zeros((16, 9), dtype=torch.float32, device="cuda")
    with pytest.raises(N.RBSMError) as e:
        api.MapTexture(buf)
    assert e.value.code == N.RBSM_ERR_ARG
    _texture(api, buf).close()


@pytest.mark.parametrize("which", ["C1", "C2", "odd"])
def test_texture_gather_path(api, which):
    """The texture-gather neighbourhood (rbsm_map_texture_create) gives
    exactly the same codes and answers as the plain loads, clamp-to-edge
    included (maps down to 1 x 1)."""
    import rbsm_scenes as sc
    cases = []
    if which == "C1":
        f = sc.config1(4)
        cases.append((f.depth, f.x, f.y, f.z))
    elif which == "C2":
        f = sc.config2(1, screen=(960, 540))
        cases.append((f.depth, f.x, f.y, f.z))
    else:
        rng = np.random.default_rng(77)
        for w, h in [(1, 1), (2, 2), (1, 9), (9, 1), (64, 48), (257, 129)]:
            cases.append(_random_case(rng, w, h, 20000, spread=0.2))
    for depth, x, y, z in cases:
        d = dev(depth)
        tex = _texture(api, d)
        for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
            ref = orc.evaluate(depth, x, y, z, mode)
            vis, cod = run_gpu(api, tex, x, y, z, mode)
            assert_parity(vis, cod, ref, mode, "texture %s %s mode %d" % (which, depth.shape, mode))
        tex.close()
