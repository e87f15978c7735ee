"""GPU parity of the shadow-map rasteriser (rbsm_shadow_map) with the
brute-force oracle: bit-exact maps (integer-exact coverage decisions and
the same double operations for the caps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api as A
    return A


def gpu_map(api, rects, rdep, sph, w, h, zs, ground=1.0):
    occ = api.DeviceOccluders(rects, rdep, sph)
    m = api.rbsm_shadow_map(occ, w, h, zs, ground)
    torch.cuda.synchronize()
    return m.cpu().numpy()


def same(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("which", ["c1", "c2", "c5_1024"])
def test_generator_scenes(api, which):
    import rbsm_scenes as sc
    if which == "c1":
        rng = np.random.default_rng(1)
        rects = np.array([[rng.uniform(32, 224), rng.uniform(32, 224), np.cos(a), np.sin(a),
                           rng.uniform(4, 32), rng.uniform(4, 32)] for a in rng.uniform(0, np.pi, 8)])
        occ = sc.Occluders(rects, rng.uniform(0.2, 0.8, 8).astype(np.float32), np.zeros((0, 4)))
        w = h = 256
    elif which == "c2":
        occ = sc._fence_scene(sc._Draw(sc._seed(2, 0)), 2048, 40, 30, 1.0)
        w = h = 2048
    else:
        occ = sc.Config5(0, size=1024, frames=4).occluders(3)
        w = h = 1024
    ref = orc.shadow_map(w, h, occ.rects, occ.rect_depth, occ.spheres, float(w))
    got = gpu_map(api, occ.rects, occ.rect_depth, occ.spheres, w, h, float(w))
    assert same(got, ref)


@pytest.mark.parametrize("w,h", [(1, 1), (31, 33), (33, 31), (100, 7), (7, 100)])
def test_odd_sizes_and_many_occluders(api, w, h):
    """Partial tiles, more occluders than one culling round (600 of each),
    occluders reaching past the map, exact ties on texel centres."""
    rng = np.random.default_rng(w * 100 + h)
    n = 600
    ang = rng.uniform(0, np.pi, n)
    rects = np.stack([rng.uniform(-10, w + 10, n), rng.uniform(-10, h + 10, n), np.cos(ang), np.sin(ang),
                      rng.uniform(0.2, 8, n), rng.uniform(0.2, 8, n)], 1)
    rects[::7, 2:4] = [1.0, 0.0]                  # axis-aligned, dyadic: edges through texel centres
    rects[::7, 0:2] = np.floor(rects[::7, 0:2])
    rects[::7, 4:6] = np.floor(rects[::7, 4:6] * 2) / 2 + 0.5
    rdep = rng.uniform(0.05, 0.95, n).astype(np.float32)
    sph = np.stack([rng.uniform(-5, w + 5, n), rng.uniform(-5, h + 5, n), rng.uniform(0.3, 6, n),
                    rng.uniform(0.4, 0.9, n)], 1)
    sph[::5, 0:2] = np.floor(sph[::5, 0:2]) + 0.5  # discs centred on texel centres with integer radii
    sph[::5, 2] = np.floor(sph[::5, 2])
    ref = orc.shadow_map(w, h, rects, rdep, sph, 16.0, ground=0.97)
    got = gpu_map(api, rects, rdep, sph, w, h, 16.0, ground=0.97)
    assert same(got, ref)


def test_only_ground_and_pitched_output(api):
    occ = api.DeviceOccluders(np.zeros((0, 6)), np.zeros(0, np.float32), np.zeros((0, 4)))
    m = api.rbsm_shadow_map(occ, 40, 30, 1.0, ground=0.5)
    assert torch.all(m == 0.5)
    big = torch.full((30, 48), 7.0, device="cuda")
    rects = [[10.0, 10.0, 0.6, 0.8, 5.0, 3.0]]
    occ2 = api.DeviceOccluders(rects, [0.25], np.zeros((0, 4)))
    api.rbsm_shadow_map(occ2, 40, 30, 40.0, out=big[:, :40])
    torch.cuda.synchronize()
    ref = orc.shadow_map(40, 30, rects, [0.25], np.zeros((0, 4)), 40.0)
    assert same(big[:, :40].cpu().numpy(), ref)
    assert torch.all(big[:, 40:] == 7.0)          # the pitch padding is untouched


def test_full_size_c5_frame(api):
    """One 8192^2 C5 map against the generator's rasteriser (bytes equal to
    the oracle's on the C5 scenes, checked on the CPU at 1024^2)."""
    import rbsm_scenes as sc
    c5 = sc.Config5(0, frames=32)
    occ = c5.occluders(17)
    ref = sc.raster(occ, c5.size, c5.size, c5.size)
    got = gpu_map(api, occ.rects, occ.rect_depth, occ.spheres, c5.size, c5.size, float(c5.size))
    assert same(got, ref)


@pytest.mark.parametrize("zs", [1024.0, 64.0, 0.5, 1000.0, 3.0])
def test_sphere_caps_against_the_oracle(api, zs):
    """Cap depths of many large and tiny discs, with centre depths that put
    caps below zero and above one, at power-of-two scales (the float-float
    evaluation with its rounding-boundary fallback) and other scales (the
    double operations throughout): bit-exact against the oracle."""
    w = h = 1024
    rng = np.random.default_rng(int(zs * 16))
    n = 300
    r = np.concatenate([rng.uniform(20, 300, 30), rng.uniform(0.3, 6, n - 30)])
    c = r / zs + rng.uniform(0.01, 0.6, n)        # caps above zero
    c[::10] = rng.uniform(-0.3, 0.3, len(c[::10]))
    c[5::10] = r[5::10] / zs                       # the cap's centre at depth zero
    sph = np.stack([rng.uniform(-50, w + 50, n), rng.uniform(-50, h + 50, n), r, c], 1)
    sph[::11, 0:2] = np.floor(sph[::11, 0:2]) + 0.5
    ref = orc.shadow_map(w, h, np.zeros((0, 6)), np.zeros(0, np.float32), sph, zs, ground=2.0)
    got = gpu_map(api, np.zeros((0, 6)), np.zeros(0, np.float32), sph, w, h, zs, ground=2.0)
    assert same(got, ref)
    assert np.mean(ref < 2.0) > 0.15 and np.mean((ref > 0) & (ref < 2.0)) > 0.01


@pytest.mark.parametrize("nr,ns", [(1100, 0), (0, 1100), (513, 1025), (256, 256), (257, 10), (384, 384)])
def test_occluders_in_several_passes(api, nr, ns):
    """More than one pass of occluders of a kind (512 each): the running
    minimum is carried through the map between passes."""
    w, h = 150, 130
    rng = np.random.default_rng(nr * 7 + ns)
    ang = rng.uniform(0, np.pi, nr)
    rects = np.stack([rng.uniform(-10, w + 10, nr), rng.uniform(-10, h + 10, nr), np.cos(ang), np.sin(ang),
                      rng.uniform(0.2, 12, nr), rng.uniform(0.2, 12, nr)], 1).reshape(-1, 6)
    rdep = rng.uniform(0.05, 0.95, nr).astype(np.float32)
    sph = np.stack([rng.uniform(-5, w + 5, ns), rng.uniform(-5, h + 5, ns), rng.uniform(0.3, 9, ns),
                    rng.uniform(0.2, 0.9, ns)], 1).reshape(-1, 4)
    ref = orc.shadow_map(w, h, rects, rdep, sph, 64.0, ground=0.99)
    got = gpu_map(api, rects, rdep, sph, w, h, 64.0, ground=0.99)
    assert same(got, ref)
    assert np.mean(ref < 0.99) > 0.5


def test_signed_zero_ties_resolve_in_definition_order(api):
    """Equal depths of different sign (+0, -0): a texel keeps the first in
    the definition's order (rectangles by index, then spheres), which the
    kernel's order-keeping gathering of survivors preserves."""
    rng = np.random.default_rng(5)
    n = 300
    rects = np.stack([rng.uniform(0, 48, n), rng.uniform(0, 48, n), np.ones(n), np.zeros(n),
                      rng.uniform(2, 10, n), rng.uniform(2, 10, n)], 1)
    rdep = np.where(rng.random(n) < 0.5, np.float32(0.0), np.float32(-0.0)).astype(np.float32)
    sph = np.stack([rng.uniform(0, 48, 40), rng.uniform(0, 48, 40), rng.uniform(1, 6, 40),
                    rng.uniform(0, 6, 40) / 16.0], 1)
    sph[:, 3] = sph[:, 2] / 16.0                   # caps reaching depth exactly 0 at their centres
    ref = orc.shadow_map(48, 48, rects, rdep, sph, 16.0, ground=1.0)
    got = gpu_map(api, rects, rdep, sph, 48, 48, 16.0, ground=1.0)
    assert same(got, ref)
    zero = ref == 0.0
    assert np.any(zero & np.signbit(ref)) and np.any(zero & ~np.signbit(ref))


def test_several_maps_in_one_call(api):
    """rbsm_shadow_maps: each map equals rbsm_shadow_map's bit for bit, with
    the maps' kernels overlapped (separate buffers) and in order (one buffer
    for all: it ends with the last map); work queued right after the call
    sees every map."""
    import rbsm_scenes as sc
    c5 = sc.Config5(0, size=1024, frames=6)
    occs = [api.DeviceOccluders(o.rects, o.rect_depth, o.spheres) for o in (c5.occluders(f) for f in range(6))]
    singles = [api.rbsm_shadow_map(o, 1024, 1024, 1024.0) for o in occs]
    torch.cuda.synchronize()
    outs = [torch.full((1024, 1024), 7.0, device="cuda") for _ in occs]
    api.rbsm_shadow_maps(occs, 1024, 1024, 1024.0, outs=outs)
    sums = torch.stack([o.double().sum() for o in outs])          # same stream, no sync before
    torch.cuda.synchronize()
    assert torch.equal(sums, torch.stack([m.double().sum() for m in singles]))
    for a, b in zip(outs, singles):
        assert same(a.cpu().numpy(), b.cpu().numpy())
    shared = torch.empty((1024, 1024), device="cuda")
    api.rbsm_shadow_maps(occs, 1024, 1024, 1024.0, outs=[shared] * len(occs))
    torch.cuda.synchronize()
    assert same(shared.cpu().numpy(), singles[-1].cpu().numpy())


@pytest.mark.parametrize("zs", [65536.0, 1000.0])
def test_far_centres_at_the_maximum_extent(api, zs):
    """Discs whose centres sit near x = 65536 (the largest map width), where
    the float-float offsets carry the centre's magnitude: bit-exact against
    the oracle at a power-of-two scale (float-float path) and another."""
    w, h = 65536, 16
    rng = np.random.default_rng(int(zs))
    n = 40
    sph = np.stack([rng.uniform(w - 3000, w + 5, n), rng.uniform(-4, h + 4, n), rng.uniform(0.6, 12, n),
                    rng.uniform(0.3, 0.8, n)], 1)
    sph[::4, 0:2] = np.floor(sph[::4, 0:2]) + 0.5
    rects = np.array([[w - 100.25, 8.0, 0.6, 0.8, 40.0, 3.0]])
    ref = orc.shadow_map(w, h, rects, [0.2], sph, zs, ground=1.0)
    got = gpu_map(api, rects, [0.2], sph, w, h, zs, ground=1.0)
    assert same(got, ref)
    assert np.sum(ref < 1.0) > 1000


def test_full_size_maps_in_one_call_as_the_bench_runs_them(api):
    """rbsm_shadow_maps over four full-size C5 maps (8192^2) in one call,
    overlapped as dependent launches (the bench's launch configuration):
    each map equals the generator's rasteriser bit for bit."""
    import rbsm_scenes as sc
    c5 = sc.Config5(0, frames=32)
    frames = (3, 11, 19, 27)
    occs = [c5.occluders(f) for f in frames]
    dev_occs = [api.DeviceOccluders(o.rects, o.rect_depth, o.spheres) for o in occs]
    outs = api.rbsm_shadow_maps(dev_occs, c5.size, c5.size, float(c5.size))
    torch.cuda.synchronize()
    for o, m in zip(occs, outs):
        ref = sc.raster(o, c5.size, c5.size, c5.size)
        assert same(m.cpu().numpy(), ref)
