"""GPU parity of RPCF (rbsm_rpcf, PCF over the RSMSS answer, §5.3) with the
oracle: every fragment within 1e-5 (the oracle sums float64 answers, the
kernel float32 ones in the same order); k = 1 equals rsmss_filter bit for
bit; plain loads and texture gathers give the same bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402
from rbsm_scenes import shapes  # noqa: E402

TOL = 1e-5


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


def gpu_rpcf(api, depth, x, y, z, k, max_dist=16, texture=False):
    from paper_1711_07793_gb300 import _native as N
    d = dev(depth) if isinstance(depth, np.ndarray) else depth
    tex = None
    if texture:
        try:
            tex = api.MapTexture(d)
        except N.RBSMError as e:
            assert e.code == N.RBSM_ERR_ARG
            return None
    v = api.rbsm_rpcf(tex or d, dev(x), dev(y), dev(z), k=k, max_dist=max_dist)
    torch.cuda.synchronize()
    out = v.cpu().numpy()
    if tex is not None:
        tex.close()
    return out


def check(api, depth, x, y, z, k, where, max_dist=16):
    ref = orc.rpcf(depth, x, y, z, k=k, max_dist=max_dist)
    got = gpu_rpcf(api, depth, x, y, z, k, max_dist)
    g = got.astype(np.float64)
    both_nan = np.isnan(g) & np.isnan(ref)
    assert not np.any(np.isnan(g) ^ np.isnan(ref)), where
    diff = np.abs(g - ref)
    diff[both_nan] = 0.0
    assert diff.max(initial=0.0) <= TOL, "%s: max |diff| %g" % (where, diff.max())
    tex = gpu_rpcf(api, depth, x, y, z, k, max_dist, texture=True)
    if tex is not None:
        assert np.array_equal(tex.view(np.uint32), got.view(np.uint32)), where + " texture"
    return got


@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_config1(api, k):
    import rbsm_scenes as sc
    f = sc.config1(0)
    got = check(api, f.depth, f.x, f.y, f.z, k, "C1 k=%d" % k)
    if k == 1:
        vis, _ = api.rsmss_filter(dev(f.depth), dev(f.x), dev(f.y), dev(f.z))
        assert np.array_equal(vis.cpu().numpy().view(np.uint32), got.view(np.uint32))


def test_config2_sampled(api):
    import rbsm_scenes as sc
    f = sc.config2(0, screen=(960, 540))
    check(api, f.depth, f.x, f.y, f.z, 3, "C2")


@pytest.mark.parametrize("n", [1, 3, 127, 129, 4097])
def test_ragged(api, n):
    rng = np.random.default_rng(n)
    depth = np.where(rng.random((40, 56)) < 0.3, np.float32(0.5), np.float32(1.0)).astype(np.float32)
    x = rng.uniform(0, 1, n).astype(np.float32)
    y = rng.uniform(0, 1, n).astype(np.float32)
    check(api, depth, x, y, np.ones_like(x), 3, "n=%d" % n)


def test_empty(api):
    v = api.rbsm_rpcf(dev(np.ones((4, 4), np.float32)), *(torch.empty(0, device="cuda") for _ in range(3)))
    assert v.shape == (0,)


@pytest.mark.parametrize("k", [3, 5, 7])
@pytest.mark.parametrize("w,h", [(1, 1), (2, 2), (1, 9), (9, 1), (3, 700), (257, 129)])
def test_odd_maps_and_borders(api, w, h, k):
    """Clamped borders and NaN / infinite coordinates: fragments outside the
    shared block, whose samples the lane walks itself, beside block
    fragments whose sums count their pending samples."""
    rng = np.random.default_rng(w * 1000 + h)
    depth = np.where(rng.random((h, w)) < 0.35, np.float32(0.25), np.float32(1.0)).astype(np.float32)
    x = rng.uniform(-0.3, 1.3, 6000).astype(np.float32)
    y = rng.uniform(-0.3, 1.3, 6000).astype(np.float32)
    x[::71] = np.nan
    y[::67] = np.inf
    check(api, depth, x, y, np.full_like(x, 0.5), k, "%dx%d k %d" % (w, h, k))


@pytest.mark.parametrize("max_dist", [1, 2, 16, 255])
def test_max_dist_and_staircases(api, max_dist):
    for run_len in (1, 3, 16):
        mask = shapes.staircase_mask(96, run_len, 4, 30)
        depth = np.where(mask, shapes.BLOCKER, shapes.LIT).astype(np.float32)
        X, Y = shapes.fragment_grid(10, 86, 10, 86, [(0.25, 0.25), (0.75, 0.6)])
        x, y = shapes.to_texcoords(X, Y, 96, 96)
        for k in (3, 5):
            check(api, depth, x, y, np.ones_like(x), k, "stair %d md %d k %d" % (run_len, max_dist, k), max_dist)


def test_rejects_bad_k(api):
    from paper_1711_07793_gb300 import _native as N
    d, x = dev(np.ones((4, 4), np.float32)), torch.zeros(8, device="cuda")
    for k in (0, 2, 9):
        with pytest.raises(N.RBSMError) as e:
            api.rbsm_rpcf(d, x, x, x, k=k)
        assert e.value.code == N.RBSM_ERR_ARG


def test_full_size_frame_sampled(api):
    """One 3840x2160 frame on an 8192^2 map at the bench's size: every
    answer of a sample of fragments against the oracle."""
    import bench
    _, host = bench.make_workload(1, 0, pin=False)
    depth = host[0]["depth"].numpy()
    x, y, z = (host[0]["xyz"][q].numpy() for q in range(3))
    got = gpu_rpcf(api, depth, x, y, z, 3)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(x.shape[0], 200000, replace=False))
    ref = orc.rpcf(depth, x[idx], y[idx], z[idx], k=3)
    assert np.abs(got[idx].astype(np.float64) - ref).max() <= TOL
    assert 0.0 < np.mean((ref > 0) & (ref < 1)) < 0.5


@pytest.mark.parametrize("k", [3, 5, 7])
def test_shared_block_conditions(api, k):
    """Fragments where u + a rounds up to the next integer (u just below a
    power of two minus a), and fragments at the map's borders, where the
    samples' texels cannot come from one shared block: the same answers as
    the oracle, and texture gathers equal to plain loads."""
    w, h = 8192, 40
    rng = np.random.default_rng(k)
    depth = np.where(rng.random((h, w)) < 0.35, np.float32(0.25), np.float32(1.0)).astype(np.float32)
    us = []
    for b in (2048.0, 4096.0, 8192.0):
        for a in range(0, 4):
            for t in range(0, 6):
                us.append(b - a - t * 2.0 ** -12)       # ulp of [2048, 4096) is 2^-12
                us.append(b - a - t * 2.0 ** -11)
    us += [0.0, 0.5, 1.0, 1.999, 2.0, 2.5, 3.0, 3.5, 4.0, 8188.5, 8189.0, 8190.25, 8191.75]
    u = np.unique(np.array(us, np.float32).astype(np.float64))   # representable texel-space positions
    u = u[(u >= 0) & (u < w)]
    vv = rng.uniform(0, h, u.size * 8)
    uu = np.repeat(u, 8)
    x = (uu / w).astype(np.float32)
    assert np.array_equal(x.astype(np.float64) * w, uu)   # u = x * 8192 exactly
    y = (vv / h).astype(np.float32)
    z = np.full_like(x, 0.5)
    check(api, depth, x, y, z, k, "block k=%d" % k)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_shared_block_at_the_maximum_extent(api, k):
    """The shared-block test at the largest map width (65536 texels): for
    positions just below 2^14, 2^15 and 2^16 minus a whole offset, u + a can
    round up while u - a stays exact (the kernel relies on the latter for
    every u below 2^16), and the far border clamps; answers equal the
    oracle's, texture gathers equal plain loads."""
    w, h = 65536, 12
    rng = np.random.default_rng(100 + k)
    depth = np.where(rng.random((h, w)) < 0.35, np.float32(0.25), np.float32(1.0)).astype(np.float32)
    us = []
    for b in (16384.0, 32768.0, 65536.0):
        ulp = b * 2.0 ** -24                      # spacing of the floats just below b
        for a in range(0, 4):
            for t in range(0, 6):
                us.append(b - a - t * ulp)
                us.append(b - a - t * 2.0 * ulp)
    us += [65529.5, 65530.0, 65532.25, 65533.0, 65534.75, 65535.0, 65535.5, 65535.99609375]
    u = np.unique(np.array(us, np.float32).astype(np.float64))
    u = u[(u >= 0) & (u < w)]
    uu = np.repeat(u, 6)
    x = (uu / w).astype(np.float32)
    assert np.array_equal(x.astype(np.float64) * w, uu)   # u = x * 65536 exactly
    y = (rng.uniform(0, h, uu.size) / h).astype(np.float32)
    z = np.full_like(x, 0.5)
    check(api, depth, x, y, z, k, "max extent k=%d" % k)


@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_workspace_schedule_gives_the_same_bits(api, k):
    """rbsm_rpcf_ws (tiles taken from a counter) against rbsm_rpcf (a fixed
    partition): the same bits on C2 at a reduced view, on odd maps with
    borders and non-finite coordinates, and twice in a row with one
    workspace (the call zeroes its counter)."""
    import rbsm_scenes as sc
    f = sc.config2(5, screen=(960, 540))
    rng = np.random.default_rng(40 + k)
    odd = np.where(rng.random((129, 257)) < 0.35, np.float32(0.25), np.float32(1.0)).astype(np.float32)
    ox = rng.uniform(-0.3, 1.3, 30000).astype(np.float32)
    oy = rng.uniform(-0.3, 1.3, 30000).astype(np.float32)
    ox[::97] = np.nan
    cases = [(f.depth, f.x, f.y, f.z), (odd, ox, oy, np.full_like(ox, 0.5))]
    ws = torch.zeros(1, dtype=torch.int64, device="cuda")
    for depth, x, y, z in cases:
        d, xs, ys, zs = dev(depth), dev(x), dev(y), dev(z)
        ref = api.rbsm_rpcf(d, xs, ys, zs, k=k, workspace=None)           # rbsm_rpcf
        for _ in range(2):
            got = api.rbsm_rpcf(d, xs, ys, zs, k=k, workspace=ws)
            auto = api.rbsm_rpcf(d, xs, ys, zs, k=k)                     # the binding's per-stream counter
            torch.cuda.synchronize()
            assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
            assert torch.equal(auto.view(torch.int32), ref.view(torch.int32))
