"""GPU tests of the stager (host-resident batches, rbsm_stager_*).

The stager copies in only the window of each map within max_dist + 1
texels of the fragments' texels, so these tests check that the answers
equal, bit for bit, those of rbsm_batch_run on device copies of the whole
batch (whose parity with the oracle the other GPU tests establish), with
one direct oracle comparison, and that the bytes it reports are the
fragment planes plus exactly those windows.
"""
import ctypes

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


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def texel_index(v, size):
    """clamp(floor(v * size)) in float32, as the kernels compute it."""
    u = np.float32(v) * np.float32(size)
    with np.errstate(invalid="ignore"):
        c = np.floor(u)
    c = np.where(np.isnan(c), np.float32(0), c)
    return np.clip(c, 0, size - 1).astype(np.int64)


def window_bytes(depth, xs, ys, max_dist):
    h, w = depth.shape
    i = np.concatenate([texel_index(x, w) for x in xs])
    j = np.concatenate([texel_index(y, h) for y in ys])
    if i.size == 0:
        return 0
    halo = max_dist + 1
    # columns widened to 4-texel boundaries (16-byte row pieces), clipped
    i0 = max(i.min() - halo, 0) // 4 * 4
    i1 = min(min(i.max() + halo, w - 1) | 3, w - 1)
    rows = min(j.max() + halo, h - 1) - max(j.min() - halo, 0) + 1
    return int(rows * (i1 - i0 + 1) * 4)


def random_map(rng, w, h):
    lv = np.array([0.25, 0.5, 0.75], np.float32)
    depth = np.ones((h, w), np.float32)
    for _ in range(max(2, w * h // 4000)):
        cx, cy = rng.integers(0, w), rng.integers(0, h)
        rx, ry = rng.integers(1, max(2, w // 6)), rng.integers(1, max(2, h // 6))
        depth[max(cy - ry, 0):cy + ry, max(cx - rx, 0):cx + rx] = lv[rng.integers(0, 3)]
    return depth


def random_frags(rng, n, lo=0.1, hi=0.6, spread=0.0):
    a, b = rng.uniform(lo, hi), rng.uniform(lo, hi)
    x = rng.uniform(a - spread, a + 0.3 + spread, n).astype(np.float32)
    y = rng.uniform(b - spread, b + 0.3 + spread, n).astype(np.float32)
    z = np.array([0.3, 0.6, 0.9, 1.0], np.float32)[rng.integers(0, 4, n)]
    return x, y, z


def device_answers(api, maps, jobs_np, max_dist, texture):
    """rbsm_batch_run on device copies of everything: the reference."""
    from paper_1711_07793_gb300 import _native as N
    dmaps = [torch.from_numpy(m).cuda() for m in maps]
    dm = list(dmaps)
    if texture:
        for k, m in enumerate(dmaps):
            try:
                dm[k] = api.MapTexture(m)
            except N.RBSMError as e:       # a pitch the texture unit refuses: plain loads
                assert e.code == N.RBSM_ERR_ARG
    jobs = [api.Job(k, *(torch.from_numpy(a).cuda() for a in (x, y, z)), mode=mode, codes=True if codes else None)
            for (k, x, y, z, mode, codes) in jobs_np]
    b = api.Batch(dm, jobs, max_dist=max_dist)
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    out = [((j.vis_silhouette.cpu().numpy() if j.vis_silhouette is not None else None),
            (j.vis_filter.cpu().numpy() if j.vis_filter is not None else None),
            (j.codes.cpu().numpy() if j.codes is not None else None)) for j in jobs]
    for t in dm:
        if isinstance(t, api.MapTexture):
            t.close()
    return out


def stager_answers(api, st, maps, jobs_np, max_dist, stream=None):
    hmaps = [pinned(m) for m in maps]
    jobs = [api.Job(k, pinned(x), pinned(y), pinned(z), mode=mode, codes=True if codes else None)
            for (k, x, y, z, mode, codes) in jobs_np]
    st.run(hmaps, jobs, max_dist=max_dist, stream=stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return [((j.vis_silhouette.numpy().copy() if j.vis_silhouette is not None else None),
             (j.vis_filter.numpy().copy() if j.vis_filter is not None else None),
             (j.codes.numpy().copy() if j.codes is not None else None)) for j in jobs]


def assert_same(a, b, where):
    for k, (ra, rb) in enumerate(zip(a, b)):
        for name, u, v in zip(("sil", "fil", "codes"), ra, rb):
            assert (u is None) == (v is None), (where, k, name)
            if u is not None:
                assert np.array_equal(u.view(np.uint32) if u.dtype == np.float32 else u,
                                      v.view(np.uint32) if v.dtype == np.float32 else v), (where, k, name)


@pytest.mark.parametrize("texture", [True, False])
def test_stager_equals_device_batch(api, texture):
    rng = np.random.default_rng(11)
    sizes = [(300, 200), (64, 64), (1024, 777), (257, 129), (2048, 2048)]
    maps = [random_map(rng, w, h) for w, h in sizes]
    jobs_np = []
    for k, (w, h) in enumerate(sizes):
        for v, n in enumerate((20000 + 37 * k, 5001, 0) if k % 2 == 0 else (77777,)):
            x, y, z = random_frags(rng, n, spread=0.05 * v)
            jobs_np.append((k, x, y, z, 1 + (k + v) % 3, (k + v) % 2 == 0))
    st = api.Stager(max_fragments=200000, max_width=2048, max_height=2048, slots=2, texture=texture)
    for rnd in range(2):          # two runs: the ring wraps and slots keep older maps' texels
        ref = device_answers(api, maps, jobs_np, 16, texture)
        got = stager_answers(api, st, maps, jobs_np, 16)
        assert_same(got, ref, "round %d" % rnd)
        maps = maps[::-1]
        jobs_np = [(len(maps) - 1 - k, x, y, z, m, c) for (k, x, y, z, m, c) in jobs_np]
    assert st.status() == 0
    st.close()


def test_stager_matches_oracle_and_counts_bytes(api):
    import rbsm_scenes as sc
    f = sc.config2(0, screen=(640, 360))
    st = api.Stager(max_fragments=f.n, max_width=2048, max_height=2048)
    jobs_np = [(0, f.x, f.y, f.z, 3, False)]
    got = stager_answers(api, st, [f.depth], jobs_np, 16)
    ref_s = orc.evaluate(f.depth, f.x, f.y, f.z, orc.MODE_SILHOUETTE)
    ref_f = orc.evaluate(f.depth, f.x, f.y, f.z, orc.MODE_FILTER)
    assert np.array_equal(got[0][0].astype(np.float64), ref_s["vis"])
    assert np.abs(got[0][1].astype(np.float64) - ref_f["vis"]).max() <= 1e-5
    b_in, b_out = st.stats()
    assert b_in == 12 * f.n + window_bytes(f.depth, [f.x], [f.y], 16)
    assert b_out == 8 * f.n
    assert b_in < 12 * f.n + f.depth.nbytes          # a window, not the whole map
    st.close()


@pytest.mark.parametrize("max_dist", [1, 255])
def test_stager_edges_of_the_map_and_max_dist(api, max_dist):
    """Fragments outside [0, 1) and NaN clamp to the border texels; the
    window then reaches the map's edges; small and large halos."""
    rng = np.random.default_rng(max_dist)
    maps = [random_map(rng, 96, 80), random_map(rng, 500, 300)]
    jobs_np = []
    for k in range(2):
        x, y, z = random_frags(rng, 30001, lo=0.0, hi=0.7, spread=0.4)
        x[::101] = np.nan
        y[::103] = np.inf
        jobs_np.append((k, x, y, z, 3, True))
        x2, y2, z2 = random_frags(rng, 999, lo=0.4, hi=0.45)
        jobs_np.append((k, x2, y2, z2, 2, False))     # a second job on the same map
    st = api.Stager(max_fragments=40000, max_width=500, max_height=300, slots=3)
    ref = device_answers(api, maps, jobs_np, max_dist, True)
    got = stager_answers(api, st, maps, jobs_np, max_dist)
    assert_same(got, ref, "max_dist %d" % max_dist)
    b_in, b_out = st.stats()
    want = sum(12 * j[1].shape[0] for j in jobs_np)
    for k, m in enumerate(maps):
        mine = [j for j in jobs_np if j[0] == k]
        want += window_bytes(m, [j[1] for j in mine], [j[2] for j in mine], max_dist)
    assert b_in == want
    st.close()


def test_stager_on_a_side_stream(api):
    rng = np.random.default_rng(5)
    maps = [random_map(rng, 128, 128)]
    x, y, z = random_frags(rng, 50000)
    jobs_np = [(0, x, y, z, 3, True)]
    st = api.Stager(max_fragments=50000, max_width=128, max_height=128)
    s = torch.cuda.Stream()
    got = stager_answers(api, st, maps, jobs_np, 16, stream=s)
    assert_same(got, device_answers(api, maps, jobs_np, 16, True), "side stream")
    st.close()


def test_stager_rejects_bad_runs(api):
    from paper_1711_07793_gb300 import _native as N
    rng = np.random.default_rng(2)
    st = api.Stager(max_fragments=1000, max_width=64, max_height=64)
    m = pinned(random_map(rng, 64, 64))
    x, y, z = (pinned(a) for a in random_frags(rng, 1000))
    with pytest.raises(N.RBSMError) as e:            # a map larger than the slots
        st.run([pinned(random_map(rng, 65, 64))], [api.Job(0, x, y, z, mode=2)])
    assert e.value.code == N.RBSM_ERR_ARG
    with pytest.raises(N.RBSMError) as e:            # more fragments on one map than a slot holds
        st.run([m], [api.Job(0, x, y, z, mode=2), api.Job(0, x, y, z, mode=2)])
    assert e.value.code == N.RBSM_ERR_ARG
    with pytest.raises(TypeError):                   # pageable planes
        st.run([m], [api.Job(0, torch.from_numpy(random_frags(rng, 10)[0]), x[:10], z[:10], mode=2)])
    # the C ABI itself refuses a pageable plane
    xs = np.ascontiguousarray(random_frags(rng, 1000)[0])
    out = pinned(np.zeros(1000, np.float32))
    md = (N.rbsm_map * 1)(N.rbsm_map(m.data_ptr(), 64, 64, 64, 0))
    jd = (N.rbsm_job * 1)(N.rbsm_job(0, 2, N.rbsm_frags(xs.ctypes.data, y.data_ptr(), z.data_ptr(), 1000),
                                     None, out.data_ptr(), None))
    b = N.rbsm_batch(md, 1, jd, 1, N.rbsm_params(16, 0), 0, 0, None, 0.0)
    assert N.lib().rbsm_stager_run(st.handle, ctypes.byref(b), None) == N.RBSM_ERR_ARG
    # a good run still works afterwards
    got = stager_answers(api, st, [random_map(rng, 64, 64)], [(0, *random_frags(rng, 1000), 2, False)], 16)
    assert got[0][1].shape == (1000,)
    st.close()
