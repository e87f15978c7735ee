"""GPU parity of the depth-buffer path (rbsm_visibility_gbuffer): p formed
in the kernel (reading R21) and then the RBSM path.  The oracle projects
the buffer (oracle_project) and evaluates the projected planes: codes and
silhouette answers bit-exact, filtering within 1e-5; the answers also equal
rbsm_visibility / rsmss_filter on the oracle-projected planes bit for bit
(the projections agree to the bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402

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


def check(api, depth, gd, m, where, modes=(1, 2, 3), max_dist=16, gd_dev=None, texture=False):
    x, y, z = orc.project(gd, m)
    refs = {md: orc.evaluate(depth, x, y, z, md, max_dist=max_dist) for md in (1, 2)}
    dmap = dev(depth)
    if texture:
        from paper_1711_07793_gb300 import _native as N
        try:
            dmap = api.MapTexture(dmap)
        except N.RBSMError:
            pass
    g = gd_dev if gd_dev is not None else dev(gd)
    for mode in modes:
        j = api.GBufferJob(dmap, g, m, mode=mode, codes=True)
        api.rbsm_visibility_gbuffer([j], mode=mode, max_dist=max_dist)
        torch.cuda.synchronize()
        sil, fil, cod = j.vis_silhouette, j.vis_filter, j.codes
        cod = cod.cpu().numpy().view(np.uint16)
        want_codes = refs[1 if mode == 1 else 2]["codes"]
        bad = np.nonzero(cod != want_codes)[0]
        assert bad.size == 0, "%s mode %d: %d code mismatches" % (where, mode, bad.size)
        if sil is not None:
            assert np.array_equal(sil.cpu().numpy().astype(np.float64), refs[1]["vis"]), where
        if fil is not None:
            f = fil.cpu().numpy().astype(np.float64)
            both = np.isnan(f) & np.isnan(refs[2]["vis"])
            diff = np.abs(f - refs[2]["vis"])
            diff[both] = 0
            assert diff.max(initial=0.0) <= TOL, where
            # the same bits as the planes path on the oracle's planes
            vis, _ = api.rsmss_filter(dmap, dev(x), dev(y), dev(z), max_dist=max_dist)
            assert np.array_equal(vis.cpu().numpy().view(np.uint32), fil.cpu().numpy().view(np.uint32)), where


def test_c5_camera_small(api):
    import rbsm_scenes as sc
    c5 = sc.Config5(0, size=1024, screen=(640, 360), frames=2)
    fr = c5.frame(1)
    d, m = c5.gbuffer(fr.z)
    check(api, fr.depth, d, m, "C5 small", texture=True)
    check(api, fr.depth, d, m, "C5 small plain loads", modes=(3,))


@pytest.mark.parametrize("w,h", [(1, 1), (3, 5), (127, 3), (129, 2), (333, 77)])
def test_odd_buffers_and_random_perspective(api, w, h):
    rng = np.random.default_rng(w * 1000 + h)
    depth = np.where(rng.random((64, 80)) < 0.3, np.float32(0.4), np.float32(1.0)).astype(np.float32)
    m = np.array([[rng.uniform(0.5, 1.5) / w, rng.uniform(-0.2, 0.2) / h, 0, rng.uniform(0, 0.2)],
                  [rng.uniform(-0.2, 0.2) / w, rng.uniform(0.5, 1.5) / h, 0, rng.uniform(0, 0.2)],
                  [rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01), 1, 0],
                  [rng.uniform(0, 0.5) / w, rng.uniform(0, 0.5) / h, 0, 1]], np.float32)
    gd = rng.uniform(0.2, 1.2, (h, w)).astype(np.float32)
    check(api, depth, gd, m, "%dx%d" % (w, h))


@pytest.mark.parametrize("max_dist", [1, 255])
def test_pitched_buffer_and_max_dist(api, max_dist):
    import rbsm_scenes as sc
    c5 = sc.Config5(1, size=1024, screen=(320, 180), frames=1)
    fr = c5.frame(0)
    d, m = c5.gbuffer(fr.z)
    big = torch.full((180, 336), 5.0, device="cuda")
    big[:, :320] = dev(d)
    check(api, fr.depth, d, m, "pitched", max_dist=max_dist, gd_dev=big[:, :320])


def test_full_size_frame_sampled(api):
    import bench
    c5, host = bench.make_workload(1, 0, pin=False)
    depth = host[0]["depth"].numpy()
    z = host[0]["xyz"][2].numpy()
    d, m = c5.gbuffer(z)
    x, y, zz = orc.project(d, m)
    j = api.GBufferJob(dev(depth), dev(d), m, mode=3, codes=True)
    api.rbsm_visibility_gbuffer([j])
    torch.cuda.synchronize()
    sil, fil, cod = j.vis_silhouette, j.vis_filter, j.codes
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(x.shape[0], 300000, replace=False))
    ref_s = orc.evaluate(depth, x[idx], y[idx], zz[idx], 1)
    ref_f = orc.evaluate(depth, x[idx], y[idx], zz[idx], 2)
    assert np.array_equal(cod.cpu().numpy().view(np.uint16)[idx], ref_f["codes"])
    assert np.array_equal(sil.cpu().numpy()[idx].astype(np.float64), ref_s["vis"])
    assert np.abs(fil.cpu().numpy()[idx].astype(np.float64) - ref_f["vis"]).max() <= TOL


def test_many_jobs_in_one_launch(api):
    """Several (map, buffer) jobs of different sizes in one launch: each
    equals its own single-job launch bit for bit."""
    rng = np.random.default_rng(4)
    jobs, singles = [], []
    for k, (w, h) in enumerate([(96, 40), (33, 17), (256, 128), (1, 1), (130, 7)]):
        depth = np.where(rng.random((50 + k, 70)) < 0.3, np.float32(0.4), np.float32(1.0)).astype(np.float32)
        m = np.array([[1.0 / w, 0.05 / h, 0, 0.01 * k], [0.03 / w, 1.0 / h, 0, 0.02],
                      [0, 0, 1, 0], [0.2 / w, 0.1 / h, 0, 1]], np.float32)
        gd = dev(rng.uniform(0.3, 1.1, (h, w)).astype(np.float32))
        jobs.append(api.GBufferJob(dev(depth), gd, m, mode=3, codes=True))
        singles.append(api.GBufferJob(dev(depth), gd, m, mode=3, codes=True))
    api.rbsm_visibility_gbuffer(jobs)
    for s_ in singles:
        api.rbsm_visibility_gbuffer([s_])
    torch.cuda.synchronize()
    for a, b in zip(jobs, singles):
        for u, v in ((a.vis_silhouette, b.vis_silhouette), (a.vis_filter, b.vis_filter), (a.codes, b.codes)):
            assert torch.equal(u, v)


def _job_set(api, rng, n, w=200, h=90, out=None):
    jobs, singles = [], []
    for k in range(n):
        depth = dev(np.where(rng.random((64, 96)) < 0.3, np.float32(0.4), np.float32(1.0)).astype(np.float32))
        m = np.array([[1.0 / w, 0.05 / h, 0, 0.01 * k], [0.03 / w, 1.0 / h, 0, 0.02],
                      [0, 0, 1, 0], [0.2 / w, 0.1 / h, 0, 1]], np.float32)
        gd = dev(rng.uniform(0.3, 1.1, (h, w)).astype(np.float32))
        jobs.append(api.GBufferJob(depth, gd, m, mode=2, vis_filter=out))
        singles.append(api.GBufferJob(depth, gd, m, mode=2))
    return jobs, singles


def test_jobs_sharing_an_output_run_in_order(api):
    """Jobs that write the same answer plane are not overlapped: the plane
    ends with the last job's answers, as launches in order leave it."""
    rng = np.random.default_rng(8)
    shared = torch.empty(200 * 90, dtype=torch.float32, device="cuda")
    jobs, singles = _job_set(api, rng, 6, out=shared)
    api.rbsm_visibility_gbuffer(jobs, mode=2)
    api.rbsm_visibility_gbuffer([singles[-1]], mode=2)
    torch.cuda.synchronize()
    assert torch.equal(shared, singles[-1].vis_filter)


def test_overlapped_jobs_are_complete_for_the_next_work_on_the_stream(api):
    """Independent jobs run as programmatic dependents of each other; work
    queued on the stream right after the call (no synchronisation between)
    sees every job's answers."""
    rng = np.random.default_rng(9)
    jobs, singles = _job_set(api, rng, 16)
    for s_ in singles:
        api.rbsm_visibility_gbuffer([s_], mode=2)
    torch.cuda.synchronize()
    for j in jobs:
        j.vis_filter.fill_(-7.0)
    api.rbsm_visibility_gbuffer(jobs, mode=2)
    sums = torch.stack([j.vis_filter.sum() for j in jobs])      # same stream, no sync before
    torch.cuda.synchronize()
    assert torch.equal(sums, torch.stack([s_.vis_filter.sum() for s_ in singles]))
    for a, b in zip(jobs, singles):
        assert torch.equal(a.vis_filter, b.vis_filter)


def test_bad_arguments(api):
    from paper_1711_07793_gb300 import _native as N
    d = dev(np.ones((8, 8), np.float32))
    with pytest.raises(N.RBSMError):
        api.rbsm_visibility_gbuffer([api.GBufferJob(d, d, np.eye(4), mode=3)], mode=4)
    with pytest.raises(N.RBSMError):        # codes for some jobs only
        api.rbsm_visibility_gbuffer([api.GBufferJob(d, d, np.eye(4), codes=True), api.GBufferJob(d, d, np.eye(4))])


def test_full_size_frames_in_one_call_as_the_bench_runs_them(api):
    """Four full-size C5 frames (3840x2160 depth buffers, 8192^2 maps) as
    jobs of one call, overlapped as dependent launches (the bench's launch
    configuration): every answer equals that frame's single-job call bit for
    bit, and a sample of one frame matches the oracle."""
    import bench
    c5, host = bench.make_workload(4, 0, pin=False)
    maps = [dev(h["depth"].numpy()) for h in host]
    bufs = []
    for h in host:
        d, m = c5.gbuffer(h["xyz"][2].numpy())
        bufs.append((dev(d), m, d))
    jobs = [api.GBufferJob(mp, g, m, mode=3, codes=True) for mp, (g, m, _) in zip(maps, bufs)]
    api.rbsm_visibility_gbuffer(jobs)
    singles = []
    for mp, (g, m, _) in zip(maps, bufs):
        j = api.GBufferJob(mp, g, m, mode=3, codes=True)
        api.rbsm_visibility_gbuffer([j])
        singles.append(j)
    torch.cuda.synchronize()
    for a, b in zip(jobs, singles):
        assert torch.equal(a.vis_silhouette, b.vis_silhouette)
        assert torch.equal(a.vis_filter, b.vis_filter)
        assert torch.equal(a.codes, b.codes)
    depth = host[2]["depth"].numpy()
    x, y, zz = orc.project(bufs[2][2], bufs[2][1])
    idx = np.sort(np.random.default_rng(2).choice(x.shape[0], 100000, replace=False))
    ref_f = orc.evaluate(depth, x[idx], y[idx], zz[idx], 2)
    assert np.array_equal(jobs[2].codes.cpu().numpy().view(np.uint16)[idx], ref_f["codes"])
    assert np.abs(jobs[2].vis_filter.cpu().numpy()[idx].astype(np.float64) - ref_f["vis"]).max() <= TOL
