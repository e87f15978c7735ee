"""GPU tests of the batched persistent launch (rbsm_batch_run).

Every job of a batch must give bit-identical answers to the single-map
entry points on the same inputs, for every launch shape the autotuner may
pick, and match the oracle.  The last test runs the benchmark's own
workload shape (8192^2 maps, 3840x2160 fragments) through the batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402
from tests.test_gpu_parity import assert_parity, dev  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def small_c3():
    import rbsm_scenes as sc
    return sc.Config3(seed=1, views=[(320, 180), (256, 144), (200, 130)], cascades=[1024, 512, 256], lights=2)


def _batch(api, scene, modes, codes=True, maps=None, **kw):
    maps = maps if maps is not None else [dev(m) for m in scene.maps]
    jobs = []
    for k, j in enumerate(scene.jobs):
        mode = modes[k % len(modes)]
        jobs.append(api.Job(j.map_index, dev(j.x), dev(j.y), dev(j.z), mode=mode, codes=True if codes else None))
    return api.Batch(maps, jobs, **kw)


def test_batch_equals_single_calls(api, small_c3):
    b = _batch(api, small_c3, modes=[3, 1, 2])
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    assert api.rbsm_batch_status(b) == 0
    for j, sj in zip(b.jobs, small_c3.jobs):
        depth = b.maps[j.map_index]
        if j.mode & 1:
            ref_v, ref_c = api.rbsm_visibility(depth, j.x, j.y, j.z, codes=True)
            assert torch.equal(j.vis_silhouette, ref_v)
            if j.mode == 1:
                assert torch.equal(j.codes, ref_c)
        if j.mode & 2:
            ref_v, ref_c = api.rsmss_filter(depth, j.x, j.y, j.z, codes=True)
            assert torch.equal(j.vis_filter, ref_v)
            assert torch.equal(j.codes, ref_c)


def test_batch_matches_oracle(api, small_c3):
    b = _batch(api, small_c3, modes=[3])
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    for j, sj in zip(b.jobs, small_c3.jobs):
        depth = small_c3.maps[sj.map_index]
        for mode, out in ((orc.MODE_SILHOUETTE, j.vis_silhouette), (orc.MODE_FILTER, j.vis_filter)):
            ref = orc.evaluate(depth, sj.x, sj.y, sj.z, mode)
            codes = j.codes.cpu().numpy().view(np.uint16) if mode == orc.MODE_FILTER else None
            assert_parity(out.cpu().numpy(), codes, ref, mode, "job %d/%d" % (sj.view, sj.cascade))


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("ctas", [0, 1, 3, 4, 5])
def test_every_launch_shape_gives_the_same_answers(api, small_c3, threads, ctas):
    """Every candidate of the autotuner (CTA size, CTAs per SM, claim size,
    texture gathers or plain loads) gives the bits of the default launch."""
    ref = _batch(api, small_c3, modes=[3], codes=False)
    api.rbsm_batch_run(ref)
    torch.cuda.synchronize()
    texs = [api.MapTexture(dev(m)) for m in small_c3.maps]
    for chunk in (1, 2, 4, 8):
        for maps, plain in ((None, False), (texs, False), (texs, True)):
            b = _batch(api, small_c3, modes=[3], codes=False, tile_threads=threads, ctas_per_sm=ctas,
                       chunk_tiles=chunk, plain_loads=plain, maps=maps)
            api.rbsm_batch_run(b)
            api.rbsm_batch_run(b)          # a second launch reuses the workspace
            torch.cuda.synchronize()
            for j, r in zip(b.jobs, ref.jobs):
                assert torch.equal(j.vis_silhouette, r.vis_silhouette), (chunk, plain, maps is None)
                assert torch.equal(j.vis_filter, r.vis_filter), (chunk, plain, maps is None)
    for t in texs:
        t.close()


def test_batch_with_empty_and_tiny_jobs(api):
    import rbsm_scenes as sc
    f = sc.config1(0)
    depth = dev(f.depth)
    x, y, z = dev(f.x), dev(f.y), dev(f.z)
    jobs = [api.Job(0, x[:0], y[:0], z[:0]), api.Job(0, x[:1], y[:1], z[:1]),
            api.Job(0, x[5:1030], y[5:1030], z[5:1030], codes=True), api.Job(0, x, y, z, codes=True)]
    b = api.Batch([depth], jobs)
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    for j, sl in zip(jobs[1:], (slice(0, 1), slice(5, 1030), slice(None))):
        ref = orc.evaluate(f.depth, f.x[sl], f.y[sl], f.z[sl], orc.MODE_FILTER)
        codes = j.codes.cpu().numpy().view(np.uint16) if j.codes is not None else None
        assert_parity(j.vis_filter.cpu().numpy(), codes, ref, orc.MODE_FILTER, "tiny")


def test_bench_workload_through_the_batch(api):
    """Three frames of the 8192^2 / 3840x2160 moving-light workload in one
    batched launch, every fragment checked against the oracle."""
    import rbsm_scenes as sc
    c5 = sc.Config5(0)
    frames = [c5.frame(f) for f in (0, 15, 31)]
    maps = [dev(fr.depth) for fr in frames]
    jobs = [api.Job(k, dev(fr.x), dev(fr.y), dev(fr.z), mode=3, codes=True) for k, fr in enumerate(frames)]
    b = api.Batch(maps, jobs)
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    assert api.rbsm_batch_status(b) == 0
    for j, fr in zip(jobs, frames):
        for mode, out in ((orc.MODE_SILHOUETTE, j.vis_silhouette), (orc.MODE_FILTER, j.vis_filter)):
            ref = orc.evaluate(fr.depth, fr.x, fr.y, fr.z, mode)
            codes = j.codes.cpu().numpy().view(np.uint16) if mode == orc.MODE_FILTER else None
            assert_parity(out.cpu().numpy(), codes, ref, mode, fr.name)


def test_graph_replay_and_autotune(api, small_c3, tmp_path):
    """The CUDA graph of a batch replays the same answers as direct launches;
    the autotuner times the candidates, keeps answers correct, and its
    choice is cached per batch signature."""
    ref = _batch(api, small_c3, modes=[3], codes=True)
    api.rbsm_batch_run(ref)
    b = _batch(api, small_c3, modes=[3], codes=True)
    g = api.BatchGraph(b)
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    for j, r in zip(b.jobs, ref.jobs):
        assert torch.equal(j.vis_silhouette, r.vis_silhouette)
        assert torch.equal(j.vis_filter, r.vis_filter)
        assert torch.equal(j.codes, r.codes)
    g.close()
    cache = str(tmp_path / "tune.json")
    t = api.rbsm_batch_autotune(b, repeats=2, cache=cache)
    # 7 (CTA size, CTAs per SM) pairs x 4 claim sizes; no map has a texture
    assert t["candidates"] == 28 and t["tile_threads"] in (128, 256, 512) and not t["cached"]
    assert t["chunk_tiles"] in (1, 2, 4, 8) and not t["plain_loads"]
    hit = api.rbsm_batch_autotune(b, cache=cache)
    assert hit["cached"] and b.desc.chunk_tiles == t["chunk_tiles"]
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    for j, r in zip(b.jobs, ref.jobs):
        assert torch.equal(j.vis_filter, r.vis_filter)
    # with map textures the tuner also weighs plain loads against the gathers
    texs = [api.MapTexture(dev(m)) for m in small_c3.maps]
    bt = _batch(api, small_c3, modes=[3], codes=True, maps=texs)
    tt = api.rbsm_batch_autotune(bt, repeats=1, cache=None)
    assert tt["candidates"] == 56
    api.rbsm_batch_run(bt)
    torch.cuda.synchronize()
    for j, r in zip(bt.jobs, ref.jobs):
        assert torch.equal(j.vis_filter, r.vis_filter) and torch.equal(j.codes, r.codes)
    for x in texs:
        x.close()


def test_batch_with_textures_matches_plain_loads(api, small_c3):
    """Maps given with textures (two gathers per fragment) give the same
    answers as the same batch with plain loads, in every mode."""
    ref = _batch(api, small_c3, modes=[3, 1, 2])
    api.rbsm_batch_run(ref)
    maps = [dev(m) for m in small_c3.maps]
    texs = [api.MapTexture(m) for m in maps]
    jobs = [api.Job(j.map_index, dev(j.x), dev(j.y), dev(j.z), mode=[3, 1, 2][k % 3], codes=True)
            for k, j in enumerate(small_c3.jobs)]
    b = api.Batch(texs, jobs)
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    for j, r in zip(b.jobs, ref.jobs):
        if j.mode & 1:
            assert torch.equal(j.vis_silhouette, r.vis_silhouette)
        if j.mode & 2:
            assert torch.equal(j.vis_filter, r.vis_filter)
        assert torch.equal(j.codes, r.codes)
    for t in texs:
        t.close()
