"""Parity at full size in the launch configuration the benchmark times:
map textures, the autotuned launch shape, a CUDA graph replay, mode BOTH.
Sampled fragments of every job are checked against the oracle (codes are
not stored in this configuration; the silhouette answer is bit-exact and
the filtering answer within 1e-5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402

TOL = 1e-5
SAMPLE = 60000


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api as A
    return A


def run_like_the_bench(api, maps_np, parts):
    dev = torch.device("cuda")
    texs = [api.MapTexture(torch.from_numpy(m).to(dev)) for m in maps_np]
    jobs = [api.Job(k, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (x, y, z)), mode=3)
            for k, x, y, z in parts]
    batch = api.Batch(texs, jobs)
    api.rbsm_batch_autotune(batch, repeats=1, cache=None)
    graph = api.BatchGraph(batch)
    graph.launch()
    graph.launch()
    torch.cuda.synchronize()
    assert api.rbsm_batch_status(batch) == 0
    out = [(j.vis_silhouette.cpu().numpy(), j.vis_filter.cpu().numpy()) for j in jobs]
    graph.close()
    for t in texs:
        t.close()
    return out


def check_sampled(maps_np, parts, out, seed):
    rng = np.random.default_rng(seed)
    for (k, x, y, z), (sil, fil) in zip(parts, out):
        n = x.shape[0]
        idx = np.sort(rng.choice(n, min(n, SAMPLE), replace=False))
        rs = orc.evaluate(maps_np[k], x[idx], y[idx], z[idx], orc.MODE_SILHOUETTE)
        rf = orc.evaluate(maps_np[k], x[idx], y[idx], z[idx], orc.MODE_FILTER)
        assert np.array_equal(sil[idx].astype(np.float64), rs["vis"])
        assert np.abs(fil[idx].astype(np.float64) - rf["vis"]).max() <= TOL


def test_c5_all_frames_as_the_bench_launches_them(api):
    import bench
    c5, host = bench.make_workload(32, 0, pin=False)
    maps_np = [h["depth"].numpy() for h in host]
    parts = [(k, h["xyz"][0].numpy(), h["xyz"][1].numpy(), h["xyz"][2].numpy()) for k, h in enumerate(host)]
    out = run_like_the_bench(api, maps_np, parts)
    check_sampled(maps_np, parts, out, 5)


def test_c3_full_size_as_the_bench_launches_it(api):
    import rbsm_scenes as sc
    c3 = sc.Config3(0)
    parts = [(j.map_index, j.x, j.y, j.z) for j in c3.jobs]
    out = run_like_the_bench(api, c3.maps, parts)
    check_sampled(c3.maps, parts, out, 3)
