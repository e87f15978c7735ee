"""Randomised GPU parity: many small seeded cases of every shape at once
(map sizes from 1 texel up, a few depth levels so that ties occur, blobs
and salt noise, fragments inside and outside the map with NaN and infinite
coordinates, every traversal cap), each against the oracle: codes and
silhouette answers bit-exact, filtering and RPCF within 1e-5, texture and
plain loads alike, and the batched launch equal to the single-map calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import rbsm as orc  # noqa: E402
from tests.test_gpu_parity import api, check_both, dev  # noqa: E402,F401
from tests.test_gpu_rpcf import check as check_rpcf  # noqa: E402

CAPS = (1, 2, 3, 5, 8, 16, 17, 64, 255)


def _case(rng):
    w, h = int(rng.integers(1, 200)), int(rng.integers(1, 200))
    levels = np.sort(rng.uniform(0.05, 1.0, size=int(rng.integers(1, 5)))).astype(np.float32)
    depth = levels[rng.integers(0, levels.size, size=(h, w))]
    bw, bh = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    blob = rng.integers(0, 2, size=((h + bh - 1) // bh, (w + bw - 1) // bw)).repeat(bh, 0).repeat(bw, 1)[:h, :w]
    depth = np.where(blob.astype(bool), depth, np.float32(1.0)).astype(np.float32)
    n = int(rng.integers(1, 4000))
    spread = float(rng.choice([0.0, 0.1, 0.5]))
    x = rng.uniform(-spread, 1 + spread, n).astype(np.float32)
    y = rng.uniform(-spread, 1 + spread, n).astype(np.float32)
    if rng.random() < 0.5:                       # texel centres and texel borders exactly
        k = n // 3
        x[:k] = (rng.integers(0, w, k) + rng.choice([0.0, 0.5], k)) / w
        y[:k] = (rng.integers(0, h, k) + rng.choice([0.0, 0.5], k)) / h
    bad = rng.random(n) < 0.01
    x[bad] = rng.choice(np.array([np.nan, np.inf, -np.inf], np.float32), int(bad.sum()))
    z = np.where(rng.random(n) < 0.5, levels[rng.integers(0, levels.size, n)],
                 rng.uniform(0.0, 1.1, n)).astype(np.float32)    # on the levels: ties
    return depth, x, y, z


@pytest.mark.parametrize("seed", range(16))
def test_random_cases_against_the_oracle(api, seed):
    rng = np.random.default_rng(7000 + seed)
    for case in range(20):
        depth, x, y, z = _case(rng)
        cap = int(rng.choice(CAPS))
        where = "seed %d case %d (%dx%d, n %d, cap %d)" % (seed, case, depth.shape[1], depth.shape[0], x.size, cap)
        check_both(api, depth, x, y, z, where, max_dist=cap, texture=bool(case % 2))
        k = int(rng.choice([1, 3, 5, 7]))
        check_rpcf(api, depth, x, y, z, k, where + " rpcf k %d" % k, max_dist=cap)


@pytest.mark.parametrize("seed", range(6))
def test_random_batches_equal_single_calls(api, seed):
    """Several random maps and fragment sets in one batched launch (both
    answers per fragment, codes on): every job equal to the single-map
    calls bit for bit, in every launch shape."""
    rng = np.random.default_rng(9100 + seed)
    maps, jobs, cases = [], [], []
    for m in range(int(rng.integers(1, 5))):
        depth, _, _, _ = _case(rng)
        maps.append(dev(depth))
        for _ in range(int(rng.integers(1, 4))):
            _, x, y, z = _case(rng)
            cases.append((m, depth, x, y, z))
    cap = int(rng.choice(CAPS))
    jobs = [api.Job(m, dev(x), dev(y), dev(z), mode=3,
                    codes=torch.empty(x.size, dtype=torch.int16, device="cuda")) for m, _, x, y, z in cases]
    for threads, ctas in ((256, 0), (128, 0), (512, 0), (256, 3), (256, 4)):
        b = api.Batch(maps, jobs, max_dist=cap, tile_threads=threads, ctas_per_sm=ctas)
        api.rbsm_batch_run(b)
        torch.cuda.synchronize()
        for j, (m, depth, x, y, z) in zip(b.jobs, cases):
            sil, _ = api.rbsm_visibility(maps[m], dev(x), dev(y), dev(z), max_dist=cap)
            fil, codes = api.rsmss_filter(maps[m], dev(x), dev(y), dev(z), codes=True, max_dist=cap)
            torch.cuda.synchronize()
            assert torch.equal(j.vis_silhouette.view(torch.int32), sil.view(torch.int32)), (threads, ctas)
            assert torch.equal(j.vis_filter.view(torch.int32), fil.view(torch.int32)), (threads, ctas)
            assert torch.equal(j.codes, codes.view(torch.int16)), (threads, ctas)
