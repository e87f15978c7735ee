"""The traversal cap as an accuracy knob (§3.1.3 caps each walk at MAXDIST
texels; runs longer than the cap are not measured to their end): on the
GPU, for staircase edges of run length L, the filtering answer is the
closed-form ramp clamp(1 + Y - X/L, 0, 1) exactly when max_dist >= L and
misses it when max_dist < L (at the first texel of each run, which a
16 x 16 in-texel grid reaches; the miss shrinks as L grows); the silhouette
is the true half-plane exactly when max_dist >= L."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from rbsm_scenes import shapes  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api as A
    return A


def staircase_errors(api, run_len, max_dist, n=512):
    """(max |filter - ramp|, silhouette mismatches) on fragments within two
    texels of the line Y - b0 = (X - a0) / L, away from the map's border."""
    a0, b0 = 8, 40
    depth = np.where(shapes.staircase_mask(n, run_len, a0, b0), shapes.BLOCKER, shapes.LIT).astype(np.float32)
    offs = [((a + 0.5) / 16, (b + 0.5) / 16) for a in range(16) for b in range(16)]
    X, Y = shapes.fragment_grid(80, n - 80, 34, n - 34, offs)
    margin = (Y - b0) - (X - a0) / run_len
    keep = (np.abs(margin) < 2.0) & (np.abs(margin) > 1e-6)
    X, Y, margin = X[keep], Y[keep], margin[keep]
    x, y = shapes.to_texcoords(X, Y, n, n)
    d = torch.from_numpy(depth).cuda()
    xs, ys, zs = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, np.ones_like(x)))
    fil, _ = api.rsmss_filter(d, xs, ys, zs, max_dist=max_dist)
    sil, _ = api.rbsm_visibility(d, xs, ys, zs, max_dist=max_dist)
    torch.cuda.synchronize()
    ramp = np.clip(1.0 + margin, 0.0, 1.0)
    err = float(np.max(np.abs(fil.cpu().numpy().astype(np.float64) - ramp)))
    bad = int(np.count_nonzero(sil.cpu().numpy() != (margin > 0)))
    return err, bad


@pytest.mark.parametrize("run_len", [4, 12, 16, 24, 40, 64])
def test_accuracy_turns_on_at_the_run_length(api, run_len):
    for max_dist in (run_len - 1, run_len, 2 * run_len):
        err, bad = staircase_errors(api, run_len, max_dist)
        if max_dist >= run_len:
            assert err < 1e-6 and bad == 0, (run_len, max_dist, err, bad)
        elif run_len <= 24:
            # the missed first texels of the runs shrink as 1 / L; past
            # L = 24 they fall between the grid's samples
            assert err > 1e-3, (run_len, max_dist, err)
