"""GPU test of rbsm_batch_run_noalloc (collected last on purpose).

rbsm_batch_run_noalloc serves callers that cannot allocate device memory,
for instance a plugin inside a host application that owns every device
allocation, or a frame loop that must not allocate while frames are in
flight.  It keeps the batched launch's scratch in a device array compiled
into the library instead of a caller workspace.  This test calls it through
the C ABI twice in a row (the array keeps the previous call's counters, so
the second call checks that they are cleared) and compares every answer
with rbsm_batch_run's on the same batch: silhouette, filtering and codes
must be identical.  It runs alone in a fresh process or after the other
tests alike.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_batch_equals_batch_run_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import rbsm_scenes as sc
    from paper_1711_07793_gb300 import _native as N
    from paper_1711_07793_gb300 import api

    frames = [sc.config1(s) for s in (0, 1, 2)]
    maps = [torch.from_numpy(f.depth).cuda() for f in frames]
    planes = [[torch.from_numpy(a).cuda() for a in (f.x, f.y, f.z)] for f in frames]

    def jobs():
        return [api.Job(k, *planes[k], mode=mode, codes=True) for k, mode in zip(range(3), (1, 2, 3))]

    ref = api.Batch(maps, jobs())
    api.rbsm_batch_run(ref)
    torch.cuda.synchronize()

    out = api.Batch(maps, jobs())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        for j in out.jobs:
            for t in (j.vis_silhouette, j.vis_filter):
                if t is not None:
                    t.fill_(float("nan"))
            j.codes.fill_(-1)
        torch.cuda.synchronize()
        rc = N.lib().rbsm_batch_run_noalloc(ctypes.byref(out.desc), stream)
        assert rc == N.RBSM_OK, N.status_string(rc)
        torch.cuda.synchronize()
        for j, r in zip(out.jobs, ref.jobs):
            if j.mode & 1:
                assert torch.equal(j.vis_silhouette, r.vis_silhouette), call
            if j.mode & 2:
                assert torch.equal(j.vis_filter, r.vis_filter), call
            assert torch.equal(j.codes, r.codes), call
    assert N.lib().rbsm_batch_run_noalloc(None, stream) == N.RBSM_ERR_ARG
