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


def test_noalloc_surrogate_counts_equal_batch_run():
    """A batch with the learned surrogate through the allocation-free call:
    the same answers as rbsm_batch_run, and the counters the library keeps
    in its own array (rbsm_batch_noalloc_counts) equal the ones
    rbsm_batch_run leaves in the caller's workspace, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import __graft_entry__
    __graft_entry__.build()
    import rbsm_scenes as sc
    from paper_1711_07793_gb300 import _native as N
    from paper_1711_07793_gb300 import api
    from paper_1711_07793_gb300.surrogate import Surrogate

    net = Surrogate.from_checkpoint(os.path.join(os.path.dirname(api.__file__), "weights", "surrogate_c4.npz"))
    f = sc.config2(5, screen=(960, 540))
    depth = torch.from_numpy(f.depth).cuda()
    x, y, z = (torch.from_numpy(a).cuda() for a in (f.x, f.y, f.z))
    ref = api.Batch([depth], [api.Job(0, x, y, z, mode=2, codes=True)], surrogate=net, guard_tau=0.01)
    api.rbsm_batch_run(ref)
    torch.cuda.synchronize()
    acc_ref, fb_ref = api.rbsm_batch_surrogate_counts(ref)
    assert acc_ref > 0 and fb_ref > 0
    out = api.Batch([depth], [api.Job(0, x, y, z, mode=2, codes=True)], surrogate=net, guard_tau=0.01)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out.jobs[0].vis_filter.fill_(float("nan"))
        torch.cuda.synchronize()
        assert N.lib().rbsm_batch_run_noalloc(ctypes.byref(out.desc), stream) == N.RBSM_OK
        torch.cuda.synchronize()
        a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
        assert N.lib().rbsm_batch_noalloc_counts(ctypes.byref(a), ctypes.byref(b)) == N.RBSM_OK
        assert (a.value, b.value) == (acc_ref, fb_ref), call
        assert torch.equal(out.jobs[0].vis_filter, ref.jobs[0].vis_filter), call
        assert torch.equal(out.jobs[0].codes, ref.jobs[0].codes), call
