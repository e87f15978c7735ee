"""CPU checks of the C ABI library and of the scene generator (no GPU needed).

The library is cross-compiled for sm_103a here; loading it and rejecting bad
arguments needs no device.  No test here launches a kernel.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_1711_07793_gb300 import build as B
    B.build()
    from paper_1711_07793_gb300 import _native as N
    N.lib()
    return N


def test_library_exports_every_header_function(native):
    names = native.header_functions()
    assert {"rbsm_visibility", "rsmss_filter", "rbsm_batch_run", "rbsm_batch_workspace_size",
            "rbsm_batch_status", "rbsm_status_string", "rbsm_last_cuda_error", "rbsm_version"} <= set(names)
    lib = native.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_struct_layouts_match_the_header(native, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and offsets."""
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "rbsm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(rbsm_map), sizeof(rbsm_frags), sizeof(rbsm_params),
         sizeof(rbsm_job), sizeof(rbsm_batch));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(rbsm_job, frags), offsetof(rbsm_job, vis_silhouette),
         offsetof(rbsm_job, codes), offsetof(rbsm_batch, jobs), offsetof(rbsm_batch, params),
         offsetof(rbsm_batch, ctas_per_sm));
  printf("%zu %zu %zu %zu\n", sizeof(rbsm_stager_desc), offsetof(rbsm_stager_desc, max_width),
         offsetof(rbsm_stager_desc, slots), offsetof(rbsm_stager_desc, flags));
  printf("%zu %zu %zu %zu %zu\n", sizeof(rbsm_rect), sizeof(rbsm_sphere), sizeof(rbsm_occluders),
         offsetof(rbsm_occluders, zscale), offsetof(rbsm_occluders, flags));
  printf("%zu %zu %zu %zu\n", sizeof(rbsm_gbuffer), offsetof(rbsm_gbuffer, m), sizeof(rbsm_gbuffer_job),
         offsetof(rbsm_gbuffer_job, vis_filter));
  printf("%zu %zu %zu %zu %zu\n", offsetof(rbsm_batch, chunk_tiles), offsetof(rbsm_batch, flags),
         sizeof(rbsm_tuning), offsetof(rbsm_tuning, chunk_tiles), offsetof(rbsm_tuning, flags));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    offs = [int(v) for v in lines[1].split()]
    N = native
    assert sizes == [ctypes.sizeof(N.rbsm_map), ctypes.sizeof(N.rbsm_frags), ctypes.sizeof(N.rbsm_params),
                     ctypes.sizeof(N.rbsm_job), ctypes.sizeof(N.rbsm_batch)]
    assert offs == [N.rbsm_job.frags.offset, N.rbsm_job.vis_silhouette.offset, N.rbsm_job.codes.offset,
                    N.rbsm_batch.jobs.offset, N.rbsm_batch.params.offset, N.rbsm_batch.ctas_per_sm.offset]
    gbl = [int(v) for v in lines[4].split()]
    assert gbl == [ctypes.sizeof(N.rbsm_gbuffer), N.rbsm_gbuffer.m.offset, ctypes.sizeof(N.rbsm_gbuffer_job),
                   N.rbsm_gbuffer_job.vis_filter.offset]
    oc = [int(v) for v in lines[3].split()]
    assert oc == [N.RBSM_RECT_BYTES, N.RBSM_SPHERE_BYTES, ctypes.sizeof(N.rbsm_occluders),
                  N.rbsm_occluders.zscale.offset, N.rbsm_occluders.flags.offset]
    bt = [int(v) for v in lines[5].split()]
    assert bt == [N.rbsm_batch.chunk_tiles.offset, N.rbsm_batch.flags.offset, ctypes.sizeof(N.rbsm_tuning),
                  N.rbsm_tuning.chunk_tiles.offset, N.rbsm_tuning.flags.offset]
    st = [int(v) for v in lines[2].split()]
    assert st == [ctypes.sizeof(N.rbsm_stager_desc), N.rbsm_stager_desc.max_width.offset,
                  N.rbsm_stager_desc.slots.offset, N.rbsm_stager_desc.flags.offset]


def test_bad_arguments_are_rejected_before_any_cuda_call(native):
    N = native
    lib = N.lib()
    buf = (ctypes.c_float * 64)()
    addr = ctypes.addressof(buf)
    good_map = N.rbsm_map(addr, 4, 4, 4)
    good_frags = N.rbsm_frags(addr, addr, addr, 4)
    p = N.rbsm_params(16, 0)
    B = ctypes.byref
    for fn in (lib.rbsm_visibility, lib.rsmss_filter):
        assert fn(None, B(good_frags), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), None, addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(N.rbsm_map(addr, 0, 4, 4)), B(good_frags), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(N.rbsm_map(addr, 4, 4, 3)), B(good_frags), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(N.rbsm_map(addr, 70000, 4, 70000)), B(good_frags), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(N.rbsm_frags(addr, None, addr, 4)), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(N.rbsm_frags(addr, addr, addr, -1)), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(N.rbsm_frags(addr + 1, addr, addr, 4)), addr, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(good_frags), None, None, B(p), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(good_frags), addr, None, B(N.rbsm_params(0, 0)), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(good_frags), addr, None, B(N.rbsm_params(256, 0)), None) == N.RBSM_ERR_ARG
        assert fn(B(good_map), B(good_frags), addr, None, B(N.rbsm_params(16, 1)), None) == N.RBSM_ERR_ARG
        # n == 0 enqueues nothing and succeeds without touching the device
        assert fn(B(good_map), B(N.rbsm_frags(None, None, None, 0)), None, None, None, None) == N.RBSM_OK
    # the surrogate's training and set-up calls (a 256-byte aligned state is required)
    big = (ctypes.c_float * 1024)()
    state = (ctypes.addressof(big) + 255) & ~255
    assert lib.rbsm_mlp_step(None, addr, addr, 8, 1, ctypes.c_float(1e-3), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_step(state + 4, addr, addr, 8, 1, ctypes.c_float(1e-3), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_step(state, None, addr, 8, 1, ctypes.c_float(1e-3), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_step(state, addr, addr, 0, 1, ctypes.c_float(1e-3), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_step(state, addr, addr, 8, 0, ctypes.c_float(1e-3), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_step(state, addr, addr, 8, 1, ctypes.c_float(0.0), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_grad(state, addr, None, 8, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_grad(state + 16, addr, addr, 8, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_forward(state + 16, addr, 4, addr, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_forward(state, None, 4, addr, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_forward(state, addr, 0, None, None) == N.RBSM_OK
    assert lib.rbsm_mlp_set_trust(None, None, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_mlp_set_trust(state + 8, None, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_batch_noalloc_counts(None, None) == N.RBSM_ERR_ARG
    words = (ctypes.c_uint64 * 4)()
    wa = ctypes.addressof(words)
    assert lib.rbsm_selftest_bounded_wait(1_000_000, None, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_selftest_bounded_wait(1_000_000, wa + 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_selftest_bounded_wait(999, wa, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_selftest_bounded_wait(1_000_000_001, wa, None) == N.RBSM_ERR_ARG
    bad_flags = N.rbsm_params(16, 2)
    counter = (ctypes.c_uint64 * 1)()
    assert lib.rbsm_mlp_dataset(B(good_map), B(good_frags), B(bad_flags), addr, 4, counter, None) == N.RBSM_ERR_ARG
    for k in (0, 2, 9, -3):
        assert lib.rbsm_rpcf(B(good_map), B(good_frags), addr, k, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_rpcf(None, B(good_frags), addr, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_rpcf(B(good_map), B(good_frags), None, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_rpcf(B(good_map), B(good_frags), addr + 2, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_rpcf(B(good_map), B(N.rbsm_frags(None, None, None, 0)), None, 3, None, None) == N.RBSM_OK
    # the output holds partial sums while the kernel runs: overlapping an input is refused
    planes = (ctypes.c_float * 64)()
    pa = ctypes.addressof(planes)
    sep_frags = N.rbsm_frags(pa, pa + 64, pa + 128, 16)
    for vis_at in (pa, pa + 96, pa + 188, addr + 60):       # over x, y, z, the map
        assert lib.rbsm_rpcf(B(good_map), B(sep_frags), vis_at, 3, B(p), None) == N.RBSM_ERR_ARG
        assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), vis_at, 3, B(p), wa, None) == N.RBSM_ERR_ARG
        for fn in (lib.rbsm_visibility, lib.rsmss_filter):
            assert fn(B(good_map), B(sep_frags), vis_at, None, B(p), None) == N.RBSM_ERR_ARG
    vis_buf = (ctypes.c_float * 32)()
    va = ctypes.addressof(vis_buf)
    assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), va, 3, B(p), None, None) == N.RBSM_ERR_ARG   # no workspace
    assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), va, 3, B(p), wa + 4, None) == N.RBSM_ERR_ARG  # unaligned
    assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), va, 3, B(p), va + 8, None) == N.RBSM_ERR_ARG  # inside vis
    assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), va, 3, B(p), pa + 8, None) == N.RBSM_ERR_ARG  # inside x
    assert lib.rbsm_rpcf_ws(B(good_map), B(sep_frags), va, 2, B(p), wa, None) == N.RBSM_ERR_ARG      # even k
    codes_buf = (ctypes.c_uint16 * 64)()
    for fn in (lib.rbsm_visibility, lib.rsmss_filter):             # codes over z
        assert fn(B(good_map), B(sep_frags), ctypes.addressof(codes_buf), pa + 150, B(p), None) == N.RBSM_ERR_ARG
    maps = (N.rbsm_map * 1)(good_map)
    jobs = (N.rbsm_job * 1)(N.rbsm_job(0, 3, good_frags, addr, addr, None))
    batch = N.rbsm_batch(maps, 1, jobs, 1, p, 0, 0)
    size = ctypes.c_size_t(0)
    assert lib.rbsm_batch_workspace_size(B(batch), B(size)) == N.RBSM_OK and size.value >= 16
    assert lib.rbsm_batch_run(B(batch), None, 0, None) == N.RBSM_ERR_WORKSPACE
    assert lib.rbsm_batch_run(B(batch), addr + 4, 4096, None) == N.RBSM_ERR_WORKSPACE
    for bad in (N.rbsm_job(1, 3, good_frags, addr, addr, None), N.rbsm_job(0, 4, good_frags, addr, addr, None),
                N.rbsm_job(0, 1, good_frags, None, addr, None), N.rbsm_job(0, 2, good_frags, addr, None, None)):
        jb = (N.rbsm_job * 1)(bad)
        assert lib.rbsm_batch_run(B(N.rbsm_batch(maps, 1, jb, 1, p, 0, 0)), addr, 4096, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_batch_run(B(N.rbsm_batch(maps, 1, jobs, 0, p, 0, 0)), addr, 4096, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_batch_run(B(N.rbsm_batch(maps, 1, jobs, 1, p, 192, 0)), addr, 4096, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_batch_run(B(N.rbsm_batch(maps, 65, jobs, 1, p, 0, 0)), addr, 4096, None) == N.RBSM_ERR_ARG
    for chunk, flags in ((3, 0), (16, 0), (-1, 0), (0, 2)):
        bad = N.rbsm_batch(maps, 1, jobs, 1, p, 0, 0, None, 0.0, chunk, flags)
        assert lib.rbsm_batch_run(B(bad), addr, 4096, None) == N.RBSM_ERR_ARG
    # the stager: descriptors are checked before any CUDA call
    h = ctypes.c_void_p(0)
    for bad in (N.rbsm_stager_desc(0, 64, 64, 0, 0, 0), N.rbsm_stager_desc(10, 0, 64, 0, 0, 0),
                N.rbsm_stager_desc(10, 64, 70000, 0, 0, 0), N.rbsm_stager_desc(10, 64, 64, 1, 0, 0),
                N.rbsm_stager_desc(10, 64, 64, 5, 0, 0), N.rbsm_stager_desc(10, 64, 64, 0, 2, 0),
                N.rbsm_stager_desc(10, 64, 64, 0, 0, 1)):
        assert lib.rbsm_stager_create(B(bad), B(h)) == N.RBSM_ERR_ARG and not h.value
    assert lib.rbsm_stager_create(None, B(h)) == N.RBSM_ERR_ARG
    assert lib.rbsm_stager_run(None, B(batch), None) == N.RBSM_ERR_ARG
    i64 = ctypes.c_int64(0)
    assert lib.rbsm_stager_stats(None, B(i64), B(i64)) == N.RBSM_ERR_ARG
    assert lib.rbsm_stager_status(None, B(ctypes.c_int(0))) == N.RBSM_ERR_ARG
    assert lib.rbsm_stager_destroy(None) == N.RBSM_ERR_ARG
    # the depth-buffer path: argument checks before any CUDA call
    m16 = (ctypes.c_float * 16)(*([1.0] + [0.0] * 4 + [1.0] + [0.0] * 4 + [1.0] + [0.0] * 4 + [1.0]))
    gb = N.rbsm_gbuffer(addr, 4, 4, 4, m16)
    GJ = lambda g=gb, sil=addr, fil=addr, cod=None: (N.rbsm_gbuffer_job * 1)(N.rbsm_gbuffer_job(good_map, g, sil,
                                                                                                fil, cod))
    assert lib.rbsm_visibility_gbuffer(None, 1, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(), 0, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(), 65, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(), 1, 0, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(sil=None), 1, 1, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(fil=None), 1, 2, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(g=N.rbsm_gbuffer(addr, 4, 4, 3, m16)), 1, 3, B(p), None) == N.RBSM_ERR_ARG
    assert lib.rbsm_visibility_gbuffer(GJ(g=N.rbsm_gbuffer(None, 4, 4, 4, m16)), 1, 3, B(p), None) == N.RBSM_ERR_ARG
    # the light pass: descriptor checks before any CUDA call
    occ = N.rbsm_occluders(None, 0, None, 0, 1.0, 1.0, 0)
    assert lib.rbsm_shadow_map(None, addr, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_map(B(occ), None, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_map(B(occ), addr, 4, 4, 3, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_map(B(occ), addr, 0, 4, 4, None) == N.RBSM_ERR_ARG
    for bad in (N.rbsm_occluders(None, 1, None, 0, 1.0, 1.0, 0), N.rbsm_occluders(None, 0, None, -1, 1.0, 1.0, 0),
                N.rbsm_occluders(None, 0, None, 0, 0.0, 1.0, 0), N.rbsm_occluders(None, 0, None, 0, 1.0, 1.0, 2)):
        assert lib.rbsm_shadow_map(B(bad), addr, 4, 4, 4, None) == N.RBSM_ERR_ARG
    occs = (N.rbsm_occluders * 2)(occ, occ)
    ptrs = (ctypes.c_void_p * 2)(addr, addr + 4096)
    assert lib.rbsm_shadow_maps(None, ptrs, 2, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_maps(occs, None, 2, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_maps(occs, ptrs, 0, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_maps(occs, ptrs, N.RBSM_SHADOW_MAPS_MAX + 1, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_maps(occs, ptrs, 2, 4, 4, 3, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_shadow_maps(occs, (ctypes.c_void_p * 2)(addr, None), 2, 4, 4, 4, None) == N.RBSM_ERR_ARG
    bad2 = (N.rbsm_occluders * 2)(occ, N.rbsm_occluders(None, 1, None, 0, 1.0, 1.0, 0))
    assert lib.rbsm_shadow_maps(bad2, ptrs, 2, 4, 4, 4, None) == N.RBSM_ERR_ARG
    assert lib.rbsm_status_string(N.RBSM_ERR_ARG) == b"invalid argument"
    assert lib.rbsm_version() >= 100


def test_generator_is_deterministic_and_in_range():
    import rbsm_scenes as sc
    a, b = sc.config1(3), sc.config1(3)
    assert np.array_equal(a.depth, b.depth) and np.array_equal(a.x, b.x) and np.array_equal(a.z, b.z)
    c = sc.config1(4)
    assert not np.array_equal(a.depth, c.depth)
    assert a.depth.shape == (256, 256) and a.n == 320 * 240
    assert np.all((a.x > 0) & (a.x < 1) & (a.y > 0) & (a.y < 1))
    assert np.all(a.z == np.float32(1.0))             # C1 fragments lie on the plane
    assert 0.01 < np.mean(a.depth < 1) < 0.6
    f = sc.config2(0, screen=(480, 270))
    assert f.depth.shape == (2048, 2048) and f.n == 480 * 270
    assert 0.0 < f.meta["sphere_fraction"] < 1.0
    # sphere receivers sit 1e-3 in front of their own surface
    assert np.all(f.z <= 1.0)


def test_generator_rasterises_exact_coverage():
    """A square occluder covers exactly the texels whose centres it contains."""
    import rbsm_scenes as sc
    occ = sc.Occluders(np.array([[10.0, 12.0, 1.0, 0.0, 3.2, 2.2]]), np.array([0.5], np.float32))
    d = sc.raster(occ, 32, 32, 32)
    ii, jj = np.meshgrid(np.arange(32) + 0.5, np.arange(32) + 0.5)
    inside = (np.abs(ii - 10) <= 3.2) & (np.abs(jj - 12) <= 2.2)
    assert np.array_equal(d < 1.0, inside)
    s = sc.Occluders(spheres=np.array([[16.0, 16.0, 5.0, 0.6]]))
    d = sc.raster(s, 32, 32, 32)
    assert d[15, 15] < 0.6 and d[0, 0] == 1.0


def test_binding_rejects_bad_light_pass_outputs(native):
    """The binding of rbsm_shadow_maps checks its outputs before the call:
    one per occluder set, CUDA float32 (height, width) planes of one pitch."""
    import torch
    from paper_1711_07793_gb300 import api

    class FakeOcc:
        def desc(self, zscale, ground=1.0):
            return native.rbsm_occluders(None, 0, None, 0, float(zscale), float(ground), 0)

    with pytest.raises(ValueError):
        api.rbsm_shadow_maps([FakeOcc(), FakeOcc()], 4, 4, 1.0, outs=[torch.zeros((4, 4))])
    with pytest.raises(ValueError):
        api.rbsm_shadow_maps([FakeOcc()], 4, 4, 1.0, outs=[torch.zeros((4, 4))])      # not a CUDA tensor
    with pytest.raises(ValueError):
        api.rbsm_shadow_maps([], 4, 4, 1.0, outs=[])
