"""Python binding of librbsm with the C ABI's names (argument marshalling only).

Tensors are torch tensors: float32 shadow maps of shape (height, width) with
unit stride along width, and float32 fragment planes x, y, z of shape (n,).
CUDA tensors are passed to the library as device pointers on the current
torch stream.  CPU tensors are accepted too: they are copied to the GPU,
evaluated there and the answers copied back (the host-buffer path); every
step of the method runs in the library's kernels either way.
"""
import ctypes
import json
import os

import torch

from . import _native as N


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_plane(name, t, n=None):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.dim() != 1:
        raise TypeError("%s must be a 1-D float32 tensor" % name)
    if not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.numel() > 1 and t.stride(0) != 1:
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.shape[0] != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.shape[0], n))


class MapTexture:
    """Texture view of a shadow map (rbsm_map_texture_create): the map's
    four-neighbourhood is then read with two texture gathers.  Keep the
    depth tensor alive while the texture is used; close() (or garbage
    collection) destroys the texture, so do that only after the launches
    that read it have completed."""

    def __init__(self, depth):
        self.depth = depth
        m = _plain_map_desc(depth)
        h = ctypes.c_uint64(0)
        N.check("rbsm_map_texture_create", N.lib().rbsm_map_texture_create(ctypes.byref(m), ctypes.byref(h)))
        self.handle = h.value

    def close(self):
        if self.handle:
            N.check("rbsm_map_texture_destroy", N.lib().rbsm_map_texture_destroy(self.handle))
        self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _plain_map_desc(depth):
    if not isinstance(depth, torch.Tensor) or depth.dtype != torch.float32 or depth.dim() != 2:
        raise TypeError("depth must be a 2-D float32 tensor")
    if not depth.is_cuda:
        raise TypeError("depth must be a CUDA tensor")
    if depth.stride(1) != 1 or depth.stride(0) < depth.shape[1]:
        raise ValueError("depth rows must be contiguous (pitch >= width)")
    return N.rbsm_map(depth.data_ptr(), depth.shape[1], depth.shape[0], depth.stride(0), 0)


def map_desc(depth):
    """rbsm_map for a (height, width) float32 CUDA tensor with unit inner
    stride, or for a MapTexture (its map with the texture attached)."""
    if isinstance(depth, MapTexture):
        m = _plain_map_desc(depth.depth)
        m.texture = depth.handle
        return m
    return _plain_map_desc(depth)


def frags_desc(x, y, z):
    _check_plane("x", x)
    n = x.shape[0]
    _check_plane("y", y, n)
    _check_plane("z", z, n)
    return N.rbsm_frags(x.data_ptr(), y.data_ptr(), z.data_ptr(), n)


def _params(max_dist):
    return N.rbsm_params(int(max_dist), 0)


def _host_roundtrip(fn, depth, x, y, z, codes, max_dist):
    dev = torch.device("cuda", torch.cuda.current_device())
    d = depth.to(dev, non_blocking=True)
    xd, yd, zd = (t.to(dev, non_blocking=True) for t in (x, y, z))
    vis, cod = fn(d, xd, yd, zd, codes=codes, max_dist=max_dist)
    vis_h = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
    vis_h.copy_(vis, non_blocking=True)
    cod_h = None
    if cod is not None:
        cod_h = torch.empty(cod.shape, dtype=cod.dtype, pin_memory=True)
        cod_h.copy_(cod, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return vis_h, cod_h


def _single(cfn, fname, depth, x, y, z, vis=None, codes=False, max_dist=N.RBSM_MAXDIST_DEFAULT, stream=None):
    if not isinstance(depth, MapTexture) and not depth.is_cuda:
        return _host_roundtrip(lambda *a, **k: _single(cfn, fname, *a, **k), depth, x, y, z, codes, max_dist)
    m = map_desc(depth)
    f = frags_desc(x, y, z)
    n = f.n
    if vis is None:
        vis = torch.empty(n, dtype=torch.float32, device=x.device)
    else:
        _check_plane("vis", vis, n)
    cod = None
    if codes is True:
        cod = torch.empty(n, dtype=torch.int16, device=x.device)
    elif isinstance(codes, torch.Tensor):
        cod = codes
        if cod.dtype not in (torch.int16, torch.uint16) or cod.numel() != n or not cod.is_cuda:
            raise TypeError("codes must be an int16/uint16 CUDA tensor of n elements")
    p = _params(max_dist)
    rc = cfn(ctypes.byref(m), ctypes.byref(f), ctypes.c_void_p(vis.data_ptr()),
             ctypes.c_void_p(cod.data_ptr() if cod is not None else 0), ctypes.byref(p), _stream_handle(stream))
    N.check(fname, rc)
    return vis, cod


def rbsm_visibility(depth, x, y, z, vis=None, codes=False, max_dist=N.RBSM_MAXDIST_DEFAULT, stream=None):
    """Silhouette recovery (Listing 4): returns (vis, codes or None).
    codes=True allocates an int16 code plane (bit layout in include/rbsm.h)."""
    return _single(N.lib().rbsm_visibility, "rbsm_visibility", depth, x, y, z, vis, codes, max_dist, stream)


def rsmss_filter(depth, x, y, z, vis=None, codes=False, max_dist=N.RBSM_MAXDIST_DEFAULT, stream=None):
    """Revectorization-based shadow filtering (Listing 5): returns (vis, codes or None)."""
    return _single(N.lib().rsmss_filter, "rsmss_filter", depth, x, y, z, vis, codes, max_dist, stream)

_RPCF_WORKSPACES = {}


def _rpcf_workspace(device, stream):
    """The 8-byte counter of rbsm_rpcf_ws kept per (device, stream): calls on
    one stream run in order, so they can share it."""
    s = stream if stream is not None else torch.cuda.current_stream(device)
    key = (device.index, s.cuda_stream)
    ws = _RPCF_WORKSPACES.get(key)
    if ws is None:
        ws = torch.zeros(1, dtype=torch.int64, device=device)
        _RPCF_WORKSPACES[key] = ws
    return ws


def rbsm_rpcf(depth, x, y, z, k=3, vis=None, max_dist=N.RBSM_MAXDIST_DEFAULT, stream=None, workspace="auto"):
    """RPCF: the mean RSMSS answer of the k x k samples shifted by whole
    texels around each fragment (PCF over Listing 5, §5.3).  CUDA tensors
    (or a MapTexture); returns vis.  workspace: "auto" (default) calls
    rbsm_rpcf_ws with a counter kept per stream; a CUDA tensor of at least 8
    bytes calls rbsm_rpcf_ws with that counter; None calls rbsm_rpcf (a
    fixed partition of the tiles).  The answers are the same bits."""
    m = map_desc(depth)
    f = frags_desc(x, y, z)
    if vis is None:
        vis = torch.empty(f.n, dtype=torch.float32, device=x.device)
    else:
        _check_plane("vis", vis, f.n)
    p = _params(max_dist)
    if isinstance(workspace, str):
        if workspace != "auto":
            raise ValueError("workspace must be 'auto', None or a CUDA tensor")
        workspace = _rpcf_workspace(x.device, stream)
    if workspace is None:
        N.check("rbsm_rpcf", N.lib().rbsm_rpcf(ctypes.byref(m), ctypes.byref(f), ctypes.c_void_p(vis.data_ptr()),
                                               int(k), ctypes.byref(p), _stream_handle(stream)))
    else:
        if not isinstance(workspace, torch.Tensor) or not workspace.is_cuda or \
                workspace.numel() * workspace.element_size() < 8:
            raise TypeError("workspace must be a CUDA tensor of at least 8 bytes")
        N.check("rbsm_rpcf_ws", N.lib().rbsm_rpcf_ws(ctypes.byref(m), ctypes.byref(f),
                                                     ctypes.c_void_p(vis.data_ptr()), int(k), ctypes.byref(p),
                                                     ctypes.c_void_p(workspace.data_ptr()),
                                                     _stream_handle(stream)))
    return vis


class Job:
    """One fragment set against one map of a batch.  Outputs are allocated
    when not given: vis_silhouette / vis_filter per the mode."""

    def __init__(self, map_index, x, y, z, mode=N.RBSM_MODE_BOTH, vis_silhouette=None, vis_filter=None,
                 codes=None):
        self.map_index, self.mode = int(map_index), int(mode)
        self.x, self.y, self.z = x, y, z
        n = x.shape[0]
        pin = not x.is_cuda      # host jobs (Stager) answer into page-locked planes
        if (mode & 1) and vis_silhouette is None:
            vis_silhouette = torch.empty(n, dtype=torch.float32, device=x.device, pin_memory=pin)
        if (mode & 2) and vis_filter is None:
            vis_filter = torch.empty(n, dtype=torch.float32, device=x.device, pin_memory=pin)
        if codes is True:
            codes = torch.empty(n, dtype=torch.int16, device=x.device, pin_memory=pin)
        self.vis_silhouette, self.vis_filter, self.codes = vis_silhouette, vis_filter, codes

    def desc(self):
        f = frags_desc(self.x, self.y, self.z)
        ptr = lambda t: t.data_ptr() if t is not None else 0
        return N.rbsm_job(self.map_index, self.mode, f, ptr(self.vis_silhouette), ptr(self.vis_filter),
                          ptr(self.codes))


class Batch:
    """Descriptor arrays of a batched launch, kept alive with their tensors."""

    def __init__(self, maps, jobs, max_dist=N.RBSM_MAXDIST_DEFAULT, tile_threads=0, ctas_per_sm=0,
                 surrogate=None, guard_tau=0.0, chunk_tiles=0, plain_loads=False):
        self.maps, self.jobs = list(maps), list(jobs)
        self.surrogate = surrogate
        self._maps = (N.rbsm_map * len(self.maps))(*[map_desc(m) for m in self.maps])
        self._jobs = (N.rbsm_job * len(self.jobs))(*[j.desc() for j in self.jobs])
        self.desc = N.rbsm_batch(self._maps, len(self.maps), self._jobs, len(self.jobs),
                                 _params(max_dist), int(tile_threads), int(ctas_per_sm),
                                 surrogate.state.data_ptr() if surrogate is not None else None,
                                 float(guard_tau), int(chunk_tiles),
                                 N.RBSM_BATCH_PLAIN_LOADS if plain_loads else 0)
        size = ctypes.c_size_t(0)
        N.check("rbsm_batch_workspace_size", N.lib().rbsm_batch_workspace_size(ctypes.byref(self.desc),
                                                                              ctypes.byref(size)))
        self.workspace_bytes = size.value
        dev = self.jobs[0].x.device
        # 256-byte aligned: the caching allocator aligns blocks to 512 bytes
        self.workspace = torch.zeros(max(self.workspace_bytes, 256) // 4, dtype=torch.int32, device=dev)

    def set_launch(self, tile_threads, ctas_per_sm, chunk_tiles=0, flags=0):
        self.desc.tile_threads = int(tile_threads)
        self.desc.ctas_per_sm = int(ctas_per_sm)
        self.desc.chunk_tiles = int(chunk_tiles)
        self.desc.flags = int(flags)


def rbsm_batch_run(batch, stream=None):
    """Enqueue one persistent launch over every job of `batch` (a Batch)."""
    rc = N.lib().rbsm_batch_run(ctypes.byref(batch.desc), ctypes.c_void_p(batch.workspace.data_ptr()),
                                batch.workspace_bytes, _stream_handle(stream))
    N.check("rbsm_batch_run", rc)
    return batch


def rbsm_batch_status(batch):
    """Status word the last completed launch of `batch` recorded."""
    st = ctypes.c_int(0)
    N.check("rbsm_batch_status", N.lib().rbsm_batch_status(ctypes.c_void_p(batch.workspace.data_ptr()),
                                                           ctypes.byref(st)))
    return st.value


class BatchGraph:
    """A CUDA graph of one batched launch of `batch` (rbsm_batch_graph_*):
    built once, replayed by launch().  It binds the batch's tensors as they
    are now; keep `batch` alive while the graph is used."""

    def __init__(self, batch):
        self.batch = batch
        h = ctypes.c_void_p(0)
        N.check("rbsm_batch_graph_create",
                N.lib().rbsm_batch_graph_create(ctypes.byref(batch.desc), ctypes.c_void_p(batch.workspace.data_ptr()),
                                                batch.workspace_bytes, ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        N.check("rbsm_batch_graph_launch", N.lib().rbsm_batch_graph_launch(self.handle, _stream_handle(stream)))

    def close(self):
        if self.handle is not None and self.handle.value:
            N.check("rbsm_batch_graph_destroy", N.lib().rbsm_batch_graph_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_signature(batch):
    """Key of a batch for the autotuner cache: device, map sizes, job sizes."""
    name = torch.cuda.get_device_name(batch.jobs[0].x.device)
    maps = [tuple(m.depth.shape) + ("tex",) if isinstance(m, MapTexture) else tuple(m.shape) for m in batch.maps]
    jobs = [(j.map_index, j.mode, int(j.x.shape[0]), j.codes is not None) for j in batch.jobs]
    return json.dumps(["v2", name, maps, jobs])


TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")


def rbsm_batch_autotune(batch, repeats=3, stream=None, cache=TUNE_CACHE):
    """Pick the batched launch shape by timing the candidates on this GPU
    (rbsm_batch_autotune), remember it per batch signature in `cache`
    (None: no file), apply it to `batch` and return the rbsm_tuning fields."""
    key = batch_signature(batch)
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table:
        hit = dict(table[key], cached=True)
        batch.set_launch(hit["tile_threads"], hit["ctas_per_sm"], hit.get("chunk_tiles", 0), hit.get("flags", 0))
        return hit
    t = N.rbsm_tuning()
    N.check("rbsm_batch_autotune",
            N.lib().rbsm_batch_autotune(ctypes.byref(batch.desc), ctypes.c_void_p(batch.workspace.data_ptr()),
                                        batch.workspace_bytes, _stream_handle(stream), int(repeats),
                                        ctypes.byref(t)))
    res = {"tile_threads": t.tile_threads, "ctas_per_sm": t.ctas_per_sm, "chunk_tiles": t.chunk_tiles,
           "flags": t.flags, "plain_loads": bool(t.flags & N.RBSM_BATCH_PLAIN_LOADS), "ms": t.ms,
           "candidates": t.candidates}
    batch.set_launch(t.tile_threads, t.ctas_per_sm, t.chunk_tiles, t.flags)
    if cache:
        table[key] = res
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return dict(res, cached=False)


def rbsm_batch_surrogate_counts(batch):
    """(surrogate answers, guard fallbacks) of the last completed launch."""
    a, f = ctypes.c_uint64(0), ctypes.c_uint64(0)
    N.check("rbsm_batch_surrogate_counts",
            N.lib().rbsm_batch_surrogate_counts(ctypes.c_void_p(batch.workspace.data_ptr()), ctypes.byref(a),
                                                ctypes.byref(f)))
    return a.value, f.value


def _host_plane(name, t, n=None, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or t.dim() != 1:
        raise TypeError("%s must be a 1-D %s tensor" % (name, dtype))
    if n is not None and t.shape[0] != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.shape[0], n))
    if t.numel() == 0:
        return None
    if t.is_cuda or not t.is_pinned():
        raise TypeError("%s must be a page-locked (pinned) CPU tensor" % name)
    if t.numel() > 1 and t.stride(0) != 1:
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.shape[0] != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.shape[0], n))
    return t.data_ptr()


def _host_map_desc(depth):
    if not isinstance(depth, torch.Tensor) or depth.dtype != torch.float32 or depth.dim() != 2:
        raise TypeError("depth must be a 2-D float32 tensor")
    if depth.is_cuda or not depth.is_pinned():
        raise TypeError("depth must be a page-locked (pinned) CPU tensor")
    if depth.stride(1) != 1 or depth.stride(0) < depth.shape[1]:
        raise ValueError("depth rows must be contiguous (pitch >= width)")
    return N.rbsm_map(depth.data_ptr(), depth.shape[1], depth.shape[0], depth.stride(0), 0)


def _host_job_desc(j):
    n = j.x.shape[0]
    f = N.rbsm_frags(_host_plane("x", j.x), _host_plane("y", j.y, n), _host_plane("z", j.z, n), n)
    sil = _host_plane("vis_silhouette", j.vis_silhouette, n) if j.vis_silhouette is not None else None
    fil = _host_plane("vis_filter", j.vis_filter, n) if j.vis_filter is not None else None
    cod = None
    if j.codes is not None:
        if j.codes.dtype not in (torch.int16, torch.uint16):
            raise TypeError("codes must be int16 or uint16")
        cod = _host_plane("codes", j.codes, n, j.codes.dtype)
    return N.rbsm_job(j.map_index, j.mode, f, sil, fil, cod)


class Stager:
    """Host-resident batches (rbsm_stager_*): shadow maps, fragment planes
    and answer planes in page-locked host memory (pinned CPU tensors; Job
    allocates pinned answers for CPU inputs).  Per map the library copies
    in the fragment planes and only the window of the map within
    max_dist + 1 texels of the fragments' texels, runs the batched kernel
    and copies the answers back, overlapping consecutive maps on its own
    streams.  Answers are those of rbsm_batch_run on device copies."""

    def __init__(self, max_fragments, max_width, max_height, slots=0, texture=True):
        d = N.rbsm_stager_desc(int(max_fragments), int(max_width), int(max_height), int(slots),
                               1 if texture else 0, 0)
        h = ctypes.c_void_p(0)
        N.check("rbsm_stager_create", N.lib().rbsm_stager_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self._inflight = []

    def run(self, maps, jobs, max_dist=N.RBSM_MAXDIST_DEFAULT, tile_threads=0, ctas_per_sm=0, surrogate=None,
            guard_tau=0.0, stream=None):
        """Enqueue one host-resident batch on `stream` (the current torch
        stream by default); the answers are in the jobs' host planes once
        the stream has passed this point.  The tensors must stay alive until
        then (the stager keeps references to the last two runs)."""
        maps, jobs = list(maps), list(jobs)
        md = (N.rbsm_map * len(maps))(*[_host_map_desc(m) for m in maps])
        jd = (N.rbsm_job * len(jobs))(*[_host_job_desc(j) for j in jobs])
        desc = N.rbsm_batch(md, len(maps), jd, len(jobs), _params(max_dist), int(tile_threads), int(ctas_per_sm),
                            surrogate.state.data_ptr() if surrogate is not None else None, float(guard_tau))
        N.check("rbsm_stager_run", N.lib().rbsm_stager_run(self.handle, ctypes.byref(desc), _stream_handle(stream)))
        self._inflight = (self._inflight + [(maps, jobs)])[-2:]

    def stats(self):
        """(bytes copied in, bytes copied out) over every run so far (waits)."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        N.check("rbsm_stager_stats", N.lib().rbsm_stager_stats(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def status(self):
        st = ctypes.c_int(0)
        N.check("rbsm_stager_status", N.lib().rbsm_stager_status(self.handle, ctypes.byref(st)))
        return st.value

    def close(self):
        if self.handle is not None and self.handle.value:
            N.check("rbsm_stager_destroy", N.lib().rbsm_stager_destroy(self.handle))
        self.handle = None
        self._inflight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceOccluders:
    """Analytic occluders of the light pass in device memory (rbsm_rect /
    rbsm_sphere arrays): rects (n, 6) float64 cx cy ux uy ha hb with depths
    (n,) float32, spheres (m, 4) float64 cx cy radius centre-depth."""

    def __init__(self, rects, rect_depth, spheres, device=None):
        import numpy as np
        rects = np.asarray(rects, np.float64).reshape(-1, 6)
        rect_depth = np.asarray(rect_depth, np.float32).reshape(-1)
        spheres = np.asarray(spheres, np.float64).reshape(-1, 4)
        if rect_depth.shape[0] != rects.shape[0]:
            raise ValueError("one depth per rectangle")
        rt = np.zeros(len(rects), np.dtype([("g", np.float64, 6), ("depth", np.float32), ("reserved", np.float32)]))
        rt["g"] = rects
        rt["depth"] = rect_depth
        assert rt.dtype.itemsize == N.RBSM_RECT_BYTES
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.n_rects, self.n_spheres = len(rects), len(spheres)
        self.rects = torch.from_numpy(rt.view(np.uint8).reshape(-1).copy()).to(dev)
        self.spheres = torch.from_numpy(np.ascontiguousarray(spheres).view(np.uint8).reshape(-1).copy()).to(dev)

    def desc(self, zscale, ground=1.0):
        return N.rbsm_occluders(self.rects.data_ptr() if self.n_rects else None, self.n_rects,
                                self.spheres.data_ptr() if self.n_spheres else None, self.n_spheres,
                                float(zscale), float(ground), 0)


def rbsm_shadow_map(occ, width, height, zscale, ground=1.0, out=None, stream=None):
    """Shadow map of DeviceOccluders `occ` (rbsm_shadow_map): a (height,
    width) float32 CUDA tensor, or `out` (rows contiguous, pitch >= width)."""
    if out is None:
        out = torch.empty((int(height), int(width)), dtype=torch.float32, device=occ.rects.device)
    elif (not out.is_cuda or out.dtype != torch.float32 or out.dim() != 2 or out.stride(1) != 1
          or tuple(out.shape) != (int(height), int(width))):
        raise ValueError("out must be a (height, width) float32 CUDA tensor with contiguous rows")
    d = occ.desc(zscale, ground)
    N.check("rbsm_shadow_map", N.lib().rbsm_shadow_map(ctypes.byref(d), ctypes.c_void_p(out.data_ptr()), int(width),
                                                       int(height), out.stride(0), _stream_handle(stream)))
    return out


def rbsm_shadow_maps(occs, width, height, zscale, ground=1.0, outs=None, stream=None):
    """Shadow maps of several DeviceOccluders sets in one call
    (rbsm_shadow_maps): a list of (height, width) float32 CUDA tensors, or
    `outs` (rows contiguous, one pitch for all); the maps' kernels overlap
    when their memory is disjoint."""
    occs = list(occs)
    if outs is None:
        outs = [torch.empty((int(height), int(width)), dtype=torch.float32, device=o.rects.device) for o in occs]
    outs = list(outs)
    if len(outs) != len(occs) or not outs:
        raise ValueError("one output per occluder set")
    for out in outs:
        if (not out.is_cuda or out.dtype != torch.float32 or out.dim() != 2 or out.stride(1) != 1
                or tuple(out.shape) != (int(height), int(width)) or out.stride(0) != outs[0].stride(0)):
            raise ValueError("outs must be (height, width) float32 CUDA tensors with contiguous rows, one pitch")
    descs = (N.rbsm_occluders * len(occs))(*[o.desc(zscale, ground) for o in occs])
    ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    N.check("rbsm_shadow_maps", N.lib().rbsm_shadow_maps(descs, ptrs, len(occs), int(width), int(height),
                                                         outs[0].stride(0), _stream_handle(stream)))
    return outs


class GBufferJob:
    """One (shadow map, depth buffer) pair of rbsm_visibility_gbuffer: `depth`
    a map tensor or MapTexture, `gdepth` a (height, width) float32 CUDA
    tensor with contiguous rows, `m` the 4 x 4 screen-to-light-clip matrix.
    Answer planes (height * width) are allocated for the mode when not given."""

    def __init__(self, depth, gdepth, m, mode=N.RBSM_MODE_BOTH, codes=False, vis_silhouette=None,
                 vis_filter=None):
        import numpy as np
        if not isinstance(gdepth, torch.Tensor) or not gdepth.is_cuda or gdepth.dtype != torch.float32 \
                or gdepth.dim() != 2 or gdepth.stride(1) != 1:
            raise TypeError("gdepth must be a 2-D float32 CUDA tensor with contiguous rows")
        self.depth, self.gdepth, self.mode = depth, gdepth, int(mode)
        self.m = np.ascontiguousarray(np.asarray(m, np.float32).reshape(16))
        n = gdepth.shape[0] * gdepth.shape[1]
        dev = gdepth.device
        if (mode & 1) and vis_silhouette is None:
            vis_silhouette = torch.empty(n, dtype=torch.float32, device=dev)
        if (mode & 2) and vis_filter is None:
            vis_filter = torch.empty(n, dtype=torch.float32, device=dev)
        if codes is True:
            codes = torch.empty(n, dtype=torch.int16, device=dev)
        self.vis_silhouette = vis_silhouette if mode & 1 else None
        self.vis_filter = vis_filter if mode & 2 else None
        self.codes = codes if isinstance(codes, torch.Tensor) else None

    def desc(self):
        h, w = self.gdepth.shape
        g = N.rbsm_gbuffer(self.gdepth.data_ptr(), w, h, self.gdepth.stride(0),
                           (ctypes.c_float * 16)(*self.m.tolist()))
        ptr = lambda t: t.data_ptr() if t is not None else None
        return N.rbsm_gbuffer_job(map_desc(self.depth), g, ptr(self.vis_silhouette), ptr(self.vis_filter),
                                  ptr(self.codes))


def rbsm_visibility_gbuffer(jobs, mode=N.RBSM_MODE_BOTH, max_dist=N.RBSM_MAXDIST_DEFAULT, stream=None):
    """Visibility of every pixel of the jobs' depth buffers in one launch
    (rbsm_visibility_gbuffer); each GBufferJob's answer planes are filled."""
    jobs = list(jobs)
    arr = (N.rbsm_gbuffer_job * len(jobs))(*[j.desc() for j in jobs])
    p = _params(max_dist)
    N.check("rbsm_visibility_gbuffer",
            N.lib().rbsm_visibility_gbuffer(arr, len(jobs), int(mode), ctypes.byref(p), _stream_handle(stream)))
    return jobs


def rbsm_selftest_bounded_wait(limit_ns=2_000_000, stream=None):
    """Runs the library's bounded mbarrier wait on a barrier nothing arrives
    at, then after one arrival (rbsm_selftest_bounded_wait); returns
    (gave_up, completed_after_arrival, waited_ns) once the stream is done."""
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    N.check("rbsm_selftest_bounded_wait",
            N.lib().rbsm_selftest_bounded_wait(int(limit_ns), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    o = out.cpu().tolist()
    return bool(o[0]), bool(o[1]), int(o[2])
