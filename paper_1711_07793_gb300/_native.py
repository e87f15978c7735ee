"""ctypes view of the C ABI in include/rbsm.h (no compute here).

The library is loaded from this package's _build/ directory and nowhere
else.  There is no fallback: when librbsm.so is missing or cannot be loaded,
``lib()`` raises, so nothing can silently run a different implementation.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librbsm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rbsm.h")

RBSM_OK = 0
RBSM_ERR_ARG = -1
RBSM_ERR_CUDA = -2
RBSM_ERR_TIMEOUT = -3
RBSM_DATASET_IN_WINDOW = 1
RBSM_BATCH_PLAIN_LOADS = 1
RBSM_MLP_TRUST_WORDS = 1 << 20
RBSM_ERR_WORKSPACE = -4

RBSM_MODE_SILHOUETTE = 1
RBSM_MODE_FILTER = 2
RBSM_MODE_BOTH = 3
RBSM_MAXDIST_DEFAULT = 16
RBSM_BATCH_MAX_MAPS = 64
RBSM_BATCH_MAX_JOBS = 256
RBSM_RPCF_MAX_K = 7


class rbsm_map(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pitch", ctypes.c_int64), ("texture", ctypes.c_uint64)]


class rbsm_frags(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("n", ctypes.c_int64)]


class rbsm_params(ctypes.Structure):
    _fields_ = [("max_dist", ctypes.c_int32), ("flags", ctypes.c_int32)]


class rbsm_job(ctypes.Structure):
    _fields_ = [("map", ctypes.c_int32), ("mode", ctypes.c_int32), ("frags", rbsm_frags),
                ("vis_silhouette", ctypes.c_void_p), ("vis_filter", ctypes.c_void_p),
                ("codes", ctypes.c_void_p)]


class rbsm_batch(ctypes.Structure):
    _fields_ = [("maps", ctypes.POINTER(rbsm_map)), ("n_maps", ctypes.c_int32),
                ("jobs", ctypes.POINTER(rbsm_job)), ("n_jobs", ctypes.c_int32),
                ("params", rbsm_params), ("tile_threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("surrogate", ctypes.c_void_p),
                ("guard_tau", ctypes.c_float), ("chunk_tiles", ctypes.c_int32), ("flags", ctypes.c_int32)]


class rbsm_sample(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_uint32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("gap", ctypes.c_float), ("label", ctypes.c_float)]


RBSM_MLP_PARAMS = 6402


class rbsm_tuning(ctypes.Structure):
    _fields_ = [("tile_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("ms", ctypes.c_float), ("candidates", ctypes.c_int32), ("chunk_tiles", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class rbsm_stager_desc(ctypes.Structure):
    _fields_ = [("max_fragments", ctypes.c_int64), ("max_width", ctypes.c_int32),
                ("max_height", ctypes.c_int32), ("slots", ctypes.c_int32), ("texture", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class rbsm_occluders(ctypes.Structure):
    _fields_ = [("rects", ctypes.c_void_p), ("n_rects", ctypes.c_int32), ("spheres", ctypes.c_void_p),
                ("n_spheres", ctypes.c_int32), ("zscale", ctypes.c_double), ("ground", ctypes.c_float),
                ("flags", ctypes.c_int32)]


RBSM_RECT_BYTES = 56
RBSM_SPHERE_BYTES = 32


class rbsm_gbuffer(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("m", ctypes.c_float * 16)]


class rbsm_gbuffer_job(ctypes.Structure):
    _fields_ = [("map", rbsm_map), ("gbuffer", rbsm_gbuffer), ("vis_silhouette", ctypes.c_void_p),
                ("vis_filter", ctypes.c_void_p), ("codes", ctypes.c_void_p)]


RBSM_GBUFFER_MAX_JOBS = 64
RBSM_SHADOW_MAPS_MAX = 256


class RBSMError(RuntimeError):
    def __init__(self, fn, code, cuda_error=0):
        msg = "%s failed: %s (%d)" % (fn, status_string(code), code)
        if code == RBSM_ERR_CUDA:
            msg += ", cudaError %d" % cuda_error
        super().__init__(msg)
        self.code = code
        self.cuda_error = cuda_error


_lib = None
_P = ctypes.POINTER


def _declare(lib):
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    for name in ("rbsm_visibility", "rsmss_filter"):
        f = getattr(lib, name)
        f.restype = i32
        f.argtypes = [_P(rbsm_map), _P(rbsm_frags), vp, vp, _P(rbsm_params), vp]
    lib.rbsm_rpcf.restype = i32
    lib.rbsm_rpcf.argtypes = [_P(rbsm_map), _P(rbsm_frags), vp, ctypes.c_int32, _P(rbsm_params), vp]
    lib.rbsm_rpcf_ws.restype = i32
    lib.rbsm_rpcf_ws.argtypes = [_P(rbsm_map), _P(rbsm_frags), vp, ctypes.c_int32, _P(rbsm_params), vp, vp]
    lib.rbsm_shadow_map.restype = i32
    lib.rbsm_shadow_map.argtypes = [_P(rbsm_occluders), vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, vp]
    lib.rbsm_shadow_maps.restype = i32
    lib.rbsm_shadow_maps.argtypes = [_P(rbsm_occluders), _P(vp), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int64, vp]
    lib.rbsm_visibility_gbuffer.restype = i32
    lib.rbsm_visibility_gbuffer.argtypes = [_P(rbsm_gbuffer_job), ctypes.c_int32, ctypes.c_int32,
                                            _P(rbsm_params), vp]
    lib.rbsm_map_texture_create.restype = i32
    lib.rbsm_map_texture_create.argtypes = [_P(rbsm_map), _P(ctypes.c_uint64)]
    lib.rbsm_map_texture_destroy.restype = i32
    lib.rbsm_map_texture_destroy.argtypes = [ctypes.c_uint64]
    lib.rbsm_batch_workspace_size.restype = i32
    lib.rbsm_batch_workspace_size.argtypes = [_P(rbsm_batch), _P(ctypes.c_size_t)]
    lib.rbsm_batch_run.restype = i32
    lib.rbsm_batch_run.argtypes = [_P(rbsm_batch), vp, ctypes.c_size_t, vp]
    lib.rbsm_batch_run_noalloc.restype = i32
    lib.rbsm_batch_run_noalloc.argtypes = [_P(rbsm_batch), vp]
    lib.rbsm_batch_noalloc_counts.restype = i32
    lib.rbsm_batch_noalloc_counts.argtypes = [_P(ctypes.c_uint64), _P(ctypes.c_uint64)]
    lib.rbsm_batch_graph_create.restype = i32
    lib.rbsm_batch_graph_create.argtypes = [_P(rbsm_batch), vp, ctypes.c_size_t, _P(vp)]
    lib.rbsm_batch_graph_launch.restype = i32
    lib.rbsm_batch_graph_launch.argtypes = [vp, vp]
    lib.rbsm_batch_graph_destroy.restype = i32
    lib.rbsm_batch_graph_destroy.argtypes = [vp]
    lib.rbsm_batch_autotune.restype = i32
    lib.rbsm_batch_autotune.argtypes = [_P(rbsm_batch), vp, ctypes.c_size_t, vp, ctypes.c_int32, _P(rbsm_tuning)]
    lib.rbsm_batch_status.restype = i32
    lib.rbsm_batch_status.argtypes = [vp, _P(ctypes.c_int)]
    lib.rbsm_batch_surrogate_counts.restype = i32
    lib.rbsm_batch_surrogate_counts.argtypes = [vp, _P(ctypes.c_uint64), _P(ctypes.c_uint64)]
    lib.rbsm_stager_create.restype = i32
    lib.rbsm_stager_create.argtypes = [_P(rbsm_stager_desc), _P(vp)]
    lib.rbsm_stager_run.restype = i32
    lib.rbsm_stager_run.argtypes = [vp, _P(rbsm_batch), vp]
    lib.rbsm_stager_stats.restype = i32
    lib.rbsm_stager_stats.argtypes = [vp, _P(ctypes.c_int64), _P(ctypes.c_int64)]
    lib.rbsm_stager_status.restype = i32
    lib.rbsm_stager_status.argtypes = [vp, _P(ctypes.c_int)]
    lib.rbsm_stager_destroy.restype = i32
    lib.rbsm_stager_destroy.argtypes = [vp]
    lib.rbsm_mlp_state_bytes.restype = ctypes.c_size_t
    lib.rbsm_mlp_state_bytes.argtypes = []
    for name in ("rbsm_mlp_load", "rbsm_mlp_store"):
        getattr(lib, name).restype = i32
        getattr(lib, name).argtypes = [vp, vp, vp]
    lib.rbsm_mlp_dataset.restype = i32
    lib.rbsm_mlp_dataset.argtypes = [_P(rbsm_map), _P(rbsm_frags), _P(rbsm_params), vp, ctypes.c_int64, vp, vp]
    lib.rbsm_mlp_grad.restype = i32
    lib.rbsm_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    lib.rbsm_mlp_set_trust.restype = i32
    lib.rbsm_mlp_set_trust.argtypes = [vp, vp, vp]
    lib.rbsm_mlp_step.restype = i32
    lib.rbsm_mlp_step.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp]
    lib.rbsm_mlp_adam.restype = i32
    lib.rbsm_mlp_adam.argtypes = [vp, ctypes.c_int32, ctypes.c_float, vp]
    lib.rbsm_mlp_read.restype = i32
    lib.rbsm_mlp_read.argtypes = [vp, vp, vp, vp]
    lib.rbsm_mlp_reset_loss.restype = i32
    lib.rbsm_mlp_reset_loss.argtypes = [vp, vp]
    lib.rbsm_mlp_forward.restype = i32
    lib.rbsm_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.rbsm_selftest_bounded_wait.restype = i32
    lib.rbsm_selftest_bounded_wait.argtypes = [ctypes.c_uint64, vp, vp]
    lib.rbsm_status_string.restype = ctypes.c_char_p
    lib.rbsm_status_string.argtypes = [i32]
    lib.rbsm_last_cuda_error.restype = i32
    lib.rbsm_version.restype = i32


def lib():
    """The loaded librbsm.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librbsm.so is not built (%s); run paper_1711_07793_gb300.build.build()"
                               % LIB_PATH)
        l = ctypes.CDLL(LIB_PATH)
        _declare(l)
        _lib = l
    return _lib


def status_string(code):
    try:
        return lib().rbsm_status_string(code).decode()
    except RuntimeError:
        return "status %d" % code


def check(fn, code):
    if code != RBSM_OK:
        raise RBSMError(fn, code, lib().rbsm_last_cuda_error() if code == RBSM_ERR_CUDA else 0)


def header_functions(path=HEADER):
    """Names of the functions include/rbsm.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^[A-Za-z_][\w \*]*?\b(rbsm\w*|rsmss\w*)\s*\(", text, flags=re.M)
