"""ctypes declarations of libvrcube.so (include/vrcube.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libvrcube.so")

VR_OK, VR_ERR_ARG, VR_ERR_OOM, VR_ERR_CUDA = 0, -1, -2, -3
VR_ERR_TIMEOUT, VR_ERR_STATE, VR_ERR_NOT_FOUND, VR_ERR_UNSUPPORTED = -4, -5, -6, -7
VR_ERR_IO = -8
VR_F32, VR_F16, VR_BF16 = 0, 1, 2
VR_HOST, VR_DEVICE = 0, 1
VR_ORTHO, VR_PERSP = 0, 1
VR_DVR, VR_MIP = 0, 1


class VrStats(C.Structure):
    _fields_ = [
        ("frames", C.c_int64), ("samples", C.c_int64), ("fragments", C.c_int64),
        ("bricks_drawn", C.c_int64), ("bricks_sampled", C.c_int64),
        ("brick_bytes_sampled", C.c_int64), ("ms_raycast", C.c_double),
        ("ms_composite", C.c_double), ("ms_frame", C.c_double), ("timed_frames", C.c_int64),
        ("bytes_streamed", C.c_int64), ("cache_hits", C.c_int64), ("cache_misses", C.c_int64),
        ("kernel_errors", C.c_int64),
    ]


class VrRequest(C.Structure):
    _fields_ = [
        ("cube_id", C.c_int), ("view", C.c_float * 16), ("proj", C.c_int), ("param", C.c_float),
        ("width", C.c_int), ("height", C.c_int), ("mode", C.c_int), ("step", C.c_float),
        ("ert_threshold", C.c_float), ("lut", C.c_void_p), ("nlut", C.c_int),
        ("vmin", C.c_float), ("vmax", C.c_float), ("arrival_ms", C.c_double),
        ("out", C.c_void_p), ("out_where", C.c_int), ("termination", C.c_int),
    ]


class VrRequestResult(C.Structure):
    _fields_ = [("status", C.c_int), ("admit_ms", C.c_double), ("done_ms", C.c_double),
                ("latency_ms", C.c_double)]


class VrView(C.Structure):
    _fields_ = [("view", C.c_float * 16), ("proj", C.c_int), ("param", C.c_float)]


class VrServeConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int)]


class VrServeSummary(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("wall_ms", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("frames_per_s", C.c_double), ("max_concurrent", C.c_int)]


# name -> (restype, argtypes); every entry point declared in include/vrcube.h
P, I, I64, F, VP = C.POINTER, C.c_int, C.c_int64, C.c_float, C.c_void_p
SIGNATURES = {
    "vr_create": (I, [P(VP), I, C.c_size_t]),
    "vr_destroy": (None, [VP]),
    "vr_load_cube": (I, [VP, VP, I, I64, I64, I64, I, P(I64), P(I64), P(I)]),
    "vr_load_cube_procedural": (I, [VP, C.c_uint64, I64, I64, I64, P(I)]),
    "vr_set_fault_injection": (I, [VP, I, I64]),
    "vr_update_cube": (I, [VP, I, VP, I, VP]),
    "vr_free_cube": (I, [VP, I]),
    "vr_compute_minmax": (I, [VP, I, P(F), P(F)]),
    "vr_set_bricking": (I, [VP, I, I, I, I, I, I]),
    "vr_set_brick_layouts": (I, [VP, I, I]),
    "vr_set_transfer_function": (I, [VP, VP, I, F, F]),
    "vr_set_camera": (I, [VP, VP, I, F, I, I]),
    "vr_set_render_params": (I, [VP, I, F, F]),
    "vr_set_termination": (I, [VP, I]),
    "vr_set_host_output_async": (I, [VP, I]),
    "vr_compress_cube": (I, [VP, I]),
    "vr_wavelet_store": (I, [VP, I, VP, P(C.c_size_t)]),
    "vr_render_frame": (I, [VP, I, VP, I, VP]),
    "vr_render_frame_noalloc": (I, [VP, I, VP, VP]),
    "vr_set_partition": (I, [VP, I, I, P(I), P(I)]),
    "vr_get_partition": (I, [VP, I, P(I), P(I), P(I)]),
    "vr_set_partition_balance": (I, [VP, I, I]),
    "vr_render_subimage": (I, [VP, I, VP, I, VP]),
    "vr_composite_subimages": (I, [VP, I, I, I, VP, I, I, I, VP, VP]),
    "vr_render_backward": (I, [VP, I, VP, VP, VP, VP]),
    "vr_render_backward_views": (I, [VP, I, I, P(VrView), VP, VP, VP, VP]),
    "vr_set_channel_mask": (I, [VP, VP, I64]),
    "vr_set_window": (I, [VP, P(I64), P(I64)]),
    "vr_set_timing": (I, [VP, I]),
    "vr_set_full_rect": (I, [VP, I]),
    "vr_get_stats": (I, [VP, P(VrStats)]),
    "vr_reset_stats": (I, [VP]),
    "vr_get_brick_grid": (I, [VP, I, P(I64), P(I)]),
    "vr_get_brick": (I, [VP, I, I64, P(I), P(I), P(I), VP]),
    "vr_serve": (I, [VP, P(VrRequest), I, P(VrServeConfig), P(VrRequestResult),
                     P(VrServeSummary)]),
    "vr_serve_open": (I, [VP, P(VrServeConfig), P(VP)]),
    "vr_serve_submit": (I, [VP, P(VrRequest), P(C.c_int64)]),
    "vr_serve_poll": (I, [VP, P(C.c_int64), P(VrRequestResult), I, P(I), I]),
    "vr_serve_close": (I, [VP, P(VrServeSummary)]),
    "vr_error_string": (C.c_char_p, [I]),
    "vr_last_error_message": (C.c_char_p, []),
}

_lib = None


def lib():
    """Loads libvrcube.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1008_0135_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
