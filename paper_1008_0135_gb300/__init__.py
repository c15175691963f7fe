"""Python binding of libvrcube.so: bricked volume ray casting + sort-last compositing on GB300.

Argument marshalling only: every step of the rendering path runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams; numpy arrays are accepted for host data.
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import (VR_BF16, VR_DEVICE, VR_DVR, VR_F16, VR_F32, VR_HOST, VR_MIP, VR_ORTHO,
                   VR_PERSP)

__all__ = ["Context", "VrError", "build", "STORAGE", "VR_DVR", "VR_MIP", "VR_ORTHO", "VR_PERSP",
           "VR_F32", "VR_F16", "VR_BF16", "VR_HOST", "VR_DEVICE"]

STORAGE = {"f32": VR_F32, "f16": VR_F16, "bf16": VR_BF16}
MODES = {"dvr": VR_DVR, "mip": VR_MIP}


def build(force: bool = False) -> str:
    from .build_ext import build as _b
    return _b(force=force)


class VrError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = _abi.lib()
        msg = L.vr_error_string(status).decode()
        detail = L.vr_last_error_message().decode()
        super().__init__(f"{where}: {msg}" + (f" [{detail}]" if detail else ""))
        self.status = status


def _check(rc: int, where: str):
    if rc != 0:
        raise VrError(rc, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_handle(stream) -> int:
    """CUDA stream handle: a torch.cuda.Stream, a raw handle, or torch's current stream."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _buffer(x):
    """(pointer, location) of a contiguous float32 numpy array or torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        loc = VR_DEVICE if x.is_cuda else VR_HOST
        return x.data_ptr(), loc
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, VR_HOST


def _fill_request(q, r, keep):
    q.cube_id = int(r["cube"])
    view = np.ascontiguousarray(r["cam"]["view"], dtype=np.float32).reshape(16)
    for j in range(16):
        q.view[j] = float(view[j])
    q.proj, q.param = int(r["cam"]["proj"]), float(r["cam"]["param"])
    q.width, q.height = int(r["cam"]["W"]), int(r["cam"]["H"])
    q.mode = MODES[r.get("mode", "dvr")]
    q.step, q.ert_threshold = float(r.get("step", 0.5)), float(r.get("tau", 0.99))
    lut = np.ascontiguousarray(r["lut"], dtype=np.float32)
    keep.append(lut)
    q.lut, q.nlut = lut.ctypes.data, lut.shape[0]
    q.vmin, q.vmax = float(r["vrange"][0]), float(r["vrange"][1])
    q.arrival_ms = float(r.get("arrival_ms", 0.0))
    ptr, loc = _buffer(r["out"])
    q.out, q.out_where = ptr, loc
    q.termination = {"segment": 0, "global": 1}[r.get("termination", "segment")]


def _result_dict(res):
    return {k: getattr(res, k) for k, _ in _abi.VrRequestResult._fields_}


class Server:
    """The online serving loop (vr_serve_open / submit / poll / close).  Keep each request's
    ``out`` alive until its ticket has been polled."""

    def __init__(self, ctx, max_inflight: int = 4):
        self._L = ctx._L
        self._h = C.c_void_p()
        cfg = _abi.VrServeConfig(int(max_inflight))
        _check(self._L.vr_serve_open(ctx._h, C.byref(cfg), C.byref(self._h)), "vr_serve_open")

    def submit(self, request: dict) -> int:
        q = _abi.VrRequest()
        keep = []
        _fill_request(q, request, keep)
        t = C.c_int64()
        _check(self._L.vr_serve_submit(self._h, C.byref(q), C.byref(t)), "vr_serve_submit")
        return t.value

    def poll(self, wait_ms: int = 0, cap: int = 64):
        """[(ticket, result dict)] of the requests finished since the last poll."""
        tk = (C.c_int64 * cap)()
        rs = (_abi.VrRequestResult * cap)()
        n = C.c_int()
        _check(self._L.vr_serve_poll(self._h, tk, rs, cap, C.byref(n), int(wait_ms)), "vr_serve_poll")
        return [(tk[i], _result_dict(rs[i])) for i in range(n.value)]

    def close(self) -> dict:
        summ = _abi.VrServeSummary()
        rc = self._L.vr_serve_close(self._h, C.byref(summ))
        self._h = None
        if rc not in (0, _abi.VR_ERR_STATE):
            raise VrError(rc, "vr_serve_close")
        return {k: getattr(summ, k) for k, _ in _abi.VrServeSummary._fields_}


class Context:
    """One library context on one CUDA device (vr_create / vr_destroy)."""

    def __init__(self, device: int = 0, cache_bytes: int = 0):
        self._L = _abi.lib()
        h = C.c_void_p()
        _check(self._L.vr_create(C.byref(h), int(device), int(cache_bytes)), "vr_create")
        self._h = h
        self.device = device
        self.cam = None
        self.mode = VR_DVR

    def close(self):
        if getattr(self, "_h", None):
            self._L.vr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------------------------- cubes
    def load_cube(self, voxels, sub_origin=None, sub_extent=None) -> int:
        """voxels: float32 [z][y][x] numpy array (host) or CUDA tensor (device)."""
        if _is_torch(voxels):
            import torch
            if voxels.dtype != torch.float32:
                raise ValueError("voxels must be float32")
        else:
            voxels = np.ascontiguousarray(voxels, dtype=np.float32)
        nz, ny, nx = voxels.shape
        ptr, loc = _buffer(voxels)
        so = (C.c_int64 * 3)(*sub_origin) if sub_origin is not None else None
        se = (C.c_int64 * 3)(*sub_extent) if sub_extent is not None else None
        cid = C.c_int()
        _check(self._L.vr_load_cube(self._h, ptr, VR_F32, nx, ny, nz, loc, so, se, C.byref(cid)),
               "vr_load_cube")
        return cid.value

    def load_cube_procedural(self, seed: int, shape_xyz) -> int:
        """Streamed procedural cube (bricks generated on host threads, cached in HBM)."""
        nx, ny, nz = shape_xyz
        cid = C.c_int()
        _check(self._L.vr_load_cube_procedural(self._h, int(seed), nx, ny, nz, C.byref(cid)),
               "vr_load_cube_procedural")
        return cid.value

    def set_fault_injection(self, kind: int, after: int = 0):
        _check(self._L.vr_set_fault_injection(self._h, int(kind), int(after)),
               "vr_set_fault_injection")

    def update_cube(self, cube_id: int, voxels, stream=None):
        ptr, loc = _buffer(voxels)
        sh = _stream_handle(stream) if loc == VR_DEVICE else 0
        _check(self._L.vr_update_cube(self._h, cube_id, ptr, loc, sh), "vr_update_cube")

    def free_cube(self, cube_id: int):
        _check(self._L.vr_free_cube(self._h, cube_id), "vr_free_cube")

    def compute_minmax(self, cube_id: int):
        lo, hi = C.c_float(), C.c_float()
        _check(self._L.vr_compute_minmax(self._h, cube_id, C.byref(lo), C.byref(hi)),
               "vr_compute_minmax")
        return lo.value, hi.value

    def set_bricking(self, cube_id: int, brick, ghost: int = 1, storage: str = "f32"):
        bx, by, bz = brick
        _check(self._L.vr_set_bricking(self._h, cube_id, bx, by, bz, ghost, STORAGE[storage]),
               "vr_set_bricking")

    def compress_cube(self, cube_id: int):
        """Encodes the cube into 8-bit Haar-wavelet blocks in HBM and releases its FP32 voxels and
        bricks; frames then decode bricks on demand into the brick cache (vr_compress_cube)."""
        _check(self._L.vr_compress_cube(self._h, cube_id), "vr_compress_cube")

    def wavelet_store_bytes(self, cube_id: int) -> int:
        n = C.c_size_t(0)
        _check(self._L.vr_wavelet_store(self._h, cube_id, None, C.byref(n)), "vr_wavelet_store")
        return n.value

    def wavelet_store(self, cube_id: int):
        """The compressed cube's block store as a uint8 numpy array (544 bytes per 8^3 block)."""
        import numpy as np
        n = C.c_size_t(0)
        _check(self._L.vr_wavelet_store(self._h, cube_id, None, C.byref(n)), "vr_wavelet_store")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(self._L.vr_wavelet_store(self._h, cube_id, buf.ctypes.data, C.byref(n)), "vr_wavelet_store")
        return buf

    def set_brick_layouts(self, cube_id: int, mask: int):
        """Keep x- (1), y- (2), z-contiguous (4) copies of the bricks (bit 0 always kept) and
        slice-atlas textures of them (8)."""
        _check(self._L.vr_set_brick_layouts(self._h, cube_id, int(mask)), "vr_set_brick_layouts")

    def brick_grid(self, cube_id: int):
        nb = (C.c_int64 * 3)()
        st = C.c_int()
        _check(self._L.vr_get_brick_grid(self._h, cube_id, nb, C.byref(st)), "vr_get_brick_grid")
        return tuple(nb), st.value

    def get_brick(self, cube_id: int, brick: int, with_data: bool = True):
        dims, org, e = (C.c_int * 3)(), (C.c_int * 3)(), C.c_int()
        _check(self._L.vr_get_brick(self._h, cube_id, brick, dims, org, C.byref(e), None),
               "vr_get_brick")
        data = None
        if with_data:
            _, st = self.brick_grid(cube_id)
            dt = np.float32 if st == VR_F32 else np.uint16
            data = np.zeros((dims[2], dims[1], dims[0]), dt)
            _check(self._L.vr_get_brick(self._h, cube_id, brick, dims, org, C.byref(e),
                                        data.ctypes.data), "vr_get_brick")
        return tuple(dims), tuple(org), e.value, data

    # ---------------------------------------------------------------------------- rendering
    def set_transfer_function(self, rgba, vmin: float, vmax: float):
        lut = np.ascontiguousarray(
            rgba.detach().cpu().numpy() if _is_torch(rgba) else rgba, dtype=np.float32)
        _check(self._L.vr_set_transfer_function(self._h, lut.ctypes.data, lut.shape[0],
                                                float(vmin), float(vmax)),
               "vr_set_transfer_function")

    def set_camera(self, view, proj: int, param: float, width: int, height: int):
        v = np.ascontiguousarray(view, dtype=np.float32).reshape(16)
        _check(self._L.vr_set_camera(self._h, v.ctypes.data, int(proj), float(param), int(width),
                                     int(height)), "vr_set_camera")
        self.cam = (int(width), int(height))

    def set_camera_dict(self, cam: dict):
        self.set_camera(cam["view"], cam["proj"], cam["param"], cam["W"], cam["H"])

    def set_render_params(self, mode: str = "dvr", step: float = 0.5, tau: float = 0.99):
        self.mode = MODES[mode]
        _check(self._L.vr_set_render_params(self._h, self.mode, float(step), float(tau)),
               "vr_set_render_params")

    def set_termination(self, scope: str = "segment"):
        """Early-termination scope for DVR: "segment" (each brick's ray segment stops on its own;
        fragments composited afterwards) or "global" (occlusion skipping: each ray walks the bricks
        front to back in one pass and stops once the whole ray is opaque)."""
        _check(self._L.vr_set_termination(self._h, {"segment": 0, "global": 1}[scope]),
               "vr_set_termination")

    def set_host_output_async(self, flag: bool = True):
        """With a host ``out``, render_frame returns once the copy into it is queued on the
        stream (read ``out`` after synchronising that stream or an event recorded after the
        call); False restores the synchronous copy."""
        _check(self._L.vr_set_host_output_async(self._h, 1 if flag else 0),
               "vr_set_host_output_async")

    def set_channel_mask(self, mask=None):
        """0/1 per spectral channel (cube z); None switches every channel on."""
        if mask is None:
            _check(self._L.vr_set_channel_mask(self._h, None, 0), "vr_set_channel_mask")
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        _check(self._L.vr_set_channel_mask(self._h, m.ctypes.data, m.size), "vr_set_channel_mask")

    def set_window(self, lo=None, hi=None):
        """Clip rendering to the voxel box [lo, hi) (x, y, z); None removes the window."""
        if lo is None:
            _check(self._L.vr_set_window(self._h, None, None), "vr_set_window")
            return
        _check(self._L.vr_set_window(self._h, (C.c_int64 * 3)(*lo), (C.c_int64 * 3)(*hi)),
               "vr_set_window")

    def set_timing(self, enable: bool):
        _check(self._L.vr_set_timing(self._h, int(bool(enable))), "vr_set_timing")

    def set_full_rect(self, enable: bool):
        _check(self._L.vr_set_full_rect(self._h, int(bool(enable))), "vr_set_full_rect")

    def render_frame(self, cube_id: int, out=None, stream=None):
        """Renders into ``out`` (CUDA tensor or numpy array; allocated as a CUDA tensor when None).
        DVR: (H, W, 4) premultiplied RGBA; MIP: (H, W)."""
        if self.cam is None:
            raise VrError(_abi.VR_ERR_STATE, "render_frame: set a camera first")
        W, H = self.cam
        if out is None:
            import torch
            shape = (H, W, 4) if self.mode == VR_DVR else (H, W)
            out = torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}")
        ptr, loc = _buffer(out)
        sh = _stream_handle(stream) if (loc == VR_DEVICE or stream is not None) else 0
        _check(self._L.vr_render_frame(self._h, cube_id, ptr, loc, sh), "vr_render_frame")
        return out

    # ------------------------------------------------------------------- sort-last partitions
    def set_partition(self, cube_id: int, counts=(), index=()):
        """Draw only one part of the cube: a recursive longest-axis split with counts[L] slabs at
        level L, keeping slab index[L] (empty counts: the whole cube)."""
        n = len(counts)
        if len(index) != n:
            raise ValueError("counts and index must have the same length")
        ca = (C.c_int * max(n, 1))(*[int(v) for v in counts])
        ia = (C.c_int * max(n, 1))(*[int(v) for v in index])
        _check(self._L.vr_set_partition(self._h, cube_id, n, ca, ia), "vr_set_partition")

    def set_partition_balance(self, cube_id: int, balanced: bool):
        """Cuts at equal layer counts (False) or balanced by the current camera's estimated cost."""
        _check(self._L.vr_set_partition_balance(self._h, cube_id, int(bool(balanced))),
               "vr_set_partition_balance")

    def partition(self, cube_id: int, nlevels: int = 8):
        """(lo, hi, axes): the part's brick index ranges per axis and the split axis per level."""
        lo, hi, ax = (C.c_int * 3)(), (C.c_int * 3)(), (C.c_int * 8)()
        _check(self._L.vr_get_partition(self._h, cube_id, lo, hi, ax), "vr_get_partition")
        return tuple(lo), tuple(hi), tuple(ax)[:nlevels]

    def render_subimage(self, cube_id: int, out=None, stream=None):
        """The part's sub-image: DVR (H, W, 4) premultiplied colour + transmittance; MIP (H, W)
        with -inf where the part has no sample."""
        if self.cam is None:
            raise VrError(_abi.VR_ERR_STATE, "render_subimage: set a camera first")
        W, H = self.cam
        if out is None:
            import torch
            shape = (H, W, 4) if self.mode == VR_DVR else (H, W)
            out = torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}")
        ptr, loc = _buffer(out)
        sh = _stream_handle(stream) if (loc == VR_DEVICE or stream is not None) else 0
        _check(self._L.vr_render_subimage(self._h, cube_id, ptr, loc, sh), "vr_render_subimage")
        return out

    def composite_subimages(self, cube_id: int, level: int, subs, row0: int, final: bool, out=None,
                            stream=None):
        """Blends the sibling parts' sub-images of `level` (CUDA tensor (n, rows, W, 4) or
        (n, rows, W)) for frame rows [row0, row0 + rows); returns (rows, W, 4) / (rows, W)."""
        if not subs.is_contiguous():
            raise ValueError("subs must be contiguous")
        n, rows = int(subs.shape[0]), int(subs.shape[1])
        if out is None:
            import torch
            out = torch.empty(tuple(subs.shape[1:]), dtype=torch.float32, device=subs.device)
        _check(self._L.vr_composite_subimages(self._h, cube_id, int(level), n, subs.data_ptr(), int(row0),
                                              rows, int(bool(final)), out.data_ptr(),
                                              _stream_handle(stream)),
               "vr_composite_subimages")
        return out

    def render_backward(self, cube_id: int, grad_out, grad_lut, grad_voxels=None, stream=None):
        gv = grad_voxels.data_ptr() if grad_voxels is not None else None
        _check(self._L.vr_render_backward(self._h, cube_id, grad_out.data_ptr(),
                                          grad_lut.data_ptr(), gv, _stream_handle(stream)),
               "vr_render_backward")

    def render_backward_views(self, cube_id: int, cams, grad_out, grad_lut, grad_voxels=None, stream=None):
        """Gradient over a batch of views (dicts with view, proj, param; the current camera's
        size): grad_out (V, H, W, 4) CUDA tensor; grad_lut (n, 4) overwritten with the batch's
        table gradient (summed over the views in FP64 by the library); grad_voxels added to."""
        n = len(cams)
        arr = (_abi.VrView * max(n, 1))()
        for i, cam in enumerate(cams):
            view = np.ascontiguousarray(cam["view"], dtype=np.float32).reshape(16)
            for j in range(16):
                arr[i].view[j] = float(view[j])
            arr[i].proj, arr[i].param = int(cam["proj"]), float(cam["param"])
        gv = grad_voxels.data_ptr() if grad_voxels is not None else None
        _check(self._L.vr_render_backward_views(self._h, cube_id, n, arr, grad_out.data_ptr(),
                                                grad_lut.data_ptr(), gv, _stream_handle(stream)),
               "vr_render_backward_views")

    def serve(self, requests, max_inflight: int = 4):
        """Runs the continuous-batching request loop (vr_serve).  ``requests``: dicts with cube,
        cam (view/proj/param/W/H), mode, step, tau, lut (n x 4), vrange, arrival_ms, out (a
        CUDA tensor or pinned host tensor) and optionally termination ("segment" or "global"),
        in arrival order.  Returns (results, summary)."""
        n = len(requests)
        arr = (_abi.VrRequest * max(n, 1))()
        keep = []
        for i, r in enumerate(requests):
            _fill_request(arr[i], r, keep)
        cfg = _abi.VrServeConfig(int(max_inflight))
        res = (_abi.VrRequestResult * max(n, 1))()
        summ = _abi.VrServeSummary()
        rc = self._L.vr_serve(self._h, arr, n, C.byref(cfg), res, C.byref(summ))
        if rc not in (0, _abi.VR_ERR_STATE):
            raise VrError(rc, "vr_serve")
        results = [_result_dict(res[i]) for i in range(n)]
        summary = {k: getattr(summ, k) for k, _ in _abi.VrServeSummary._fields_}
        return results, summary

    def serve_online(self, max_inflight: int = 4) -> "Server":
        """An online request loop (vr_serve_open): submit requests as they arrive, poll results."""
        return Server(self, max_inflight)

    def stats(self) -> dict:
        s = _abi.VrStats()
        _check(self._L.vr_get_stats(self._h, C.byref(s)), "vr_get_stats")
        return {k: getattr(s, k) for k, _ in _abi.VrStats._fields_}

    def reset_stats(self):
        _check(self._L.vr_reset_stats(self._h), "vr_reset_stats")
