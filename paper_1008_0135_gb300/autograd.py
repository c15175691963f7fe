"""torch.autograd.Function over the library's forward and adjoint ray casting.

``render_views`` renders a batch of views of one cube with a transfer-function table that may
require gradients, and optionally with voxels that require gradients (they are copied into the
cube's bricks before rendering).  Backward is one vr_render_backward_views call: the library
replays every ray of every view from its stored segment colour and transmittance (no per-sample
storage) and sums the views' table gradients in FP64.
"""
from __future__ import annotations

import torch


class _RenderViews(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lut, voxels, vctx, cube_id, cams, vrange, step, tau):
        if voxels is not None:
            vctx.update_cube(cube_id, voxels.detach().contiguous())
        vctx.set_transfer_function(lut.detach(), vrange[0], vrange[1])
        vctx.set_render_params("dvr", step, tau)
        outs = []
        for cam in cams:
            vctx.set_camera_dict(cam)
            outs.append(vctx.render_frame(cube_id))
        fctx.vctx, fctx.cube_id, fctx.cams = vctx, cube_id, cams
        fctx.vrange, fctx.step, fctx.tau = vrange, step, tau
        fctx.lut_host = lut.detach().cpu()
        fctx.vox_shape = None if voxels is None else voxels.shape
        fctx.dev = lut.device if lut.is_cuda else torch.device(f"cuda:{vctx.device}")
        return torch.stack(outs)

    @staticmethod
    def backward(fctx, gout):
        vctx = fctx.vctx
        vctx.set_transfer_function(fctx.lut_host, fctx.vrange[0], fctx.vrange[1])
        vctx.set_render_params("dvr", fctx.step, fctx.tau)
        n = fctx.lut_host.shape[0]
        glut = torch.empty((n, 4), dtype=torch.float32, device=fctx.dev)
        need_vox = fctx.needs_input_grad[1] and fctx.vox_shape is not None
        gvox = torch.zeros(fctx.vox_shape, dtype=torch.float32, device=fctx.dev) if need_vox else None
        vctx.set_camera_dict(fctx.cams[-1])      # the batch's frame size; last view's fragments reused
        vctx.render_backward_views(fctx.cube_id, fctx.cams, gout.contiguous(), glut, gvox)
        glut_out = glut if fctx.needs_input_grad[0] else None
        return glut_out, gvox, None, None, None, None, None, None


def render_views(vctx, cube_id: int, lut: torch.Tensor, cams, vrange, voxels=None,
                 step: float = 0.5, tau: float = 0.99) -> torch.Tensor:
    """(V, H, W, 4) premultiplied RGBA of each camera in ``cams`` (dicts with view, proj, param,
    W, H; all the same size).  Differentiable w.r.t. ``lut`` (n x 4) and ``voxels``
    ([z][y][x] float32 CUDA tensor, FP32 bricks)."""
    return _RenderViews.apply(lut, voxels, vctx, cube_id, list(cams), tuple(vrange), float(step),
                              float(tau))
