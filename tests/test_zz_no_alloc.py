"""vr_render_frame_noalloc: the frame renderer for callers that cannot allocate device memory while
they render (their GPU memory belongs to another allocator or a fixed budget, or their frame
loop must not stall on cudaMalloc's device-wide synchronisation).  It must give the same image
as vr_render_frame, call after call, although every call reuses one static scratch array.

This file is collected last so that a run stopping at the first failure has run everything
else first; it creates its own context, so it also passes alone in a fresh process."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import ATOL_F32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1008_0135_gb300 as P
    from paper_1008_0135_gb300 import _abi
    P.build()
    ctx = P.Context(0)
    cube = synth.pr1_cube(seed=0)
    cid = ctx.load_cube(cube)
    ctx.set_brick_layouts(cid, 15)
    ctx.set_bricking(cid, (32, 32, 32), 1, "f32")
    ctx.set_transfer_function(synth.ramp_lut(alpha=0.5), -3.0, 20.0)
    yield torch, ctx, _abi.lib(), cid
    ctx.close()


def _noalloc(torch, ctx, L, cid, like):
    out = torch.full_like(like, float("nan"))
    rc = L.vr_render_frame_noalloc(ctx._h, cid, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.vr_last_error_message().decode()
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_render_frame_on_consecutive_calls(setup):
    torch, ctx, L, cid = setup
    views = [
        (synth.pr1_camera(), "dvr"),
        (dict(view=synth.look_at((90.0, 70.0, -40.0), (32.0, 30.0, 34.0)), proj=1,
              param=math.radians(55.0), W=200, H=150), "dvr"),
        (synth.pr1_camera(W=128, H=96, angle_deg=75.0), "mip"),
    ]
    refs = []
    for cam, mode in views:
        ctx.set_camera_dict(cam)
        ctx.set_render_params(mode, 0.5, 0.99)
        refs.append(ctx.render_frame(cid).clone())
    torch.cuda.synchronize()
    # two (here three, then a repeat) calls in a row, each against the allocating entry point
    for k in [0, 1, 2, 0]:
        cam, mode = views[k]
        ctx.set_camera_dict(cam)
        ctx.set_render_params(mode, 0.5, 0.99)
        out = _noalloc(torch, ctx, L, cid, refs[k])
        assert not torch.isnan(out).any()
        if mode == "dvr":
            assert (out - refs[k]).abs().max().item() <= ATOL_F32
        else:
            assert torch.equal(out, refs[k])


def test_noalloc_rejects_frames_beyond_its_scratch(setup):
    torch, ctx, L, cid = setup
    cube = synth.pr1_cube(seed=1, n=64)
    big = ctx.load_cube(cube)
    ctx.set_bricking(big, (4, 4, 4), 1, "f32")          # 4096 bricks: fragments far above 64 MiB
    ctx.set_camera_dict(synth.pr1_camera(W=2048, H=2048))
    ctx.set_render_params("dvr", 0.5, 0.99)
    out = torch.zeros((2048, 2048, 4), device="cuda")
    rc = L.vr_render_frame_noalloc(ctx._h, big, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert "64 MiB" in L.vr_last_error_message().decode()
    ctx.free_cube(big)
