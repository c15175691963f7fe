"""vr_render_frame_noalloc: the frame renderer for callers that cannot allocate device memory while
they render (their GPU memory belongs to another allocator or a fixed budget, or their frame
loop must not stall on cudaMalloc's device-wide synchronisation).  It runs the same kernels on
the same work-list as vr_render_frame, so its frames must be the same bits, call after call,
although every call reuses one static scratch array.

This file is collected last so that a run stopping at the first failure has run everything
else first; it creates its own context, so it also passes alone in a fresh process."""
import math

import pytest

import synth

pytestmark = pytest.mark.gpu

VR_ERR_UNSUPPORTED = -7


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


VIEWS = [
    (synth.pr1_camera(), "dvr"),
    (dict(view=synth.look_at((90.0, 70.0, -40.0), (32.0, 30.0, 34.0)), proj=1,
          param=math.radians(55.0), W=200, H=150), "dvr"),
    (synth.pr1_camera(W=128, H=96, angle_deg=75.0), "mip"),
]


def _set_view(ctx, k):
    cam, mode = VIEWS[k]
    ctx.set_camera_dict(cam)
    ctx.set_render_params(mode, 0.5, 0.99)


def _call(torch, ctx, L, cid, out):
    rc = L.vr_render_frame_noalloc(ctx._h, cid, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.vr_last_error_message().decode()


def _references(torch, ctx, cid):
    refs = []
    for k in range(len(VIEWS)):
        _set_view(ctx, k)
        refs.append(ctx.render_frame(cid).clone())
    torch.cuda.synchronize()
    return refs


def test_noalloc_matches_render_frame_on_consecutive_calls(setup):
    torch, ctx, L, cid = setup
    refs = _references(torch, ctx, cid)
    # calls one after the other (each waited for), against the allocating entry point
    for k in [0, 1, 2, 0]:
        _set_view(ctx, k)
        out = torch.full_like(refs[k], float("nan"))
        _call(torch, ctx, L, cid, out)
        torch.cuda.synchronize()
        assert torch.equal(out, refs[k]), k


@pytest.mark.parametrize("storage,layouts", [("f16", 41), ("bf16", 9)])
def test_noalloc_matches_render_frame_with_16bit_bricks(setup, storage, layouts):
    """16-bit bricks read through slice atlases or pair atlases (one gather per sample): the same
    bits as the allocating entry point."""
    torch, ctx, L, _ = setup
    cid = ctx.load_cube(synth.pr1_cube(seed=1))
    ctx.set_brick_layouts(cid, layouts)
    ctx.set_bricking(cid, (24, 32, 20), 1, storage)
    try:
        refs = _references(torch, ctx, cid)
        for k in range(len(VIEWS)):
            _set_view(ctx, k)
            out = torch.full_like(refs[k], float("nan"))
            _call(torch, ctx, L, cid, out)
            torch.cuda.synchronize()
            assert torch.equal(out, refs[k]), (storage, k)
    finally:
        ctx.free_cube(cid)


def test_noalloc_calls_queued_on_one_stream_allocate_nothing(setup):
    """Calls queued back to back on one stream (each one's upload overwrites the scratch the one
    before it read, in stream order) give every frame its own bits; across them neither the
    device's free memory nor torch's allocator changes."""
    torch, ctx, L, cid = setup
    refs = _references(torch, ctx, cid)
    order = [0, 1, 2, 1, 0, 2, 0]
    outs = [torch.full_like(refs[k], float("nan")) for k in order]
    _set_view(ctx, 0)
    _call(torch, ctx, L, cid, torch.empty_like(refs[0]))     # warm-up: every kernel loaded
    _set_view(ctx, 2)
    _call(torch, ctx, L, cid, torch.empty_like(refs[2]))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for k, out in zip(order, outs):
        _set_view(ctx, k)
        _call(torch, ctx, L, cid, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
    for k, out in zip(order, outs):
        assert torch.equal(out, refs[k]), k


def test_noalloc_refuses_what_needs_the_allocating_path(setup):
    """Streamed cubes need the brick cache, and global termination its own pass: both are
    refused with VR_ERR_UNSUPPORTED, and the next frame renders normally."""
    torch, ctx, L, cid = setup
    import paper_1008_0135_gb300 as P
    refs = _references(torch, ctx, cid)
    _set_view(ctx, 0)
    out = torch.empty_like(refs[0])
    ctx.set_termination("global")
    rc = L.vr_render_frame_noalloc(ctx._h, cid, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == VR_ERR_UNSUPPORTED
    ctx.set_termination("segment")
    with P.Context(0, cache_bytes=64 * 34 ** 3 * 4) as sc:
        sid = sc.load_cube_procedural(4, (64, 64, 64))
        sc.set_bricking(sid, (32, 32, 32), 1, "f32")
        sc.set_transfer_function(synth.ramp_lut(alpha=0.5), -3.0, 20.0)
        sc.set_camera_dict(VIEWS[0][0])
        sc.set_render_params("dvr", 0.5, 0.99)
        rc = L.vr_render_frame_noalloc(sc._h, sid, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == VR_ERR_UNSUPPORTED
    _call(torch, ctx, L, cid, out)
    torch.cuda.synchronize()
    assert torch.equal(out, refs[0])


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
