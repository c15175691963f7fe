"""Streamed (out-of-core) cubes: bricks produced on host threads, cached in HBM, LRU eviction,
chunked frames, host-side fault injection -- checked against the oracle's own procedural cube."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import compare_dvr, gpu_ctx, render

pytestmark = pytest.mark.gpu

SEED = 4
SMALL = (300, 270, 260)          # three 128^3 bricks per axis (the last ones partial)
BRICK = (128, 128, 128)
F32_BRICK_BYTES = 130 ** 3 * 4


@pytest.fixture(scope="module")
def big_ctx():
    import paper_1008_0135_gb300 as P
    c = gpu_ctx()
    c.close()
    c = P.Context(0, cache_bytes=64 * F32_BRICK_BYTES)
    yield c
    c.close()


def _cam(shape, W=96, H=80, seed=0):
    return synth.random_camera(np.random.default_rng(seed), shape, W, H, proj=1)


def test_streamed_bricks_match_the_oracle_generator(big_ctx, orc):
    ctx = big_ctx
    cid = ctx.load_cube_procedural(SEED, SMALL)
    ctx.set_bricking(cid, BRICK, 1, "f32")
    for b in (0, 4, 26):                            # interior-touching and border bricks
        dims, org, e, data = ctx.get_brick(cid, b)
        ref = orc.proc_region(SEED, SMALL, org, dims)
        assert e == 0 and np.array_equal(data.view(np.uint32), ref.view(np.uint32))
    ctx.free_cube(cid)


@pytest.mark.parametrize("mode", ["dvr", "mip"])
def test_streamed_render_matches_oracle(big_ctx, orc, mode):
    ctx = big_ctx
    cid = ctx.load_cube_procedural(SEED, SMALL)
    ctx.set_bricking(cid, BRICK, 1, "f32")
    lut = synth.ramp_lut(alpha=0.4)
    cam = _cam(SMALL, seed=3)
    g = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
    proc = orc.Procedural(SEED, SMALL)
    if mode == "dvr":
        ref, flags, _ = orc.render(proc, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=BRICK)
        compare_dvr(g, ref, flags, 0.99)
    else:
        ref, _, _ = orc.render(proc, lut, (-3, 20), cam, mode="mip32", step=0.5, brick=BRICK)
        assert np.array_equal(g, ref.astype(np.float32))
    ctx.free_cube(cid)


def test_cache_hits_and_chunked_frames_agree():
    """A cache of 5 slots forces a 27-brick frame into chunks and evictions; the image equals
    the one rendered with a cache that holds every brick, and a repeated frame hits."""
    import paper_1008_0135_gb300 as P
    lut = synth.ramp_lut(alpha=0.3)
    cam = dict(view=synth.look_at((150.0, 135.0, -300.0), (150.0, 135.0, 130.0)), proj=1,
               param=math.radians(70.0), W=120, H=100)
    imgs, stats = [], []
    for slots in (64, 5):
        with P.Context(0, cache_bytes=slots * F32_BRICK_BYTES) as ctx:
            cid = ctx.load_cube_procedural(SEED, SMALL)
            ctx.set_bricking(cid, BRICK, 1, "f32")
            ctx.reset_stats()
            imgs.append(render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99))
            s1 = ctx.stats()
            imgs.append(render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99))
            s2 = ctx.stats()
            stats.append((s1, s2))
    assert np.array_equal(imgs[0], imgs[2]) and np.array_equal(imgs[0], imgs[1])
    assert np.array_equal(imgs[2], imgs[3])
    big1, big2 = stats[0]
    assert big1["cache_misses"] == big1["bricks_drawn"] and big1["cache_hits"] == 0
    assert big2["cache_hits"] - big1["cache_hits"] == big1["bricks_drawn"]      # all hits
    assert big2["cache_misses"] == big1["cache_misses"]
    small1, small2 = stats[1]
    assert small2["cache_misses"] > small1["cache_misses"]       # 5 slots: evicted, re-streamed
    assert small1["bytes_streamed"] > 0


def test_streamed_frames_are_timed():
    """vr_set_timing covers streamed frames too: frame, ray-cast (with residency) and compositing."""
    import paper_1008_0135_gb300 as P
    lut = synth.ramp_lut(alpha=0.3)
    cam = dict(view=synth.look_at((150.0, 135.0, -300.0), (150.0, 135.0, 130.0)), proj=1,
               param=math.radians(70.0), W=120, H=100)
    with P.Context(0, cache_bytes=8 * F32_BRICK_BYTES) as ctx:
        cid = ctx.load_cube_procedural(SEED, SMALL)
        ctx.set_bricking(cid, BRICK, 1, "f32")
        ctx.reset_stats()
        ctx.set_timing(True)
        render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        st = ctx.stats()
        ctx.set_timing(False)
    assert st["timed_frames"] == 2
    assert st["ms_frame"] >= st["ms_raycast"] + st["ms_composite"] - 1e-3 > 0


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_streamed_16bit_equals_resident_16bit(orc, storage):
    """Host-encoded streamed bricks equal device-encoded resident bricks of the same voxels."""
    import paper_1008_0135_gb300 as P
    shape = (200, 150, 130)
    vox = orc.proc_region(SEED, shape, (0, 0, 0), shape)
    lut = synth.ramp_lut(alpha=0.4)
    cam = _cam(shape, seed=5)
    with P.Context(0, cache_bytes=40 * 66 ** 3 * 2) as ctx:
        sid = ctx.load_cube_procedural(SEED, shape)
        ctx.set_bricking(sid, (64, 64, 64), 1, storage)
        rid = ctx.load_cube(vox)
        ctx.set_bricking(rid, (64, 64, 64), 1, storage)
        for b in (0, 11, 23):
            d1, o1, e1, c1 = ctx.get_brick(sid, b)
            d2, o2, e2, c2 = ctx.get_brick(rid, b)
            assert (d1, o1, e1) == (d2, o2, e2) and np.array_equal(c1, c2)
        a = render(ctx, sid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        b = render(ctx, rid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        assert np.array_equal(a, b)


def test_virtual_cube_close_up_matches_oracle(orc):
    """The 4096x4096x4800 virtual cube (322 GB as FP32, above HBM) through a small cache:
    a close-up view, checked on seeded sampled rays."""
    import paper_1008_0135_gb300 as P
    shape = (4096, 4096, 4800)
    brick = (256, 256, 256)
    lut = synth.ramp_lut()
    cam = dict(view=synth.look_at((2100.0, 1900.0, -60.0), (2050.0, 2000.0, 300.0)), proj=1,
               param=math.radians(12.0), W=256, H=256)
    with P.Context(0, cache_bytes=48 * 258 ** 3 * 4) as ctx:
        cid = ctx.load_cube_procedural(SEED, shape)
        ctx.set_bricking(cid, brick, 1, "f32")
        ctx.reset_stats()
        g = render(ctx, cid, lut, (-3, 100), cam, step=1.0, tau=0.99)
        st = ctx.stats()
    assert st["bricks_drawn"] > 48                                  # more than the cache holds
    pix = synth.sample_pixels(44, 256, 256, 384)
    ref, flags, _ = orc.render(orc.Procedural(SEED, shape), lut, (-3, 100), cam, step=1.0,
                               tau=0.99, brick=brick, pix=pix)
    compare_dvr(g[pix], ref, flags, 0.99)


def test_fault_injection_leaves_the_context_usable(big_ctx):
    import paper_1008_0135_gb300 as P
    ctx = big_ctx
    lut = synth.ramp_lut(alpha=0.3)
    cam = _cam(SMALL, seed=9)
    cid = ctx.load_cube_procedural(SEED + 1, SMALL)
    ctx.set_bricking(cid, BRICK, 1, "f32")
    ctx.set_fault_injection(1, after=ctx.stats()["cache_misses"] + 3)
    with pytest.raises(P.VrError) as e:
        render(ctx, cid, lut, (-3, 20), cam, step=0.5)
    assert e.value.status == -8                                    # VR_ERR_IO
    ctx.set_fault_injection(0)
    ok1 = render(ctx, cid, lut, (-3, 20), cam, step=0.5)
    with P.Context(0, cache_bytes=64 * F32_BRICK_BYTES) as fresh:
        fid = fresh.load_cube_procedural(SEED + 1, SMALL)
        fresh.set_bricking(fid, BRICK, 1, "f32")
        ok2 = render(fresh, fid, lut, (-3, 20), cam, step=0.5)
    assert np.array_equal(ok1, ok2)
    with P.Context(0, cache_bytes=64 * F32_BRICK_BYTES) as bad:
        bad.set_fault_injection(2)
        bid = bad.load_cube_procedural(SEED, SMALL)
        bad.set_bricking(bid, BRICK, 1, "f32")
        with pytest.raises(P.VrError) as e:
            render(bad, bid, lut, (-3, 20), cam, step=0.5)
        assert e.value.status == -2                                # VR_ERR_OOM
    with P.Context(0, cache_bytes=64 * F32_BRICK_BYTES) as slow:
        slow.set_fault_injection(3)
        sid = slow.load_cube_procedural(SEED, SMALL)
        slow.set_bricking(sid, (32, 32, 32), 1, "f32")             # many misses per frame
        with pytest.raises(P.VrError) as e:
            render(slow, sid, lut, (-3, 20), _cam(SMALL, W=200, H=200, seed=2), step=0.5)
        assert e.value.status == -4                                # VR_ERR_TIMEOUT
    ctx.free_cube(cid)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", ["dvr", "mip"])
def test_slot_atlases_give_identical_images(storage, mode):
    """Mask 9 on a streamed cube: cache slots also hold slice atlases, read by texture gathers;
    the image equals the one read from the slots' linear bricks, bit for bit, for a frame that
    fits the cache and for one chunked through a cache of 5 slots (evictions re-pack atlases)."""
    import paper_1008_0135_gb300 as P
    lut = synth.ramp_lut(alpha=0.3)
    cam = dict(view=synth.look_at((150.0, 135.0, -300.0), (150.0, 135.0, 130.0)), proj=1,
               param=math.radians(70.0), W=120, H=100)
    esz = 4 if storage == "f32" else 2
    for slots in (64, 5):
        with P.Context(0, cache_bytes=slots * 130 ** 3 * esz) as ctx:
            cid = ctx.load_cube_procedural(SEED, SMALL)
            ctx.set_bricking(cid, BRICK, 1, storage)
            lin = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            ctx.set_brick_layouts(cid, 9)
            at1 = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)   # packs hits
            at2 = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            ctx.set_brick_layouts(cid, 1)
            lin2 = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            assert np.array_equal(lin, at1) and np.array_equal(lin, at2) and np.array_equal(lin, lin2)
            assert np.count_nonzero(lin) > 0
            with pytest.raises(P.VrError):
                ctx.set_brick_layouts(cid, 15)


@pytest.mark.parametrize("layouts", [1, 9])
def test_global_termination_of_a_streamed_cube(orc, layouts):
    """Occlusion skipping on a streamed cube: the frame's bricks made resident together, one
    ray-march over the brick grid; the image equals the resident cube's global-termination frame
    of the same voxels (bit for bit), repeats from cache hits, and a cache smaller than the
    frame's bricks refuses (VR_ERR_UNSUPPORTED)."""
    import paper_1008_0135_gb300 as P
    vox = orc.proc_region(SEED, SMALL, (0, 0, 0), SMALL)
    lut = synth.ramp_lut(alpha=1.0)                  # opaque: rays stop early
    cams = [_cam(SMALL, W=96, H=80, seed=s) for s in (3, 8)]
    cams.append(dict(view=synth.look_at((150.0, 135.0, -300.0), (150.0, 135.0, 130.0)), proj=1,
                     param=math.radians(70.0), W=120, H=100))
    with P.Context(0, cache_bytes=40 * F32_BRICK_BYTES) as ctx:
        sid = ctx.load_cube_procedural(SEED, SMALL)
        ctx.set_bricking(sid, BRICK, 1, "f32")
        ctx.set_brick_layouts(sid, layouts)
        rid = ctx.load_cube(vox)
        ctx.set_brick_layouts(rid, layouts)
        ctx.set_bricking(rid, BRICK, 1, "f32")
        ctx.set_termination("global")
        try:
            for cam in cams:
                a = render(ctx, sid, lut, (-3, 20), cam, step=0.5, tau=0.99)
                b = render(ctx, rid, lut, (-3, 20), cam, step=0.5, tau=0.99)
                again = render(ctx, sid, lut, (-3, 20), cam, step=0.5, tau=0.99)
                assert np.array_equal(a, b) and np.array_equal(a, again)
                assert np.count_nonzero(a) > 0
        finally:
            ctx.set_termination("segment")
    with P.Context(0, cache_bytes=5 * F32_BRICK_BYTES) as small:
        sid = small.load_cube_procedural(SEED, SMALL)
        small.set_bricking(sid, BRICK, 1, "f32")
        small.set_termination("global")
        with pytest.raises(P.VrError) as e:
            render(small, sid, lut, (-3, 20), cams[2], step=0.5, tau=0.99)
        assert e.value.status == -7


def test_async_host_output_of_streamed_frames():
    """Asynchronous host output for streamed frames (DVR and MIP, chunked through 5 slots):
    the queued copies, read after an event, equal the synchronous frames."""
    import torch
    import paper_1008_0135_gb300 as P
    lut = synth.ramp_lut(alpha=0.3)
    cam = dict(view=synth.look_at((150.0, 135.0, -300.0), (150.0, 135.0, 130.0)), proj=1,
               param=math.radians(70.0), W=120, H=100)
    with P.Context(0, cache_bytes=5 * F32_BRICK_BYTES) as ctx:
        cid = ctx.load_cube_procedural(SEED, SMALL)
        ctx.set_bricking(cid, BRICK, 1, "f32")
        for mode in ["dvr", "mip"]:
            want = render(ctx, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            shape = (cam["H"], cam["W"], 4) if mode == "dvr" else (cam["H"], cam["W"])
            bufs = [torch.full(shape, -1.0).pin_memory() for _ in range(2)]
            ev = [torch.cuda.Event() for _ in range(2)]
            ctx.set_host_output_async(True)
            try:
                for k in range(2):
                    ctx.render_frame(cid, bufs[k])
                    ev[k].record()
                for k in range(2):
                    ev[k].synchronize()
                    assert np.array_equal(bufs[k].numpy().reshape(want.shape), want)
            finally:
                ctx.set_host_output_async(False)


@pytest.mark.parametrize("term", ["segment", "global"])
def test_streamed_atlas_frames_with_mask_and_window(orc, term):
    """A streamed cube with slot atlases, a spectral-channel mask and a render window, per-segment
    and global termination, DVR and MIP: every frame equals the resident cube's of the same
    voxels with the same settings, bit for bit."""
    import paper_1008_0135_gb300 as P
    vox = orc.proc_region(SEED, SMALL, (0, 0, 0), SMALL)
    lut = synth.ramp_lut(alpha=0.6)
    rng = np.random.default_rng(7)
    mask = (rng.uniform(size=SMALL[2]) > 0.3).astype(np.uint8)
    cams = [_cam(SMALL, W=96, H=80, seed=s) for s in (2, 9)]
    with P.Context(0, cache_bytes=40 * F32_BRICK_BYTES) as ctx:
        sid = ctx.load_cube_procedural(SEED, SMALL)
        ctx.set_bricking(sid, BRICK, 1, "f32")
        ctx.set_brick_layouts(sid, 9)
        rid = ctx.load_cube(vox)
        ctx.set_brick_layouts(rid, 9)
        ctx.set_bricking(rid, BRICK, 1, "f32")
        ctx.set_channel_mask(mask)
        ctx.set_window((20, 31, 11), (260, 240, 250))
        ctx.set_termination(term)
        try:
            for cam in cams:
                for mode in ["dvr", "mip"]:
                    a = render(ctx, sid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
                    b = render(ctx, rid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
                    assert np.array_equal(a, b) and np.count_nonzero(a) > 0
        finally:
            ctx.set_termination("segment")
            ctx.set_window()
            ctx.set_channel_mask()
