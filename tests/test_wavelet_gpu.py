"""Wavelet-compressed cubes on the GPU against the oracle's block store: the store itself
(bit for bit), the bricks decoded from it into the brick cache (bit for bit) and the frames
rendered from them (the usual 1e-4 / bit-exact MIP bars, against the oracle rendering the
oracle-decoded cube)."""
import numpy as np
import pytest

import synth
from gpu_helpers import compare_dvr, render

pytestmark = pytest.mark.gpu


def _ctx(cache_bytes):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1008_0135_gb300 as P
    P.build()
    return P.Context(0, cache_bytes=cache_bytes)


@pytest.fixture(scope="module")
def ctx():
    c = _ctx(256 << 20)
    yield c
    c.close()


def _cube(seed, shape):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(shape) * 1.5).astype(np.float32)
    nz, ny, nx = shape
    for _ in range(6):                             # bright compact sources
        c = rng.uniform(0, 1, 3) * np.array([nz, ny, nx])
        z, y, w = np.ogrid[:nz, :ny, :nx]
        r2 = (z - c[0]) ** 2 + (y - c[1]) ** 2 + (w - c[2]) ** 2
        x += (rng.uniform(5, 18) * np.exp(-r2 / (2 * rng.uniform(1.5, 4) ** 2))).astype(np.float32)
    x[: min(8, nz), : min(8, ny), : min(8, nx)] = 0.0  # an all-zero block
    return x


def test_store_matches_the_oracle_bit_for_bit(ctx, orc):
    cube = _cube(1, (37, 29, 45))                  # ragged blocks on every axis
    cid = ctx.load_cube(cube)
    ctx.compress_cube(cid)
    st = ctx.wavelet_store(cid)
    ref = orc.wavelet_encode(cube)
    assert st.size == ref.size == 5 * 4 * 6 * 544
    assert np.array_equal(st, ref)
    ctx.free_cube(cid)


def test_decoded_bricks_match_the_oracle(ctx, orc):
    cube = _cube(2, (40, 36, 50))
    nz, ny, nx = cube.shape
    dec = orc.wavelet_decode(orc.wavelet_encode(cube), cube.shape)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (16, 16, 16), 1, "f32")
    ctx.compress_cube(cid)
    nb, storage = ctx.brick_grid(cid)
    total = nb[0] * nb[1] * nb[2]
    for b in sorted({0, 1, nb[0], total // 2, total - 1}):
        dims, org, e, data = ctx.get_brick(cid, b)
        zi = np.clip(org[2] + np.arange(dims[2]), 0, nz - 1)
        yi = np.clip(org[1] + np.arange(dims[1]), 0, ny - 1)
        xi = np.clip(org[0] + np.arange(dims[0]), 0, nx - 1)
        assert e == 0 and np.array_equal(data, dec[np.ix_(zi, yi, xi)]), b
    ctx.free_cube(cid)


@pytest.mark.parametrize("brick", [(16, 16, 16), (24, 20, 32)])
def test_frames_from_a_compressed_cube(ctx, orc, brick):
    cube = synth.pr1_cube(seed=3)
    dec = orc.wavelet_decode(orc.wavelet_encode(cube), cube.shape)
    lut = synth.ramp_lut(alpha=0.4)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, brick, 1, "f32")
    ctx.compress_cube(cid)
    rng = np.random.default_rng(17)
    for cam in [synth.pr1_camera(W=96, H=80), synth.random_camera(rng, (64, 64, 64), 72, 64)]:
        g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        ref, flags, _ = orc.render(dec, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=brick)
        compare_dvr(g, ref, flags, 0.99)
        m = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
        rm, _, _ = orc.render(dec, lut, (-3, 20), cam, mode="mip32", step=0.5, brick=brick)
        assert np.array_equal(m, rm.astype(np.float32))
        # the lossy store changes the image by little next to the FP32 cube's
        full, _, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=brick)
        assert np.abs(g.astype(np.float64) - full).max() < 0.05
    ctx.free_cube(cid)


def test_frames_larger_than_the_cache(orc):
    """A cache of 4 bricks: frames decode their 27 bricks chunk by chunk."""
    c = _ctx(4 * 18 ** 3 * 4 + 1024)
    try:
        cube = synth.pr1_cube(seed=4, n=48)
        dec = orc.wavelet_decode(orc.wavelet_encode(cube), cube.shape)
        lut = synth.ramp_lut(alpha=0.4)
        cid = c.load_cube(cube)
        c.set_bricking(cid, (16, 16, 16), 1, "f32")
        c.compress_cube(cid)
        cam = synth.pr1_camera(n=48, W=64, H=64)
        for _ in range(2):
            g = render(c, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
            ref, flags, _ = orc.render(dec, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(16, 16, 16))
            compare_dvr(g, ref, flags, 0.99)
        st = c.stats()
        assert st["cache_misses"] > 27
    finally:
        c.close()


def test_compressed_cube_refusals(ctx):
    import paper_1008_0135_gb300 as P
    cube = synth.pr1_cube(seed=5, n=32)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (16, 16, 16), 1, "f16")
    ctx.compress_cube(cid)                         # bricks become FP32
    assert ctx.brick_grid(cid)[1] == 0
    ctx.compress_cube(cid)                         # no-op
    with pytest.raises(P.VrError) as e:
        ctx.set_bricking(cid, (16, 16, 16), 1, "bf16")
    assert e.value.status == -7
    with pytest.raises(P.VrError) as e:
        ctx.compute_minmax(cid)
    assert e.value.status == -7
    vid = ctx.load_cube_procedural(3, (64, 64, 64))
    with pytest.raises(P.VrError) as e:
        ctx.compress_cube(vid)
    assert e.value.status == -7
    other = ctx.load_cube(cube)
    with pytest.raises(P.VrError) as e:
        ctx.wavelet_store(other)
    assert e.value.status == -5
    for i in (cid, vid, other):
        ctx.free_cube(i)


def test_compressed_frames_with_slot_atlases(orc):
    """Mask 9 on a compressed cube: decoded bricks are also packed into the cache slots' slice
    atlases; frames (fitting the cache, and chunked through 4 slots) equal the linear slots'."""
    cube = synth.pr1_cube(seed=4, n=48)
    lut = synth.ramp_lut(alpha=0.4)
    cam = synth.pr1_camera(n=48, W=64, H=64)
    for cache in (64 * 18 ** 3 * 4, 4 * 18 ** 3 * 4 + 1024):
        c = _ctx(cache)
        try:
            cid = c.load_cube(cube)
            c.set_bricking(cid, (16, 16, 16), 1, "f32")
            c.compress_cube(cid)
            for mode in ["dvr", "mip"]:
                c.set_brick_layouts(cid, 1)
                lin = render(c, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
                c.set_brick_layouts(cid, 9)
                at = render(c, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
                again = render(c, cid, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
                assert np.array_equal(lin, at) and np.array_equal(lin, again)
        finally:
            c.close()


def test_compressed_cube_global_termination(orc):
    """Occlusion skipping on a compressed cube equals the resident cube of the oracle-decoded
    voxels under the same termination, bit for bit (slot atlases and linear slots)."""
    cube = synth.pr1_cube(seed=4, n=48)
    dec = orc.wavelet_decode(orc.wavelet_encode(cube), cube.shape).astype(np.float32)
    lut = synth.ramp_lut(alpha=1.0)
    cam = synth.pr1_camera(n=48, W=64, H=64)
    c = _ctx(64 * 18 ** 3 * 4)
    try:
        cid = c.load_cube(cube)
        c.set_bricking(cid, (16, 16, 16), 1, "f32")
        c.compress_cube(cid)
        rid = c.load_cube(dec)
        c.set_bricking(rid, (16, 16, 16), 1, "f32")
        c.set_termination("global")
        try:
            for mask in (1, 9):
                c.set_brick_layouts(cid, mask)
                c.set_brick_layouts(rid, mask)
                a = render(c, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
                b = render(c, rid, lut, (-3, 20), cam, step=0.5, tau=0.99)
                assert np.array_equal(a, b) and np.count_nonzero(a) > 0
        finally:
            c.set_termination("segment")
    finally:
        c.close()
