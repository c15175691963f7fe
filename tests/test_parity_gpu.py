"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import ATOL_F32, BOUND_16, compare_dvr, gpu_ctx, render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


@pytest.fixture(scope="module")
def pr1(ctx):
    cube = synth.pr1_cube(seed=0)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (32, 32, 32), 1, "f32")
    return cube, cid


# ---------------------------------------------------------------------------------------------
# PR1 (64^3, 256^2, 2x2x2 bricks of 32^3 + ghost 1)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [0.1, 0.9])
def test_pr1_dvr_matches_oracle(ctx, orc, pr1, alpha):
    cube, cid = pr1
    cam = synth.pr1_camera()
    lut = synth.ramp_lut(alpha=alpha)
    g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    ref, flags, ns = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32))
    compare_dvr(g, ref, flags, 0.99)
    assert not np.any(flags & 4)


def test_pr1_dvr_ert_off_matches_unbricked_oracle(ctx, orc, pr1):
    cube, cid = pr1
    cam = synth.pr1_camera()
    lut = synth.ramp_lut(alpha=0.5)
    g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=1.0)
    ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=1.0)
    compare_dvr(g, ref, flags, 1.0)


def test_pr1_sample_count_matches_oracle(ctx, orc, pr1):
    cube, cid = pr1
    cam = synth.pr1_camera()
    lut = synth.ramp_lut()
    ctx.reset_stats()
    render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
    st = ctx.stats()
    _, _, ns = orc.render(cube, lut, (-3, 20), cam, mode="mip", step=0.5)
    assert st["samples"] == ns          # integer work: every lattice sample exactly once


def test_pr1_mip_bit_exact(ctx, orc, pr1):
    cube, cid = pr1
    cam = synth.pr1_camera()
    g = render(ctx, cid, synth.ramp_lut(), (-3, 20), cam, mode="mip", step=0.5)
    ref32, _, _ = orc.render(cube, synth.ramp_lut(), (-3, 20), cam, mode="mip32", step=0.5,
                             brick=(32, 32, 32))
    assert np.array_equal(g.view(np.uint32), ref32.astype(np.float32).view(np.uint32))
    ref64, _, _ = orc.render(cube, synth.ramp_lut(), (-3, 20), cam, mode="mip", step=0.5)
    assert np.abs(g - ref64).max() < 1e-4 * max(1.0, np.abs(ref64).max())


def test_mip_axis_aligned_is_column_max(ctx):
    cube = synth.pr1_cube(seed=4, n=32)[:20].copy()
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (8, 16, 6), 1, "f32")
    cam = synth.axis_ortho_camera((32, 32, 20))
    g = render(ctx, cid, synth.ramp_lut(), (-3, 20), cam, mode="mip", step=0.5)
    expect = cube.max(axis=0)[::-1, ::-1].ravel()
    assert np.array_equal(g, expect)
    ctx.free_cube(cid)


def test_rays_and_samples_on_brick_faces(ctx, orc):
    """Orthographic rays along z through integer x and y (every ray lies in voxel faces, and in
    brick faces every 8 voxels) with samples on integer z (brick faces every 8 slices): every
    lattice sample is owned by exactly one brick (the sample count equals the oracle's), DVR per
    segment and with global termination matches the oracle, MIP bit for bit."""
    cube = synth.pr1_cube(seed=6, n=32)[:20].copy()          # nz=20, ny=32, nx=32
    nx, ny, nz = 32, 32, 20
    c = np.array([nx / 2.0 - 0.5, ny / 2.0 - 0.5, nz / 2.0])
    cam = dict(view=synth.look_at(c - np.array([0.0, 0.0, nz + 8.0]), c), proj=0, param=64.0,
               W=64, H=64)                                       # pixel centres on integer x, y
    o, _, _ = orc.rays(cam, (nx, ny, nz), step=0.5)
    assert np.array_equal(o[:, :2], np.round(o[:, :2]))          # exactly, in FP32
    assert (np.isin(o[:, 0], (8.0, 16.0, 24.0)) | np.isin(o[:, 1], (8.0, 16.0, 24.0))).sum() > 300
    lut = synth.random_lut(23, n=40, alpha_max=0.4)
    cid = ctx.load_cube(cube)
    try:
        for layouts in (1, 9):
            ctx.set_brick_layouts(cid, layouts)
            ctx.set_bricking(cid, (8, 8, 8), 1, "f32")
            ctx.reset_stats()
            m = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
            m32, _, ns = orc.render(cube, lut, (-3, 20), cam, mode="mip32", step=0.5, brick=(8, 8, 8))
            assert ctx.stats()["samples"] == ns
            assert np.array_equal(m, m32.astype(np.float32))
            for scope, tau in (("segment", 1.0), ("segment", 0.9), ("global", 0.9)):
                ctx.set_termination(scope)
                g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=tau)
                ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=tau, brick=(8, 8, 8),
                                           term=scope)
                compare_dvr(g, ref, flags, tau)
            ctx.set_termination("segment")
    finally:
        ctx.set_termination("segment")
        ctx.free_cube(cid)


def test_bricked_equals_unbricked(ctx, pr1):
    cube, _ = pr1
    lut = synth.ramp_lut(alpha=0.4)
    cam = synth.pr1_camera()
    one = ctx.load_cube(cube)
    ctx.set_bricking(one, (64, 64, 64), 1, "f32")
    many = ctx.load_cube(cube)
    ctx.set_bricking(many, (16, 8, 32), 1, "f32")
    a = render(ctx, one, lut, (-3, 20), cam, step=0.5, tau=1.0)
    b = render(ctx, many, lut, (-3, 20), cam, step=0.5, tau=1.0)
    assert np.abs(a - b).max() <= 1e-5
    ma = render(ctx, one, lut, (-3, 20), cam, mode="mip", step=0.5)
    mb = render(ctx, many, lut, (-3, 20), cam, mode="mip", step=0.5)
    assert np.array_equal(ma, mb)
    ctx.free_cube(one)
    ctx.free_cube(many)


@pytest.mark.parametrize("mode", ["dvr", "mip"])
def test_rendering_rectangle_does_not_change_image(ctx, pr1, mode):
    _, cid = pr1
    rng = np.random.default_rng(5)
    for _ in range(3):
        cam = synth.random_camera(rng, (64, 64, 64), 200, 120)
        a = render(ctx, cid, synth.ramp_lut(alpha=0.3), (-3, 20), cam, mode=mode, step=0.5)
        b = render(ctx, cid, synth.ramp_lut(alpha=0.3), (-3, 20), cam, mode=mode, step=0.5,
                   full_rect=True)
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------------------------
# random geometry, tiny cubes, ragged bricks
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_random_tiny_cubes(ctx, orc, seed):
    rng = np.random.default_rng(200 + seed)
    shape = tuple(int(x) for x in rng.integers(2, 10, 3))
    nx, ny, nz = shape
    cube = rng.uniform(-1, 3, (nz, ny, nx)).astype(np.float32)
    lut = synth.random_lut(seed, n=int(rng.integers(2, 64)), alpha_max=0.7)
    W, H = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    cam = synth.random_camera(rng, shape, W, H)
    step = float(rng.choice([0.5, 0.25, 0.3, 1.0, 0.7]))
    tau = float(rng.choice([1.0, 0.9, 0.6, 0.99]))
    brick = tuple(int(x) for x in rng.integers(1, 5, 3))
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, brick, 1, "f32")
    g = render(ctx, cid, lut, (-1, 3), cam, step=step, tau=tau)
    ref, flags, _ = orc.render(cube, lut, (-1, 3), cam, step=step, tau=tau, brick=brick)
    compare_dvr(g, ref, flags, tau)
    m = render(ctx, cid, lut, (-1, 3), cam, mode="mip", step=step)
    m32, _, _ = orc.render(cube, lut, (-1, 3), cam, mode="mip32", step=step, brick=brick)
    assert np.array_equal(m, m32.astype(np.float32))
    ctx.free_cube(cid)


@pytest.mark.parametrize("step", [3.0, 7.5, 13.0])
def test_steps_longer_than_bricks(ctx, orc, step):
    """Lattice steps longer than a brick: most rays take no sample in most bricks they cross
    (empty slab ranges), a brick's segment is one sample or none, and the global walk crosses
    bricks without sampling them.  DVR per segment and with global termination against the oracle
    (FP32 bricks, and FP16 bricks against the oracle on the same codes; linear copies and slice
    atlases), MIP bit for bit."""
    rng = np.random.default_rng(int(step * 10))
    nz, ny, nx = 44, 36, 40
    cube = rng.uniform(-1.0, 3.0, (nz, ny, nx)).astype(np.float32)
    cube += synth.pr1_cube(seed=9, n=44, n_sources=5, sigma=(2.0, 5.0))[:nz, :ny, :nx]
    lut = synth.random_lut(17, n=48, alpha_max=0.6)
    brick = (6, 5, 7)
    cams = [synth.random_camera(rng, (nx, ny, nz), 48, 40),
            dict(view=synth.look_at((20.0, 18.0, -70.0), (20.0, 18.0, 22.0)), proj=0, param=60.0, W=40, H=44)]
    cid = ctx.load_cube(cube)
    try:
        for layouts, storage in ((1, "f32"), (9, "f32"), (9, "f16")):
            ctx.set_brick_layouts(cid, layouts)
            ctx.set_bricking(cid, brick, 1, storage)
            for cam in cams:
                for scope, tau in (("segment", 1.0), ("segment", 0.8), ("global", 0.8)):
                    ctx.set_termination(scope)
                    g = render(ctx, cid, lut, (-1, 8), cam, step=step, tau=tau)
                    # 16-bit bricks: against the oracle reading the same rounded bricks
                    ref, flags, _ = orc.render(cube, lut, (-1, 8), cam, step=step, tau=tau, brick=brick,
                                               term=scope, quant=storage)
                    compare_dvr(g, ref, flags, tau)
                ctx.set_termination("segment")
                if storage == "f32":
                    m = render(ctx, cid, lut, (-1, 8), cam, mode="mip", step=step)
                    m32, _, _ = orc.render(cube, lut, (-1, 8), cam, mode="mip32", step=step, brick=brick)
                    assert np.array_equal(m, m32.astype(np.float32))
    finally:
        ctx.set_termination("segment")
        ctx.free_cube(cid)


def test_eye_inside_volume(ctx, orc, pr1):
    cube, cid = pr1
    lut = synth.ramp_lut(alpha=0.3)
    for k, (eye, tgt) in enumerate([((30.0, 33.0, 31.0), (60.0, 10.0, 40.0)),
                                    ((32.0, 32.0, 32.0), (0.0, 64.0, 0.0)),
                                    ((1.0, 63.5, 17.0), (64.0, 0.0, 64.0))]):
        cam = dict(view=synth.look_at(eye, tgt), proj=1, param=math.radians(80.0), W=96, H=64)
        g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32))
        compare_dvr(g, ref, flags, 0.99)


def test_ragged_bricks(ctx, orc):
    cube = synth.pr1_cube(seed=6, n=64)[:61, :50, :].copy()        # 64 x 50 x 61
    lut = synth.ramp_lut(alpha=0.5)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (24, 20, 28), 1, "f32")
    nb, _ = ctx.brick_grid(cid)
    assert nb == (3, 3, 3)
    rng = np.random.default_rng(8)
    for _ in range(3):
        cam = synth.random_camera(rng, (64, 50, 61), 70, 90)
        g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.95)
        ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.95, brick=(24, 20, 28))
        compare_dvr(g, ref, flags, 0.95)
    ctx.free_cube(cid)


def test_empty_and_degenerate_frames(ctx, pr1):
    _, cid = pr1
    lut = synth.ramp_lut()
    away = dict(view=synth.look_at((-10.0, -10.0, -10.0), (-20.0, -30.0, -40.0)), proj=1,
                param=0.5, W=33, H=17)
    g = render(ctx, cid, lut, (-3, 20), away, step=0.5)
    assert np.all(g == 0)
    m = render(ctx, cid, lut, (-3, 20), away, mode="mip", step=0.5)
    assert np.all(m == np.float32(-3))
    one = dict(view=synth.look_at((32.0, 32.0, -50.0), (32.0, 32.0, 32.0)), proj=0, param=1.0,
               W=1, H=1)
    g1 = render(ctx, cid, lut, (-3, 20), one, step=0.5)
    assert g1.shape == (1, 4) and g1[0, 3] > 0
    big_step = render(ctx, cid, lut, (-3, 20), synth.pr1_camera(W=40, H=30), step=500.0)
    assert big_step.shape == (1200, 4)


# ---------------------------------------------------------------------------------------------
# cube operations
# ---------------------------------------------------------------------------------------------
def test_minmax_exact_and_subcube(ctx, orc):
    cube = synth.pr1_cube(seed=7, n=40)
    cid = ctx.load_cube(cube)
    assert ctx.compute_minmax(cid) == orc.minmax(cube)
    sid = ctx.load_cube(cube, sub_origin=(3, 5, 7), sub_extent=(20, 11, 30))
    sub = cube[7:37, 5:16, 3:23]
    assert ctx.compute_minmax(sid) == orc.minmax(sub)
    ctx.set_bricking(sid, (8, 8, 8), 1, "f32")
    dims, org, e, data = ctx.get_brick(sid, 0)
    assert dims == (10, 10, 10) and org == (-1, -1, -1) and e == 0
    idx = np.clip(np.arange(-1, 9), 0, None)
    assert np.array_equal(data, sub[np.ix_(idx, idx, idx)])
    ctx.free_cube(cid)
    ctx.free_cube(sid)


def test_update_cube_rebuilds_bricks(ctx, orc):
    import torch
    cube = synth.pr1_cube(seed=1, n=32)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (16, 16, 16), 1, "f32")
    cube2 = (cube * 0.5 + 1.0).astype(np.float32)
    ctx.update_cube(cid, torch.from_numpy(cube2).cuda())
    cam = synth.pr1_camera(n=32, W=64, H=64)
    lut = synth.ramp_lut(alpha=0.4)
    g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    ref, flags, _ = orc.render(cube2, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(16, 16, 16))
    compare_dvr(g, ref, flags, 0.99)
    ctx.free_cube(cid)


def test_error_statuses(ctx):
    import paper_1008_0135_gb300 as P
    with pytest.raises(P.VrError) as e:
        ctx.set_bricking(12345, (8, 8, 8))
    assert e.value.status == -6
    cube = synth.pr1_cube(seed=2, n=16)
    cid = ctx.load_cube(cube)
    with pytest.raises(P.VrError) as e:
        ctx.set_camera_dict(synth.pr1_camera(n=16, W=8, H=8))
        ctx.render_frame(cid)
    assert e.value.status == -5            # no bricking yet
    with pytest.raises(P.VrError) as e:
        ctx.set_bricking(cid, (0, 8, 8))
    assert e.value.status == -1
    with pytest.raises(P.VrError):
        ctx.set_transfer_function(synth.ramp_lut(), 5.0, 5.0)
    with pytest.raises(P.VrError):
        ctx.load_cube(cube, sub_origin=(0, 0, 0), sub_extent=(17, 1, 1))
    with pytest.raises(P.VrError) as e:
        ctx.set_brick_layouts(cid, 16)
    assert e.value.status == -1
    ctx.free_cube(cid)


def test_slice_atlas_refuses_bricks_beyond_the_gather_limit(ctx):
    """A 4002 x 4 x 4002 stored brick would need a 64 x 4002 = 256128 texel wide atlas, beyond
    the device's 2D-gather limit: the bricking is refused (VR_ERR_UNSUPPORTED), and the same
    bricking without atlases is fine."""
    import torch
    import paper_1008_0135_gb300 as P
    cid = ctx.load_cube(torch.zeros((4000, 2, 4000), device="cuda"))
    ctx.set_brick_layouts(cid, 9)
    with pytest.raises(P.VrError) as e:
        ctx.set_bricking(cid, (4000, 2, 4000))
    assert e.value.status == -7 and "slice atlas" in str(e.value)
    ctx.set_brick_layouts(cid, 1)
    ctx.set_bricking(cid, (4000, 2, 4000))
    ctx.free_cube(cid)


# ---------------------------------------------------------------------------------------------
# 16-bit bricks
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_bricks(ctx, orc, storage):
    cube = synth.pr1_cube(seed=0)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (32, 32, 32), 1, storage)
    exps = orc.brick_exponents(cube, (32, 32, 32), 1, storage)
    # stored codes, bit for bit (integer work), ghost included
    for b in (0, 5, 7):
        dims, org, e, data = ctx.get_brick(cid, b)
        cz, cy, cx = b // 4, (b // 2) % 2, b % 2
        assert e == exps[cz, cy, cx]
        iz = np.clip(np.arange(org[2], org[2] + dims[2]), 0, 63)
        iy = np.clip(np.arange(org[1], org[1] + dims[1]), 0, 63)
        ix = np.clip(np.arange(org[0], org[0] + dims[0]), 0, 63)
        region = cube[np.ix_(iz, iy, ix)]
        scaled = np.ldexp(region, -e).astype(np.float32)
        want = (orc.round_fp16(scaled) if storage == "f16" else orc.round_bf16(scaled))
        if storage == "f16":
            bits = want.astype(np.float16).view(np.uint16)
        else:
            bits = (want.view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal(data.ravel(), bits)
    cam = synth.pr1_camera()
    lut = synth.ramp_lut(alpha=0.5)
    g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    # against the oracle reading the same rounded bricks: the kernel's own error
    refq, flq, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32),
                              quant=storage)
    compare_dvr(g, refq, flq, 0.99)
    # against the FP32 cube: the stated bound for 16-bit storage
    ref, fl, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32))
    compare_dvr(g, ref, fl, 0.99, atol=BOUND_16)
    m = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
    m32, _, _ = orc.render(cube, lut, (-3, 20), cam, mode="mip32", step=0.5, brick=(32, 32, 32),
                           quant=storage)
    assert np.array_equal(m, m32.astype(np.float32))
    ctx.free_cube(cid)


# ---------------------------------------------------------------------------------------------
# brick layouts: the gathered addresses change, the arithmetic does not.  Mask 7 keeps x-, y- and
# z-contiguous copies; 9 and 15 add slice atlases (texture gathers) that every frame then reads;
# 41 and 47 make a 16-bit cube's atlases pair atlases (one gather per sample; FP32 keeps slices).
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,layouts", [("f32", 7), ("f16", 7), ("f32", 9), ("f16", 15),
                                             ("bf16", 9), ("f16", 41), ("bf16", 41), ("f16", 47),
                                             ("f32", 41)])
def test_brick_layouts_give_identical_images(ctx, orc, storage, layouts):
    cube = synth.pr1_cube(seed=2)
    lut = synth.ramp_lut(alpha=0.5)
    one = ctx.load_cube(cube)
    ctx.set_bricking(one, (24, 32, 20), 1, storage)
    many = ctx.load_cube(cube)
    ctx.set_brick_layouts(many, layouts)
    ctx.set_bricking(many, (24, 32, 20), 1, storage)
    rng = np.random.default_rng(21)
    cams = [synth.pr1_camera(W=100, H=90), synth.random_camera(rng, (64, 64, 64), 90, 110),
            dict(view=synth.look_at((32.0, 150.0, 30.0), (32.0, 32.0, 32.0), up=(1.0, 0.0, 0.0)),
                 proj=1, param=0.9, W=64, H=80),       # up along x: warps along image y = world x
            dict(view=synth.look_at((150.0, 30.0, 32.0), (32.0, 32.0, 32.0), up=(0.0, 0.0, 1.0)),
                 proj=0, param=100.0, W=72, H=64)]     # up along z
    for cam in cams:
        for mode in ("dvr", "mip"):
            a = render(ctx, one, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            b = render(ctx, many, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.99)
            assert np.array_equal(a, b)
        if storage == "f32":
            ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99,
                                       brick=(24, 32, 20))
            compare_dvr(render(ctx, many, lut, (-3, 20), cam, step=0.5, tau=0.99), ref, flags, 0.99)
    dims, org, e, data = ctx.get_brick(many, 3)
    dims1, org1, e1, data1 = ctx.get_brick(one, 3)
    assert np.array_equal(data, data1)                  # get_brick returns the x-contiguous copy
    ctx.free_cube(one)
    ctx.free_cube(many)


def test_fp16_atlas_keeps_subnormal_codes(ctx):
    """A brick whose maximum (1000) sets the FP16 scale 2^-4 turns values of 1e-7..2e-6 into
    subnormal codes; the slice atlas (half texels widened by the texture unit) must give the
    same frames as the linear copy, bit for bit, so no code may be flushed to zero."""
    rng = np.random.default_rng(99)
    cube = (rng.uniform(1e-7, 2e-6, (32, 32, 32)) * rng.choice([-1.0, 1.0], (32, 32, 32))).astype(np.float32)
    cube[16, 16, 16] = 1000.0
    lut = synth.ramp_lut(alpha=0.5)
    one = ctx.load_cube(cube)
    ctx.set_bricking(one, (32, 32, 32), 1, "f16")
    atl = ctx.load_cube(cube)
    ctx.set_brick_layouts(atl, 9)
    ctx.set_bricking(atl, (32, 32, 32), 1, "f16")
    assert ctx.get_brick(one, 0)[2] == -4
    codes = ctx.get_brick(one, 0)[3]
    assert np.count_nonzero((codes & 0x7C00) == 0) > 1000         # subnormal (or zero) codes
    rng2 = np.random.default_rng(3)
    for cam in [synth.pr1_camera(n=32, W=64, H=64), synth.random_camera(rng2, (32, 32, 32), 48, 40)]:
        a = render(ctx, one, lut, (-1e-5, 1e-5), cam, step=0.5, tau=1.0)
        b = render(ctx, atl, lut, (-1e-5, 1e-5), cam, step=0.5, tau=1.0)
        assert np.abs(a).max() > 0 and np.array_equal(a, b)
    ctx.free_cube(one)
    ctx.free_cube(atl)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_pair_atlas_frames_equal_slice_atlas_frames(ctx, storage):
    """Pair atlases (layout bit 5) hold the codes of slices z and z + 1 in one 32-bit texel: DVR
    with per-segment and global termination, MIP, a channel mask and a render window give the
    slice atlases' frames bit for bit, on ragged bricks (the last z layer 5 slices deep) and with
    FP16 subnormal codes; bit 5 without bit 3 is refused."""
    import paper_1008_0135_gb300 as P
    rng = np.random.default_rng(61)
    cube = synth.pr1_cube(seed=7, n=64)[:45].copy()
    cube[:, :20, :20] *= 1e-7                       # tiny values: subnormal FP16 codes there
    cube[3, 3, 3] = 50.0
    lut = synth.ramp_lut(alpha=0.5)
    sl = ctx.load_cube(cube)
    ctx.set_brick_layouts(sl, 9)
    ctx.set_bricking(sl, (20, 24, 20), 1, storage)
    pr = ctx.load_cube(cube)
    with pytest.raises(P.VrError) as e:
        ctx.set_brick_layouts(pr, 33)
    assert e.value.status == -1
    ctx.set_brick_layouts(pr, 41)
    ctx.set_bricking(pr, (20, 24, 20), 1, storage)
    mask = (rng.uniform(size=45) > 0.3).astype(np.uint8)
    cams = [synth.pr1_camera(W=80, H=72), synth.random_camera(rng, (64, 64, 45), 70, 66),
            dict(view=synth.look_at((32.0, 150.0, 22.0), (32.0, 32.0, 22.0), up=(1.0, 0.0, 0.0)),
                 proj=1, param=0.9, W=64, H=70)]
    try:
        for scope in ("segment", "global"):
            ctx.set_termination(scope)
            for cam in cams:
                for extra in (False, True):
                    ctx.set_channel_mask(mask if extra else None)
                    if extra:
                        ctx.set_window((3, 5, 2), (60, 57, 40))
                    else:
                        ctx.set_window()
                    for mode in ("dvr", "mip"):
                        a = render(ctx, sl, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.95)
                        b = render(ctx, pr, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.95)
                        assert np.abs(a).max() > 0 and np.array_equal(a, b), (scope, mode, extra)
    finally:
        ctx.set_termination("segment")
        ctx.set_channel_mask(None)
        ctx.set_window()
        ctx.free_cube(sl)
        ctx.free_cube(pr)


# ---------------------------------------------------------------------------------------------
# empty-space skipping (a noise-suppressing table: zero opacity below a threshold)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_empty_space_skipping_is_exact(ctx, orc, storage):
    cube = synth.pr1_cube(seed=0)
    lut = synth.ramp_lut(alpha=0.6)
    x = np.linspace(-3, 20, 256)
    lut[x < 4.0, 3] = 0.0                     # bricks of pure N(0,1) noise become invisible
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (16, 16, 16), 1, storage)
    cam = synth.pr1_camera()
    ctx.reset_stats()
    a = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    skipped = ctx.stats()["bricks_drawn"]
    ctx.reset_stats()
    b = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99, full_rect=True)
    full = ctx.stats()["bricks_drawn"]
    assert full == 64 and skipped < full          # some bricks were dropped ...
    assert np.array_equal(a, b)                   # ... without changing a single bit
    if storage == "f32":
        ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(16, 16, 16))
        compare_dvr(a, ref, flags, 0.99)
    m1 = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
    m2 = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5, full_rect=True)
    assert np.array_equal(m1, m2)                 # MIP never skips
    ctx.free_cube(cid)


# ---------------------------------------------------------------------------------------------
# spectral-channel masks and render windows (Section 2.3)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,layouts", [("f32", 7), ("f16", 7), ("f32", 9), ("bf16", 9)])
def test_channel_mask_and_window(ctx, orc, storage, layouts):
    rng = np.random.default_rng(77)
    cube = synth.pr1_cube(seed=8)
    mask = (rng.uniform(size=64) > 0.3).astype(np.uint8)
    win = ((5, 9, 3), (57, 50, 61))
    lut = synth.ramp_lut(alpha=0.4)
    lut[:20, 3] = 0.05                        # vmin itself visible: masked slices show
    cid = ctx.load_cube(cube)
    ctx.set_brick_layouts(cid, layouts)
    ctx.set_bricking(cid, (16, 32, 24), 1, storage)
    q = "f32" if storage == "f32" else storage
    try:
        for k, (m, w) in enumerate([(mask, None), (None, win), (mask, win)]):
            ctx.set_channel_mask(m)
            if w is None:
                ctx.set_window()
            else:
                ctx.set_window(*w)
            cam = synth.random_camera(rng, (64, 64, 64), 90, 70)
            g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
            ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99,
                                       brick=(16, 32, 24), quant=q, channels=m, window=w)
            compare_dvr(g, ref, flags, 0.99)
            gm = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)
            rm, _, _ = orc.render(cube, lut, (-3, 20), cam, mode="mip32", step=0.5,
                                  brick=(16, 32, 24), quant=q, channels=m, window=w)
            assert np.array_equal(gm, rm.astype(np.float32))
    finally:
        ctx.set_channel_mask(None)
        ctx.set_window()
        ctx.free_cube(cid)


def test_channel_mask_gradient(ctx, orc):
    import torch
    rng = np.random.default_rng(78)
    n = 20
    cube = synth.pr1_cube(seed=9, n=n, amp=(1.0, 4.0))
    mask = (rng.uniform(size=n) > 0.4).astype(np.uint8)
    lut = synth.random_lut(5, n=32, alpha_max=0.4)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (8, 8, 8), 1, "f32")
    cam = synth.random_camera(rng, (n, n, n), 40, 32, proj=1)
    ctx.set_channel_mask(mask)
    try:
        render(ctx, cid, lut, (-3, 8), cam, step=0.5, tau=1.0)
        gout = rng.standard_normal((40 * 32, 4)).astype(np.float32)
        glut = torch.zeros((32, 4), device="cuda")
        gvox = torch.zeros(cube.shape, device="cuda")
        ctx.render_backward(cid, torch.from_numpy(gout.reshape(32, 40, 4)).cuda(), glut, gvox)
        rl, rv = orc.render_grad(cube, lut, (-3, 8), cam, gout.astype(np.float64), step=0.5,
                                 tau=1.0, brick=(8, 8, 8), channels=mask)
        gv = gvox.cpu().numpy()
        assert np.all(gv[mask == 0] == 0)
        assert np.abs(glut.cpu().numpy() - rl).max() <= 2e-4 * np.abs(rl).max()
        assert np.abs(gv - rv).max() <= 2e-4 * np.abs(rv).max()
    finally:
        ctx.set_channel_mask(None)
        ctx.free_cube(cid)


# ---------------------------------------------------------------------------------------------
# global termination (occlusion skipping): front-to-back waves into per-pixel accumulators
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,layouts,brick", [("f32", 1, (16, 16, 16)), ("f32", 9, (24, 32, 20)),
                                                   ("f16", 7, (16, 16, 16)), ("bf16", 9, (32, 16, 24))])
def test_global_termination_matches_the_whole_ray(ctx, orc, storage, layouts, brick):
    """The image is the oracle's with the whole ray's termination (bricking only sets the 16-bit
    scales); it is within 1 - tau of per-segment termination and takes no more samples; with
    an opaque table it takes far fewer."""
    cube = synth.pr1_cube(seed=4)
    lut = synth.ramp_lut(alpha=0.6)
    cid = ctx.load_cube(cube)
    ctx.set_brick_layouts(cid, layouts)
    ctx.set_bricking(cid, brick, 1, storage)
    rng = np.random.default_rng(31)
    cams = [synth.pr1_camera(W=96, H=80), synth.random_camera(rng, (64, 64, 64), 90, 70),
            dict(view=synth.look_at((30.0, 35.0, 28.0), (64.0, 10.0, 60.0)), proj=1, param=1.2,
                 W=80, H=64)]                                   # eye inside the cube
    fewer = 0
    try:
        for cam in cams:
            for tau in (0.95, 1.0):
                ctx.set_termination("global")
                ctx.reset_stats()
                g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=tau)
                st_g = ctx.stats()
                ctx.set_termination("segment")
                ctx.reset_stats()
                s = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=tau)
                st_s = ctx.stats()
                ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=tau, brick=brick,
                                           quant=storage, term="global")
                compare_dvr(g, ref, flags, tau)
                assert st_g["fragments"] == 0 and st_g["samples"] <= st_s["samples"]
                assert np.abs(g.astype(np.float64) - s).max() <= (1.0 - min(tau, 1.0)) + 2e-4
                if tau >= 1.0:
                    assert st_g["samples"] == st_s["samples"]
                else:
                    fewer += st_g["samples"] < 0.8 * st_s["samples"]
        assert fewer >= 2
    finally:
        ctx.set_termination("segment")
        ctx.free_cube(cid)


def test_global_termination_with_mask_window_and_mip(ctx, orc):
    rng = np.random.default_rng(41)
    cube = synth.pr1_cube(seed=5)
    mask = (rng.uniform(size=64) > 0.25).astype(np.uint8)
    win = ((4, 6, 2), (60, 52, 58))
    lut = synth.ramp_lut(alpha=0.5)
    cid = ctx.load_cube(cube)
    ctx.set_brick_layouts(cid, 9)
    ctx.set_bricking(cid, (16, 16, 16), 1, "f32")
    cam = synth.random_camera(rng, (64, 64, 64), 72, 64)
    try:
        ctx.set_termination("global")
        ctx.set_channel_mask(mask)
        ctx.set_window(*win)
        g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.9)
        ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.9, brick=(16, 16, 16),
                                   channels=mask, window=win, term="global")
        compare_dvr(g, ref, flags, 0.9)
        m = render(ctx, cid, lut, (-3, 20), cam, mode="mip", step=0.5)    # MIP ignores the scope
        rm, _, _ = orc.render(cube, lut, (-3, 20), cam, mode="mip32", step=0.5, brick=(16, 16, 16),
                              channels=mask, window=win)
        assert np.array_equal(m, rm.astype(np.float32))
    finally:
        ctx.set_termination("segment")
        ctx.set_channel_mask(None)
        ctx.set_window()
        ctx.free_cube(cid)


def test_global_termination_refusals(ctx):
    """The adjoint and the no-allocation path need per-segment termination; a streamed cube
    needs a brick cache (this context has none: VR_ERR_OOM, as for its per-segment frames)."""
    import torch
    import paper_1008_0135_gb300 as P
    from paper_1008_0135_gb300 import _abi
    cube = synth.pr1_cube(seed=6, n=32)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (16, 16, 16), 1, "f32")
    cam = synth.pr1_camera(n=32, W=48, H=40)
    lut = synth.ramp_lut(alpha=0.4)
    vid = ctx.load_cube_procedural(7, (64, 64, 64))
    ctx.set_bricking(vid, (32, 32, 32), 1, "f32")
    try:
        ctx.set_termination("global")
        img = torch.from_numpy(render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)).cuda()
        with pytest.raises(P.VrError) as e:
            ctx.render_backward(cid, img.reshape(40, 48, 4).contiguous(),
                                torch.zeros((256, 4), device="cuda"), None)
        assert e.value.status == -7
        out = torch.zeros((40, 48, 4), device="cuda")
        rc = _abi.lib().vr_render_frame_noalloc(ctx._h, cid, out.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
        assert rc == -7
        with pytest.raises(P.VrError) as e:
            ctx.render_frame(vid)
        assert e.value.status == -2
        assert _abi.lib().vr_set_termination(ctx._h, 5) == -1
    finally:
        ctx.set_termination("segment")
        ctx.free_cube(cid)
        ctx.free_cube(vid)


# ---------------------------------------------------------------------------------------------
# asynchronous host output (a viewer queues frame k while it reads frame k - 1)
# ---------------------------------------------------------------------------------------------
def test_async_host_output_pipelined_frames(ctx, pr1):
    import torch
    _, cid = pr1
    lut = synth.ramp_lut()
    ctx.set_transfer_function(lut, -3.0, 20.0)
    ctx.set_render_params("dvr", 0.5, 0.99)
    cams = [synth.pr1_camera(W=64 + 8 * k, H=48 + 4 * k) for k in range(4)]
    want = []
    for cam in cams:                                   # synchronous copies: the reference
        ctx.set_camera_dict(cam)
        h = np.empty((cam["H"], cam["W"], 4), np.float32)
        ctx.render_frame(cid, h)
        want.append(h)
    bufs = [torch.full((c["H"], c["W"], 4), -1.0, dtype=torch.float32).pin_memory() for c in cams]
    ev = [torch.cuda.Event() for _ in cams]
    ctx.set_host_output_async(True)
    try:
        for k, cam in enumerate(cams):
            ctx.set_camera_dict(cam)
            ctx.render_frame(cid, bufs[k])                 # queued on the default stream
            ev[k].record()
            if k > 0:                                      # frame k - 1 is read while k renders
                ev[k - 1].synchronize()
                assert np.array_equal(bufs[k - 1].numpy(), want[k - 1])
        ev[-1].synchronize()
        assert np.array_equal(bufs[-1].numpy(), want[-1])
    finally:
        ctx.set_host_output_async(False)
    assert _abi_status(ctx, 2) == -1


def _abi_status(ctx, flag):
    from paper_1008_0135_gb300 import _abi
    return _abi.lib().vr_set_host_output_async(ctx._h, flag)


def test_device_cube_source_is_read_after_queued_writes(ctx):
    """vr_load_cube from device memory sees every write already queued on the caller's stream
    (the library copies on its own stream): a chain of in-place adds still running at the call
    is complete in the loaded cube."""
    import torch
    x = torch.zeros((256, 512, 512), device="cuda")        # 256 MB: the adds take a while
    for _ in range(24):
        x.add_(1.0)
    cid = ctx.load_cube(x)
    vmin, vmax = ctx.compute_minmax(cid)
    assert vmin == 24.0 and vmax == 24.0
    ctx.free_cube(cid)


@pytest.mark.parametrize("layouts", [1, 9])
def test_maximum_table_and_frame_sizes(ctx, orc, pr1, layouts):
    """The largest table the library takes (4096 entries, two shared-memory arrays of 64 KB per
    block) and the widest / tallest frames (16384 pixels) against the oracle; one past each
    limit is refused."""
    import paper_1008_0135_gb300 as P
    cube, cid = pr1
    ctx.set_brick_layouts(cid, layouts)
    try:
        # smooth across its 4096 entries: the 1e-4 bar covers FP32 rounding of the sampled value
        # times the table's slope, and a random table of 4096 entries has slopes of ~180 colour
        # units per data unit (measured 1.3e-4 there)
        t = np.arange(4096) / 4095.0
        lut = np.stack([0.5 + 0.5 * np.sin(6 * np.pi * t), t * t, 1.0 - t, 0.3 * t], 1).astype(np.float32)
        cam = synth.pr1_camera(W=96, H=64)
        g = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
        ref, flags, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32))
        compare_dvr(g, ref, flags, 0.99)
        for W, H in ((16384, 2), (2, 16384)):
            cam = synth.pr1_camera(W=W, H=H)
            g = render(ctx, cid, synth.ramp_lut(), (-3, 20), cam, step=0.5, tau=0.99)
            pix = np.arange(0, W * H, 97)
            ref, flags, _ = orc.render(cube, synth.ramp_lut(), (-3, 20), cam, step=0.5, tau=0.99,
                                       brick=(32, 32, 32), pix=pix)
            compare_dvr(g[pix], ref, flags, 0.99)
        with pytest.raises(P.VrError):
            ctx.set_transfer_function(synth.random_lut(31, n=4097), -3.0, 20.0)
        with pytest.raises(P.VrError):
            ctx.set_camera_dict(synth.pr1_camera(W=16385, H=2))
    finally:
        ctx.set_brick_layouts(cid, 1)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 17, 9), (13, 1, 1), (6, 1, 11)])
def test_degenerate_cube_extents(ctx, orc, shape):
    """Cubes one voxel thin along some axes (the stencil clamps to the edge there): DVR within
    the bar and MIP bit-exact against the oracle, bricked into 1- to 4-voxel bricks."""
    rng = np.random.default_rng(sum(shape))
    nx, ny, nz = shape
    cube = rng.uniform(-1, 3, (nz, ny, nx)).astype(np.float32)
    lut = synth.random_lut(5, n=48, alpha_max=0.6)
    for k in range(3):
        cam = synth.random_camera(rng, shape, 24, 20)
        brick = tuple(int(x) for x in rng.integers(1, 5, 3))
        cid = ctx.load_cube(cube)
        ctx.set_bricking(cid, brick, 1, "f32")
        g = render(ctx, cid, lut, (-1, 3), cam, step=0.3, tau=0.99)
        ref, flags, _ = orc.render(cube, lut, (-1, 3), cam, step=0.3, tau=0.99, brick=brick)
        compare_dvr(g, ref, flags, 0.99)
        m = render(ctx, cid, lut, (-1, 3), cam, mode="mip", step=0.3)
        m32, _, _ = orc.render(cube, lut, (-1, 3), cam, mode="mip32", step=0.3, brick=brick)
        assert np.array_equal(m, m32.astype(np.float32))
        ctx.free_cube(cid)


def test_contexts_created_later_render_the_largest_table(ctx, pr1):
    """Launch attributes (the 128 KB shared-memory limit a 4096-entry table needs, the carveout)
    belong to a device and are remembered per device: two more contexts on the same device,
    created after frames were rendered, render 4096-entry tables (fragment and one-pass kernels)
    bit for bit like the first context."""
    import paper_1008_0135_gb300 as P
    cube, cid = pr1
    t = np.arange(4096) / 4095.0
    lut = np.stack([t, 1.0 - t, t * t, 0.2 * t], 1).astype(np.float32)
    cam = synth.pr1_camera(W=80, H=72)
    refs = {}
    for term in ("segment", "global"):
        ctx.set_termination(term)
        refs[term] = render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    ctx.set_termination("segment")
    with P.Context(0) as a, P.Context(0) as b:
        for c in (a, b):
            k = c.load_cube(cube)
            c.set_bricking(k, (32, 32, 32), 1, "f32")
            for term in ("segment", "global"):
                c.set_termination(term)
                g = render(c, k, lut, (-3, 20), cam, step=0.5, tau=0.99)
                assert np.array_equal(g, refs[term]), term
            c.free_cube(k)


def _layouts_frame(ctx, cid, mask, lut, vr, cam, mode="dvr", step=0.5, tau=0.99):
    ctx.set_brick_layouts(cid, mask)
    return render(ctx, cid, lut, vr, cam, mode=mode, step=step, tau=tau)


@pytest.mark.parametrize("seed", range(4))
def test_staged_slabs_equal_the_linear_path_and_the_oracle(ctx, orc, seed):
    """Layout bit 4 keeps copies with 16-byte rows; DVR frames of FP32 bricks then read their
    stencils from slabs of the brick staged in shared memory by bulk copies.  They are the linear
    copies' frames bit for bit (the same voxels through the same arithmetic; stencils outside a
    slab come from global memory) and within the oracle's bar: random cameras, ragged bricks,
    tables of 2..4096 entries, a channel mask, a window, MIP frames (not staged) unchanged."""
    rng = np.random.default_rng(300 + seed)
    shape = tuple(int(v) for v in rng.integers(37, 71, 3))
    nx, ny, nz = shape
    cube = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    cube += synth.pr1_cube(seed=seed, n=max(shape), n_sources=6, sigma=(2.0, 5.0))[:nz, :ny, :nx]
    brick = tuple(int(v) for v in rng.integers(9, 33, 3))
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, brick, 1, "f32")
    nl = [2, 64, 256, 4096][seed]
    t = np.arange(nl) / max(nl - 1, 1)
    lut = np.stack([t, 1.0 - t, t * t, 0.25 * t], 1).astype(np.float32)
    try:
        for k in range(3):
            cam = synth.random_camera(rng, shape, int(rng.integers(40, 97)), int(rng.integers(30, 81)))
            lin = _layouts_frame(ctx, cid, 7, lut, (-3.0, 12.0), cam)
            stg = _layouts_frame(ctx, cid, 7 | 16, lut, (-3.0, 12.0), cam)
            assert np.array_equal(stg, lin), (k, np.abs(stg - lin).max())
            if k == 0:
                ref, flags, _ = orc.render(cube, lut, (-3.0, 12.0), cam, step=0.5, tau=0.99, brick=brick)
                compare_dvr(stg, ref, flags, 0.99)
            m_lin = _layouts_frame(ctx, cid, 7, lut, (-3.0, 12.0), cam, mode="mip")
            m_stg = _layouts_frame(ctx, cid, 7 | 16, lut, (-3.0, 12.0), cam, mode="mip")
            assert np.array_equal(m_lin, m_stg)
        # a spectral-channel mask and a render window
        mask = np.ones(nz, np.uint8)
        mask[nz // 3:nz // 3 + 4] = 0
        ctx.set_channel_mask(mask)
        ctx.set_window((2, 3, 1), (nx - 4, ny - 2, nz - 3))
        cam = synth.random_camera(rng, shape, 64, 48, proj=1)
        lin = _layouts_frame(ctx, cid, 7, lut, (-3.0, 12.0), cam)
        stg = _layouts_frame(ctx, cid, 7 | 16, lut, (-3.0, 12.0), cam)
        assert np.array_equal(stg, lin)
    finally:
        ctx.set_channel_mask(None)
        ctx.set_window()
        ctx.free_cube(cid)
    assert ctx.stats()["kernel_errors"] == 0


def test_staged_slabs_on_large_bricks_and_frames(ctx):
    """64^3 bricks of a 192x160x128 cube in 384^2 perspective frames from around the cube: many
    chunks per brick, slabs that overflow a stage near the eye (those chunks read global memory),
    rays of a tile crossing the march axis both ways; frames equal to the linear copies'."""
    rng = np.random.default_rng(77)
    shape = (192, 160, 128)
    nx, ny, nz = shape
    cube = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (64, 64, 64), 1, "f32")
    lut = synth.ramp_lut(alpha=0.02)
    try:
        c = np.array(shape, np.float64) / 2
        for j, dist in ((0, 400.0), (3, 260.0), (5, 150.0)):
            cam = dict(view=synth.orbit_view(360.0 * j / 8 + 10.0, c, dist), proj=1, param=math.radians(55.0),
                       W=384, H=384)
            lin = _layouts_frame(ctx, cid, 1 | 2, lut, (-3.0, 12.0), cam, step=0.7)
            stg = _layouts_frame(ctx, cid, 1 | 2 | 16, lut, (-3.0, 12.0), cam, step=0.7)
            assert np.array_equal(stg, lin), j
    finally:
        ctx.free_cube(cid)
    assert ctx.stats()["kernel_errors"] == 0
