"""Sort-last rendering on the GPU: longest-axis parts (Section 2.2), their sub-images and the
staged depth-ordered compositing (Section 2.5) equal the whole cube's frame, and the oracle."""
import math
import os
import socket
import sys

import numpy as np
import pytest

import synth
from gpu_helpers import compare_dvr, gpu_ctx

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (96, 64, 40)                      # x, y, z
BRICK = (16, 16, 16)                      # 6 x 4 x 3 bricks (the last z layer 8 deep)


@pytest.fixture(scope="module")
def setup():
    c = gpu_ctx()
    rng = np.random.default_rng(42)
    nx, ny, nz = SHAPE
    cube = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    cube += synth.pr1_cube(seed=5, n=96, n_sources=12, sigma=(3.0, 8.0))[:nz, :ny, :nx]
    cid = c.load_cube(cube)
    c.set_bricking(cid, BRICK, 1, "f32")
    yield c, cube, cid
    c.close()


def test_partition_boxes_follow_the_longest_axis(setup):
    ctx, cube, cid = setup
    for k, want in enumerate([(0, 2), (2, 4), (4, 6)]):   # x (96) is longest: 6 layers in 3
        ctx.set_partition(cid, (3,), (k,))
        lo, hi, ax = ctx.partition(cid, 1)
        assert ax == (0,) and (lo[0], hi[0]) == want and lo[1:] == (0, 0) and hi[1:] == (4, 3)
    # two nodes of two GPUs: x first (96), then each 48 x 64 x 40 half along y (64)
    ctx.set_partition(cid, (2, 2), (1, 0))
    lo, hi, ax = ctx.partition(cid, 2)
    assert ax == (0, 1) and lo == (3, 0, 0) and hi == (6, 2, 3)
    ctx.set_partition(cid, (8,), (7,))                 # more slabs than layers: some parts empty
    lo, hi, _ = ctx.partition(cid, 1)
    assert hi[0] - lo[0] in (0, 1)
    ctx.set_partition(cid)
    lo, hi, _ = ctx.partition(cid, 0)
    assert lo == (0, 0, 0) and hi == (6, 4, 3)


def _blend(ctx, cid, counts):
    """The library's blend for one process holding every part: the split axis of a level
    depends on the parent part, so the context takes the partition of one of the siblings."""
    from paper_1008_0135_gb300 import sortlast as SL

    def f(level, stack, row0, final, members):
        ctx.set_partition(cid, counts, SL.digits(members[0], counts))
        return ctx.composite_subimages(cid, level, stack, row0, final)
    return f


def _sortlast_local(ctx, cid, counts):
    from paper_1008_0135_gb300 import sortlast as SL
    world = int(np.prod(counts))
    subs = []
    for r in range(world):
        ctx.set_partition(cid, counts, SL.digits(r, counts))
        subs.append(ctx.render_subimage(cid).clone())
    frame = SL.composite_parts_local(subs, counts, _blend(ctx, cid, counts))
    ctx.set_partition(cid)
    return frame


CAMS = [
    dict(view=synth.look_at((150.0, 90.0, -60.0), (48.0, 32.0, 20.0)), proj=1, param=math.radians(50.0), W=72, H=56),
    dict(view=synth.look_at((48.0, 32.0, 20.0 - 140.0), (48.0, 32.0, 20.0)), proj=0, param=110.0, W=64, H=48),
    # eye inside the cube's x range: rays cross the x slabs in both directions
    dict(view=synth.look_at((40.0, 30.0, -90.0), (50.0, 34.0, 20.0)), proj=1, param=math.radians(80.0), W=80, H=60),
]


@pytest.mark.parametrize("counts,balanced", [((2,), False), ((3,), False), ((2, 2), False), ((4,), False),
                                             ((3, 2), False), ((3,), True), ((2, 2), True)])
def test_sortlast_frame_equals_the_whole_cube(setup, orc, counts, balanced):
    """Sub-images of every part composited in stages equal the whole cube's frame (DVR to FP32
    re-association, 1e-6; MIP bit for bit) and the oracle within the 1e-4 bar, for equal and
    camera-balanced cuts."""
    ctx, cube, cid = setup
    ctx.set_partition_balance(cid, balanced)
    lut = synth.random_lut(3, n=64, alpha_max=0.35)
    ctx.set_transfer_function(lut, -3.0, 12.0)
    for cam in CAMS:
        ctx.set_camera_dict(cam)
        for mode in ("dvr", "mip"):
            ctx.set_render_params(mode, 0.5, 0.99)
            whole = ctx.render_frame(cid).cpu().numpy()
            parts = _sortlast_local(ctx, cid, counts).cpu().numpy()
            if mode == "mip":
                assert np.array_equal(parts, whole)
                continue
            assert np.abs(parts - whole).max() <= 1e-6
            ref, flags, _ = orc.render(cube, lut, (-3.0, 12.0), cam, step=0.5, tau=0.99, brick=BRICK)
            compare_dvr(parts.reshape(-1, 4), ref, flags, 0.99)
    ctx.set_partition_balance(cid, False)


def test_balanced_cuts_even_out_the_parts_work(setup):
    """A perspective view from close to one end of the cube's longest axis: equal cuts give the
    near slab most of the samples; camera-balanced cuts spread them (the slowest part renders
    fewer samples), and the parts still tile the brick grid."""
    ctx, cube, cid = setup
    ctx.set_transfer_function(synth.ramp_lut(alpha=0.05), -3.0, 12.0)
    cam = dict(view=synth.look_at((-25.0, 32.0, 20.0), (96.0, 32.0, 20.0)), proj=1, param=math.radians(70.0),
               W=96, H=96)
    ctx.set_camera_dict(cam)
    ctx.set_render_params("dvr", 0.5, 1.0)
    worst = {}
    for balanced in (False, True):
        ctx.set_partition_balance(cid, balanced)
        per, spans = [], []
        for k in range(3):
            ctx.set_partition(cid, (3,), (k,))
            lo, hi, _ = ctx.partition(cid, 1)
            spans.append((lo[0], hi[0]))
            ctx.reset_stats()
            ctx.render_subimage(cid)
            per.append(ctx.stats()["samples"])
        assert spans[0][0] == 0 and spans[-1][1] == 6
        assert all(spans[i][1] == spans[i + 1][0] for i in range(2))
        worst[balanced] = max(per) / (sum(per) / 3.0)
    ctx.set_partition(cid)
    ctx.set_partition_balance(cid, False)
    assert worst[True] < worst[False]


def test_balanced_cuts_follow_the_render_state(setup):
    """The bricks' estimated costs behind balanced cuts are kept per render state: after camera,
    table and window changes, and between the parts' own calls, every part's box equals the one
    a fresh context computes for the same state."""
    ctx, cube, cid = setup
    near = dict(view=synth.look_at((-25.0, 32.0, 20.0), (96.0, 32.0, 20.0)), proj=1,
                param=math.radians(70.0), W=96, H=96)
    far = dict(view=synth.look_at((121.0, 32.0, 20.0), (0.0, 32.0, 20.0)), proj=1,
               param=math.radians(70.0), W=96, H=96)
    states = [(near, synth.ramp_lut(alpha=0.05), None), (far, synth.ramp_lut(alpha=0.05), None),
              (far, synth.random_lut(5, n=32, alpha_max=0.3), None),
              (far, synth.random_lut(5, n=32, alpha_max=0.3), ((40, 0, 0), (96, 64, 40))),
              (near, synth.ramp_lut(alpha=0.05), None)]

    def boxes(c, k_cube, cam, lut, win):
        c.set_camera_dict(cam)
        c.set_transfer_function(lut, -3.0, 12.0)
        c.set_render_params("dvr", 0.5, 1.0)
        if win is None:
            c.set_window()
        else:
            c.set_window(*win)
        c.set_partition_balance(k_cube, True)
        out = []
        for k in range(3):
            c.set_partition(k_cube, (3,), (k,))
            out.append(c.partition(k_cube, 1)[:2])
        c.set_partition(k_cube)
        c.set_partition_balance(k_cube, False)
        c.set_window()
        return out

    got = [boxes(ctx, cid, *st) for st in states]
    assert got[0] != got[1]                               # the view moves the cuts
    for st, g in zip(states, got):
        fresh = gpu_ctx()
        try:
            fid = fresh.load_cube(cube)
            fresh.set_bricking(fid, BRICK, 1, "f32")
            assert boxes(fresh, fid, *st) == g
        finally:
            fresh.close()


def test_subimage_keeps_transmittance_and_refuses_global_termination(setup):
    import paper_1008_0135_gb300 as P
    ctx, cube, cid = setup
    ctx.set_transfer_function(synth.ramp_lut(alpha=0.3), -3.0, 12.0)
    ctx.set_camera_dict(CAMS[0])
    ctx.set_render_params("dvr", 0.5, 0.99)
    frame = ctx.render_frame(cid)
    sub = ctx.render_subimage(cid)                      # whole cube: T in place of 1 - T
    assert (sub[..., :3] == frame[..., :3]).all()
    assert ((1.0 - sub[..., 3]) - frame[..., 3]).abs().max().item() <= 1e-7
    ctx.set_partition(cid, (2,), (0,))
    ctx.set_termination("global")
    with pytest.raises(P.VrError):
        ctx.render_frame(cid)
    with pytest.raises(P.VrError):
        ctx.render_subimage(cid)
    ctx.set_termination("segment")
    ctx.set_partition(cid)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q, backend="gloo"):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from datetime import timedelta
    import torch.distributed as dist
    import paper_1008_0135_gb300 as P
    from paper_1008_0135_gb300.sortlast import SortLast
    if backend == "nccl":
        import torch
        torch.cuda.set_device(0)
    dist.init_process_group(backend, rank=rank, world_size=world, timeout=timedelta(seconds=120))
    rng = np.random.default_rng(42)
    nx, ny, nz = SHAPE
    cube = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    cube += synth.pr1_cube(seed=5, n=96, n_sources=12, sigma=(3.0, 8.0))[:nz, :ny, :nx]
    with P.Context(0) as ctx:
        cid = ctx.load_cube(cube)
        ctx.set_bricking(cid, BRICK, 1, "f32")
        ctx.set_transfer_function(synth.random_lut(3, n=64, alpha_max=0.35), -3.0, 12.0)
        ctx.set_camera_dict(CAMS[2])
        ctx.set_render_params("dvr", 0.5, 0.99)
        # NCCL groups with the bench's bounded wait
        tmo = timedelta(seconds=120) if backend == "nccl" else None
        frame = SortLast(ctx, cid, (world,), rank, backend=backend, timeout=tmo).render().cpu().numpy()
    q.put((rank, frame))
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_exchange_subimages_over_gloo(setup):
    """Two ranks (processes sharing cuda:0; no kernel waits on the other's), each rendering one
    half of the cube and exchanging sub-image bands over gloo, end with the frame the stages
    give in one process, bit for bit."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx, cube, cid = setup
    ctx.set_transfer_function(synth.random_lut(3, n=64, alpha_max=0.35), -3.0, 12.0)
    ctx.set_camera_dict(CAMS[2])
    ctx.set_render_params("dvr", 0.5, 0.99)
    local = _sortlast_local(ctx, cid, (2,)).cpu().numpy()
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    port = _free_port()
    procs = [mpc.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert np.array_equal(got[r], local), r


def test_one_rank_over_nccl(setup):
    """The exchange's NCCL path (groups created with the NCCL backend, the bands gathered with
    all_gather_into_tensor on CUDA tensors) with one rank on cuda:0 -- one GPU, so no kernel
    waits on another rank: the frame equals the one-part composite made in this process."""
    import torch.distributed as dist
    if not dist.is_nccl_available():
        pytest.skip("torch built without NCCL")
    mp = pytest.importorskip("torch.multiprocessing")
    ctx, cube, cid = setup
    ctx.set_transfer_function(synth.random_lut(3, n=64, alpha_max=0.35), -3.0, 12.0)
    ctx.set_camera_dict(CAMS[2])
    ctx.set_render_params("dvr", 0.5, 0.99)
    local = _sortlast_local(ctx, cid, (1,)).cpu().numpy()
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    p = mpc.Process(target=_rank, args=(0, 1, _free_port(), q, "nccl"))
    p.start()
    rank, got = q.get(timeout=300)
    p.join(timeout=120)
    assert p.exitcode == 0 and rank == 0
    assert np.array_equal(got, local)


def test_sortlast_with_16bit_bricks_mask_window_and_streamed_cube(setup, orc):
    """Parts compose the whole frame for FP16 bricks with a channel mask and a render window
    (DVR within 1e-6, MIP bit for bit), and for a streamed (procedural) cube, whose parts make
    only their own bricks resident."""
    import paper_1008_0135_gb300 as P
    ctx, cube, cid = setup
    lut = synth.random_lut(9, n=48, alpha_max=0.3)
    ctx.set_transfer_function(lut, -3.0, 12.0)
    ctx.set_bricking(cid, BRICK, 1, "f16")
    try:
        mask = np.ones(SHAPE[2], np.uint8)
        mask[5:9] = 0
        ctx.set_channel_mask(mask)
        ctx.set_window((10, 4, 2), (90, 60, 37))
        for cam in CAMS[:2]:
            ctx.set_camera_dict(cam)
            for mode in ("dvr", "mip"):
                ctx.set_render_params(mode, 0.5, 0.99)
                whole = ctx.render_frame(cid).cpu().numpy()
                parts = _sortlast_local(ctx, cid, (3,)).cpu().numpy()
                if mode == "mip":
                    assert np.array_equal(parts, whole)
                else:
                    assert np.abs(parts - whole).max() <= 1e-6
    finally:
        ctx.set_channel_mask(None)
        ctx.set_window()
        ctx.set_bricking(cid, BRICK, 1, "f32")
    with P.Context(0, cache_bytes=40 * 66 ** 3 * 4) as sc:
        shape = (200, 140, 120)
        sid = sc.load_cube_procedural(4, shape)
        sc.set_bricking(sid, (64, 64, 64), 1, "f32")
        sc.set_transfer_function(lut, -3.0, 12.0)
        cam = synth.random_camera(np.random.default_rng(5), shape, 64, 48, proj=1)
        sc.set_camera_dict(cam)
        sc.set_render_params("dvr", 0.5, 0.99)
        whole = sc.render_frame(sid).cpu().numpy()
        parts = _sortlast_local(sc, sid, (2, 2)).cpu().numpy()
        assert np.abs(parts - whole).max() <= 1e-6
        ref, flags, _ = orc.render(orc.Procedural(4, shape), lut, (-3.0, 12.0), cam, step=0.5, tau=0.99,
                                   brick=(64, 64, 64))
        compare_dvr(parts.reshape(-1, 4), ref, flags, 0.99)
