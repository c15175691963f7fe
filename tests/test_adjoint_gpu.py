"""Adjoint ray casting on the GPU against the FP64 oracle gradient and finite differences."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import gpu_ctx, render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _setup(ctx, seed, n=24, brick=(8, 8, 8), W=48, H=40, nlut=32):
    rng = np.random.default_rng(seed)
    cube = synth.pr1_cube(seed=seed, n=n, amp=(1.0, 4.0))
    lut = synth.random_lut(seed, n=nlut, alpha_max=0.4)
    cam = synth.random_camera(rng, (n, n, n), W, H)
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, brick, 1, "f32")
    return rng, cube, lut, cam, cid


def _gpu_grad(ctx, cid, cube, lut, vr, cam, gout, step, tau):
    import torch
    render(ctx, cid, lut, vr, cam, step=step, tau=tau)
    g = torch.from_numpy(gout.astype(np.float32).reshape(cam["H"], cam["W"], 4)).cuda()
    glut = torch.zeros((lut.shape[0], 4), device="cuda")
    gvox = torch.zeros(cube.shape, device="cuda")
    ctx.render_backward(cid, g.contiguous(), glut, gvox)
    return glut.cpu().numpy().astype(np.float64), gvox.cpu().numpy().astype(np.float64)


# the table gradient accumulates in 8 shared-memory copies for small tables, 1 for 2048 entries;
# an opacity above 1 (transmittance can turn negative) is followed as written
@pytest.mark.parametrize("seed,tau,layouts,nlut,over", [(0, 0.95, 1, 32, False), (1, 1.0, 1, 32, False),
                                                        (2, 0.9, 7, 32, False), (3, 0.9, 9, 32, False),
                                                        (4, 0.95, 1, 2048, False), (5, 0.95, 1, 32, True)])
def test_adjoint_matches_oracle_gradient(ctx, orc, seed, tau, layouts, nlut, over):
    rng, cube, lut, cam, cid = _setup(ctx, seed, nlut=nlut)
    if over:
        lut[7, 3] = 1.05
    if layouts != 1:
        ctx.set_brick_layouts(cid, layouts)
    vr = (-3.0, 8.0)
    step = 0.5
    gout = rng.standard_normal((cam["W"] * cam["H"], 4))
    _, flags, _ = orc.render(cube, lut, vr, cam, step=step, tau=tau, brick=(8, 8, 8))
    # pixels that stop at the threshold, or with a sample on a table entry (where the
    # derivative jumps), have two valid gradients: left out
    gout[(flags & 9).astype(bool)] = 0.0
    gl, gv = _gpu_grad(ctx, cid, cube, lut, vr, cam, gout, step, tau)
    rl, rv = orc.render_grad(cube, lut, vr, cam, gout.astype(np.float32).astype(np.float64),
                             step=step, tau=tau, brick=(8, 8, 8))
    assert np.abs(rl).max() > 0 and np.abs(rv).max() > 0
    assert np.abs(gl - rl).max() <= 2e-4 * np.abs(rl).max(), np.abs(gl - rl).max()
    assert np.abs(gv - rv).max() <= 2e-4 * np.abs(rv).max(), np.abs(gv - rv).max()
    ctx.free_cube(cid)


def test_adjoint_matches_gpu_finite_differences(ctx):
    """Central differences of the GPU forward itself (no early termination, so no stop moves)."""
    import torch
    rng, cube, lut, cam, cid = _setup(ctx, 7, n=16, brick=(8, 8, 8), W=24, H=24)
    vr = (-3.0, 8.0)
    gout = rng.standard_normal((cam["W"] * cam["H"], 4))
    gl, _ = _gpu_grad(ctx, cid, cube, lut, vr, cam, gout, 0.5, 1.0)

    def loss(l):
        img = render(ctx, cid, l, vr, cam, step=0.5, tau=1.0).astype(np.float64)
        return float((img * gout).sum())

    checked = 0
    for i in rng.choice(lut.shape[0], 10, replace=False):
        ch = int(rng.integers(0, 4))
        h = 1e-2
        lp, lm = lut.copy(), lut.copy()
        lp[i, ch] += h
        lm[i, ch] -= h
        fd = (loss(lp) - loss(lm)) / (float(lp[i, ch]) - float(lm[i, ch]))
        if abs(gl[i, ch]) < 1e-3:
            continue
        assert abs(fd - gl[i, ch]) <= 2e-2 * abs(gl[i, ch]) + 1e-3, (i, ch, fd, gl[i, ch])
        checked += 1
    assert checked >= 4
    ctx.free_cube(cid)


def test_autograd_function_sums_views(ctx, orc):
    import torch
    from paper_1008_0135_gb300.autograd import render_views
    n = 20
    cube = synth.pr1_cube(seed=11, n=n, amp=(1.0, 4.0))
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, (10, 10, 10), 1, "f32")
    lut = torch.from_numpy(synth.random_lut(4, n=16, alpha_max=0.3)).cuda().requires_grad_(True)
    vox = torch.from_numpy(cube).cuda().requires_grad_(True)
    c = np.array([n / 2] * 3)
    cams = [dict(view=synth.orbit_view(a, c, 40.0), proj=1, param=math.radians(50), W=32, H=32)
            for a in (0.0, 100.0)]
    imgs = render_views(ctx, cid, lut, cams, (-3.0, 8.0), voxels=vox, step=0.5, tau=1.0)
    w = np.random.default_rng(0).standard_normal(imgs.shape).astype(np.float32)
    for k, cam in enumerate(cams):             # no weight on pixels with an ambiguous gradient
        _, flags, _ = orc.render(cube, lut.detach().cpu().numpy(), (-3.0, 8.0), cam, step=0.5,
                                 tau=1.0, brick=(10, 10, 10))
        w[k].reshape(-1, 4)[(flags & 8).astype(bool)] = 0.0
    w = torch.from_numpy(w).cuda()
    (imgs * w).sum().backward()
    wl = w.cpu().numpy().reshape(2, -1, 4).astype(np.float64)
    rl = np.zeros((16, 4))
    rv = np.zeros(cube.shape)
    for k, cam in enumerate(cams):
        a, b = orc.render_grad(cube, lut.detach().cpu().numpy(), (-3.0, 8.0), cam, wl[k],
                               step=0.5, tau=1.0, brick=(10, 10, 10))
        rl += a
        rv += b
    assert np.abs(lut.grad.cpu().numpy() - rl).max() <= 2e-4 * np.abs(rl).max()
    assert np.abs(vox.grad.cpu().numpy() - rv).max() <= 2e-4 * np.abs(rv).max()
    ctx.free_cube(cid)


def test_adjoint_at_the_benchmark_size_on_sampled_pixels(ctx, orc):
    """The differentiation workload as the bench times it (256^3 cube, 128^3 bricks, 512^2
    views, step 0.5, ERT 0.99, ramp table): pixel gradients on 512 seeded pixels of two orbit
    views (zero elsewhere), so the oracle traces only those rays; table and voxel gradients
    against it."""
    import torch
    cfg = synth.DIFF
    cube = synth.diff_cube(seed=cfg["seed"])
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, cfg["brick"], 1, "f32")
    lut = synth.ramp_lut()
    vr = cfg["vrange"]
    c = np.array(cfg["shape"], np.float64) / 2
    rng = np.random.default_rng(31)
    for j in (1, 6):
        cam = dict(view=synth.orbit_view(45.0 * j, c, 1.5 * 0.5 * math.sqrt(3) * cfg["shape"][0]),
                   proj=1, param=math.radians(60.0), W=cfg["W"], H=cfg["H"])
        pix = synth.sample_pixels(700 + j, cam["W"], cam["H"], 512)
        _, flags, _ = orc.render(cube, lut, vr, cam, step=cfg["step"], tau=cfg["tau"],
                                 brick=cfg["brick"], pix=pix)
        g = rng.standard_normal((len(pix), 4))
        g[(flags & 9).astype(bool)] = 0.0
        g = g.astype(np.float32).astype(np.float64)
        full = np.zeros((cam["H"] * cam["W"], 4), np.float32)
        full[pix] = g
        render(ctx, cid, lut, vr, cam, step=cfg["step"], tau=cfg["tau"])
        gl = torch.zeros((lut.shape[0], 4), device="cuda")
        gv = torch.zeros(cube.shape, device="cuda")
        ctx.render_backward(cid, torch.from_numpy(full.reshape(cam["H"], cam["W"], 4)).cuda(), gl, gv)
        rl, rv = orc.render_grad(cube, lut, vr, cam, g, step=cfg["step"], tau=cfg["tau"],
                                 brick=cfg["brick"], pix=pix)
        gl = gl.cpu().numpy().astype(np.float64)
        gv = gv.cpu().numpy().astype(np.float64)
        assert np.abs(rl).max() > 0 and np.abs(rv).max() > 0
        assert np.abs(gl - rl).max() <= 2e-4 * np.abs(rl).max(), np.abs(gl - rl).max()
        assert np.abs(gv - rv).max() <= 2e-4 * np.abs(rv).max(), np.abs(gv - rv).max()
    ctx.free_cube(cid)


@pytest.mark.parametrize("layouts", [1, 9])
def test_backward_reuses_the_frames_fragments_only_when_valid(ctx, layouts):
    """vr_render_backward right after the frame it differentiates reuses that frame's fragments;
    after any call that can change a frame, or another frame, it ray-casts again.  All three
    orders give the same gradients (to the atomics' summation order)."""
    import torch
    rng, cube, lut, cam, cid = _setup(ctx, 21)
    ctx.set_brick_layouts(cid, layouts)
    other = synth.random_camera(rng, cube.shape, cam["W"], cam["H"])
    g = torch.from_numpy(rng.standard_normal((cam["H"], cam["W"], 4)).astype(np.float32)).cuda()

    def grads():
        glut = torch.zeros((lut.shape[0], 4), device="cuda")
        gvox = torch.zeros(cube.shape, device="cuda")
        ctx.render_backward(cid, g, glut, gvox)
        return glut.cpu().numpy(), gvox.cpu().numpy()

    render(ctx, cid, lut, (-3, 20), cam, step=0.5, tau=0.99)
    a = grads()                                      # reuses the frame's fragments
    ctx.set_camera_dict(cam)                         # a setter: the next backward ray-casts
    b = grads()
    render(ctx, cid, lut, (-3, 20), other, step=0.5, tau=0.99)
    ctx.set_camera_dict(cam)                         # another frame's fragments are held
    c = grads()
    for x, y in ((a, b), (a, c)):
        for u, v in zip(x, y):
            assert np.allclose(u, v, rtol=1e-5, atol=1e-6 * np.abs(u).max())
    assert np.abs(a[0]).max() > 0
    ctx.free_cube(cid)
