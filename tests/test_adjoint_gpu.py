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


# small tables and a 2048-entry one (the table gradient's per-CTA partial rows in L2 scale with
# it); an opacity above 1 (transmittance can turn negative) is followed as written
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


def test_adjoint_with_channel_mask_and_window_matches_oracle_gradient(ctx, orc):
    """Disabled channels read as vmin and receive no voxel gradient; a render window clips the
    rays (voxels outside it still feed the stencils at its faces): the GPU gradients follow the
    oracle's with both set."""
    import torch
    rng, cube, lut, cam, cid = _setup(ctx, 11)
    vr = (-3.0, 8.0)
    step, tau = 0.5, 0.95
    mask = (rng.uniform(size=cube.shape[0]) > 0.3).astype(np.uint8)
    win = ((2, 3, 1), (21, 20, 22))
    gout = rng.standard_normal((cam["W"] * cam["H"], 4))
    try:
        ctx.set_channel_mask(mask)
        ctx.set_window(*win)
        _, flags, _ = orc.render(cube, lut, vr, cam, step=step, tau=tau, brick=(8, 8, 8),
                                 channels=mask, window=win)
        gout[(flags & 9).astype(bool)] = 0.0
        gl, gv = _gpu_grad(ctx, cid, cube, lut, vr, cam, gout, step, tau)
    finally:
        ctx.set_channel_mask(None)
        ctx.set_window()
    rl, rv = orc.render_grad(cube, lut, vr, cam, gout.astype(np.float32).astype(np.float64),
                             step=step, tau=tau, brick=(8, 8, 8), channels=mask, window=win)
    assert np.abs(rl).max() > 0 and np.abs(rv).max() > 0
    assert np.abs(gl - rl).max() <= 2e-4 * np.abs(rl).max(), np.abs(gl - rl).max()
    assert np.abs(gv - rv).max() <= 2e-4 * np.abs(rv).max(), np.abs(gv - rv).max()
    off = mask == 0                       # disabled channels: no voxel gradient at all
    assert np.all(gv[off] == 0.0)
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
    """vr_render_backward right after the frame it differentiates reuses that frame's fragments
    (setting the same camera, table or parameters again changes nothing); after a change of
    camera, or another frame, it ray-casts again.  All three
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
    ctx.set_camera_dict(other)                       # the camera changed and back: the next
    ctx.set_camera_dict(cam)                         # backward ray-casts
    b = grads()
    render(ctx, cid, lut, (-3, 20), other, step=0.5, tau=0.99)
    ctx.set_camera_dict(cam)                         # another frame's fragments are held
    c = grads()
    for x, y in ((a, b), (a, c)):
        for u, v in zip(x, y):
            assert np.allclose(u, v, rtol=1e-5, atol=1e-6 * np.abs(u).max())
    assert np.abs(a[0]).max() > 0
    ctx.free_cube(cid)


def test_adjoint_finite_differences_at_the_differentiation_config(ctx, orc):
    """The differentiation workload: 256^3 cube (seed 3), 128^3 bricks, 8 orbit views 45 degrees
    apart at 512^2, step 0.5, ERT 0.99, ramp table; loss = squared difference against a target
    rendered with the ramp shifted by +3, on 2048 seeded pixels per view (no weight elsewhere).
    The GPU gradient, one autograd backward through vr_render_backward_views, against FP64
    central differences (h = 1e-3) of the oracle's loss for 64 seeded table entries and 64
    seeded voxels, relative tolerance 1e-3.  The image is piecewise smooth: a pixel that some
    checked +-h perturbation moves across a table entry, clamp edge or termination stop (its
    oracle piece signature changes), or whose gradient is ambiguous at the unperturbed input, gets
    no weight in the loss, so every checked difference stays inside one piece."""
    import torch
    from paper_1008_0135_gb300.autograd import render_views
    cfg = synth.DIFF
    cube = synth.diff_cube(seed=cfg["seed"])
    lut = synth.ramp_lut()
    target_lut = synth.shifted_ramp_lut(shift=3.0, vrange=cfg["vrange"])
    vr, step, tau, brick = cfg["vrange"], cfg["step"], cfg["tau"], cfg["brick"]
    c = np.array(cfg["shape"], np.float64) / 2
    dist = 1.5 * 0.5 * math.sqrt(3) * cfg["shape"][0]
    cams = [dict(view=synth.orbit_view(45.0 * j, c, dist), proj=1, param=math.radians(60.0),
                 W=cfg["W"], H=cfg["H"]) for j in range(cfg["n_views"])]
    V, npx = len(cams), cfg["W"] * cfg["H"]
    kw = dict(step=step, tau=tau, brick=brick)
    S, tgt, sig0 = [], [], []
    for v, cam in enumerate(cams):
        pix = synth.sample_pixels(900 + v, cam["W"], cam["H"], 2048)
        _, flags, _, sg = orc.render_sig(cube, lut, vr, cam, pix=pix, **kw)
        keep = (flags & 9) == 0
        t, _, _ = orc.render(cube, target_lut, vr, cam, pix=pix[keep], **kw)
        S.append(pix[keep])
        tgt.append(t)
        sig0.append(sg[keep])
    # the oracle's analytic gradient picks entries the loss depends on
    rl, rv = np.zeros((lut.shape[0], 4)), np.zeros(cube.shape)
    for v, cam in enumerate(cams):
        out, _, _ = orc.render(cube, lut, vr, cam, pix=S[v], **kw)
        a, b = orc.render_grad(cube, lut, vr, cam, 2.0 * (out - tgt[v]), pix=S[v], **kw)
        rl += a
        rv += b
    rng = np.random.default_rng(cfg["seed"])
    h = 1e-3
    cand = np.argwhere(np.abs(rl) > 1e-3 * np.abs(rl).max())
    lut_entries = cand[rng.choice(len(cand), 64, replace=False)]
    cand = np.argwhere(np.abs(rv) > 1e-2 * np.abs(rv).max())
    vox_entries = cand[rng.choice(len(cand), 64, replace=False)]
    rays = [orc.rays(cam, cfg["shape"], step=step, pix=S[v]) for v, cam in enumerate(cams)]
    excluded = [np.zeros(len(S[v]), bool) for v in range(V)]

    def perturbed(cb, lt, sel_of_view):
        """Oracle images of the selected loss pixels (index arrays into S per view); marks the
        pixels whose piece signature differs from the unperturbed one."""
        res = {}
        for v, sel in sel_of_view.items():
            out, _, _, sg = orc.render_sig(cb, lt, vr, cams[v], pix=S[v][sel], **kw)
            excluded[v][sel[sg != sig0[v][sel]]] = True
            res[v] = (sel, out)
        return res

    runs = []
    everything = {v: np.arange(len(S[v])) for v in range(V)}
    for i, ch in lut_entries:
        lp, lm = lut.astype(np.float64).copy(), lut.astype(np.float64).copy()
        lp[i, ch] += h
        lm[i, ch] -= h
        lp32, lm32 = lp.astype(np.float32), lm.astype(np.float32)
        runs.append(("lut", (i, ch), float(lp32[i, ch]) - float(lm32[i, ch]),
                     perturbed(cube, lp32, everything), perturbed(cube, lm32, everything)))
    for z, y, x in vox_entries:
        p = np.array([x + 0.5, y + 0.5, z + 0.5])
        near = {}
        for v, (o, d, _) in enumerate(rays):       # rays within the stencil's reach of the voxel
            dd = np.linalg.norm(np.cross(p[None, :] - o.astype(np.float64), d.astype(np.float64)), axis=1)
            sel = np.nonzero(dd < 2.0)[0]
            if len(sel):
                near[v] = sel
        cp, cm = cube.copy(), cube.copy()
        cp[z, y, x] = np.float32(float(cube[z, y, x]) + h)
        cm[z, y, x] = np.float32(float(cube[z, y, x]) - h)
        runs.append(("vox", (z, y, x), float(cp[z, y, x]) - float(cm[z, y, x]),
                     perturbed(cp, lut, near), perturbed(cm, lut, near)))
    kept = sum(int((~e).sum()) for e in excluded)
    assert kept > 0.8 * sum(len(p) for p in S), kept
    # GPU gradient of the loss over the kept pixels, through the autograd function
    mask = np.zeros((V, npx), np.float32)
    target = np.zeros((V, npx, 4), np.float32)
    for v in range(V):
        mask[v, S[v][~excluded[v]]] = 1.0
        target[v, S[v]] = tgt[v]
    cid = ctx.load_cube(cube)
    ctx.set_bricking(cid, brick, 1, "f32")
    lut_t = torch.from_numpy(lut).cuda().requires_grad_(True)
    vox_t = torch.from_numpy(cube).cuda().requires_grad_(True)
    imgs = render_views(ctx, cid, lut_t, cams, vr, voxels=vox_t, step=step, tau=tau)
    m = torch.from_numpy(mask).cuda().reshape(V, cfg["H"], cfg["W"], 1)
    tt = torch.from_numpy(target).cuda().reshape(V, cfg["H"], cfg["W"], 4)
    (((imgs - tt) ** 2) * m).sum().backward()
    gl = lut_t.grad.cpu().numpy().astype(np.float64)
    gv = vox_t.grad.cpu().numpy().astype(np.float64)
    checked = {"lut": 0, "vox": 0}
    for kind, idx, den, plus, minus in runs:
        num = 0.0
        for v, (sel, op) in plus.items():
            om = minus[v][1]
            w = ~excluded[v][sel]
            t = tgt[v][sel][w]
            num += float(((op[w] - t) ** 2).sum() - ((om[w] - t) ** 2).sum())
        fd = num / den
        g = gl[idx] if kind == "lut" else gv[idx]
        if fd == 0.0 and g == 0.0:
            continue                        # every pixel the entry reaches was left out
        assert abs(g - fd) <= 1e-3 * abs(fd), (kind, idx, g, fd)
        checked[kind] += 1
    assert checked["lut"] >= 48 and checked["vox"] >= 48, checked
    ctx.free_cube(cid)
