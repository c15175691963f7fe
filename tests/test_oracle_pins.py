"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* closed forms: constant opacity (alpha = 1-(1-a)^n), per-column max of an axis-aligned MIP;
* library routines: scipy's trilinear ``map_coordinates`` (clamp-to-edge = mode 'nearest') and
  numpy's ``interp`` for the table, composited by a textbook loop, on tiny cubes;
* numpy/torch float16/bfloat16 casts for the brick rounding;
* hand-computed ray/box intersections and a matrix-inverse check of the ray generation;
* finite differences of the oracle's own forward for its analytic gradient;
* invariants: early termination moves the result by at most 1 - tau per channel; with it
  off, per-brick segmentation changes nothing; the brick partition of the samples is exact.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# rounding to the 16-bit brick formats
# ---------------------------------------------------------------------------------------------
def _special_values():
    rng = np.random.default_rng(11)
    v = np.concatenate([
        rng.standard_normal(3000).astype(np.float32) * 10.0 ** rng.integers(-9, 5, 3000),
        np.array([0.0, -0.0, 1.0, 65504.0, 65519.0, 65520.0, 6.1035156e-05, 5.9604645e-08,
                  2.9802322e-08, 2.9802326e-08, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11,
                  2049.0, 2051.0, -2049.0, 0.1, 1e-30], np.float32),
    ])
    return v.astype(np.float32)


def test_round_fp16_matches_numpy(orc):
    v = _special_values()
    ours = orc.round_fp16(v)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).astype(np.float32)
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


def test_round_bf16_matches_torch(orc):
    torch = pytest.importorskip("torch")
    v = _special_values()
    v = np.concatenate([v, np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38], np.float32)])
    ours = orc.round_bf16(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).float().numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("m", [100.0, 2.0 ** 14, 0.5, 3.0e-3, 7.0, 65504.0, 1e-20])
def test_scale_exponent_tight(orc, m):
    e16 = orc.scale_exponent(m, "f16")
    assert m * 2.0 ** -e16 <= 2.0 ** 14 < 2 * m * 2.0 ** -e16
    eb = orc.scale_exponent(m, "bf16")
    assert m * 2.0 ** -eb <= 1.0 < 2 * m * 2.0 ** -eb
    assert orc.scale_exponent(0.0, "f16") == 0


def test_brick_exponents_cover_ghost_region(orc):
    cube = synth.pr1_cube(seed=5, n=16)
    cube[0, 0, 8] = 1000.0          # inside brick (1,0,0)'s core, in brick (0,0,0)'s ghost
    e = orc.brick_exponents(cube, (8, 8, 8), 1, "f16")
    assert e.shape == (2, 2, 2)
    assert e[0, 0, 1] == orc.scale_exponent(1000.0, "f16")
    assert e[0, 0, 0] == orc.scale_exponent(1000.0, "f16")
    assert e[1, 1, 1] == orc.scale_exponent(np.abs(cube[7:, 7:, 7:]).max(), "f16")


def test_minmax(orc):
    v = synth.pr1_cube(seed=2, n=20)
    assert orc.minmax(v) == (float(v.min()), float(v.max()))


# ---------------------------------------------------------------------------------------------
# rays
# ---------------------------------------------------------------------------------------------
def test_rays_axis_ortho_hand_computed(orc):
    shape = (8, 6, 5)
    cam = synth.axis_ortho_camera(shape)        # eye plane at z = 2.5 - 13 = -10.5, looking +z
    o, d, k = orc.rays(cam, shape, step=0.5)
    assert np.all(d == np.array([0, 0, 1], np.float32))
    ii, jj = np.meshgrid(np.arange(8), np.arange(6))
    assert np.array_equal(o[:, 0], (8 - ii.ravel() - 0.5).astype(np.float32))
    assert np.array_equal(o[:, 1], (6 - jj.ravel() - 0.5).astype(np.float32))
    assert np.all(o[:, 2] == -10.5)
    # enters at t = 10.5, leaves at 15.5: k in [21, 31)
    assert np.all(k[:, 0] == 21) and np.all(k[:, 1] == 31)


def test_rays_corner_and_miss(orc):
    shape = (4, 4, 4)
    view = synth.look_at((-2.0, -2.0, -2.0), (2.0, 2.0, 2.0), up=(0.0, 1.0, 0.0))
    cam = dict(view=view, proj=1, param=math.radians(1.0), W=1, H=1)
    o, d, k = orc.rays(cam, shape, step=0.25)
    # the centre ray runs along the diagonal: enters the corner at t = 2*sqrt(3)
    t0 = 2 * math.sqrt(3)
    t1 = 6 * math.sqrt(3)
    assert abs(k[0, 0] - math.ceil(t0 / 0.25)) <= 1 and abs(k[0, 1] - math.ceil(t1 / 0.25)) <= 1
    assert np.allclose(d[0], np.ones(3) / math.sqrt(3), atol=1e-6)
    view2 = synth.look_at((-2.0, -2.0, -2.0), (-3.0, -3.0, -3.0), up=(0.0, 1.0, 0.0))
    cam2 = dict(view=view2, proj=1, param=math.radians(10.0), W=3, H=3)
    o2, d2, k2 = orc.rays(cam2, shape, step=0.25)
    assert np.all(k2[:, 0] == k2[:, 1])        # looking away: no samples


def test_rays_match_inverse_view(orc):
    rng = np.random.default_rng(1)
    for _ in range(6):
        cam = synth.random_camera(rng, (20, 30, 40), 17, 11)
        o, d, _ = orc.rays(cam, (20, 30, 40), step=0.5)
        V = cam["view"].astype(np.float64)
        Vi = np.linalg.inv(V)
        jj, ii = np.divmod(np.arange(17 * 11), 17)
        sx = (ii + 0.5) / 17 * 2 - 1
        sy = 1 - (jj + 0.5) / 11 * 2
        if cam["proj"] == 0:
            hh = cam["param"] / 2
            e = np.stack([sx * hh * 17 / 11, sy * hh, np.zeros_like(sx), np.ones_like(sx)], 1)
            dref = np.tile(-V[2, :3], (len(sx), 1))
        else:
            th = math.tan(cam["param"] / 2)
            de = np.stack([sx * th * 17 / 11, sy * th, -np.ones_like(sx)], 1)
            de /= np.linalg.norm(de, axis=1, keepdims=True)
            e = np.tile([0, 0, 0, 1.0], (len(sx), 1))
            dref = de @ V[:3, :3]
        oref = (e @ Vi.T)[:, :3]
        assert np.allclose(o, oref, atol=2e-4 * (1 + np.abs(oref)))
        assert np.allclose(d, dref, atol=2e-6)


# ---------------------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------------------
def test_golden_constant_cube(orc):
    g = json.load(open(os.path.join(GOLDEN, "constant_cube_ortho.json")))
    cube = synth.constant_cube(g["shape_xyz"], g["voxel_value"])
    lut = synth.constant_lut(g["lut_rgba"])
    c = g["camera"]
    cam = dict(view=synth.look_at(c["eye"], c["target"]), proj=c["proj"], param=c["param"],
               W=c["W"], H=c["H"])
    out, flags, ns = orc.render(cube, lut, g["vrange"], cam, step=g["step"], tau=g["tau"])
    assert ns == g["n_samples_per_pixel"] * c["W"] * c["H"]
    assert np.allclose(out, np.array(g["expected_rgba"])[None, :], atol=1e-8)


def _slab64(o, d, n):
    """FP64 entry/exit of the box [0, n) (t >= 0) -- independent of the oracle's FP32 path."""
    t0, t1 = 0.0, math.inf
    for a in range(3):
        if d[a] == 0:
            if not (0 <= o[a] < n[a]):
                return None
            continue
        ta, tb = (0 - o[a]) / d[a], (n[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return (t0, t1) if t1 > t0 else None


def test_table_kink_flag_marks_samples_on_table_entries(orc):
    """Bit 3 of the flags: a composited sample's table coordinate x = (v - vmin)/(vmax - vmin)
    (N - 1) within 1e-4 of an entry.  A constant cube whose value sits on entry 10 of a
    32-entry table flags every pixel with samples; half-way between entries flags none; the
    bit changes nothing else."""
    rng = np.random.default_rng(5)
    shape = (9, 8, 7)
    lut = synth.random_lut(1, n=32, alpha_max=0.2)
    cam = synth.random_camera(rng, shape, 20, 18)
    on = synth.constant_cube(shape, -3.0 + 11.0 * 10.0 / 31.0)
    half = synth.constant_cube(shape, -3.0 + 11.0 * 10.5 / 31.0)
    o1, f1, _ = orc.render(on, lut, (-3, 8), cam, step=0.5, tau=1.0)
    o2, f2, _ = orc.render(half, lut, (-3, 8), cam, step=0.5, tau=1.0)
    hit = (f1 & 2) == 0
    assert hit.sum() > 100
    assert np.all(f1[hit] & 8) and not np.any(f1[~hit] & 8)
    assert not np.any(f2 & 8)
    assert np.all((f1 & ~np.uint8(8)) == (f2 & ~np.uint8(8)))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_constant_cube_alpha_closed_form(orc, seed):
    rng = np.random.default_rng(seed)
    shape = (7, 5, 9)
    cube = synth.constant_cube(shape, 0.7)
    lut = synth.constant_lut([0.3, 0.6, 0.9, 0.13])
    rgba = lut[0].astype(np.float64)              # the table holds float32 entries
    cam = synth.random_camera(rng, shape, 24, 20)
    step = [0.5, 0.25, 0.37, 1.0][seed]
    out, _, _ = orc.render(cube, lut, (0, 1), cam, step=step, tau=1.0)
    o, d, _ = orc.rays(cam, shape, step=step)
    checked = 0
    for p in range(24 * 20):
        tt = _slab64(o[p].astype(np.float64), d[p].astype(np.float64), shape)
        if tt is None:
            n = 0
        else:
            t0, t1 = tt
            # skip rays whose boundary falls within FP32 rounding of a lattice point
            if min(abs(t0 / step - round(t0 / step)), abs(t1 / step - round(t1 / step))) < 1e-3:
                continue
            n = max(0, math.ceil(t1 / step) - math.ceil(t0 / step))
        A = 1 - (1 - rgba[3]) ** n
        assert abs(out[p, 3] - A) < 1e-12
        assert np.allclose(out[p, :3], rgba[:3] * A, atol=1e-12)
        checked += 1
    assert checked > 300


@pytest.mark.parametrize("mode", ["mip", "mip32"])
def test_axis_aligned_mip_is_column_max(orc, mode):
    # power-of-two square frame: pixel centres map exactly onto voxel centres in FP32
    cube = synth.pr1_cube(seed=4, n=32)[:20].copy()       # nz=20, ny=32, nx=32
    shape = (32, 32, 20)
    cam = synth.axis_ortho_camera(shape)
    m, _, _ = orc.render(cube, synth.ramp_lut(), (-3, 20), cam, mode=mode, step=0.5)
    colmax = cube.max(axis=0)                               # [y][x]
    expect = colmax[::-1, ::-1].ravel()                     # image row j <-> y = ny-1-j, col i <-> x = nx-1-i
    assert np.array_equal(m.astype(np.float32), expect)


def test_linear_field_reproduced(orc):
    """Trilinear interpolation reproduces a linear field exactly away from the clamped border."""
    shape = (12, 12, 12)
    coef = (0.25, -0.5, 0.125)
    cube = synth.linear_cube(shape, coef, 1.0).astype(np.float64).astype(np.float32)
    cam = dict(view=synth.look_at((6.2, 5.9, -20.0), (6.1, 6.05, 6.0)), proj=1,
               param=math.radians(6.0), W=5, H=5)
    m, _, _ = orc.render(cube, synth.ramp_lut(), (-20, 20), cam, mode="mip", step=0.5)
    o, d, k = orc.rays(cam, shape, step=0.5)
    for p in range(25):
        ks = np.arange(k[p, 0], k[p, 1])
        pos = o[p].astype(np.float64)[None, :] + (ks[:, None] * 0.5) * d[p].astype(np.float64)
        inner = np.all((pos >= 0.5) & (pos <= 11.5), axis=1)
        lin = pos @ np.array(coef) + 1.0
        # clamped samples (first/last half voxel) are not linear; they never exceed the max here
        assert abs(m[p] - lin[inner].max()) < 1e-5 or lin[~inner].size


# ---------------------------------------------------------------------------------------------
# brute force against library routines on tiny cubes
# ---------------------------------------------------------------------------------------------
def _brute(cube, lut, vrange, o, d, k0, k1, step, tau, seg_of=None):
    """Textbook front-to-back compositing from scipy trilinear + numpy interp of the table."""
    if k1 <= k0:
        return np.zeros(4)
    ks = np.arange(k0, k1)
    pos = o.astype(np.float64)[None, :] + (ks[:, None] * float(step)) * d.astype(np.float64)
    coords = np.stack([pos[:, 2] - 0.5, pos[:, 1] - 0.5, pos[:, 0] - 0.5])
    v = map_coordinates(cube.astype(np.float64), coords, order=1, mode="nearest")
    u = np.clip((v - vrange[0]) / (vrange[1] - vrange[0]), 0, 1) * (len(lut) - 1)
    rgba = np.stack([np.interp(u, np.arange(len(lut)), lut[:, c].astype(np.float64))
                     for c in range(4)], 1)
    thr = float(np.float32(1.0) - np.float32(min(tau, 1.0)))
    C = np.zeros(3)
    T = 1.0
    Tseg = 1.0
    cur = None
    stop = False
    for m in range(len(ks)):
        s = seg_of[m] if seg_of is not None else 0
        if s != cur:
            cur, Tseg, stop = s, 1.0, False
        if stop:
            continue
        a = rgba[m, 3]
        C += T * a * rgba[m, :3]
        T *= 1 - a
        Tseg *= 1 - a
        if Tseg <= thr:
            stop = True
    return np.array([*C, 1 - T])


@pytest.mark.parametrize("seed", range(8))
def test_bruteforce_tiny_cubes(orc, seed):
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(x) for x in rng.integers(2, 9, 3))
    nx, ny, nz = shape
    cube = rng.uniform(-1, 3, (nz, ny, nx)).astype(np.float32)
    lut = synth.random_lut(seed, n=int(rng.integers(2, 40)), alpha_max=0.6)
    cam = synth.random_camera(rng, shape, 9, 7)
    step = float(rng.choice([0.5, 0.25, 0.3, 1.0]))
    tau = float(rng.choice([1.0, 0.9, 0.6]))
    brick = tuple(int(x) for x in rng.integers(1, 5, 3))
    for b in (None, brick):
        out, flags, _ = orc.render(cube, lut, (-1, 3), cam, step=step, tau=tau, brick=b)
        o, d, k = orc.rays(cam, shape, step=step)
        for p in range(63):
            seg = None
            if b is not None and k[p, 1] > k[p, 0]:
                own = orc.sample_owners(shape, cam, p, step, b)
                seg = [tuple(r) for r in own]
            ref = _brute(cube, lut, (-1, 3), o[p], d[p], k[p, 0], k[p, 1], step, tau, seg)
            if flags[p] & 1:
                assert np.all(np.abs(out[p] - ref) <= (1 - tau) + 1e-9)
            else:
                assert np.allclose(out[p], ref, atol=1e-12), (p, out[p], ref)
        assert not np.any(flags & 4)


def test_sample_owner_is_geometric_brick(orc):
    """Away from brick faces, the FP32 ownership decision is the brick holding the sample."""
    rng = np.random.default_rng(7)
    shape = (20, 17, 23)
    b = (4, 6, 5)
    for _ in range(4):
        cam = synth.random_camera(rng, shape, 8, 8)
        o, d, k = orc.rays(cam, shape, step=0.5)
        for p in range(0, 64, 3):
            own = orc.sample_owners(shape, cam, p, 0.5, b)
            ks = np.arange(k[p, 0], k[p, 1])
            assert len(own) == len(ks)
            if len(ks) == 0:
                continue
            pos = o[p].astype(np.float64) + (ks[:, None] * 0.5) * d[p].astype(np.float64)
            geo = np.floor(pos / np.array(b)).astype(np.int64)
            frac = pos / np.array(b) - np.floor(pos / np.array(b))
            safe = np.all((frac > 1e-4) & (frac < 1 - 1e-4), axis=1)
            assert np.array_equal(own[safe], geo[safe])
            assert np.all(own >= 0)


# ---------------------------------------------------------------------------------------------
# early ray termination and segmentation
# ---------------------------------------------------------------------------------------------
def test_ert_bounds_and_off(orc):
    cube = synth.pr1_cube(seed=0)
    lut = synth.ramp_lut(alpha=0.9)
    cam = synth.pr1_camera(W=96, H=96)
    off, _, n_off = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=1.0)
    off_b, _, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=1.0, brick=(32, 32, 32))
    assert np.array_equal(off, off_b)           # segmentation alone changes nothing
    glob, fg, n_g = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99)
    loc, fl, n_l = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.99, brick=(32, 32, 32))
    assert n_g < n_l < n_off                      # termination saves samples
    assert np.abs(glob - off).max() <= 0.01 + 1e-12
    assert np.abs(loc - off).max() <= 0.01 + 1e-12
    assert np.abs(loc - glob).max() <= 0.01 + 1e-12
    assert (glob[:, 3] >= 0).all() and np.any(glob[:, 3] >= 0.99)


def test_global_termination_ignores_the_bricking(orc):
    """term="global": the ray keeps its transmittance across bricks, so the bricked image is
    the unbricked one sample for sample (bit-identical, FP64), for any brick size; and it takes
    no more samples than per-segment termination."""
    rng = np.random.default_rng(9)
    cube = synth.pr1_cube(seed=3, n=32)
    lut = synth.ramp_lut(alpha=0.8)
    for _ in range(3):
        cam = synth.random_camera(rng, (32, 32, 32), 40, 36)
        b = tuple(int(x) for x in rng.integers(3, 17, 3))
        ref, fr, nr = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.95)
        g, fgl, ng = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.95, brick=b, term="global")
        _, _, ns = orc.render(cube, lut, (-3, 20), cam, step=0.5, tau=0.95, brick=b)
        assert np.array_equal(g, ref) and np.array_equal(fgl, fr) and ng == nr
        assert ng <= ns


def test_no_partition_errors_random(orc):
    rng = np.random.default_rng(3)
    cube = synth.pr1_cube(seed=1, n=24)
    for _ in range(5):
        cam = synth.random_camera(rng, (24, 24, 24), 32, 32)
        b = tuple(int(x) for x in rng.integers(1, 13, 3))
        _, flags, _ = orc.render(cube, synth.ramp_lut(), (-3, 20), cam, step=0.5, brick=b)
        assert not np.any(flags & 4)


# ---------------------------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------------------------
def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(9)
    shape = (10, 9, 8)
    cube = synth.pr1_cube(seed=9, n=10, amp=(1.0, 3.0))[:8, :9, :10].copy()
    lut = synth.random_lut(3, n=16, alpha_max=0.5)
    cam = synth.random_camera(rng, shape, 12, 10, proj=1)
    vr = (-3.0, 8.0)
    gout = rng.standard_normal((120, 4))
    kw = dict(step=0.5, tau=0.95, brick=(4, 5, 3))
    glut, gvox = orc.render_grad(cube, lut, vr, cam, gout, **kw)

    def loss(c, l):
        out, _, ns = orc.render(c, l, vr, cam, **kw)
        return float((out * gout).sum()), ns

    _, ns0 = loss(cube, lut)
    checked = 0
    for _ in range(24):
        i, ch = int(rng.integers(0, 16)), int(rng.integers(0, 4))
        h = 2.0 ** -14
        lp, lm = lut.astype(np.float64).copy(), lut.astype(np.float64).copy()
        lp[i, ch] += h
        lm[i, ch] -= h
        # the oracle reads float32 tables: use exactly representable perturbations
        lp32, lm32 = lp.astype(np.float32), lm.astype(np.float32)
        (fp, np_), (fm, nm) = loss(cube, lp32), loss(cube, lm32)
        if np_ != ns0 or nm != ns0:
            continue                    # the perturbation moved an early-termination stop
        fd = (fp - fm) / (float(lp32[i, ch]) - float(lm32[i, ch]))
        assert abs(fd - glut[i, ch]) <= 1e-6 + 1e-5 * abs(fd), (i, ch, fd, glut[i, ch])
        checked += 1
    assert checked >= 12
    nz_idx = np.argwhere(np.abs(gvox) > 1e-6)
    checked = 0
    for q in nz_idx[rng.choice(len(nz_idx), 24, replace=False)]:
        z, y, x = q
        h = 2.0 ** -10
        cp, cm = cube.copy(), cube.copy()
        cp[z, y, x] += h
        cm[z, y, x] -= h
        (fp, np_), (fm, nm) = loss(cp, lut), loss(cm, lut)
        if np_ != ns0 or nm != ns0:
            continue
        fd = (fp - fm) / (float(cp[z, y, x]) - float(cm[z, y, x]))
        # a table knot or a clamp crossed inside [-h, h] shows as a large mismatch; allow that
        # for at most a few entries
        if abs(fd - gvox[z, y, x]) <= 1e-5 + 1e-4 * abs(fd):
            checked += 1
    assert checked >= 20


# ---------------------------------------------------------------------------------------------
# procedural cube (input generator of the out-of-core tests)
# ---------------------------------------------------------------------------------------------
SEED = 4


def test_procedural_noise_is_standard_normal(orc):
    """Box-Muller of SplitMix64 hashes gives independent standard normals."""
    stats = pytest.importorskip("scipy.stats")
    vals = np.array([orc.proc_noise(SEED, (4096, 4096, 4800), x, 17, 33) for x in range(20000)])
    assert abs(vals.mean()) < 0.03 and abs(vals.std() - 1.0) < 0.02
    assert stats.kstest(vals, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(vals[0::2], vals[1::2])[0, 1]) < 0.03   # Box-Muller pairs independent


def test_procedural_sources_add_gaussian_bumps(orc):
    """Away from its noise, a voxel holds the sum of the sources' Gaussian terms: the brightest
    voxel of a region exceeds what N(0,1) noise reaches there, and the field minus its noise is
    non-negative (sources only add)."""
    shape = (700, 600, 520)
    lo, dim = (0, 0, 0), (64, 64, 64)
    v = orc.proc_region(SEED, shape, lo, (700, 600, 4))
    z, y, x = np.unravel_index(np.argmax(v), v.shape)
    noise = orc.proc_noise(SEED, shape, x, y, z)
    assert v[z, y, x] - noise > 2.5                 # amplitudes are at least 3
    for (xx, yy, zz) in [(5, 7, 1), (300, 200, 2), (699, 599, 3)]:
        assert v[zz, yy, xx] - orc.proc_noise(SEED, shape, xx, yy, zz) >= -1e-6


# ---------------------------------------------------------------------------------------------
# spectral-channel masks and render windows (Section 2.3)
# ---------------------------------------------------------------------------------------------
def test_channel_mask_equals_cube_with_vmin_slices(orc):
    """A disabled channel holds vmin: the same as editing those z-slices of the cube."""
    rng = np.random.default_rng(31)
    cube = synth.pr1_cube(seed=31, n=24)
    mask = (rng.uniform(size=24) > 0.4).astype(np.uint8)
    edited = cube.copy()
    edited[mask == 0] = np.float32(-3.0)
    lut = synth.random_lut(2, n=40, alpha_max=0.4)
    for proj in (0, 1):
        cam = synth.random_camera(rng, (24, 24, 24), 30, 26, proj=proj)
        for mode in ("dvr", "mip", "mip32"):
            a, _, _ = orc.render(cube, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.95,
                                 brick=(8, 8, 8), channels=mask)
            b, _, _ = orc.render(edited, lut, (-3, 20), cam, mode=mode, step=0.5, tau=0.95,
                                 brick=(8, 8, 8))
            assert np.array_equal(a, b)
    ones = np.ones(24, np.uint8)
    a, _, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5, channels=ones)
    b, _, _ = orc.render(cube, lut, (-3, 20), cam, step=0.5)
    assert np.array_equal(a, b)
    # gradient: disabled channels receive none
    gout = rng.standard_normal((30 * 26, 4))
    _, gv = orc.render_grad(cube, lut, (-3, 20), cam, gout, step=0.5, tau=1.0, channels=mask)
    assert np.all(gv[mask == 0] == 0) and np.abs(gv[mask == 1]).max() > 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_window_clips_the_lattice(orc, seed):
    """Samples are the lattice points inside the window box (checked in FP64 away from its
    faces); the field is still the whole cube's (no clamping at the window)."""
    rng = np.random.default_rng(40 + seed)
    shape = (9, 8, 7)
    nx, ny, nz = shape
    cube = rng.uniform(-1, 3, (nz, ny, nx)).astype(np.float32)
    lut = synth.random_lut(seed, n=20, alpha_max=0.5)
    win = ((1, 2, 1), (7, 6, 5))
    cam = synth.random_camera(rng, shape, 11, 9)
    out, _, _ = orc.render(cube, lut, (-1, 3), cam, step=0.5, tau=1.0, window=win)
    o, d, _ = orc.rays(cam, shape, step=0.5)
    checked = 0
    for p in range(11 * 9):
        tt = _slab64(o[p].astype(np.float64) - np.array(win[0]), d[p].astype(np.float64),
                     np.subtract(win[1], win[0]))
        if tt is None:
            k0 = k1 = 0
        else:
            t0, t1 = tt
            if min(abs(t0 / 0.5 - round(t0 / 0.5)), abs(t1 / 0.5 - round(t1 / 0.5))) < 1e-3:
                continue
            k0, k1 = math.ceil(t0 / 0.5), math.ceil(t1 / 0.5)
        ref = _brute(cube, lut, (-1, 3), o[p], d[p], k0, k1, 0.5, 1.0)
        assert np.allclose(out[p], ref, atol=1e-12)
        checked += 1
    assert checked > 60
    whole, _, _ = orc.render(cube, lut, (-1, 3), cam, step=0.5, window=((0, 0, 0), shape))
    plain, _, _ = orc.render(cube, lut, (-1, 3), cam, step=0.5)
    assert np.array_equal(whole, plain)
