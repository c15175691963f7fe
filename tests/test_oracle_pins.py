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


@pytest.mark.parametrize("step,brick", [(2.3, (2, 3, 2)), (5.0, (1, 2, 3)), (3.7, (3, 3, 3))])
def test_long_steps_closed_form_and_bricking(orc, step, brick):
    """Steps longer than a brick (most bricks take no sample of a ray, some take one): the
    constant cube still gives 1 - (1 - a)^n with n the lattice points in [t0, t1), unbricked and
    bricked alike (no early termination); the brute-force sum over owned segments agrees on a
    random cube with early termination."""
    rng = np.random.default_rng(int(step * 10))
    shape = (9, 7, 11)
    cube = synth.constant_cube(shape, 0.7)
    lut = synth.constant_lut([0.3, 0.6, 0.9, 0.13])
    rgba = lut[0].astype(np.float64)
    cam = synth.random_camera(rng, shape, 20, 18)
    out, _, _ = orc.render(cube, lut, (0, 1), cam, step=step, tau=1.0)
    outb, _, _ = orc.render(cube, lut, (0, 1), cam, step=step, tau=1.0, brick=brick)
    assert np.allclose(outb, out, atol=1e-12)
    o, d, _ = orc.rays(cam, shape, step=step)
    st = float(np.float32(step))                  # the lattice spacing the library is given
    checked = 0
    for p in range(20 * 18):
        tt = _slab64(o[p].astype(np.float64), d[p].astype(np.float64), shape)
        if tt is None:
            n = 0
        else:
            t0, t1 = tt
            if min(abs(t0 / st - round(t0 / st)), abs(t1 / st - round(t1 / st))) < 1e-3:
                continue
            n = max(0, math.ceil(t1 / st) - math.ceil(t0 / st))
        A = 1 - (1 - rgba[3]) ** n
        assert abs(out[p, 3] - A) < 1e-12
        checked += 1
    assert checked > 250
    # random values, bricked with early termination, against the brute-force sum
    nx, ny, nz = shape
    cube = rng.uniform(-1, 3, (nz, ny, nx)).astype(np.float32)
    lut = synth.random_lut(7, n=24, alpha_max=0.8)
    out, flags, _ = orc.render(cube, lut, (-1, 3), cam, step=step, tau=0.7, brick=brick)
    o, d, k = orc.rays(cam, shape, step=step)
    for p in range(0, 20 * 18, 3):
        seg = None
        if k[p, 1] > k[p, 0]:
            seg = [tuple(r) for r in orc.sample_owners(shape, cam, p, step, brick)]
        # the library's step is a binary32 parameter: 2.3 and 3.7 are not exact
        ref = _brute(cube, lut, (-1, 3), o[p], d[p], k[p, 0], k[p, 1], float(np.float32(step)), 0.7, seg)
        if flags[p] & 1:
            assert np.all(np.abs(out[p] - ref) <= 0.3 + 1e-9)
        else:
            assert np.allclose(out[p], ref, atol=1e-12), (p, out[p], ref)


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
            ref = _brute(cube, lut, (-1, 3), o[p], d[p], k[p, 0], k[p, 1], float(np.float32(step)), tau, seg)
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


# ---------------------------------------------------------------------------------------------
# wavelet block store (lossy compression of the cube kept in GPU memory)
# ---------------------------------------------------------------------------------------------
def _rec(store, i):
    r = store[544 * i: 544 * (i + 1)]
    return r[:512].view(np.int8), r[512:516].view(np.float32)[0], r[516:537].view(np.int8), r[537:]


def test_wavelet_constant_block(orc):
    """A constant block has no detail: every subband empty (-128), codes 0, average = value."""
    c = np.full((8, 8, 8), -7.375, np.float32)
    st = orc.wavelet_encode(c)
    codes, avg, e, pad = _rec(st, 0)
    assert st.size == 544 and avg == np.float32(-7.375)
    assert np.all(e == -128) and not codes.any() and not pad.any()
    assert np.array_equal(orc.wavelet_decode(st, c.shape), c)


@pytest.mark.parametrize("k", [5, -3])
def test_wavelet_delta_block_by_hand(orc, k):
    """A single voxel 2^k at (0,0,0): each Haar level halves it per axis, so level L leaves the
    value 2^(k - 3L) in every subband at the subband's first position, (bx, by, bz) * 8/2^L,
    and 2^(k-9) as the average.  The step is the smallest 2^e with 2^j <= 127 2^e: e = j - 6, so
    every code is 2^j / 2^(j-6) = 64 and the block decodes exactly."""
    x = np.zeros((8, 8, 8), np.float32)
    x[0, 0, 0] = 2.0 ** k
    st = orc.wavelet_encode(x)
    codes, avg, e, _ = _rec(st, 0)
    want = np.zeros(512, np.int8)
    want_e = np.zeros(21, np.int8)
    for L in (1, 2, 3):
        h = 8 >> L
        for sb in range(1, 8):
            bx, by, bz = sb & 1, (sb >> 1) & 1, sb >> 2
            want[bx * h + 8 * by * h + 64 * bz * h] = 64
            want_e[7 * (L - 1) + sb - 1] = (k - 3 * L) - 6
    assert np.array_equal(codes, want) and np.array_equal(e, want_e)
    assert avg == np.float32(2.0 ** (k - 9))
    assert np.array_equal(orc.wavelet_decode(st, x.shape), x)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_wavelet_linear_ramp_by_hand(orc, axis):
    """v = coordinate along one axis: level L's detail along that axis is -2^(L-2) everywhere in
    its subband (a difference of averages 2^(L-1) apart, halved), all other subbands are empty,
    the average is 3.5; steps 2^(L-8), codes -64; lossless."""
    g = np.arange(8, dtype=np.float32)
    x = np.broadcast_to(g.reshape([8 if a == 2 - axis else 1 for a in range(3)]), (8, 8, 8)).copy()
    st = orc.wavelet_encode(x)
    codes, avg, e, _ = _rec(st, 0)
    sb = 1 << axis
    for L in (1, 2, 3):
        for s in range(1, 8):
            assert e[7 * (L - 1) + s - 1] == ((L - 8) if s == sb else -128)
    assert avg == np.float32(3.5)
    assert set(np.unique(codes[1:]).tolist()) == {0, -64}
    assert (codes == -64).sum() == 64 + 8 + 1
    assert np.array_equal(orc.wavelet_decode(st, x.shape), x)


def test_wavelet_error_within_half_steps(orc):
    """Lossy bound: a voxel is the average plus, at each level, one coefficient of each of the
    7 subbands with sign +-1, so its error is at most the sum of half a step over the block's
    21 subbands, plus binary32 rounding in the 9 add/subtract stages (<= 9 ulp of 2 max|v|)."""
    rng = np.random.default_rng(12)
    shape = (19, 21, 27)                         # ragged: partial blocks on every axis
    x = (rng.standard_normal(shape) * 2.0).astype(np.float32)
    x[3:9, 4:12, 5:13] += 60.0 * rng.uniform(size=(6, 8, 8)).astype(np.float32)
    x[16:, :, :8] = 0.0                          # whole blocks of zeros: empty subbands
    st = orc.wavelet_encode(x)
    y = orc.wavelet_decode(st, x.shape)
    nb = ((27 + 7) // 8, (21 + 7) // 8, (19 + 7) // 8)
    worst = 0.0
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                i = bx + nb[0] * (by + nb[1] * bz)
                _, _, e, _ = _rec(st, i)
                bound = sum(2.0 ** (int(v) - 1) for v in e if v != -128)
                sl = np.s_[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
                m = float(np.abs(x[sl]).max())
                slack = 9 * 2.0 * m * 2.0 ** -23
                err = float(np.abs(y[sl].astype(np.float64) - x[sl]).max())
                assert err <= bound + slack, (bx, by, bz, err, bound)
                worst = max(worst, err / max(bound, 1e-30))
    assert 0.05 < worst <= 1.0 + 1e-6               # the bound is reached, not vacuous
    assert np.array_equal(y[16:, :, :8], x[16:, :, :8])   # an all-zero block decodes exactly


def test_wavelet_edge_blocks_repeat_the_border(orc):
    """Blocks that stick out of the cube see the edge voxels repeated: the store of a 13x11x9
    cube equals that of the same cube padded to 16x16x16 by edge replication."""
    rng = np.random.default_rng(13)
    x = rng.standard_normal((9, 11, 13)).astype(np.float32)
    pad = np.pad(x, ((0, 7), (0, 5), (0, 3)), mode="edge")
    assert np.array_equal(orc.wavelet_encode(x), orc.wavelet_encode(pad))
    assert np.array_equal(orc.wavelet_decode(orc.wavelet_encode(x), x.shape),
                          orc.wavelet_decode(orc.wavelet_encode(pad), pad.shape)[:9, :11, :13])


# ---------------------------------------------------------------------------------------------
# 16-bit bricks: a sample reads the voxels as stored in the brick that owns it
# ---------------------------------------------------------------------------------------------
def _ceil_log2(m):
    """ceil(log2 m) of a positive float from numpy's exact frexp (m = f 2^e, f in [0.5, 1))."""
    f, e = np.frexp(np.float64(m))
    return int(e) - 1 if f == 0.5 else int(e)


def _round16(x32, quant):
    """Round-to-nearest-even to binary16 (numpy cast) or bfloat16 (torch cast), as FP64."""
    x32 = np.asarray(x32, np.float32)
    if quant == "f16":
        with np.errstate(over="ignore"):
            return x32.astype(np.float16).astype(np.float64)
    torch = pytest.importorskip("torch")
    return torch.from_numpy(x32).to(torch.bfloat16).double().numpy()


def _brick_exp_np(cube, b, cell, quant):
    """The brick's scale exponent from numpy: max|v| over its core plus one ghost voxel per side
    (clamped to the cube); FP16 maps it to at most 2^14, BF16 to at most 1."""
    nz, ny, nx = cube.shape
    lo = [max(0, cell[a] * b[a] - 1) for a in range(3)]
    hi = [min((nx, ny, nz)[a], (cell[a] + 1) * b[a] + 1) for a in range(3)]
    m = float(np.abs(cube[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]).max())
    if m == 0.0:
        return 0
    return _ceil_log2(m) - 14 if quant == "f16" else _ceil_log2(m)


def _composite_np(rgba, tau, seg):
    """Front-to-back over with per-segment termination (seg: segment id of every sample)."""
    thr = float(np.float32(1.0) - np.float32(min(tau, 1.0)))
    C, T, Tseg, cur, stop = np.zeros(3), 1.0, 1.0, None, False
    for m in range(len(rgba)):
        if seg[m] != cur:
            cur, Tseg, stop = seg[m], 1.0, False
        if stop:
            continue
        a = rgba[m, 3]
        C += T * a * rgba[m, :3]
        T *= 1 - a
        Tseg *= 1 - a
        stop = Tseg <= thr
    return np.array([*C, 1 - T])


def _quant_brute(cube, lut, vrange, cam, step, tau, b, quant, owner_rule=True):
    """Every pixel of the frame from scipy trilinear interpolation of a copy of the cube rounded
    with the exponent of the brick that owns the sample (owner_rule) or, for comparison, with
    each voxel's home-brick exponent."""
    nz, ny, nx = cube.shape
    shape = (nx, ny, nz)
    nb = [-(-shape[a] // b[a]) for a in range(3)]
    exps = {}
    for cz in range(nb[2]):
        for cy in range(nb[1]):
            for cx in range(nb[0]):
                exps[(cx, cy, cz)] = _brick_exp_np(cube, b, (cx, cy, cz), quant)
    rounded = {}

    def at_exp(e):
        if e not in rounded:
            rounded[e] = np.ldexp(_round16(np.ldexp(cube, -e).astype(np.float32), quant), e)
        return rounded[e]

    if not owner_rule:
        z, y, x = np.meshgrid(np.arange(nz) // b[2], np.arange(ny) // b[1], np.arange(nx) // b[0],
                              indexing="ij")
        home = np.empty(cube.shape, np.float64)
        for (cx, cy, cz), e in exps.items():
            sel = (x == cx) & (y == cy) & (z == cz)
            home[sel] = at_exp(e)[sel]
    o, d, k = orc_rays_cached(cam, shape, step)
    out = np.zeros((cam["W"] * cam["H"], 4))
    for p in range(len(out)):
        if k[p, 1] <= k[p, 0]:
            continue
        ks = np.arange(k[p, 0], k[p, 1])
        own = ORC.sample_owners(shape, cam, p, step, b)
        pos = o[p].astype(np.float64)[None, :] + (ks[:, None] * float(step)) * d[p].astype(np.float64)
        coords = np.stack([pos[:, 2] - 0.5, pos[:, 1] - 0.5, pos[:, 0] - 0.5])
        v = np.empty(len(ks))
        for m in range(len(ks)):
            src = at_exp(exps[tuple(int(c) for c in own[m])]) if owner_rule else home
            v[m] = map_coordinates(src, coords[:, m:m + 1], order=1, mode="nearest")[0]
        u = np.clip((v - vrange[0]) / (vrange[1] - vrange[0]), 0, 1) * (len(lut) - 1)
        rgba = np.stack([np.interp(u, np.arange(len(lut)), lut[:, c].astype(np.float64))
                         for c in range(4)], 1)
        out[p] = _composite_np(rgba, tau, [tuple(r) for r in own])
    return out


ORC = None


def orc_rays_cached(cam, shape, step):
    return ORC.rays(cam, shape, step=step)


@pytest.mark.parametrize("quant", ["f16", "bf16"])
def test_16bit_samples_read_the_owner_bricks_copy(orc, quant):
    """Reading 10 (16-bit storage): a sample reads the 8 voxels of its stencil as stored in the
    brick that owns it, ghost copies included, each rounded with that brick's exponent.  Two
    bricks along x; brick 1 holds one bright voxel away from the shared face, so its exponent
    is 2 (FP16 codes of its faint voxels are subnormal), brick 0's is -29: the face voxels x = 7
    and x = 8 round differently in the two copies.  The oracle equals the owner-rule reference
    and (FP16) differs from the home-brick rule."""
    global ORC
    ORC = orc
    rng = np.random.default_rng(21)
    nx, ny, nz = 16, 6, 5
    cube = (rng.uniform(-3e-5, 3e-5, (nz, ny, nx))).astype(np.float32)
    cube[2, 3, 13] = 60000.0
    b = (8, 8, 8)
    assert _brick_exp_np(cube, b, (1, 0, 0), "f16") == 2
    assert _brick_exp_np(cube, b, (0, 0, 0), "f16") == -29
    lut = synth.random_lut(4, n=24, alpha_max=0.3)
    vr = (-2.0 ** -15, 2.0 ** -15)           # binary32 values (the table range is binary32)
    e_home = e_owner = 0.0
    for trial in range(3):
        cam = synth.random_camera(rng, (nx, ny, nz), 12, 9)
        out, flags, _ = orc.render(cube, lut, vr, cam, step=0.5, tau=0.97, brick=b, quant=quant)
        ref = _quant_brute(cube, lut, vr, cam, 0.5, 0.97, b, quant)
        ok = (flags & 1) == 0
        assert ok.sum() > 40
        e_owner = max(e_owner, float(np.abs(out[ok] - ref[ok]).max()))
        if quant == "f16":
            alt = _quant_brute(cube, lut, vr, cam, 0.5, 0.97, b, quant, owner_rule=False)
            e_home = max(e_home, float(np.abs(out[ok] - alt[ok]).max()))
    assert e_owner < 1e-12
    if quant == "f16":
        assert e_home > 1e-4       # the home-brick rule is a different image: the pin can tell


# ---------------------------------------------------------------------------------------------
# FP32-order MIP at non-zero fractions
# ---------------------------------------------------------------------------------------------
def test_mip32_single_sample_by_hand(orc):
    """Reading 9: one sample at p = (1.25, 1.0, 1.25) of a 2x2x2 cube (fractions 0.75, 0.5, 0.75),
    interpolated as a + f (b - a) along x, then y, then z, each operation rounded to binary32.
    Values chosen so that other orders (z first, or b + (1 - f)(a - b)) round differently."""
    cube = np.array([1.0 / 3, 7.1, -2.3, 1e3 + 1.0 / 7,
                     0.3, -5.0 / 3, 11.0 / 13, 2.0 ** -9 + 3.0], np.float32)
    c = cube.reshape(2, 2, 2)                       # [z][y][x]
    view = synth.look_at((1.25, 1.0, -8.75), (1.25, 1.0, 0.0))
    cam = dict(view=view, proj=0, param=1.0, W=1, H=1)
    o, d, k = orc.rays(cam, (2, 2, 2), step=10.0)
    assert o[0].tolist() == [1.25, 1.0, -8.75] and d[0].tolist() == [0.0, 0.0, 1.0]
    assert k[0].tolist() == [1, 2]                  # t = 10: p = (1.25, 1.0, 1.25)
    f32 = np.float32
    fx, fy, fz = f32(0.75), f32(0.5), f32(0.75)

    def lerp(a, b, f):
        return f32(f32(a) + f32(f32(f) * f32(f32(b) - f32(a))))

    x00 = lerp(c[0, 0, 0], c[0, 0, 1], fx)
    x10 = lerp(c[0, 1, 0], c[0, 1, 1], fx)
    x01 = lerp(c[1, 0, 0], c[1, 0, 1], fx)
    x11 = lerp(c[1, 1, 0], c[1, 1, 1], fx)
    expect = lerp(lerp(x00, x10, fy), lerp(x01, x11, fy), fz)
    z_first = lerp(lerp(lerp(c[0, 0, 0], c[1, 0, 0], fz), lerp(c[0, 1, 0], c[1, 1, 0], fz), fy),
                   lerp(lerp(c[0, 0, 1], c[1, 0, 1], fz), lerp(c[0, 1, 1], c[1, 1, 1], fz), fy), fx)

    def lerp_rev(a, b, f):
        return f32(f32(b) + f32(f32(f32(1) - f32(f)) * f32(f32(a) - f32(b))))

    rev = lerp_rev(lerp_rev(lerp_rev(c[0, 0, 0], c[0, 0, 1], fx), lerp_rev(c[0, 1, 0], c[0, 1, 1], fx), fy),
                   lerp_rev(lerp_rev(c[1, 0, 0], c[1, 0, 1], fx), lerp_rev(c[1, 1, 0], c[1, 1, 1], fx), fy), fz)
    assert expect != z_first and expect != rev
    m32, _, _ = orc.render(cube.reshape(2, 2, 2), synth.ramp_lut(), (-3, 20), cam, mode="mip32", step=10.0)
    assert np.float32(m32[0]) == expect
    # the FP64 MIP of the same sample: the trilinear weights written out
    w = np.array([(1 - 0.75) * (1 - 0.5) * (1 - 0.75), 0.75 * 0.5 * 0.25, 0.25 * 0.5 * 0.25,
                  0.75 * 0.5 * 0.25, 0.25 * 0.5 * 0.75, 0.75 * 0.5 * 0.75, 0.25 * 0.5 * 0.75,
                  0.75 * 0.5 * 0.75])
    w[1] = 0.75 * (1 - 0.5) * (1 - 0.75)
    m64, _, _ = orc.render(cube.reshape(2, 2, 2), synth.ramp_lut(), (-3, 20), cam, mode="mip", step=10.0)
    assert abs(m64[0] - float(w @ cube.astype(np.float64))) < 1e-12


def test_mip32_equals_fp64_mip_to_rounding_at_random_views(orc):
    """On random views every fraction is non-zero; the FP32-order MIP stays within FP32 rounding
    of the FP64 MIP (a swapped weight or lerp would be off by O(1) of the data range)."""
    rng = np.random.default_rng(31)
    cube = rng.uniform(-1, 3, (11, 9, 13)).astype(np.float32)
    shape = (13, 9, 11)
    worst = 0.0
    for _ in range(4):
        cam = synth.random_camera(rng, shape, 16, 14)
        step = float(rng.choice([0.37, 0.5, 0.71]))
        m64, f, _ = orc.render(cube, synth.ramp_lut(), (-1, 3), cam, mode="mip", step=step, brick=(5, 4, 6))
        m32, _, _ = orc.render(cube, synth.ramp_lut(), (-1, 3), cam, mode="mip32", step=step, brick=(5, 4, 6))
        hit = (f & 2) == 0
        assert hit.sum() > 40
        worst = max(worst, float(np.abs(m32[hit] - m64[hit]).max()))
    # positions rounded to binary32 (|p| < 40: 4e-6) times a slope below 4 per voxel, plus
    # 7 lerps of values below 3 rounded to binary32
    assert worst < 3e-5


def test_piece_signature_changes_exactly_across_piece_boundaries(orc):
    """render_sig's per-pixel hash: a constant cube on a table entry moved by +-h lands in two
    different intervals (signatures differ); half-way between entries they are equal, and equal
    to the unmoved cube's; a change of the termination stop (more opacity) changes it."""
    rng = np.random.default_rng(8)
    shape = (7, 6, 9)
    lut = synth.random_lut(2, n=32, alpha_max=0.2)
    cam = synth.random_camera(rng, shape, 16, 12)
    vr = (-3.0, 8.0)
    on = -3.0 + 11.0 * 10.0 / 31.0
    half = -3.0 + 11.0 * 10.5 / 31.0
    sig = {}
    for name, v in (("on+", on + 1e-3), ("on-", on - 1e-3), ("half", half), ("half+", half + 1e-3),
                    ("half-", half - 1e-3)):
        _, f, _, s = orc.render_sig(synth.constant_cube(shape, v), lut, vr, cam, step=0.5, tau=1.0)
        sig[name] = s
    hit = (f & 2) == 0
    assert hit.sum() > 30
    assert np.all(sig["on+"][hit] != sig["on-"][hit])
    assert np.array_equal(sig["half"], sig["half+"]) and np.array_equal(sig["half"], sig["half-"])
    # termination: an opaque table stops every segment early, a faint one never
    _, _, n1, s1 = orc.render_sig(synth.constant_cube(shape, half), synth.constant_lut([1, 1, 1, 0.6], 32),
                                  vr, cam, step=0.5, tau=0.9)
    _, _, n2, s2 = orc.render_sig(synth.constant_cube(shape, half), synth.constant_lut([1, 1, 1, 0.01], 32),
                                  vr, cam, step=0.5, tau=0.9)
    # (rays with only a few samples stop nowhere in either)
    assert n1 < n2 and np.mean(s1[hit] != s2[hit]) > 0.5
