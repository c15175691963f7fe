"""ctypes wrapper of the FP64 CPU oracle (``vr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  The renderer never imports it, and it imports nothing from the
renderer.  ``build()`` compiles the C file with gcc into ``liborc.so`` beside it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle (plain C, OpenMP over pixels, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-std=gnu11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Args(C.Structure):
    _fields_ = [
        ("vox", C.c_void_p), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("lut", C.c_void_p), ("nlut", C.c_int32), ("vmin", C.c_float), ("vmax", C.c_float),
        ("view", C.c_float * 16), ("proj", C.c_int32), ("param", C.c_float),
        ("W", C.c_int32), ("H", C.c_int32), ("mode", C.c_int32), ("step", C.c_float),
        ("tau", C.c_float), ("bx", C.c_int64), ("by", C.c_int64), ("bz", C.c_int64),
        ("quant", C.c_int32), ("ghost", C.c_int32), ("nthreads", C.c_int32),
        ("procedural", C.c_int32), ("proc_seed", C.c_uint64),
        ("channels", C.c_void_p), ("win_lo", C.c_int64 * 3), ("win_hi", C.c_int64 * 3),
        ("term_global", C.c_int32), ("sig", C.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        L.orc_render.argtypes = [P(Args), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                 P(C.c_int64)]
        L.orc_render_grad.argtypes = [P(Args), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
        L.orc_rays.argtypes = [P(Args), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                               C.c_void_p]
        L.orc_sample_owners.argtypes = [P(Args), C.c_int64, C.c_void_p, C.c_int64]
        L.orc_sample_owners.restype = C.c_int64
        L.orc_round_fp16.argtypes = [C.c_float]
        L.orc_round_fp16.restype = C.c_float
        L.orc_round_bf16.argtypes = [C.c_float]
        L.orc_round_bf16.restype = C.c_float
        L.orc_scale_exponent.argtypes = [C.c_float, C.c_int]
        L.orc_brick_exponents.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                          C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int,
                                          C.c_void_p]
        L.orc_minmax.argtypes = [C.c_void_p, C.c_int64, P(C.c_float), P(C.c_float)]
        L.orc_proc_voxel.argtypes = [C.c_uint64] + [C.c_int64] * 6
        L.orc_proc_voxel.restype = C.c_float
        L.orc_proc_noise.argtypes = [C.c_uint64] + [C.c_int64] * 5
        L.orc_proc_noise.restype = C.c_double
        L.orc_proc_region.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                      C.c_void_p, C.c_void_p]
        L.orc_wavelet_bytes.argtypes = [C.c_int64] * 3
        L.orc_wavelet_bytes.restype = C.c_int64
        L.orc_wavelet_encode.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p]
        L.orc_wavelet_decode.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p]
        _lib = L
    return _lib


MODES = {"dvr": 0, "mip": 1, "mip32": 2}
QUANT = {"f32": 0, "f16": 1, "bf16": 2}


class Procedural:
    """The procedural cube of a seed and a size (voxels evaluated on demand)."""

    def __init__(self, seed: int, shape_xyz):
        self.seed = int(seed)
        self.shape_xyz = tuple(int(v) for v in shape_xyz)


TERM = {"segment": 0, "global": 1}


def _args(cube, lut, vrange, cam, mode="dvr", step=0.5, tau=0.99, brick=None, quant="f32",
          ghost=1, nthreads=0, channels=None, window=None, term="segment"):
    lut = np.ascontiguousarray(lut, dtype=np.float32)
    a = Args()
    a.term_global = TERM[term]
    if isinstance(cube, Procedural):
        nx, ny, nz = cube.shape_xyz
        a.vox = None
        a.procedural, a.proc_seed = 1, cube.seed
    else:
        cube = np.ascontiguousarray(cube, dtype=np.float32)
        nz, ny, nx = cube.shape
        a.vox = cube.ctypes.data
    a.nx, a.ny, a.nz = nx, ny, nz
    a.lut = lut.ctypes.data
    a.nlut = lut.shape[0]
    a.vmin, a.vmax = float(vrange[0]), float(vrange[1])
    view = np.ascontiguousarray(cam["view"], dtype=np.float32).reshape(16)
    for i in range(16):
        a.view[i] = float(view[i])
    a.proj, a.param, a.W, a.H = int(cam["proj"]), float(cam["param"]), int(cam["W"]), int(cam["H"])
    a.mode = MODES[mode]
    a.step, a.tau = float(step), float(tau)
    b = brick or (0, 0, 0)
    a.bx, a.by, a.bz = int(b[0]), int(b[1]), int(b[2])
    a.quant = QUANT[quant]
    a.ghost = int(ghost)
    a.nthreads = int(nthreads)
    ch = None
    if channels is not None:
        ch = np.ascontiguousarray(channels, dtype=np.uint8)
        a.channels = ch.ctypes.data
    if window is not None:
        for i in range(3):
            a.win_lo[i], a.win_hi[i] = int(window[0][i]), int(window[1][i])
    return a, (cube, lut, ch)  # keep the arrays alive


def _pix(pix):
    if pix is None:
        return None, None
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    return pix, pix.ctypes.data


def render(cube, lut, vrange, cam, mode="dvr", step=0.5, tau=0.99, brick=None, quant="f32",
           pix=None, ghost=1, nthreads=0, channels=None, window=None, term="segment"):
    """Returns (out, flags, nsamples).  out: (npix, 4) premultiplied RGBA for DVR, (npix,) for
    MIP; float64.  pix: flat pixel indices (row*W + col) or None for the whole frame.
    channels: per-z 0/1 enable mask; window: ((x0,y0,z0), (x1,y1,z1)) voxel box.
    term: DVR early termination per brick segment ("segment") or of the whole ray ("global";
    the bricking then only sets the 16-bit scales).
    flags per pixel: bit 0 early-termination decision within 2e-4 (relative) of the threshold,
    bit 1 no samples, bit 2 broken sample partition (never expected), bit 3 a composited DVR
    sample's table coordinate within 1e-4 of a table entry (the image's derivative with respect
    to that sample's value jumps there)."""
    out, flags, ns, _ = _render(cube, lut, vrange, cam, mode, step, tau, brick, quant, pix, ghost,
                                nthreads, channels, window, term, False)
    return out, flags, ns


def render_sig(cube, lut, vrange, cam, step=0.5, tau=0.99, brick=None, pix=None, channels=None,
               window=None):
    """DVR render plus, per pixel, a uint64 hash of its piecewise structure: the table interval
    (or clamp side) of every composited sample and the number of composited samples.  Two inputs
    with equal hashes at every pixel lie, almost surely, in one piece of the image as a function
    of the table and the voxels (no table entry, clamp edge or termination stop between them).
    Returns (out, flags, nsamples, sig)."""
    return _render(cube, lut, vrange, cam, "dvr", step, tau, brick, "f32", pix, 1, 0, channels,
                   window, "segment", True)


def _render(cube, lut, vrange, cam, mode, step, tau, brick, quant, pix, ghost, nthreads, channels,
            window, term, want_sig):
    a, keep = _args(cube, lut, vrange, cam, mode, step, tau, brick, quant, ghost, nthreads,
                    channels, window, term)
    pixa, pp = _pix(pix)
    npix = cam["W"] * cam["H"] if pix is None else len(pixa)
    stride = 4 if mode == "dvr" else 1
    out = np.zeros((npix, stride), np.float64)
    flags = np.zeros(npix, np.uint8)
    sig = np.zeros(npix, np.uint64) if want_sig else None
    if want_sig:
        a.sig = sig.ctypes.data
    ns = C.c_int64(0)
    rc = lib().orc_render(C.byref(a), pp, npix, out.ctypes.data, flags.ctypes.data, C.byref(ns))
    if rc != 0:
        raise ValueError(f"orc_render failed ({rc})")
    del keep
    return (out if stride == 4 else out[:, 0]), flags, int(ns.value), sig


def proc_region(seed, shape_xyz, lo, dim):
    """Voxels [z][y][x] of the procedural cube in the box [lo, lo+dim) (coordinates clamped)."""
    lo = np.ascontiguousarray(lo, dtype=np.int64)
    dim = np.ascontiguousarray(dim, dtype=np.int64)
    out = np.zeros((int(dim[2]), int(dim[1]), int(dim[0])), np.float32)
    nx, ny, nz = shape_xyz
    lib().orc_proc_region(int(seed), nx, ny, nz, lo.ctypes.data, dim.ctypes.data, out.ctypes.data)
    return out


def proc_noise(seed, shape_xyz, x, y, z) -> float:
    nx, ny, nz = shape_xyz
    return float(lib().orc_proc_noise(int(seed), nx, ny, int(x), int(y), int(z)))


def proc_voxel(seed, shape_xyz, x, y, z) -> float:
    nx, ny, nz = shape_xyz
    return float(lib().orc_proc_voxel(int(seed), nx, ny, nz, int(x), int(y), int(z)))


def render_grad(cube, lut, vrange, cam, gout, step=0.5, tau=0.99, brick=None, pix=None,
                want_vox=True, channels=None, window=None):
    """Gradient of sum(gout * out) w.r.t. (lut, cube) in FP64; DVR only."""
    a, keep = _args(cube, lut, vrange, cam, "dvr", step, tau, brick, "f32", channels=channels,
                    window=window)
    pixa, pp = _pix(pix)
    npix = cam["W"] * cam["H"] if pix is None else len(pixa)
    g = np.ascontiguousarray(gout, dtype=np.float64).reshape(npix, 4)
    glut = np.zeros((a.nlut, 4), np.float64)
    gvox = np.zeros(np.asarray(cube).shape, np.float64) if want_vox else None
    rc = lib().orc_render_grad(C.byref(a), pp, npix, g.ctypes.data, glut.ctypes.data,
                               gvox.ctypes.data if want_vox else None)
    if rc != 0:
        raise ValueError(f"orc_render_grad failed ({rc})")
    del keep
    return glut, gvox


def rays(cam, shape_xyz, step=0.5, pix=None):
    """FP32 rays (o, d) and lattice range k=(k0,k1) of the listed pixels."""
    nx, ny, nz = shape_xyz
    dummy = np.zeros((1, 1, 1), np.float32)
    lut = np.zeros((2, 4), np.float32)
    a, keep = _args(dummy, lut, (0, 1), cam, step=step)
    a.nx, a.ny, a.nz = nx, ny, nz
    pixa, pp = _pix(pix)
    npix = cam["W"] * cam["H"] if pix is None else len(pixa)
    o = np.zeros((npix, 3), np.float32)
    d = np.zeros((npix, 3), np.float32)
    k = np.zeros((npix, 2), np.int64)
    lib().orc_rays(C.byref(a), pp, npix, o.ctypes.data, d.ctypes.data, k.ctypes.data)
    del keep
    return o, d, k


def sample_owners(cube_shape_xyz, cam, pixel, step, brick):
    nx, ny, nz = cube_shape_xyz
    dummy = np.zeros((1, 1, 1), np.float32)
    lut = np.zeros((2, 4), np.float32)
    a, keep = _args(dummy, lut, (0, 1), cam, step=step, brick=brick)
    a.nx, a.ny, a.nz = nx, ny, nz
    cap = 4 * (nx + ny + nz) * int(2 / step + 2)
    own = np.zeros((cap, 3), np.int64)
    n = lib().orc_sample_owners(C.byref(a), int(pixel), own.ctypes.data, cap)
    del keep
    return own[:n]


def round_fp16(x):
    f = lib().orc_round_fp16
    return np.array([f(float(v)) for v in np.asarray(x, np.float32).ravel()], np.float32)


def round_bf16(x):
    f = lib().orc_round_bf16
    return np.array([f(float(v)) for v in np.asarray(x, np.float32).ravel()], np.float32)


def scale_exponent(maxabs: float, quant: str) -> int:
    return int(lib().orc_scale_exponent(float(maxabs), QUANT[quant]))


def brick_exponents(cube, brick, ghost, quant):
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    nz, ny, nx = cube.shape
    bx, by, bz = brick
    nb = (-(-nx // bx), -(-ny // by), -(-nz // bz))
    e = np.zeros(nb[0] * nb[1] * nb[2], np.int32)
    lib().orc_brick_exponents(cube.ctypes.data, nx, ny, nz, bx, by, bz, ghost, QUANT[quant],
                              e.ctypes.data)
    return e.reshape(nb[2], nb[1], nb[0])


def quantize(cube, exps_zyx, brick, quant):
    """Codes (as float) of every voxel as stored in its own core brick (no ghost)."""
    cube = np.asarray(cube, np.float32)
    bx, by, bz = brick
    nz, ny, nx = cube.shape
    z, y, x = np.meshgrid(np.arange(nz) // bz, np.arange(ny) // by, np.arange(nx) // bx,
                          indexing="ij")
    e = exps_zyx[z, y, x].astype(np.int32)
    scaled = np.ldexp(cube, -e).astype(np.float32)
    r = round_fp16(scaled) if quant == "f16" else round_bf16(scaled)
    return r.reshape(cube.shape), e


def minmax(v):
    v = np.ascontiguousarray(v, dtype=np.float32).ravel()
    lo, hi = C.c_float(0), C.c_float(0)
    lib().orc_minmax(v.ctypes.data, v.size, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


WAVELET_RECORD = 544


def wavelet_encode(cube):
    """The 8-bit Haar-wavelet block store of a [z][y][x] FP32 cube (544 bytes per 8^3 block,
    x-fastest block order; format in ``orc_wavelet_encode``)."""
    cube = np.ascontiguousarray(cube, dtype=np.float32)
    nz, ny, nx = cube.shape
    out = np.zeros(int(lib().orc_wavelet_bytes(nx, ny, nz)), np.uint8)
    lib().orc_wavelet_encode(cube.ctypes.data, nx, ny, nz, out.ctypes.data)
    return out


def wavelet_decode(store, shape_zyx):
    """The FP32 cube a block store decodes to."""
    store = np.ascontiguousarray(store, dtype=np.uint8)
    nz, ny, nx = shape_zyx
    assert store.size == int(lib().orc_wavelet_bytes(nx, ny, nz))
    out = np.zeros((nz, ny, nx), np.float32)
    lib().orc_wavelet_decode(store.ctypes.data, nx, ny, nz, out.ctypes.data)
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())
