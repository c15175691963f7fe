"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the rendering method: it only draws cubes, transfer-function
tables, view matrices, pixel samples and request streams from fixed seeds.  Both sides of every
parity check receive the arrays produced here; neither side's arithmetic lives here.

Shapes follow the datasets of the paper (Table 3: HIPASS 1721x1721x1024, GASS 2502x2501x1093),
which are not available; the generators stand in for them:

* ``pr1_cube``     64^3, N(0,1) background + 8 Gaussian sources (sigma 2-6, amplitude 5-20).
* ``diff_cube``    256^3, the same recipe with sigma scaled 4x (seed 3).
* ``hipass_cube``  1720x1720x1024 (x, y, z), N(0,1) + 20 000 sources elongated along the spectral
                   axis ("short bars", Section 1.2) with log-uniform amplitude 3-100, plus a
                   smooth band of emission at z in [480, 544].
* ``gass_cube``    2048x2048x1600, N(0, 0.5) + a Gaussian random field with power spectrum
                   P(k) ~ k^-3 confined to a 200-voxel slab (z in [700, 900)).

Cubes are stored ``[z][y][x]`` (x fastest), float32.  Voxel (x, y, z) sits at world position
(x+0.5, y+0.5, z+0.5); the volume box is [0,nx] x [0,ny] x [0,nz].
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "pr1_cube", "diff_cube", "hipass_cube", "gass_cube", "constant_cube", "linear_cube",
    "ramp_lut", "shifted_ramp_lut", "constant_lut", "random_lut",
    "look_at", "orbit_view", "pr1_camera", "axis_ortho_camera", "random_camera",
    "sample_pixels", "poisson_arrivals",
    "PR1", "HIPASS", "HIPASS_SMALL", "HIPASS_SLAB", "GASS", "GASS_SLAB", "DIFF", "orbit_camera",
]

# ----------------------------------------------------------------------------------------------
# workload descriptions (sizes from the configs the method is measured on)
# ----------------------------------------------------------------------------------------------
PR1 = dict(name="PR1 64^3", shape=(64, 64, 64), seed=0, W=256, H=256, step=0.5, tau=0.99,
           vrange=(-3.0, 20.0), brick=(32, 32, 32), ghost=1)
HIPASS = dict(name="HIPASS-scale 1720x1720x1024", shape=(1720, 1720, 1024), seed=1, W=1024,
              H=1024, step=1.0, tau=0.99, vrange=(-3.0, 100.0), brick=(256, 256, 256), ghost=1,
              n_views=64, fov_deg=60.0, eye_factor=1.5)
# the HIPASS recipe at 768x768x512 (1.2 GB, still above L2): the case hardware counters are
# captured on (a full-size capture would replay a 12 GB working set dozens of times)
HIPASS_SMALL = dict(HIPASS, name="HIPASS-recipe 768x768x512", shape=(768, 768, 512), n_sources=1000)
# the HIPASS recipe 256 channels deep (3.0 GB): the full cube's sky extent, so its rays are as
# far apart as the full frame's (the case the sparse-ray counters are captured on)
HIPASS_SLAB = dict(HIPASS, name="HIPASS-recipe 1720x1720x256", shape=(1720, 1720, 256), n_sources=5000)
GASS = dict(name="GASS-scale 2048x2048x1600", shape=(2048, 2048, 1600), seed=2, W=1024,
            H=1024, step=0.5, tau=0.99, vrange=(-2.0, 8.0), brick=(256, 256, 256), ghost=1,
            n_views=64, fov_deg=60.0, eye_factor=1.5)
# the GASS recipe 256 channels deep (4.3 GB): the full cube's sky extent with its 200-voxel
# emission slab, so its rays are as far apart and its bricks as varied as the full frame's
# (the case DRAM counters of GASS frames are captured on)
GASS_SLAB = dict(GASS, name="GASS-recipe 2048x2048x256", shape=(2048, 2048, 256), slab=(28, 228))
DIFF = dict(name="Diff 256^3", shape=(256, 256, 256), seed=3, W=512, H=512, step=0.5, tau=0.99,
            vrange=(-3.0, 20.0), brick=(128, 128, 128), ghost=1, n_views=8)


def _gauss_sources_np(shape_xyz, rng, n_src, sigma_rng, amp_rng, cube):
    nx, ny, nz = shape_xyz
    xs = np.arange(nx, dtype=np.float64) + 0.5
    ys = np.arange(ny, dtype=np.float64) + 0.5
    zs = np.arange(nz, dtype=np.float64) + 0.5
    for _ in range(n_src):
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        sig = rng.uniform(*sigma_rng)
        amp = rng.uniform(*amp_rng)
        gx = np.exp(-((xs - cx) ** 2) / (2 * sig * sig))
        gy = np.exp(-((ys - cy) ** 2) / (2 * sig * sig))
        gz = np.exp(-((zs - cz) ** 2) / (2 * sig * sig))
        cube += (amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).astype(cube.dtype)
    return cube


def pr1_cube(seed: int = 0, n: int = 64, n_sources: int = 8, sigma=(2.0, 6.0),
             amp=(5.0, 20.0)) -> np.ndarray:
    """64^3 N(0,1) background plus Gaussian sources (uniform centres). Returns [z][y][x] f32."""
    rng = np.random.default_rng(seed)
    cube = rng.standard_normal((n, n, n), dtype=np.float32)
    return _gauss_sources_np((n, n, n), rng, n_sources, sigma, amp, cube)


def diff_cube(seed: int = 3, n: int = 256) -> np.ndarray:
    """The PR1 recipe at n^3 with the source widths scaled by n/64."""
    s = n / 64.0
    return pr1_cube(seed=seed, n=n, n_sources=8, sigma=(2.0 * s, 6.0 * s))


def constant_cube(shape_xyz, value: float) -> np.ndarray:
    nx, ny, nz = shape_xyz
    return np.full((nz, ny, nx), value, dtype=np.float32)


def linear_cube(shape_xyz, coef=(0.25, -0.5, 0.125), offset=1.0) -> np.ndarray:
    """Voxel (x,y,z) holds a*(x+.5) + b*(y+.5) + c*(z+.5) + offset, rounded to float32."""
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    return (coef[0] * x + coef[1] * y + coef[2] * z + offset).astype(np.float32)


def _torch_gen(device, seed):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _splat_sources_torch(cube, cx, cy, cz, sxy, sz, amp, chunk=512):
    """Adds amp*exp(-r^2/2) (anisotropic sigma) inside +-3 sigma boxes, in chunks of sources."""
    import torch
    nz, ny, nx = cube.shape
    dev = cube.device
    flat = cube.view(-1)
    rxy = int(math.ceil(3 * float(sxy.max())))
    rz = int(math.ceil(3 * float(sz.max())))
    oxy = torch.arange(-rxy, rxy + 1, device=dev)
    oz = torch.arange(-rz, rz + 1, device=dev)
    for s0 in range(0, cx.numel(), chunk):
        sl = slice(s0, s0 + chunk)
        ix = torch.floor(cx[sl]).long()[:, None] + oxy[None, :]          # (c, bx)
        iy = torch.floor(cy[sl]).long()[:, None] + oxy[None, :]
        iz = torch.floor(cz[sl]).long()[:, None] + oz[None, :]
        gx = torch.exp(-((ix.double() + 0.5 - cx[sl, None]) ** 2) / (2 * sxy[sl, None] ** 2))
        gy = torch.exp(-((iy.double() + 0.5 - cy[sl, None]) ** 2) / (2 * sxy[sl, None] ** 2))
        gz = torch.exp(-((iz.double() + 0.5 - cz[sl, None]) ** 2) / (2 * sz[sl, None] ** 2))
        gx = torch.where((ix >= 0) & (ix < nx), gx, torch.zeros_like(gx))
        gy = torch.where((iy >= 0) & (iy < ny), gy, torch.zeros_like(gy))
        gz = torch.where((iz >= 0) & (iz < nz), gz, torch.zeros_like(gz))
        val = (amp[sl, None, None, None] * gz[:, :, None, None] * gy[:, None, :, None]
               * gx[:, None, None, :]).float()
        idx = ((iz.clamp(0, nz - 1)[:, :, None, None] * ny
                + iy.clamp(0, ny - 1)[:, None, :, None]) * nx
               + ix.clamp(0, nx - 1)[:, None, None, :])
        flat.index_put_((idx.reshape(-1),), val.reshape(-1), accumulate=True)
        del val, idx


def hipass_cube(seed: int = 1, shape_xyz=(1720, 1720, 1024), n_sources: int = 20000,
                device: str = "cuda"):
    """HIPASS-shaped cube (torch tensor on ``device``): N(0,1) + bar-like sources + a band."""
    import torch
    nx, ny, nz = shape_xyz
    g = _torch_gen(device, seed)
    cube = torch.randn((nz, ny, nx), generator=g, device=device, dtype=torch.float32)
    u = torch.rand((6, n_sources), generator=g, device=device, dtype=torch.float64)
    cx, cy, cz = u[0] * nx, u[1] * ny, u[2] * nz
    sxy = 1.0 + 3.0 * u[3]                       # sigma on the sky axes in [1, 4]
    sz = sxy * (2.0 + 3.0 * u[4])                # elongated along the spectral axis
    amp = torch.exp(math.log(3.0) + (math.log(100.0) - math.log(3.0)) * u[5])
    _splat_sources_torch(cube, cx, cy, cz, sxy, sz, amp)
    zc = torch.arange(nz, device=device, dtype=torch.float64) + 0.5
    band = (2.0 * torch.exp(-((zc - 512.0) ** 2) / (2 * 16.0 ** 2))).float()
    cube += band[:, None, None]
    return cube


def gass_cube(seed: int = 2, shape_xyz=(2048, 2048, 1600), slab=(700, 900), amp: float = 2.0,
              device: str = "cuda"):
    """GASS-shaped cube: N(0, 0.5) + a power-law (k^-3) Gaussian random field in a z-slab."""
    import torch
    nx, ny, nz = shape_xyz
    g = _torch_gen(device, seed)
    cube = torch.randn((nz, ny, nx), generator=g, device=device, dtype=torch.float32)
    cube *= 0.5
    z0, z1 = slab
    tz = z1 - z0
    white = torch.randn((tz, ny, nx), generator=g, device=device, dtype=torch.float32)
    f = torch.fft.rfftn(white)
    del white
    kz = torch.fft.fftfreq(tz, device=device)[:, None, None]
    ky = torch.fft.fftfreq(ny, device=device)[None, :, None]
    kx = torch.fft.rfftfreq(nx, device=device)[None, None, :]
    k = torch.sqrt(kz * kz + ky * ky + kx * kx)
    k[0, 0, 0] = 1.0
    f *= k.pow(-1.5)                             # amplitude ~ sqrt(P(k)), P ~ k^-3
    f[0, 0, 0] = 0
    del k
    grf = torch.fft.irfftn(f, s=(tz, ny, nx))
    del f
    grf = grf / grf.std()
    w = torch.ones(tz, device=device)
    taper = 20
    ramp = 0.5 - 0.5 * torch.cos(math.pi * (torch.arange(taper, device=device) + 0.5) / taper)
    w[:taper] = ramp
    w[-taper:] = ramp.flip(0)
    cube[z0:z1] += amp * grf * w[:, None, None]
    return cube


# ----------------------------------------------------------------------------------------------
# transfer-function tables (N x 4 RGBA, non-premultiplied)
# ----------------------------------------------------------------------------------------------
def ramp_lut(n: int = 256, alpha: float = 0.1) -> np.ndarray:
    t = np.arange(n, dtype=np.float64) / (n - 1)
    return np.stack([t, t, t, alpha * t], axis=1).astype(np.float32)


def shifted_ramp_lut(n: int = 256, shift: float = 3.0, vrange=(-3.0, 20.0),
                     alpha: float = 0.1) -> np.ndarray:
    """The ramp moved by ``shift`` data units (the target table of the differentiation config)."""
    v = vrange[0] + np.arange(n, dtype=np.float64) / (n - 1) * (vrange[1] - vrange[0])
    t = np.clip((v - shift - vrange[0]) / (vrange[1] - vrange[0]), 0.0, 1.0)
    return np.stack([t, t, t, alpha * t], axis=1).astype(np.float32)


def constant_lut(rgba, n: int = 256) -> np.ndarray:
    return np.tile(np.asarray(rgba, dtype=np.float32)[None, :], (n, 1))


def random_lut(seed: int, n: int = 256, alpha_max: float = 0.3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lut = rng.uniform(0.0, 1.0, (n, 4))
    lut[:, 3] *= alpha_max
    return lut.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# cameras: 4x4 row-major world->eye matrices (eye looks down -z, x right, y up)
# ----------------------------------------------------------------------------------------------
def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = r, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m.astype(np.float32)


def orbit_view(theta_deg: float, center, distance: float) -> np.ndarray:
    """Camera on a circle about the y axis through ``center``, looking at the centre."""
    th = math.radians(theta_deg)
    c = np.asarray(center, np.float64)
    eye = c + distance * np.array([math.sin(th), 0.0, math.cos(th)])
    return look_at(eye, c)


def pr1_camera(n: int = 64, W: int = 256, H: int = 256, angle_deg: float = 30.0):
    """Orthographic view along +z rotated ``angle_deg`` about y; height = cube diagonal."""
    c = np.array([n / 2.0] * 3)
    th = math.radians(angle_deg)
    d = np.array([math.sin(th), 0.0, math.cos(th)])
    diag = n * math.sqrt(3.0)
    view = look_at(c - diag * d, c)
    return dict(view=view, proj=0, param=float(diag), W=W, H=H)


def axis_ortho_camera(shape_xyz):
    """Orthographic camera looking along +z with one pixel per voxel column (W=nx, H=ny)."""
    nx, ny, nz = shape_xyz
    c = np.array([nx / 2.0, ny / 2.0, nz / 2.0])
    view = look_at(c - np.array([0.0, 0.0, nz + 8.0]), c)
    return dict(view=view, proj=0, param=float(ny), W=nx, H=ny)


def random_camera(rng: np.random.Generator, shape_xyz, W: int, H: int, proj=None):
    nx, ny, nz = shape_xyz
    c = np.array([nx, ny, nz], np.float64) / 2.0
    diag = float(np.linalg.norm([nx, ny, nz]))
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    if proj is None:
        proj = int(rng.integers(0, 2))
    up = (0.0, 1.0, 0.0) if abs(v[1]) < 0.9 else (1.0, 0.0, 0.0)
    if proj == 0:
        view = look_at(c + diag * v, c, up)
        return dict(view=view, proj=0, param=float(diag * rng.uniform(0.6, 1.1)), W=W, H=H)
    dist = diag * rng.uniform(0.8, 1.6)
    view = look_at(c + dist * v, c, up)
    return dict(view=view, proj=1, param=float(math.radians(rng.uniform(30, 70))), W=W, H=H)


def orbit_camera(cfg: dict, j: int, W=None, H=None):
    """View j of the n_views orbit about y (theta_j = 360 j / n_views), perspective."""
    nx, ny, nz = cfg["shape"]
    c = np.array([nx, ny, nz], np.float64) / 2.0
    half_diag = 0.5 * math.sqrt(nx * nx + ny * ny + nz * nz)
    view = orbit_view(360.0 * j / cfg["n_views"], c, cfg["eye_factor"] * half_diag)
    return dict(view=view, proj=1, param=math.radians(cfg["fov_deg"]),
                W=W or cfg["W"], H=H or cfg["H"])


def sample_pixels(seed: int, W: int, H: int, n: int) -> np.ndarray:
    """``n`` distinct pixel indices (row*W + col) drawn from a WxH frame."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(W * H, size=min(n, W * H), replace=False)).astype(np.int64)


def poisson_arrivals(seed: int, rate_hz: float, n: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
