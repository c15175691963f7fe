"""Full-size workloads in the bench's launch configuration, checked on seeded sampled rays.

HIPASS-scale: 1720x1720x1024 (12.1 GB), 256^3 bricks, 1024^2 perspective orbit, step 1.
GASS-scale:   2048x2048x1600 (26.8 GB), 256^3 bricks, 1024^2 perspective orbit, step 0.5,
              FP32 / FP16 / BF16 bricks, error against the FP64 oracle on 4096 sampled rays.
Both keep the bench's brick layouts (slice atlases + the x-contiguous copy), so every frame
here gathers from the atlases as the timed frames do; HIPASS also checks global termination
with the occlusion leg's opaque table, and GASS's 16-bit frames are rendered again through pair
atlases (the bench's `*_pair_atlas` frames), which must give the same frame bit for bit.
The measured maximum errors are written as JSON to the file named by VR_LARGE_ERRORS, if set.
"""
import json
import os

import numpy as np
import pytest

import synth
from gpu_helpers import ATOL_F32, BOUND_16, compare_dvr, gpu_ctx

pytestmark = pytest.mark.gpu
RESULTS = {}


def _record(key, val):
    RESULTS[key] = val
    path = os.environ.get("VR_LARGE_ERRORS")
    if path:
        with open(path, "w") as f:
            json.dump(RESULTS, f, indent=1)


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _check_config(ctx, orc, cfg, cube_t, storages, views, n_rays, tag, pair_storages=()):
    import torch
    cube = cube_t.cpu().numpy()
    cid = ctx.load_cube(cube_t)
    del cube_t
    torch.cuda.empty_cache()
    ctx.set_brick_layouts(cid, 9)
    lut = synth.ramp_lut()
    vr = cfg["vrange"]
    for storage in storages:
        ctx.set_bricking(cid, cfg["brick"], 1, storage)
        ctx.set_transfer_function(lut, *vr)
        ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
        for j in views:
            cam = synth.orbit_camera(cfg, j)
            ctx.set_camera_dict(cam)
            img = ctx.render_frame(cid).cpu().numpy().reshape(-1, 4)
            pix = synth.sample_pixels(cfg["seed"] * 100 + j, cam["W"], cam["H"], n_rays)
            ref, flags, _ = orc.render(cube, lut, vr, cam, step=cfg["step"], tau=cfg["tau"],
                                       brick=cfg["brick"], pix=pix)
            tol = ATOL_F32 if storage == "f32" else BOUND_16
            err = compare_dvr(img[pix], ref, flags, cfg["tau"], atol=tol)
            _record(f"{tag} {storage} view{j}", {"max_abs_err": err, "rays": int(len(pix)),
                                                 "fragile": int((flags & 1).sum())})
            # MIP at full size: the sampled pixels against the FP32-order oracle, bit for bit
            if storage == "f32" and j == views[0]:
                ctx.set_render_params("mip", cfg["step"], cfg["tau"])
                m = ctx.render_frame(cid).cpu().numpy().reshape(-1)
                m32, _, _ = orc.render(cube, lut, vr, cam, mode="mip32", step=cfg["step"],
                                       brick=cfg["brick"], pix=pix[:512])
                assert np.array_equal(m[pix[:512]], m32.astype(np.float32))
                ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
            # global termination (occlusion skipping) with an opaque table, as timed
            if tag == "hipass" and storage == "f32" and j == views[0]:
                opaque = synth.ramp_lut(alpha=1.0)
                ctx.set_transfer_function(opaque, *vr)
                ctx.set_termination("global")
                g = ctx.render_frame(cid).cpu().numpy().reshape(-1, 4)
                ctx.set_termination("segment")
                ctx.set_transfer_function(lut, *vr)
                refg, flg, _ = orc.render(cube, opaque, vr, cam, step=cfg["step"], tau=cfg["tau"],
                                          brick=cfg["brick"], pix=pix, term="global")
                errg = compare_dvr(g[pix], refg, flg, cfg["tau"])
                _record(f"{tag} f32 global-termination view{j}", {"max_abs_err": errg, "rays": int(len(pix))})
        # 16-bit bricks through pair atlases (layout bit 5), as the bench times GASS-scale frames:
        # the whole last frame equals the slice atlases' bit for bit
        if storage in pair_storages:
            ctx.set_brick_layouts(cid, 41)
            ctx.set_bricking(cid, cfg["brick"], 1, storage)
            ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
            pimg = ctx.render_frame(cid).cpu().numpy().reshape(-1, 4)
            ctx.set_brick_layouts(cid, 9)
            same = bool(np.array_equal(pimg, img))
            _record(f"{tag} {storage} pair-atlas frame view{views[-1]}", {"bit_equal": same})
            assert same
    ctx.free_cube(cid)


def test_hipass_scale(ctx, orc):
    cfg = synth.HIPASS
    _check_config(ctx, orc, cfg, synth.hipass_cube(device="cuda"), ["f32", "f16"], [0, 13, 40],
                  1024, "hipass")


def test_gass_scale(ctx, orc):
    cfg = synth.GASS
    _check_config(ctx, orc, cfg, synth.gass_cube(device="cuda"), ["f32", "f16", "bf16"], [5],
                  4096, "gass", pair_storages=("f16", "bf16"))
