"""Benchmark of the bricked ray-cast + sort-last composite path on GB300.

One step = one frame of the hot path: work-list (rendering rectangles, order, bins), the brick
ray-cast launch and the compositing launch, for view j of a 64-view orbit about y (Fig. 7 of
the paper sweeps the rotation angle the same way).  Default workload: the HIPASS-shaped cube,
1720 x 1720 x 1024 float32 (12.1 GB, larger than L2, so no flush is needed between steps),
256^3 bricks + 1 ghost voxel, 1024^2 perspective frames (60 deg), step 1 voxel, early ray
termination at 0.99, 256-entry ramp table over [-3, 100].

Prints one JSON line.  ``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ms per 1024² frame & Gsamples/s (FP32 vs FP16 bricks); adjoint ms; p99 latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=128)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="hipass", choices=["hipass", "hipass_small", "hipass_slab", "gass", "gass_slab",
                                                           "pr1"])
    ap.add_argument("--no-extras", action="store_true", help="skip FP16, adjoint and CPU legs")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="brick storage of the main leg (the headline line uses f32)")
    ap.add_argument("--cpu-rays", type=int, default=1 << 20)
    ap.add_argument("--layouts", type=int, default=9,
                    help="brick layout mask of the main leg (9: x-contiguous copy + slice atlases; "
                         "19: x- and y-contiguous copies + their 16-byte-row copies, staged slabs)")
    ap.add_argument("--frame", type=int, default=0,
                    help="frame edge in pixels of --leg runs (0: the config's); a smaller frame of a "
                         "small cube spaces its rays as far apart as the full cube's (for profiling)")
    ap.add_argument("--leg", default=None, choices=["adjoint", "occlusion", "mip", "subcube", "compressed", "serving",
                                                         "sortlast"],
                    help="run one extra leg alone and print its JSON (for profiling)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# distributed plumbing (replicas: every rank renders its own frames; no data-path collective)
# ---------------------------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            import datetime
            dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=900))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(name: str):
    """dram bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(name)
    if not d:
        return None
    src = os.path.join(ROOT, "paper_1008_0135_gb300", "csrc", "vr_raycast.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if d.get("source_sha") != h:
        return None
    return d.get("dram_bytes_per_launch")


def make_cube(cfg_name: str, device: str):
    if cfg_name == "hipass":
        return synth.hipass_cube(device=device), synth.HIPASS
    if cfg_name in ("hipass_small", "hipass_slab"):
        c = synth.HIPASS_SMALL if cfg_name == "hipass_small" else synth.HIPASS_SLAB
        return synth.hipass_cube(seed=c["seed"], shape_xyz=c["shape"], n_sources=c["n_sources"],
                                 device=device), c
    if cfg_name == "gass":
        return synth.gass_cube(device=device), synth.GASS
    if cfg_name == "gass_slab":
        c = synth.GASS_SLAB
        return synth.gass_cube(seed=c["seed"], shape_xyz=c["shape"], slab=c["slab"], device=device), c
    import torch
    return torch.from_numpy(synth.pr1_cube(seed=0)).to(device), dict(synth.PR1, n_views=64,
                                                                       fov_deg=60.0, eye_factor=1.5)


def cameras(cfg, n):
    return [synth.orbit_camera(cfg, j) for j in range(n)]


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
def timed_frames(ctx, cid, cams, lut, vr, cfg, steps, warmup, dist, out, clocks=None, mode="dvr"):
    import torch
    ctx.set_transfer_function(lut, *vr)
    ctx.set_render_params(mode, cfg["step"], cfg["tau"])
    stream = torch.cuda.current_stream()
    for w in range(warmup):
        ctx.set_camera_dict(cams[w % len(cams)])
        ctx.render_frame(cid, out)
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True)
    dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        ctx.set_camera_dict(cams[(warmup + k) % len(cams)])
        ctx.render_frame(cid, out)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop() if clocks else None
    ctx.set_timing(False)
    ms = e0.elapsed_time(e1)
    st = ctx.stats()
    return ms, st, clk


def mip_leg(ctx, cid, cfg, cams, dist, out, steps, warmup):
    """Maximum-intensity projection (Section 2.4's second mode) of the bench's orbit frames: every
    lattice sample of every brick segment (no early termination), one FP32 maximum per (brick,
    pixel) fragment, the fragments' maximum per pixel.  Its roofline counts the sampled bricks'
    stored bytes and 4 B per fragment."""
    peak, psrc = peaks()
    ms, st, _ = timed_frames(ctx, cid, cams, synth.ramp_lut(), cfg["vrange"], cfg, steps, warmup, dist,
                             out, mode="mip")
    t = dist.max(ms)
    ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
    return {"workload": cfg["name"] + f", {cfg['W']}x{cfg['H']} orbit, step {cfg['step']}, MIP",
            "ms_per_frame": round(t / steps, 4), "samples_per_frame": int(st["samples"] // max(steps, 1)),
            "Gsamples_per_s": round(dist.sum(st["samples"]) / (t * 1e-3) / 1e9, 3),
            "roofline": roofline(st, steps, peak, psrc, "k_raycast<f32,MIP>", 32, 4)}


def subcube_leg(ctx, cid, cfg, cams, dist, out, steps, warmup):
    """Render-time selections (Section 2.3's spectral-channel choice and sub-cube windows): the
    bench's orbit frames with only a band of channels enabled (the others read as the bottom of
    the table range), and clipped to a sub-cube window, beside the full frame."""
    nx, ny, nz = cfg["shape"]
    lut = synth.ramp_lut()
    res = {"workload": cfg["name"] + f", {cfg['W']}x{cfg['H']} orbit, step {cfg['step']}, DVR"}

    def run(tag):
        ms, st, _ = timed_frames(ctx, cid, cams, lut, cfg["vrange"], cfg, steps, warmup, dist, out)
        t = dist.max(ms)
        res[tag] = {"ms_per_frame": round(t / steps, 4), "samples_per_frame": int(st["samples"] // max(steps, 1)),
                    "Gsamples_per_s": round(dist.sum(st["samples"]) / (t * 1e-3) / 1e9, 3)}

    run("full")
    lo, hi = int(nz * 0.40), int(nz * 0.60)
    mask = np.zeros(nz, np.uint8)
    mask[lo:hi] = 1
    ctx.set_channel_mask(mask)
    try:
        run("channel_band")
    finally:
        ctx.set_channel_mask(None)
    res["channel_band"]["channels"] = [lo, hi]
    wlo, whi = (nx // 4, ny // 4, nz // 4), (3 * nx // 4, 3 * ny // 4, nz // 2)
    ctx.set_window(wlo, whi)
    try:
        run("window")
    finally:
        ctx.set_window()
    res["window"]["box"] = [list(wlo), list(whi)]
    return res


def occlusion_leg(ctx, cid, cfg, cams, dist, out, steps, warmup):
    """Occlusion skipping on the bench's cube with an opaque table (opacity = the ramp itself,
    so a ray through the noise is opaque after a few hundred samples): per-segment termination
    (every brick runs its own segment of a ray down to 1 - tau) against global termination
    (one pass in which each ray walks the bricks front to back and stops once the whole ray is
    opaque)."""
    lut = synth.ramp_lut(alpha=1.0)
    res = {"workload": cfg["name"] + f", {cfg['W']}x{cfg['H']} orbit, step {cfg['step']}, "
                       f"ramp table with opacity = ramp (x10 the bench table), ERT {cfg['tau']}"}
    for scope in ("segment", "global"):
        ctx.set_termination(scope)
        ms, st, _ = timed_frames(ctx, cid, cams, lut, cfg["vrange"], cfg, steps, warmup, dist, out)
        t = dist.max(ms)
        res[scope] = {"ms_per_frame": round(t / steps, 4),
                      "samples_per_frame": int(st["samples"] // max(steps, 1)),
                      "Gsamples_per_s": round(dist.sum(st["samples"]) / (t * 1e-3) / 1e9, 3)}
    ctx.set_termination("segment")
    res["speedup"] = round(res["segment"]["ms_per_frame"] / res["global"]["ms_per_frame"], 2)
    return res


def sortlast_leg(ctx, cid, cfg, cams, lut, vr, dist, steps, warmup):
    """N > 1 ranks: the same orbit frames rendered sort-last (Sections 2.2 and 2.5): rank r
    draws its slab of a longest-axis cut of the cube into a sub-image, the sub-images are
    exchanged by screen band over NCCL (direct send) and blended in depth order by the library,
    and every rank gathers the frame.  One frame is split over all ranks ("strong")."""
    import torch
    from paper_1008_0135_gb300.sortlast import SortLast
    ctx.set_transfer_function(lut, *vr)
    ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
    import datetime
    # a rank that fails or stalls ends the others' collectives within two minutes
    sl = SortLast(ctx, cid, (dist.world,), dist.rank, backend="nccl", timeout=datetime.timedelta(seconds=120))
    for w in range(warmup):
        ctx.set_camera_dict(cams[w % len(cams)])
        sl.render()
    torch.cuda.synchronize()
    ctx.reset_stats()
    dist.barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        ctx.set_camera_dict(cams[(warmup + k) % len(cams)])
        sl.render()
    torch.cuda.synchronize()
    t = dist.max(time.perf_counter() - t0)
    samples = dist.sum(ctx.stats()["samples"])
    ctx.set_partition(cid)
    return {"value": round(samples / t / 1e9, 3), "unit": "Gsamples/s", "scaling": "strong",
            "ms_per_frame": round(1e3 * t / steps, 4), "ranks": dist.world,
            "what": "one frame per step split over all ranks: longest-axis slabs, sub-image bands "
                    "exchanged over NCCL, staged depth-ordered compositing, frame gathered on every rank"}


def sortlast_projection_leg(ctx, cid, cfg, cams, lut, vr, views=8,
                            counts_list=((2,), (4,), (2, 2), (8,), (2, 2, 2)), fine_brick=128):
    """Sort-last on one GPU, part by part (Sections 2.2, 2.5, 3): for N parts of a longest-axis cut
    (equal layer counts, and cuts balanced by the view's estimated cost) every part's sub-image
    of the same orbit views is rendered and timed alone (CUDA events around each part's frame),
    for one cut into N slabs (key "N") and for the paper's nested cuts (Fig. 3: nodes, then each
    node's GPUs, every level along its part's longest axis; key "2x2", "2x2x2"),
    then the staged composite of all parts is timed.  With one part per GPU the frame would take
    the slowest part plus a rank's share of the compositing plus the exchange (each rank sends
    and receives (N - 1)/N of a frame of (C, T) per stage, not timed here): the projection is
    that sum without the exchange, its speedup over the whole frame, and the parts' imbalance
    (slowest / mean), the paper's limit on speedup.  With fine_brick set, 4 and 8 parts are
    projected again on bricks of that size (more layers to place the cuts between)."""
    import torch
    from paper_1008_0135_gb300 import sortlast as SL
    ctx.set_transfer_function(lut, *vr)
    ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ev[0].record(st)
        r = fn()
        ev[1].record(st)
        torch.cuda.synchronize()
        return r, ev[0].elapsed_time(ev[1])

    def project(counts_list):
        whole = []
        for v in range(views):
            ctx.set_camera_dict(cams[v * len(cams) // views])
            ctx.render_frame(cid)                              # warm
            whole.append(timed(lambda: ctx.render_frame(cid))[1])
        res = {"whole_ms_per_frame": round(float(np.mean(whole)), 4), "views": views}
        for counts in counts_list:
            world = int(np.prod(counts))
            for balanced in (False, True):
                ctx.set_partition_balance(cid, balanced)
                proj, imb, comp_share = [], [], []
                for v in range(views):
                    ctx.set_camera_dict(cams[v * len(cams) // views])
                    subs, times = [], []
                    for r in range(world):
                        ctx.set_partition(cid, counts, SL.digits(r, counts))
                        ctx.render_subimage(cid)               # warm (and the cuts for this view)
                        sub, ms = timed(lambda: ctx.render_subimage(cid))
                        subs.append(sub)
                        times.append(ms)

                    def blend(level, stack, row0, final, members):
                        ctx.set_partition(cid, counts, SL.digits(members[0], counts))
                        return ctx.composite_subimages(cid, level, stack, row0, final)

                    SL.composite_parts_local(subs, counts, blend)              # warm (scratch)
                    _, cms = timed(lambda: SL.composite_parts_local(subs, counts, blend))
                    proj.append(max(times) + cms / world)
                    imb.append(max(times) / (sum(times) / world))
                    comp_share.append(cms / world)
                key = f"{'x'.join(map(str, counts))}_{'balanced' if balanced else 'equal'}"
                res[key] = {"projected_ms_per_frame": round(float(np.mean(proj)), 4),
                            "speedup_vs_whole": round(res["whole_ms_per_frame"] / float(np.mean(proj)), 2),
                            "imbalance_slowest_over_mean": round(float(np.mean(imb)), 3),
                            "composite_ms_per_rank": round(float(np.mean(comp_share)), 4),
                            "exchange_bytes_per_rank": int(cfg["W"] * cfg["H"] * 16 * (world - 1) / world)}
        ctx.set_partition(cid)
        ctx.set_partition_balance(cid, False)
        return res

    res = project(counts_list)
    if fine_brick:
        # the same frames with bricks of fine_brick^3: more brick layers per axis, so cuts (equal
        # or balanced by the view's cost) can even the parts out; the cube is re-bricked after
        ctx.set_bricking(cid, (fine_brick,) * 3, 1, "f32")
        res[f"bricks_{fine_brick}"] = project(((4,), (8,)))
        ctx.set_bricking(cid, cfg["brick"], 1, "f32")
    ctx.set_partition(cid)
    ctx.set_partition_balance(cid, False)
    return res


def compressed_leg(ctx, cid, cfg, cams, lut, vr, out, cube_np, frames=16):
    """The bench's cube compressed into 8-bit Haar-wavelet blocks in HBM (the FP32 voxels, brick
    pool and atlases released), then rendered with its bricks decoded on demand into the brick
    cache: store size, encode time, decoded-voxel error on sampled bricks, the first frame
    (every brick decoded) and warm frames (bricks cached), and the image change against the
    FP32 frame of the same view."""
    import torch
    ctx.set_transfer_function(lut, *vr)
    ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
    ctx.set_camera_dict(cams[0])
    ref = ctx.render_frame(cid, out).clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.compress_cube(cid)
    enc_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.set_brick_layouts(cid, 9)      # cache slots also hold slice atlases of the decoded bricks
    atlas_s = time.perf_counter() - t0
    n_store = int(ctx.wavelet_store_bytes(cid))
    nx, ny, nz = cfg["shape"]
    res = {"workload": cfg["name"] + ": 8x8x8 Haar blocks, 3 levels, int8 codes, power-of-two "
                                     "step per subband, decoded on demand into the brick cache "
                                     "(slots with slice atlases)",
           "store_bytes": n_store, "fp32_bytes": 4 * nx * ny * nz,
           "ratio_vs_fp32": round(4 * nx * ny * nz / n_store, 3), "encode_s": round(enc_s, 3),
           "slot_atlas_setup_s": round(atlas_s, 3)}
    # decoded voxels against the FP32 cube on sampled bricks
    nb, _ = ctx.brick_grid(cid)
    total = nb[0] * nb[1] * nb[2]
    errs, sq, cnt, peak = 0.0, 0.0, 0, 0.0
    for b in np.linspace(0, total - 1, 6).astype(int):
        dims, org, _, data = ctx.get_brick(cid, int(b))
        zi = np.clip(org[2] + np.arange(dims[2]), 0, nz - 1)
        yi = np.clip(org[1] + np.arange(dims[1]), 0, ny - 1)
        xi = np.clip(org[0] + np.arange(dims[0]), 0, nx - 1)
        want = cube_np[np.ix_(zi, yi, xi)]
        d = data.astype(np.float64) - want
        errs = max(errs, float(np.abs(d).max()))
        sq += float((d * d).sum())
        cnt += d.size
        peak = max(peak, float(np.abs(want).max()))
    rms = (sq / cnt) ** 0.5
    res["voxel_error"] = {"max_abs": round(errs, 5), "rms": round(rms, 5),
                          "psnr_db": round(20 * np.log10(peak / rms), 2), "bricks_sampled": 6}
    ctx.reset_stats()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    img = ctx.render_frame(cid, out)
    e1.record()
    torch.cuda.synchronize()
    st = ctx.stats()
    res["first_frame"] = {"ms": round(e0.elapsed_time(e1), 3), "bricks_decoded": st["cache_misses"],
                          "bytes_decoded": st["bytes_streamed"]}
    diff = (img - ref).abs()
    res["image_change_vs_fp32"] = {"max_abs": round(float(diff.max()), 5),
                                   "mean_abs": round(float(diff.mean()), 7)}
    ctx.reset_stats()
    e0.record()
    for k in range(frames):
        ctx.set_camera_dict(cams[k % len(cams)])
        ctx.render_frame(cid, out)
    e1.record()
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.set_timing(False)
    ms = e0.elapsed_time(e1) / frames
    res["warm_frames"] = {"ms_per_frame": round(ms, 4), "Gsamples_per_s": round(st["samples"] / frames / (ms * 1e-3) / 1e9, 3),
                          "cache_misses": st["cache_misses"], "frames": frames}
    return res


def traffic_entry(name: str):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    return json.load(open(p)).get(name) if os.path.exists(p) else None


def roofline(st, steps, peak, src, name, texel_bytes=32, frag_bytes=16):
    """The HBM roofline of the ray-cast launch, and beside it the texture unit's texel writeback:
    the texel bytes its gathers return per second (`texel_bytes` per sample: two gathers of four
    texels, 32 B for FP32 texels and 16 B for 16-bit ones -- the writeback's busy cycles follow
    the texel size, not the widened registers) against the L1TEX writeback rate derived from ncu
    (32 B per cycle per SM)."""
    nl = max(st["timed_frames"], 1)
    per_launch = (st["brick_bytes_sampled"] + frag_bytes * st["fragments"]) / nl
    ms = st["ms_raycast"] / nl
    achieved = per_launch / (ms * 1e-3) / 1e9
    rl = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
          "frac": round(achieved / peak, 4), "traffic": kernel_traffic(name),
          "peak_source": src, "kernel": name, "algorithmic_bytes_per_launch": int(per_launch),
          "launch_ms": round(ms, 4)}
    wb = traffic_entry("l1tex_texel_writeback_peak_gbs")
    if wb:
        tex = float(texel_bytes) * st["samples"] / nl / (ms * 1e-3) / 1e9
        rl["l1tex"] = {"bound": "l1tex texel writeback", "achieved": round(tex, 1), "peak": wb["value"],
                       "unit": "GB/s", "frac": round(tex / wb["value"], 4),
                       "peak_source": "derived from ncu (profiles/traffic.json)"}
    return rl


def adjoint_leg(ctx, device):
    """Differentiation workload: 256^3 cube, 8 views at 512^2, L2 loss vs a target rendered with
    a shifted ramp; timed forward (8 frames) and backward (8 adjoint passes)."""
    import torch
    cfg = synth.DIFF
    cube = torch.from_numpy(synth.diff_cube(seed=cfg["seed"])).to(device)
    cid = ctx.load_cube(cube)
    ctx.set_brick_layouts(cid, 9)      # forward and replay read the slice atlases
    ctx.set_bricking(cid, cfg["brick"], 1, "f32")
    lut = synth.ramp_lut()
    target_lut = synth.shifted_ramp_lut()
    c = np.array(cfg["shape"], np.float64) / 2
    cams = []
    for j in range(cfg["n_views"]):
        view = synth.orbit_view(45.0 * j, c, 1.5 * 0.5 * math.sqrt(3) * cfg["shape"][0])
        cams.append(dict(view=view, proj=1, param=math.radians(60.0), W=cfg["W"], H=cfg["H"]))
    ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
    targets = []
    ctx.set_transfer_function(target_lut, *cfg["vrange"])
    for cam in cams:
        ctx.set_camera_dict(cam)
        targets.append(ctx.render_frame(cid).clone())
    ctx.set_transfer_function(lut, *cfg["vrange"])
    glut = torch.zeros((256, 4), device=device)
    gvox = torch.zeros_like(cube)
    acc = torch.zeros_like(glut)

    def step():
        acc.zero_()
        gvox.zero_()
        for cam, tgt in zip(cams, targets):
            ctx.set_camera_dict(cam)
            img = ctx.render_frame(cid)
            g = 2.0 * (img - tgt)
            ctx.render_backward(cid, g.contiguous(), glut, gvox)
            acc.add_(glut)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.free_cube(cid)
    return {"workload": "256^3, 8 views x 512^2, L2 loss, grads w.r.t. 256x4 table and voxels (slice atlases)",
            "ms_per_batch_fwd_bwd": round(ms, 3), "ms_per_view_fwd_bwd": round(ms / len(cams), 3)}


def serving_leg(ctx, hip_cid, device, rates=(10.0, 20.0, 40.0), n_req=60, seed=4):
    """Continuous batching through the online server (vr_serve_open / submit / poll): requests
    are submitted by this process at Poisson arrival times while earlier ones render, over three
    cubes -- the resident HIPASS-scale cube (1024^2 or 512^2 orbit views), a resident 256^3 cube
    (512^2 orbit views) and the 4096x4096x4800 virtual cube (322 GB as FP32, above HBM),
    streamed through the HBM brick cache: its 512^2 requests come from two viewers flying
    across it (the eye moves 16 voxels sideways per request, so each frame needs some bricks the
    cache does not hold) and occasional jumps to a random region.  Rates are swept; latency is
    submission to completion, per request kind; cache misses and bytes streamed are counted
    inside each timed run."""
    import torch
    rng = np.random.default_rng(seed)
    diff = synth.DIFF
    dcid = ctx.load_cube(torch.from_numpy(synth.diff_cube(seed=diff["seed"])).to(device))
    ctx.set_bricking(dcid, diff["brick"], 1, "f32")
    vshape = (4096, 4096, 4800)
    vcid = ctx.load_cube_procedural(seed, vshape)
    ctx.set_bricking(vcid, (256, 256, 256), 1, "f32")
    ctx.set_brick_layouts(vcid, 9)     # cache slots also hold slice atlases of its bricks
    luts = [synth.ramp_lut(), synth.shifted_ramp_lut(vrange=(-3.0, 100.0))]
    # two viewers strafing across the cube (the eye moves sideways, so each frame's frustum
    # takes in bricks at its leading edge that earlier frames did not need)
    paths = [dict(eye=np.array([-200.0, 300.0, 1800.0]), step=np.array([0.0, 16.0, 0.0]), look=np.array([1.0, 0.05, 0.1])),
             dict(eye=np.array([300.0, 2900.0, -200.0]), step=np.array([16.0, 0.0, 0.0]), look=np.array([0.08, -0.05, 1.0]))]
    fly = [0, 0]

    def virtual_cam():
        if rng.uniform() < 0.1:                        # a jump to a random region
            tgt = rng.uniform((256, 256, 256), (3840, 3840, 4544))
            eye = tgt - np.array([0.0, 0.0, 400.0])
            kind = "virtual_jump"
        else:
            v = int(rng.integers(0, 2))
            p = paths[v]
            eye = p["eye"] + fly[v] * p["step"]
            tgt = eye + p["look"] * 500.0
            fly[v] += 1
            kind = "virtual_fly"
        return dict(view=synth.look_at(eye, tgt), proj=1, param=math.radians(8.0), W=512, H=512), kind

    def make_request(arrival_ms):
        u = rng.uniform()
        if u < 0.4:
            res = 1024 if rng.uniform() < 0.5 else 512
            cam = synth.orbit_camera(synth.HIPASS, int(rng.integers(0, 64)), W=res, H=res)
            cube, vr, step, kind = hip_cid, (-3.0, 100.0), 1.0, f"hipass{res}"
        elif u < 0.85:
            c = np.array(diff["shape"], np.float64) / 2
            view = synth.orbit_view(45.0 * int(rng.integers(0, 8)), c, 1.5 * 0.5 * math.sqrt(3) * 256)
            cam = dict(view=view, proj=1, param=math.radians(60.0), W=512, H=512)
            cube, vr, step, kind = dcid, diff["vrange"], diff["step"], "diff512"
        else:
            cam, kind = virtual_cam()
            cube, vr, step = vcid, (-3.0, 100.0), 1.0
        out = torch.empty((cam["H"], cam["W"], 4), dtype=torch.float32, device=device)
        return dict(cube=cube, cam=cam, mode="dvr", step=step, tau=0.99,
                    lut=luts[int(rng.integers(0, 2))], vrange=vr, arrival_ms=arrival_ms, out=out), kind

    # each viewer's first view once, outside the request loop (its whole frustum is a cold start:
    # every brick generated on the host threads and streamed into the cache)
    stc = ctx.stats()
    t_cold = time.perf_counter()
    for p in paths:
        ctx.set_transfer_function(luts[0], -3.0, 100.0)
        ctx.set_camera_dict(dict(view=synth.look_at(p["eye"], p["eye"] + p["look"] * 500.0), proj=1,
                                 param=math.radians(8.0), W=512, H=512))
        ctx.set_render_params("dvr", 1.0, 0.99)
        ctx.render_frame(vcid)
    torch.cuda.synchronize()
    cold_s = time.perf_counter() - t_cold
    stc1 = ctx.stats()
    cold_bricks = stc1["cache_misses"] - stc["cache_misses"]
    cold_bytes = stc1["bytes_streamed"] - stc["bytes_streamed"]
    cold = {"bricks": int(cold_bricks), "GB": round(cold_bytes / 1e9, 2), "seconds": round(cold_s, 2),
            "bricks_per_s": round(cold_bricks / cold_s, 1), "GB_per_s": round(cold_bytes / cold_s / 1e9, 2),
            "what": "the two viewers' first frames from an empty cache: bricks generated on the "
                    "host worker threads (each brick's z-slabs in parallel), staged in pinned "
                    "memory, copied on the side stream and packed into the slots' atlases"}
    runs = []
    for ri, rate in enumerate(rates):
        arrivals = synth.poisson_arrivals(seed + ri, rate, n_req) * 1e3
        reqs = [make_request(float(a)) for a in arrivals]
        st0 = ctx.stats()
        srv = ctx.serve_online(max_inflight=4)
        done = {}
        t0 = time.perf_counter()
        for i, (r, _) in enumerate(reqs):
            while (time.perf_counter() - t0) * 1e3 < r["arrival_ms"]:
                for t, res in srv.poll(wait_ms=0):
                    done[t] = res
                time.sleep(0.0002)
            srv.submit(r)
        while len(done) < len(reqs):
            for t, res in srv.poll(wait_ms=200):
                done[t] = res
        summ = srv.close()
        st1 = ctx.stats()
        by_kind = {}
        for i, (_, kind) in enumerate(reqs):
            if done[i]["status"] == 0:
                by_kind.setdefault(kind, []).append(done[i]["latency_ms"])
        runs.append({
            "rate_hz": rate, "requests": n_req, "completed": summ["completed"], "failed": summ["failed"],
            "p50_ms": round(summ["p50_ms"], 3), "p99_ms": round(summ["p99_ms"], 3),
            "max_ms": round(summ["max_ms"], 3), "frames_per_s": round(summ["frames_per_s"], 2),
            "max_concurrent": summ["max_concurrent"],
            "by_kind": {k: {"n": len(v), "p50_ms": round(float(np.percentile(v, 50)), 3),
                            "p99_ms": round(float(np.percentile(v, 99)), 3)} for k, v in sorted(by_kind.items())},
            "cache_misses": st1["cache_misses"] - st0["cache_misses"],
            "cache_hits": st1["cache_hits"] - st0["cache_hits"],
            "bytes_streamed": st1["bytes_streamed"] - st0["bytes_streamed"]})
        del reqs
    ctx.free_cube(dcid)
    ctx.free_cube(vcid)
    return {"workload": f"{n_req} Poisson requests per rate, submitted online while frames run: "
                        "HIPASS-scale 1024^2/512^2 (40 %), 256^3 cube 512^2 (45 %), 4096x4096x4800 "
                        "virtual cube (322 GB, streamed through a 64 GB brick cache with slice-atlas "
                        "slots) 512^2 views, 8 deg, of two viewers strafing 16 voxels per request and "
                        "jumps to random regions (15 %); two tables",
            "max_inflight": 4, "virtual_first_views_s": round(cold_s, 2), "cold_stream": cold,
            "rates": runs,
            "p50_ms": runs[0]["p50_ms"], "p99_ms": runs[0]["p99_ms"]}


def empty_space_leg(ctx, device, steps=16):
    """Empty-space skipping on the GASS-scale cube (2048x2048x1600, 26.8 GB): its emission lies
    in a 200-voxel slab and N(0, 0.5) noise fills the rest.  A noise-suppressing table (zero
    opacity below 3.0) lets whole bricks drop out; the same table with opacity 1e-7 instead of
    0 keeps every brick and gives the time without skipping."""
    import torch
    cfg = synth.GASS
    cube = synth.gass_cube(device=device)
    cid = ctx.load_cube(cube)
    del cube
    torch.cuda.empty_cache()
    ctx.set_brick_layouts(cid, 9)
    ctx.set_bricking(cid, cfg["brick"], 1, "f32")
    x = np.linspace(cfg["vrange"][0], cfg["vrange"][1], 256)
    out = torch.empty((cfg["H"], cfg["W"], 4), dtype=torch.float32, device=device)
    cams = [synth.orbit_camera(cfg, j) for j in range(64)]
    res = {}
    for name, floor_alpha in (("skipping", 0.0), ("no_skipping", 1e-7)):
        lut = synth.ramp_lut(alpha=0.05)
        lut[x < 3.0, 3] = floor_alpha
        ctx.set_transfer_function(lut, *cfg["vrange"])
        ctx.set_render_params("dvr", cfg["step"], cfg["tau"])
        for j in range(3):
            ctx.set_camera_dict(cams[j])
            ctx.render_frame(cid, out)
        torch.cuda.synchronize()
        ctx.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            ctx.set_camera_dict(cams[(3 + 4 * k) % 64])
            ctx.render_frame(cid, out)
        e1.record()
        torch.cuda.synchronize()
        st = ctx.stats()
        res[name] = {"ms_per_frame": round(e0.elapsed_time(e1) / steps, 3),
                     "bricks_drawn_per_frame": round(st["bricks_drawn"] / steps, 1),
                     "Gsamples_per_s": round(st["samples"] / (e0.elapsed_time(e1) * 1e-3) / 1e9, 2)}
    # the GASS-scale configuration itself: the ramp table, FP32 / FP16 / BF16 bricks through
    # slice atlases, and the 16-bit bricks again through pair atlases (layout bit 5)
    frames = {}
    ctx.set_transfer_function(synth.ramp_lut(), *cfg["vrange"])
    for storage, layouts, tag in (("f32", 9, "f32"), ("f16", 9, "f16"), ("bf16", 9, "bf16"),
                                  ("f16", 41, "f16_pair_atlas"), ("bf16", 41, "bf16_pair_atlas")):
        ctx.set_brick_layouts(cid, layouts)
        ctx.set_bricking(cid, cfg["brick"], 1, storage)
        for j in range(3):
            ctx.set_camera_dict(cams[j])
            ctx.render_frame(cid, out)
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.set_timing(True)
        e0.record()
        for k in range(steps):
            ctx.set_camera_dict(cams[(3 + 4 * k) % 64])
            ctx.render_frame(cid, out)
        e1.record()
        torch.cuda.synchronize()
        st = ctx.stats()
        ctx.set_timing(False)
        ms = e0.elapsed_time(e1) / steps
        alg = (st["brick_bytes_sampled"] + 16 * st["fragments"]) / max(st["timed_frames"], 1)
        rc_ms = st["ms_raycast"] / max(st["timed_frames"], 1)
        frames[tag] = {"ms_per_frame": round(ms, 3),
                           "Gsamples_per_s": round(st["samples"] / (ms * steps * 1e-3) / 1e9, 2),
                           "raycast_GB_per_s_upper_bound": round(alg / (rc_ms * 1e-3) / 1e9, 1)}
        g = traffic_entry("k_raycast<f32,DVR>@GASS")
        if storage == "f32" and g:
            dram = g["traffic_over_algorithmic"] * alg / (rc_ms * 1e-3) / 1e9
            frames[tag]["raycast_dram_GB_per_s"] = round(dram, 1)
            frames[tag]["hbm_frac_of_measured"] = round(dram / peaks()[0], 4)
    res["gass_frames"] = dict(frames, table=f"ramp over [{cfg['vrange'][0]}, {cfg['vrange'][1]}], "
                                            f"step {cfg['step']}, slice atlases (pair atlases where named)",
                              bytes="upper bound: stored bytes of every drawn brick / ray-cast time "
                                    "(segments stop early, so a drawn brick is not read whole); "
                                    "dram: that times the DRAM traffic / algorithmic bytes ratio of "
                                    "the GASS-recipe slab capture (0.663)")
    ctx.free_cube(cid)
    res["workload"] = (f"GASS-scale 2048x2048x1600, {cfg['W']}x{cfg['H']} orbit, step "
                       f"{cfg['step']}, table with zero opacity below 3.0 (noise sd 0.5)")
    res["speedup"] = round(res["no_skipping"]["ms_per_frame"] / res["skipping"]["ms_per_frame"], 2)
    return res


def cpu_baseline(cube_np, cfg, lut, vr, n_rays, samples_per_frame=None):
    import oracle
    cam = synth.orbit_camera(cfg, 0)
    pix = synth.sample_pixels(cfg["seed"], cam["W"], cam["H"], n_rays)
    t0 = time.perf_counter()
    _, _, ns = oracle.render(cube_np, lut, vr, cam, step=cfg["step"], tau=cfg["tau"],
                             brick=cfg["brick"], pix=pix)
    dt = time.perf_counter() - t0
    res = {"value": round(ns / dt / 1e9, 6), "unit": "Gsamples/s", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": f"{len(pix)} seeded pixels of orbit view 0 ({ns} samples, {dt:.2f} s wall)"}
    if samples_per_frame:            # a whole frame at the sample's rate
        res["ms_per_frame_extrapolated"] = round(1e3 * samples_per_frame / (ns / dt), 1)
    return res


def run_ours(args, dist):
    import torch
    import paper_1008_0135_gb300 as P
    P.build()
    dev = dist.local
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    cube, cfg = make_cube(args.config, device)
    nz, ny, nx = cube.shape
    lut = synth.ramp_lut()
    vr = cfg["vrange"]
    cams = cameras(cfg, cfg.get("n_views", 64))
    W, H = cfg["W"], cfg["H"]
    ctx = P.Context(dev, cache_bytes=64 << 30)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    cid = ctx.load_cube(cube)
    load_s = time.perf_counter() - t_setup
    cube_np = None
    if dist.world == 1 and not args.no_extras:
        cube_np = cube.cpu().numpy()
    del cube
    torch.cuda.empty_cache()
    ctx.set_brick_layouts(cid, args.layouts)   # default: slice atlases (gathers) + the x copy
    t_setup = time.perf_counter()
    ctx.set_bricking(cid, cfg["brick"], 1, args.storage)
    brick_s = time.perf_counter() - t_setup
    out = torch.empty((H, W, 4), dtype=torch.float32, device=device)
    peak, psrc = peaks()
    clocks = Clocks(dev)
    ms, st, clk = timed_frames(ctx, cid, cams, lut, vr, cfg, args.steps, args.warmup, dist, out,
                               clocks)
    t_max = dist.max(ms)
    samples_all = dist.sum(st["samples"])
    value = samples_all / (t_max * 1e-3) / 1e9
    rl = roofline(st, args.steps, peak, psrc, f"k_raycast<{args.storage},DVR>",
                  32 if args.storage == "f32" else 16)
    sortlast = None
    if dist.world > 1:
        try:
            sortlast = sortlast_leg(ctx, cid, cfg, cams, lut, vr, dist, min(args.steps, 32), args.warmup)
        except Exception as e:                 # the replicas' line stands without it
            sortlast = {"error": f"{type(e).__name__}: {e}"[:300]}
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gsamples/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded stand-in for the HIPASS cube; no dataset available)",
        "config": {"workload": cfg["name"] + f", {W}x{H} perspective 64-view orbit, step "
                   f"{cfg['step']}, 256^3 bricks + ghost 1, {args.storage.upper()} bricks, ERT 0.99",
                   "cube_xyz": [nx, ny, nz], "frame": [W, H], "bricks": list(cfg["brick"]),
                   "l2": f"inputs larger than L2 ({4 * nx * ny * nz / 1e9:.1f} GB cube); no flush",
                   "brick_layouts": ("slice-atlas textures (2 gathers per sample) + x-contiguous copy"
                                     if args.layouts == 9 else f"layout mask {args.layouts}"),
                   "parallelism": f"replicas x{dist.world}"},
        "ms_per_frame": round(t_max / args.steps, 4),
        "samples_per_frame": st["samples"] // max(args.steps, 1),
        "roofline": rl,
        "clocks": clk,
        "gpu_launches": 2 * args.steps,
        "sortlast": sortlast,
        "setup": {"load_cube_s": round(load_s, 3), "bricking_s": round(brick_s, 3),
                  "what": "cube copied in from device memory; bricking = bricks with ghost voxels, "
                          "their value ranges and the slice atlases (one-time)"},
    }
    if not args.no_extras:
        ctx.set_bricking(cid, cfg["brick"], 1, "f16")   # same layouts as the FP32 leg
        ms16, st16, _ = timed_frames(ctx, cid, cams, lut, vr, cfg, args.steps, args.warmup, dist,
                                     out)
        t16 = dist.max(ms16)
        res["fp16_bricks"] = {
            "value": round(dist.sum(st16["samples"]) / (t16 * 1e-3) / 1e9, 3),
            "unit": "Gsamples/s", "ms_per_frame": round(t16 / args.steps, 4),
            "roofline": roofline(st16, args.steps, peak, psrc, "k_raycast<f16,DVR>", 16)}
        ctx.set_bricking(cid, cfg["brick"], 1, "f32")
        res["occlusion"] = occlusion_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 32),
                                         args.warmup)
        res["mip"] = mip_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 32), args.warmup)
        res["subcube"] = subcube_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 16), args.warmup)
        # end to end through the C ABI with host buffers: table + camera in, frame out.  A
        # viewer's loop: frame k is queued (asynchronous copy into one of two pinned frames)
        # before frame k - 1 is read, so the host's work for a frame overlaps the GPU's
        host_out = [torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        lut_h = torch.from_numpy(lut).pin_memory()
        ctx.set_host_output_async(True)

        def viewer_frames(first, count):
            for k in range(count):
                ctx.set_transfer_function(lut_h.numpy(), *vr)
                ctx.set_camera_dict(cams[(first + k) % len(cams)])
                ctx.render_frame(cid, host_out[k % 2])
                done[k % 2].record()
                if k > 0:
                    done[(k - 1) % 2].synchronize()
                    _ = float(host_out[(k - 1) % 2][H // 2, W // 2, 3])
            done[(count - 1) % 2].synchronize()
            _ = float(host_out[(count - 1) % 2][H // 2, W // 2, 3])

        viewer_frames(0, max(args.warmup, 1))
        ctx.reset_stats()
        dist.barrier()
        t0 = time.perf_counter()
        viewer_frames(args.warmup, args.steps)
        e2e_s = dist.max(time.perf_counter() - t0)
        ctx.set_host_output_async(False)
        ste = ctx.stats()
        res["e2e"] = {"value": round(dist.sum(ste["samples"]) / e2e_s / 1e9, 3),
                      "unit": "Gsamples/s", "h2d_bytes_per_step": 64 + lut.nbytes,
                      "d2h_bytes_per_step": W * H * 16,
                      "ms_per_frame": round(1e3 * e2e_s / args.steps, 4),
                      "loop": "table + camera set, frame queued with an asynchronous copy into "
                              "one of two pinned host frames, previous frame read"}
        if dist.world == 1:
            # the one-GPU legs (and the CPU baseline) run in the N = 1 line only: a scaling run's
            # other GPUs are not held while they run
            res["sortlast_projection"] = sortlast_projection_leg(ctx, cid, cfg, cams, lut, vr)
            res["adjoint"] = adjoint_leg(ctx, device)
            res["serving"] = serving_leg(ctx, cid, device)
            res["compressed"] = compressed_leg(ctx, cid, cfg, cams, lut, vr, out, cube_np)
            ctx.free_cube(cid)
            cid = None
            res["empty_space"] = empty_space_leg(ctx, device)
            res["cpu_baseline"] = cpu_baseline(cube_np, cfg, lut, vr, args.cpu_rays, res["samples_per_frame"])
    ctx.close()
    if dist.rank == 0:
        print(json.dumps(res))


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores, a bounded sample per step
# ---------------------------------------------------------------------------------------------
def run_reference(args, dist):
    if dist.rank != 0:
        return
    import torch
    import oracle
    oracle.build()
    device = "cuda:0" if torch.cuda.is_available() else "cpu"
    cube, cfg = make_cube(args.config, device)
    cube_np = cube.cpu().numpy()
    del cube
    lut = synth.ramp_lut()
    cams = cameras(cfg, cfg.get("n_views", 64))
    rays = 16384                       # per step: large enough that the call's fixed cost is small
    total, t_all = 0, 0.0
    for k in range(args.warmup + args.steps):
        cam = cams[k % len(cams)]
        pix = synth.sample_pixels(cfg["seed"] + k, cam["W"], cam["H"], rays)
        t0 = time.perf_counter()
        _, _, ns = oracle.render(cube_np, lut, cfg["vrange"], cam, step=cfg["step"],
                                 tau=cfg["tau"], brick=cfg["brick"], pix=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            total += ns
            t_all += dt
    value = total / t_all / 1e9
    res = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gsamples/s",
           "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * t_all / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded stand-in for the HIPASS cube)",
           "config": {"workload": cfg["name"] + f" {cfg['W']}x{cfg['H']} orbit; per step "
                      f"{rays} seeded pixels of one view (FP64 CPU oracle)"},
           "cpu_baseline": {"value": round(value, 6), "unit": "Gsamples/s",
                            "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{rays} pixels per step, {args.steps} steps"},
           "e2e": {"value": round(value, 6), "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def main():
    args = parse()
    dist = Dist()
    if args.leg == "adjoint":
        import torch
        import paper_1008_0135_gb300 as P
        P.build()
        torch.cuda.set_device(dist.local)
        ctx = P.Context(dist.local)
        print(json.dumps({"leg": "adjoint", **adjoint_leg(ctx, f"cuda:{dist.local}")}))
        ctx.close()
        return
    if args.leg in ("occlusion", "mip", "subcube", "compressed", "serving", "sortlast"):
        import torch
        import paper_1008_0135_gb300 as P
        P.build()
        torch.cuda.set_device(dist.local)
        device = f"cuda:{dist.local}"
        cube, cfg = make_cube(args.config, device)
        if args.frame > 0:
            cfg = dict(cfg, W=args.frame, H=args.frame)
        ctx = P.Context(dist.local, cache_bytes=64 << 30)
        cid = ctx.load_cube(cube)
        cube_np = cube.cpu().numpy() if args.leg == "compressed" else None
        del cube
        torch.cuda.empty_cache()
        ctx.set_brick_layouts(cid, 9)
        ctx.set_bricking(cid, cfg["brick"], 1, "f32")
        out = torch.empty((cfg["H"], cfg["W"], 4), dtype=torch.float32, device=device)
        cams = cameras(cfg, cfg.get("n_views", 64))
        if args.leg == "occlusion":
            res = occlusion_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 32), args.warmup)
        elif args.leg == "mip":
            res = mip_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 32), args.warmup)
        elif args.leg == "subcube":
            res = subcube_leg(ctx, cid, cfg, cams, dist, out, min(args.steps, 16), args.warmup)
        elif args.leg == "serving":
            res = serving_leg(ctx, cid, device)
        elif args.leg == "sortlast":
            res = sortlast_projection_leg(ctx, cid, cfg, cams, synth.ramp_lut(), cfg["vrange"])
        else:
            res = compressed_leg(ctx, cid, cfg, cams, synth.ramp_lut(), cfg["vrange"], out, cube_np)
        print(json.dumps({"leg": args.leg, **res}))
        ctx.close()
        return
    if args.impl == "reference":
        run_reference(args, dist)
    else:
        run_ours(args, dist)


if __name__ == "__main__":
    main()
