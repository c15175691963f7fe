"""Continuous-batching serving loop: requests for several cubes at different resolutions arrive
over time, overlap on the device, and each result equals the frame rendered alone."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    import paper_1008_0135_gb300 as P
    c = gpu_ctx()
    c.close()
    ctx = P.Context(0, cache_bytes=24 * 130 ** 3 * 4)
    a = ctx.load_cube(synth.pr1_cube(seed=0))
    ctx.set_bricking(a, (32, 32, 32), 1, "f32")
    b = ctx.load_cube(synth.pr1_cube(seed=3, n=96))
    ctx.set_bricking(b, (32, 48, 40), 1, "f16")
    v = ctx.load_cube_procedural(4, (300, 270, 260))
    ctx.set_bricking(v, (128, 128, 128), 1, "f32")
    yield ctx, {"pr1": (a, (64, 64, 64)), "b96": (b, (96, 96, 96)), "proc": (v, (300, 270, 260))}
    ctx.close()


def _requests(cubes, n, rate_hz, seed, device):
    import torch
    rng = np.random.default_rng(seed)
    arrivals = synth.poisson_arrivals(seed, rate_hz, n) * 1e3
    luts = [synth.ramp_lut(alpha=0.3), synth.random_lut(7, n=64, alpha_max=0.2)]
    names = list(cubes)
    reqs = []
    for i in range(n):
        name = names[int(rng.integers(0, len(names)))]
        cid, shape = cubes[name]
        W, H = [(128, 128), (96, 80), (160, 120)][int(rng.integers(0, 3))]
        cam = synth.random_camera(rng, shape, W, H)
        mode = "mip" if rng.uniform() < 0.25 else "dvr"
        out = torch.full((H, W, 4) if mode == "dvr" else (H, W), float("nan"), device=device)
        reqs.append(dict(cube=cid, cam=cam, mode=mode, step=0.5, tau=0.99,
                         lut=luts[int(rng.integers(0, 2))], vrange=(-3.0, 20.0),
                         arrival_ms=float(arrivals[i]), out=out))
    return reqs


def _alone(ctx, r):
    ctx.set_transfer_function(r["lut"], *r["vrange"])
    ctx.set_camera_dict(r["cam"])
    ctx.set_render_params(r["mode"], r["step"], r["tau"])
    ctx.set_termination(r.get("termination", "segment"))
    try:
        return ctx.render_frame(r["cube"])
    finally:
        ctx.set_termination("segment")


def test_each_result_is_the_same_alone_and_in_the_mix(world):
    import torch
    ctx, cubes = world
    reqs = _requests(cubes, 40, 400.0, 11, "cuda")
    results, summary = ctx.serve(reqs, max_inflight=6)
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in results), results
    assert summary["completed"] == 40 and summary["failed"] == 0
    assert summary["p99_ms"] >= summary["p50_ms"] > 0
    for r, res in zip(reqs, results):
        assert res["admit_ms"] >= r["arrival_ms"] - 1e-6
        assert res["latency_ms"] > 0
        alone = _alone(ctx, r)
        _same(r, alone)


def _same(r, alone):
    import torch
    if torch.equal(r["out"], alone):
        return
    d = (r["out"] - alone).abs()
    bad = ~(d == 0)
    raise AssertionError(f"cube {r['cube']} mode {r['mode']} {tuple(alone.shape)}: {int(bad.sum())} values "
                         f"differ, max {float(torch.nan_to_num(d, nan=float('inf')).max()):.3e}, "
                         f"nan in mix {int(torch.isnan(r['out']).sum())}")


def test_burst_overlaps_on_the_device(world):
    import torch
    ctx, cubes = world
    reqs = _requests({"pr1": cubes["pr1"], "b96": cubes["b96"]}, 24, 1e9, 12, "cuda")
    for r in reqs:
        r["arrival_ms"] = 0.0
    results, summary = ctx.serve(reqs, max_inflight=8)
    torch.cuda.synchronize()
    assert summary["failed"] == 0
    assert summary["max_concurrent"] >= 4
    for r in reqs:
        _same(r, _alone(ctx, r))


def test_pinned_host_outputs_and_errors(world):
    import torch
    ctx, cubes = world
    reqs = _requests({"pr1": cubes["pr1"]}, 6, 1000.0, 13, "cuda")
    for r in reqs:
        r["out"] = torch.zeros(r["out"].shape, pin_memory=True)
    bad = dict(reqs[0])
    bad["cam"] = dict(bad["cam"], W=0)                 # an invalid request fails alone
    bad["out"] = torch.zeros(4, pin_memory=True)
    reqs.insert(3, bad)
    for i in range(1, len(reqs)):
        reqs[i]["arrival_ms"] = max(reqs[i]["arrival_ms"], reqs[i - 1]["arrival_ms"])
    results, summary = ctx.serve(reqs, max_inflight=3)
    assert results[3]["status"] == -1 and summary["failed"] == 1
    for i, (r, res) in enumerate(zip(reqs, results)):
        if i == 3:
            continue
        assert res["status"] == 0
        assert torch.equal(r["out"].cuda(), _alone(ctx, r))


def test_slot_atlases_in_the_mix(world):
    """The streamed cube with slice atlases in its cache slots (mask 9): frames of the mix pack
    and gather slot atlases on several streams at once (24 slots for 27 bricks: evictions and
    re-packs during the run); each result equals the frame alone, and the frame from the linear
    slots."""
    import torch
    ctx, cubes = world
    v = cubes["proc"][0]
    ctx.set_brick_layouts(v, 9)
    try:
        reqs = _requests({"proc": cubes["proc"], "pr1": cubes["pr1"]}, 32, 400.0, 21, "cuda")
        results, summary = ctx.serve(reqs, max_inflight=6)
        torch.cuda.synchronize()
        assert all(r["status"] == 0 for r in results), results
        for r in reqs:
            _same(r, _alone(ctx, r))
        ctx.set_brick_layouts(v, 1)
        for r in reqs:
            if r["cube"] == v:
                _same(r, _alone(ctx, r))
    finally:
        ctx.set_brick_layouts(v, 1)


def test_soak_mixed_requests_with_evictions():
    """A longer soak: 240 requests over a resident FP32 cube, a resident FP16 cube, a streamed
    FP32 cube with slot atlases and a streamed FP16 cube through a 10-slot cache (evictions and
    re-packs all the time), up to 8 frames in flight, device and pinned host outputs; every
    result equals the frame alone."""
    import torch
    import paper_1008_0135_gb300 as P
    with P.Context(0, cache_bytes=10 * 130 ** 3 * 4) as ctx:
        a = ctx.load_cube(synth.pr1_cube(seed=0))
        ctx.set_bricking(a, (32, 32, 32), 1, "f32")
        b = ctx.load_cube(synth.pr1_cube(seed=3, n=96))
        ctx.set_brick_layouts(b, 9)
        ctx.set_bricking(b, (32, 48, 40), 1, "f16")
        v = ctx.load_cube_procedural(4, (300, 270, 260))
        ctx.set_bricking(v, (128, 128, 128), 1, "f32")
        ctx.set_brick_layouts(v, 9)
        w = ctx.load_cube_procedural(5, (200, 150, 130))
        ctx.set_bricking(w, (64, 64, 64), 1, "f16")
        cubes = {"pr1": (a, (64, 64, 64)), "b96": (b, (96, 96, 96)), "proc": (v, (300, 270, 260)),
                 "proc16": (w, (200, 150, 130))}
        reqs = _requests(cubes, 240, 2000.0, 31, "cuda")
        for i, r in enumerate(reqs):
            if i % 3 == 0:
                r["out"] = torch.zeros(r["out"].shape, pin_memory=True)
        results, summary = ctx.serve(reqs, max_inflight=8)
        torch.cuda.synchronize()
        assert all(r["status"] == 0 for r in results), [r for r in results if r["status"] != 0][:3]
        assert summary["completed"] == 240 and summary["max_concurrent"] >= 2
        for r in reqs:
            out = r["out"] if r["out"].is_cuda else r["out"].cuda()
            _same(dict(r, out=out), _alone(ctx, r))


def test_global_termination_requests_in_the_mix(world):
    """Requests that ask for global termination (occlusion skipping) run beside per-segment ones
    (the same cubes, opaque and transparent tables); each result equals the frame alone with
    its own termination scope."""
    import torch
    ctx, cubes = world
    reqs = _requests({"pr1": cubes["pr1"], "b96": cubes["b96"]}, 40, 400.0, 41, "cuda")
    opaque = synth.ramp_lut(alpha=1.0)
    for i, r in enumerate(reqs):
        if i % 2 == 0:
            r["termination"] = "global"
            r["lut"] = opaque
    results, summary = ctx.serve(reqs, max_inflight=6)
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in results), results
    for r in reqs:
        _same(r, _alone(ctx, r))


def test_online_server_takes_requests_while_frames_run(world):
    """vr_serve_open / submit / poll / close: requests handed over one at a time while earlier
    ones render (resident and streamed cubes, DVR and MIP), results collected as they finish;
    every ticket comes back once, each result equals the frame rendered alone, and a request
    submitted after others completed is still served by the same loop."""
    import time

    import torch
    ctx, cubes = world
    reqs = _requests(cubes, 48, 400.0, 23, "cuda")
    srv = ctx.serve_online(max_inflight=5)
    got = {}
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        while (time.perf_counter() - t0) * 1e3 < r["arrival_ms"]:
            for t, res in srv.poll(wait_ms=0):
                got[t] = res
            time.sleep(0.0002)
        tickets.append(srv.submit(r))
    assert tickets == list(range(len(reqs)))
    deadline = time.perf_counter() + 120
    while len(got) < len(reqs) - 1 and time.perf_counter() < deadline:
        for t, res in srv.poll(wait_ms=100):
            assert t not in got
            got[t] = res
    late = _requests(cubes, 1, 1.0, 99, "cuda")[0]       # after the loop went idle
    tickets.append(srv.submit(late))
    while len(got) < len(reqs) + 1 and time.perf_counter() < deadline:
        for t, res in srv.poll(wait_ms=100):
            got[t] = res
    summary = srv.close()
    torch.cuda.synchronize()
    assert sorted(got) == tickets
    assert all(res["status"] == 0 for res in got.values()), got
    assert summary["completed"] == len(reqs) + 1 and summary["failed"] == 0
    for t, r in enumerate(reqs + [late]):
        assert got[t]["latency_ms"] > 0 and got[t]["done_ms"] >= got[t]["admit_ms"]
        _same(r, _alone(ctx, r))


def test_online_server_from_several_threads_and_its_errors(world):
    """Submissions from four host threads at once each get their own ticket and result; poll
    returns at most `cap` results per call; a request for an unknown cube is refused at submit;
    results not polled before close are dropped without harm; a closed server takes nothing."""
    import threading

    import paper_1008_0135_gb300 as P
    import torch
    ctx, cubes = world
    reqs = _requests({"pr1": cubes["pr1"], "b96": cubes["b96"]}, 32, 1e9, 31, "cuda")
    srv = ctx.serve_online(max_inflight=4)
    tickets = {}
    lock = threading.Lock()

    def worker(part):
        for i in part:
            t = srv.submit(reqs[i])
            with lock:
                tickets[t] = i

    ths = [threading.Thread(target=worker, args=(list(range(k, 32, 4)),)) for k in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert sorted(tickets) == list(range(32))
    bad = dict(reqs[0], cube=12345)
    with pytest.raises(P.VrError):
        srv.submit(bad)
    got = {}
    import time
    deadline = time.perf_counter() + 120
    while len(got) < 30 and time.perf_counter() < deadline:
        batch = srv.poll(wait_ms=50, cap=3)
        assert len(batch) <= 3
        for t, res in batch:
            got[t] = res
    summary = srv.close()                       # the last results may never be polled
    torch.cuda.synchronize()
    assert summary["completed"] == 32 and summary["failed"] == 0
    with pytest.raises(P.VrError):
        srv.submit(reqs[0])
    for t, res in got.items():
        assert res["status"] == 0
        r = reqs[tickets[t]]
        _same(r, _alone(ctx, r))
