"""Sort-last exchange on CPU (gloo ranks): the partition paths, the row bands of the compositing
stages and the all-to-all / all-gather plumbing of paper_1008_0135_gb300.sortlast.  The blend of
a stage is the library's kernel on the GPU; here a plain CPU "over" in part-index order stands
in for it, so these tests check the exchange, not the blending (tests/test_sortlast_gpu.py does)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1008_0135_gb300 import sortlast as SL  # noqa: E402


def test_paths_and_bands():
    for counts in [(1,), (3,), (2, 2), (2, 3, 2), (5, 1, 2)]:
        world = int(np.prod(counts))
        paths = [SL.digits(r, counts) for r in range(world)]
        assert [SL.rank_of(p, counts) for p in paths] == list(range(world))
        assert len({tuple(p) for p in paths}) == world
        for H in (1, 7, 64, 1000):
            spans = sorted(SL.band_of(p, counts, H) for p in paths)
            # the final bands tile the frame: disjoint, in order, covering [0, H)
            assert spans[0][0] == 0 and spans[-1][1] == H
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
        for level in range(len(counts)):
            for r in range(world):
                g = SL.group_ranks(paths[r], level, counts)
                assert len(g) == counts[level] and r in g
                assert [SL.digits(q, counts)[level] for q in g] == list(range(counts[level]))
    assert SL.bands(3, 10, 3) == [(3, 5), (5, 7), (7, 10)]


def _over(stack):
    """CPU stand-in blend: (n, rows, W, 4) (C, T) sub-images, front to back in index order."""
    import torch
    c = torch.zeros(stack.shape[1:3] + (3,), dtype=torch.float64)
    T = torch.ones(stack.shape[1:3], dtype=torch.float64)
    for k in range(stack.shape[0]):
        f = stack[k].double()
        c = c + T[..., None] * f[..., :3]
        T = T * f[..., 3]
    return torch.cat([c, T[..., None]], -1).float()


def _subimage(rank, H, W):
    import torch
    g = torch.Generator().manual_seed(1000 + rank)
    s = torch.rand((H, W, 4), generator=g)
    s[..., :3] *= 0.5
    return s


def _reference(counts, H, W):
    """Nested blend of all parts' sub-images, deepest cut first, in index order."""
    import torch
    world = int(np.prod(counts))
    subs = {tuple(SL.digits(r, counts)): _subimage(r, H, W) for r in range(world)}
    for level in reversed(range(len(counts))):
        nxt = {}
        for path in {p[:level] for p in subs}:
            stack = torch.stack([subs[path + (k,)] for k in range(counts[level])])
            nxt[path] = _over(stack)
        subs = nxt
    return subs[()]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, counts, H, W, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from datetime import timedelta
    from paper_1008_0135_gb300 import sortlast as S
    world = int(np.prod(counts))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    # the nested split's groups with a bounded wait (the bench passes one to its NCCL groups)
    ex = S.TorchExchange(counts, None, timedelta(seconds=30)) if len(counts) > 1 else S.TorchExchange(counts)
    frame = S.composite_frame(_subimage(rank, H, W), counts, rank, ex,
                              lambda level, stack, row0, final, members: _over(stack))
    q.put((rank, frame.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("counts,H,W", [((2,), 9, 4), ((3,), 10, 3), ((2, 2), 13, 5)])
def test_gloo_ranks_composite_the_frame(counts, H, W):
    """Every rank ends with the frame of the nested blend of all parts, bit for bit; the
    in-process emulation (composite_parts_local) gives the same bits."""
    mp = pytest.importorskip("torch.multiprocessing")
    import torch
    world = int(np.prod(counts))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, counts, H, W, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _reference(counts, H, W).numpy()
    local = SL.composite_parts_local([_subimage(r, H, W) for r in range(world)], counts,
                                     lambda level, stack, row0, final, members: _over(stack)).numpy()
    assert np.array_equal(local, ref)
    for r in range(world):
        assert np.array_equal(got[r], ref), r


def _rank_stalls(rank, port, q):
    """Rank 1 creates the exchange's groups, then never takes part in a frame; rank 0's
    composite, with the groups' bounded wait, must fail instead of waiting for it."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import time
    import torch.distributed as dist
    from datetime import timedelta
    from paper_1008_0135_gb300 import sortlast as S
    dist.init_process_group("gloo", rank=rank, world_size=2, timeout=timedelta(seconds=60))
    ex = S.TorchExchange((2,), None, timedelta(seconds=3))
    if rank == 1:
        time.sleep(12.0)                      # alive, but not in the exchange
        q.put((1, "stalled", 0.0))
        return
    t0 = time.perf_counter()
    try:
        S.composite_frame(_subimage(0, 8, 4), (2,), 0, ex,
                          lambda level, stack, row0, final, members: _over(stack))
        q.put((0, "completed", time.perf_counter() - t0))
    except Exception as e:                    # the collective's timeout
        q.put((0, type(e).__name__, time.perf_counter() - t0))


def test_stalled_rank_ends_the_others_exchange_within_its_timeout():
    """Failure detection on the host: a rank that stops taking part (alive, holding no GPU work)
    makes the other rank's collective fail after the exchange's timeout, not hang."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_stalls, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, what, t = q.get(timeout=120)
        got[r] = (what, t)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    what, t = got[0]
    assert what != "completed", "the exchange completed without its peer"
    assert t < 11.0, f"the failure took {t:.1f} s (timeout 3 s)"
    assert got[1][0] == "stalled"
