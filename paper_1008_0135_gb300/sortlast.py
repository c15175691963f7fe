"""Sort-last rendering over several processes, one per GPU (Section 2.2: object-space partition
of the cube, cut along the current longest axis at every level; Section 2.5, Fig. 4: the parts'
sub-images composited in depth order in stages).

Every rank holds a context with the cube loaded and bricked.  Rank r's part is the leaf of the
partition tree whose path is r written in the mixed radix of ``counts`` (digit 0, the first
cut, most significant), so ``counts = (world,)`` is one cut into world slabs and ``(2, 2)`` is
two nodes of two GPUs.  A frame is:

1. each rank renders its part's sub-image (C, T) with ``vr_render_subimage``;
2. the stages run from the last cut to the first: the siblings of a cut (ranks whose paths
   differ only in that digit) split the frame rows they hold into one band per sibling, send
   each sibling its band of their sub-images (direct send: one all-to-all in the siblings'
   group), and blend the received bands with ``vr_composite_subimages`` (the library orders
   them per pixel along the cut's axis); after the first cut every rank holds one band of the
   final frame;
3. the bands are gathered on every rank.

The exchange moves raw (C, T) sub-image rows: "over" is associative but not commutative, so no
built-in reduction of a collective library applies.  Collectives go through torch.distributed
(NCCL for CUDA tensors; gloo exchanges host copies).  This module holds no arithmetic of the
method: the sub-images and their blending are the library's kernels.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple


def digits(rank: int, counts: Sequence[int]) -> List[int]:
    """Rank as partition path: mixed radix over ``counts``, digit 0 most significant."""
    out = []
    for c in reversed(counts):
        out.append(rank % c)
        rank //= c
    if rank != 0:
        raise ValueError("rank outside the partition")
    return out[::-1]


def rank_of(path: Sequence[int], counts: Sequence[int]) -> int:
    r = 0
    for d, c in zip(path, counts):
        r = r * c + d
    return r


def bands(r0: int, r1: int, n: int) -> List[Tuple[int, int]]:
    """[r0, r1) cut into n consecutive bands of as equal a row count as possible."""
    rows = r1 - r0
    return [(r0 + rows * k // n, r0 + rows * (k + 1) // n) for k in range(n)]


def group_ranks(path: Sequence[int], level: int, counts: Sequence[int]) -> List[int]:
    """Ranks whose paths equal ``path`` except at ``level``, in that digit's order."""
    out = []
    for k in range(counts[level]):
        p = list(path)
        p[level] = k
        out.append(rank_of(p, counts))
    return out


def band_of(path: Sequence[int], counts: Sequence[int], H: int) -> Tuple[int, int]:
    """Final frame rows a rank holds after every stage (the last cut's band first)."""
    r0, r1 = 0, H
    for level in reversed(range(len(counts))):
        r0, r1 = bands(r0, r1, counts[level])[path[level]]
    return r0, r1


class TorchExchange:
    """The collectives of a frame over torch.distributed: one process group per sibling set
    (created once, by every rank, in the same order) and the world group for the gather."""

    def __init__(self, counts: Sequence[int], backend: str = None, timeout=None):
        """backend: that of the groups this exchange creates ("nccl": CUDA tensors move
        GPU to GPU; "gloo": host copies); None: the default group's.  timeout (a
        datetime.timedelta, or None for the backend's default): how long a collective of these
        groups waits for the other ranks before it fails."""
        import torch.distributed as dist
        self.dist = dist
        self.counts = list(counts)
        world = 1
        for c in counts:
            world *= c
        if dist.get_world_size() != world:
            raise ValueError(f"the partition has {world} parts for {dist.get_world_size()} ranks")
        backend = backend or dist.get_backend()
        self.host = backend == "gloo"                     # gloo moves host tensors
        kw = {"backend": backend} if timeout is None else {"backend": backend, "timeout": timeout}
        self.world_group = dist.new_group(list(range(world)), **kw)
        self.groups: Dict[Tuple[int, Tuple[int, ...]], object] = {}
        for level in range(len(counts)):
            seen = set()
            for r in range(world):
                g = tuple(group_ranks(digits(r, counts), level, counts))
                if g in seen:
                    continue
                seen.add(g)
                self.groups[(level, g)] = dist.new_group(list(g), **kw) if len(g) > 1 else None

    def _to(self, t):
        return t.cpu() if self.host else t

    def all_to_all(self, level: int, members: List[int], send: List, recv_rows: List[int], row_elems: int):
        """send[j]: rows for member j; returns the rows received from each member."""
        import torch
        g = self.groups[(level, tuple(members))]
        if g is None:
            return [send[0]]
        dev = send[0].device
        flat_in = self._to(torch.cat([s.reshape(-1) for s in send]))
        flat_out = torch.empty(sum(recv_rows) * row_elems, dtype=flat_in.dtype, device=flat_in.device)
        self.dist.all_to_all_single(flat_out, flat_in,
                                    output_split_sizes=[r * row_elems for r in recv_rows],
                                    input_split_sizes=[s.numel() for s in send], group=g)
        flat_out = flat_out.to(dev)
        out, o = [], 0
        for r in recv_rows:
            out.append(flat_out[o:o + r * row_elems])
            o += r * row_elems
        return out

    def all_gather(self, mine, max_rows: int, row_elems: int):
        """Every rank's final band (padded to max_rows) from every rank."""
        import torch
        dev = mine.device
        pad = torch.zeros(max_rows * row_elems, dtype=mine.dtype, device=dev)
        pad[:mine.numel()] = mine.reshape(-1)
        src = self._to(pad)
        out = torch.empty(self.dist.get_world_size() * src.numel(), dtype=src.dtype, device=src.device)
        self.dist.all_gather_into_tensor(out, src, group=self.world_group)
        return out.to(dev)


def composite_frame(sub, counts: Sequence[int], rank: int, exchange,
                    blend: Callable[[int, object, int, bool, List[int]], object]):
    """Stages 2 and 3 of a frame from this rank's sub-image ``sub`` ((H, W, 4) or (H, W)).
    ``blend(level, stack, row0, final, members)`` composites a (n, rows, ...) stack of the
    bands of sibling parts ``members`` (ranks, in part-index order); returns the full frame."""
    import torch
    path = digits(rank, counts)
    H = int(sub.shape[0])
    tail = tuple(sub.shape[1:])
    row_elems = 1
    for v in tail:
        row_elems *= int(v)
    cur, r0, r1 = sub, 0, H
    for level in reversed(range(len(counts))):
        members = group_ranks(path, level, counts)
        bl = bands(r0, r1, counts[level])
        send = [cur[a - r0:b - r0].contiguous() for a, b in bl]
        mine = bl[path[level]]
        rows = mine[1] - mine[0]
        recv = exchange.all_to_all(level, members, send, [rows] * len(members), row_elems)
        stack = torch.stack([t.reshape((rows,) + tail) for t in recv]) if rows > 0 else \
            torch.empty((len(members), 0) + tail, dtype=sub.dtype, device=sub.device)
        cur = blend(level, stack.contiguous(), mine[0], level == 0, members)
        r0, r1 = mine
    world = 1
    for c in counts:
        world *= c
    spans = [band_of(digits(q, counts), counts, H) for q in range(world)]
    max_rows = max(b - a for a, b in spans)
    allb = exchange.all_gather(cur, max_rows, row_elems).reshape(world, max_rows * row_elems)
    frame = torch.empty((H,) + tail, dtype=sub.dtype, device=sub.device)
    flat = frame.reshape(H, row_elems)
    for q, (a, b) in enumerate(spans):
        flat[a:b] = allb[q, :(b - a) * row_elems].reshape(b - a, row_elems)
    return frame


def composite_parts_local(subs: Sequence, counts: Sequence[int],
                          blend: Callable[[int, object, int, bool, List[int]], object]):
    """The stages of composite_frame for every part at once, in one process: ``subs[r]`` is the
    sub-image of the part with rank r.  Each rank's band is blended from the same rows of the
    same siblings as over the network, so the frame is the distributed frame bit for bit."""
    import torch
    world = len(subs)
    H = int(subs[0].shape[0])
    paths = [digits(r, counts) for r in range(world)]
    cur = {r: (subs[r], 0, H) for r in range(world)}
    for level in reversed(range(len(counts))):
        nxt = {}
        for r in range(world):
            members = group_ranks(paths[r], level, counts)
            _, r0, r1 = cur[r]
            a, b = bands(r0, r1, counts[level])[paths[r][level]]
            stack = torch.stack([cur[q][0][a - cur[q][1]:b - cur[q][1]] for q in members]).contiguous()
            nxt[r] = (blend(level, stack, a, level == 0, members) if b > a else stack[0], a, b)
        cur = nxt
    frame = torch.empty_like(subs[0])
    for r in range(world):
        img, a, b = cur[r]
        frame[a:b] = img
    return frame


class SortLast:
    """Sort-last frames of one cube over the ranks of torch.distributed (one GPU each)."""

    def __init__(self, ctx, cube_id: int, counts: Sequence[int], rank: int, exchange=None,
                 backend: str = None, balanced: bool = False, timeout=None):
        self.ctx, self.cube_id, self.counts, self.rank = ctx, cube_id, list(counts), rank
        ctx.set_partition(cube_id, self.counts, digits(rank, self.counts))
        ctx.set_partition_balance(cube_id, balanced)
        self.exchange = exchange if exchange is not None else TorchExchange(self.counts, backend, timeout)

    def render(self, stream=None):
        """The full frame ((H, W, 4) premultiplied RGBA, or (H, W) MIP) on every rank."""
        sub = self.ctx.render_subimage(self.cube_id, stream=stream)

        def blend(level, stack, row0, final, members):
            if stack.shape[1] == 0:
                return stack[0]
            return self.ctx.composite_subimages(self.cube_id, level, stack, row0, final, stream=stream)

        return composite_frame(sub, self.counts, self.rank, self.exchange, blend)
