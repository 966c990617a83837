"""Sharded map-reduce across processes (one per GPU): the host side.

A map-reduce over [0, n) (Sec. 3.2.5) is cut into contiguous shards, one per
rank.  Each rank folds its shard on its own GPU into a 16-byte accumulator
record (``pyc_reduce_shard``), the ranks exchange their records once (an
all-gather of 16 bytes per rank), and every rank folds the K records in rank
order with the handle's reduce expression (``pyc_reduce_combine``).  The
exchange is the one collective of the path; maps and segmented batches shard
with none.

Segmented batches shard by whole segments (:func:`segment_bounds`, balanced by
elements) and need no exchange at all.

The three steps are methods of :class:`ShardedReduce` so that each can be
checked on its own: ``partial`` and ``combine`` are C-ABI calls on the GPU,
``exchange`` is a plain ``torch.distributed`` all-gather (NCCL between GPUs,
gloo between CPU processes).
"""
from __future__ import annotations

from . import pyc


def shard_bounds(n_total: int, world: int) -> list:
    """Boundaries b[0] = 0 <= b[1] <= ... <= b[world] = n_total; rank r holds
    [b[r], b[r + 1]).  Shard lengths differ by at most one element."""
    if world < 1 or n_total < 0:
        raise ValueError("need world >= 1 and n_total >= 0")
    return [(n_total * r) // world for r in range(world + 1)]


def segment_bounds(seg_offsets, world: int) -> list:
    """Split a segment table across ranks for pyc_reduce_batched with no
    exchange: rank r takes the whole segments [b[r], b[r + 1]) (b[0] = 0,
    b[world] = nseg), the cut after segment s placed where the elements before
    it come closest to r / world of the total, so that ranks get about equal
    bytes; a rank may get no segment.  Each rank reduces its segments into its
    own results; nothing is combined."""
    import numpy as np
    off = np.asarray(seg_offsets, dtype=np.int64)
    if off.ndim != 1 or off.size < 1 or world < 1:
        raise ValueError("need seg_offsets of nseg + 1 entries and world >= 1")
    nseg = off.size - 1
    start = off - off[0]
    total = int(start[-1])
    b = [0]
    for r in range(1, world):
        target = total * r / world
        # the segment boundary nearest the target, never before the previous cut
        k = int(np.searchsorted(start, target, side="left"))
        if k > 0 and k <= nseg and abs(start[k - 1] - target) <= abs(start[min(k, nseg)] - target):
            k -= 1
        b.append(max(b[-1], min(k, nseg)))
    b.append(nseg)
    return b


class ShardedReduce:
    """One map-reduce handle reduced over a range partitioned across ranks."""

    def __init__(self, handle, n_total: int, rank: int = 0, world: int = 1, group=None):
        if not 0 <= rank < world:
            raise ValueError("rank must be in [0, world)")
        self.h = handle
        self.n_total = int(n_total)
        self.rank, self.world, self.group = rank, world, group
        b = shard_bounds(self.n_total, world)
        self.i0, self.n = b[rank], b[rank + 1] - b[rank]

    def partial(self, ptrs, scalars, stream=None):
        """This rank's record (a 16-byte uint8 tensor on the current GPU);
        ptrs point at this rank's shard (global element i0)."""
        import torch
        rec = torch.empty(pyc.PYC_RECORD_BYTES, dtype=torch.uint8, device="cuda")
        pyc.pyc_reduce_shard(self.h, self.n_total, self.i0, self.n, ptrs, scalars,
                             rec.data_ptr(), stream)
        return rec

    def exchange(self, rec):
        """All ranks' records in rank order (world x 16 bytes, on rec's device)."""
        import torch
        if self.world == 1:
            return rec.reshape(1, -1)
        import torch.distributed as dist
        parts = [torch.empty_like(rec) for _ in range(self.world)]
        dist.all_gather(parts, rec, group=self.group)
        return torch.stack(parts)

    def combine(self, recs, d_out, stream=None):
        """Fold the gathered records into one result at d_out (device)."""
        recs = recs.contiguous()
        pyc.pyc_reduce_combine(self.h, recs.shape[0], recs.data_ptr(), d_out, stream)

    def __call__(self, ptrs, scalars, d_out, stream=None):
        """partial -> exchange -> combine.  The C-ABI steps run on `stream`
        (default: torch's current stream); the all-gather is ordered after the
        partial and before the combine by stream waits, with no host sync."""
        import torch
        cur = torch.cuda.current_stream()
        ext = torch.cuda.ExternalStream(stream) if stream else cur
        rec = self.partial(ptrs, scalars, ext.cuda_stream)
        if self.world > 1:
            other = ext.cuda_stream != cur.cuda_stream
            if other:
                cur.wait_stream(ext)
            recs = self.exchange(rec)
            if other:
                ext.wait_stream(cur)
        else:
            recs = rec.reshape(1, -1)
        if ext.cuda_stream != cur.cuda_stream:  # allocated on cur, used on ext
            rec.record_stream(ext)
            recs.record_stream(ext)
        self.combine(recs, d_out, ext.cuda_stream)
