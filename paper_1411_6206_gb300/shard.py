"""x-slab sharding of one reconstruction problem over several plans (one per GPU).

Once the k-space samples are moved to the hybrid (x, ky, kz) space, every step of Algorithm 1
(Sec. 3) except the singular-value thresholding acts on each x-plane alone: the data
consistency of step (4) plane by plane, the soft thresholding of step (3) on Haar tiles that
are 8 planes wide. Step (1) needs the Casorati Gram (X - S)^H (X - S), a sum over all planes;
the statistics of the stopping rule are sums too, and lambda_S is fixed from a maximum over
all planes. So a volume splits into slabs of whole tiles, each iteration every slab leaves its
share of those sums in a small record (lps_slab_* in the C ABI), the records are reduced (a
sum and a max), and every slab repeats the nz x nz eigendecomposition from the reduced record.

This module holds no arithmetic of the method: it partitions the planes, orders the calls and
reduces the records (in a fixed order over the slabs of a process, then across processes with
torch.distributed: NCCL for device records, gloo for host ones).
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple


def slab_ranges(nx_total: int, parts: int, align: int = 8) -> List[Tuple[int, int]]:
    """Split nx_total planes into `parts` contiguous slabs of whole `align`-plane tiles, as
    even as the tiles allow (the first slabs take one tile more): [(x0, nx), ...]."""
    if nx_total % align:
        raise ValueError(f"nx_total = {nx_total} is not a multiple of {align}")
    tiles = nx_total // align
    if not 1 <= parts <= tiles:
        raise ValueError(f"cannot split {tiles} tiles of {align} planes into {parts} slabs")
    base, extra = divmod(tiles, parts)
    out, x0 = [], 0
    for r in range(parts):
        n = (base + (1 if r < extra else 0)) * align
        out.append((x0, n))
        x0 += n
    return out


class Reducer:
    """Reduces slab records: the first `nsum` entries are added, the rest maximised.

    The records of the slabs held by this process are combined in list order into the first
    one; with `distributed` the result is then all-reduced across the processes of `group`
    (SUM and MAX), and copied back into every local record."""

    def __init__(self, nsum: int, distributed: bool = False, group=None):
        self.nsum = nsum
        self.distributed = distributed
        self.group = group

    def __call__(self, recs: Sequence) -> None:
        import torch
        acc = recs[0]
        for r in recs[1:]:
            acc[:self.nsum] += r[:self.nsum]
            torch.maximum(acc[self.nsum:], r[self.nsum:], out=acc[self.nsum:])
        if self.distributed:
            import torch.distributed as dist
            s = acc[:self.nsum].contiguous()
            m = acc[self.nsum:].contiguous()
            dist.all_reduce(s, op=dist.ReduceOp.SUM, group=self.group)
            dist.all_reduce(m, op=dist.ReduceOp.MAX, group=self.group)
            acc[:self.nsum].copy_(s)
            acc[self.nsum:].copy_(m)
        for r in recs[1:]:
            r.copy_(acc)


class LibrarySlab:
    """One slab held by a library plan (created with nx_total, x0); its record is a device
    tensor on the plan's stream (the binding's Plan must use the current torch stream so that
    the reduction is ordered between the calls)."""

    def __init__(self, lps, plan, device):
        import torch
        self.lps = lps
        self.plan = plan
        nsum, nmax = lps.slab_reduction_size(plan.handle)
        self.nsum = nsum
        self.rec = torch.zeros(nsum + nmax, dtype=torch.float32, device=device)

    def begin(self):
        self.lps.slab_begin(self.plan.handle, self.rec)

    def iterate(self, k: int):
        self.lps.slab_iterate(self.plan.handle, self.rec, k)

    def end(self):
        return self.lps.slab_end(self.plan.handle, self.rec)


def reconstruct_frame(slabs: Sequence, reduce: Callable[[Sequence], None], iters: int) -> list:
    """One time instance over all slabs: step (0), `iters` iterations, the frame's outputs
    (Algorithm 1, Sec. 3). Each slab exposes begin(), iterate(k), end() and a record `rec`;
    `reduce` combines the records after every call. Returns what each slab's end() returns."""
    for s in slabs:
        s.begin()
    reduce([s.rec for s in slabs])
    for k in range(1, iters + 1):
        for s in slabs:
            s.iterate(k)
        reduce([s.rec for s in slabs])
    return [s.end() for s in slabs]
