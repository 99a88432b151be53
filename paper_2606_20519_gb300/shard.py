"""Sharding a batch of cones across ranks.

The projection acts cone by cone (App. D.2 projects each PSD block on its
own), so a batch splits across GPUs with no exchange on the data path: each
rank projects its own cones.  ``partition`` balances the ranks by work
(the eigensolver's cost grows as n^3) with a deterministic greedy rule, the
same on every rank; ``pack`` and ``unpack`` move between the full svec
buffer and a rank's local buffer; ``gather`` assembles the full output on
every rank for callers that want it (one all_gather of the local outputs,
after the projections, outside the projection itself).
"""
from __future__ import annotations

import numpy as np


def svec_len(n: int) -> int:
    return n * (n + 1) // 2


def offsets_of(sides) -> np.ndarray:
    s = np.asarray(sides, dtype=np.int64)
    off = np.zeros(s.size + 1, dtype=np.int64)
    np.cumsum(s * (s + 1) // 2, out=off[1:])
    return off


def partition(sides, world: int) -> list[list[int]]:
    """Cone indices per rank: largest cones first, each to the least-loaded
    rank (ties to the lower rank); every rank gets its cones in batch order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sides = [int(n) for n in sides]
    order = sorted(range(len(sides)), key=lambda i: (-sides[i], i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(sides[i]) ** 3
    for p in parts:
        p.sort()
    return parts


def pack(x, sides, idx):
    """The local svec buffer of cones ``idx`` (in that order) and their sides."""
    off = offsets_of(sides)
    pieces = [x[int(off[i]):int(off[i + 1])] for i in idx]
    local_sides = [int(sides[i]) for i in idx]
    if not pieces:
        return x[:0], local_sides
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return torch.cat(pieces), local_sides
    except ImportError:  # pragma: no cover
        pass
    return np.concatenate(pieces), local_sides


def unpack(y_local, sides, idx, out):
    """Write a rank's local outputs back into the full buffer ``out``."""
    off = offsets_of(sides)
    pos = 0
    for i in idx:
        ln = int(off[i + 1] - off[i])
        out[int(off[i]):int(off[i + 1])] = y_local[pos:pos + ln]
        pos += ln
    return out


def gather(y_local, sides, parts, group=None):
    """Full output on every rank from each rank's local outputs (torch.distributed)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    lens = [int(sum(svec_len(int(sides[i])) for i in p)) for p in parts]
    maxlen = max(lens) if lens else 0
    buf = torch.zeros(maxlen, dtype=y_local.dtype, device=y_local.device)
    buf[: y_local.numel()] = y_local
    got = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(got, buf, group=group)
    out = torch.empty(int(offsets_of(sides)[-1]), dtype=y_local.dtype, device=y_local.device)
    for r, p in enumerate(parts):
        unpack(got[r][: lens[r]], sides, p, out)
    return out
