"""One join sharded over the ranks of a torch.distributed group (one GPU per rank).

Every rank holds a slice of R and a slice of S.  Each rank groups its slices by
the sharding hash (``hj_split``: group g of every rank is meant for rank g), one
all-to-all of R and one of S deliver the groups, and each rank joins what it
received with ``hj_join``: equal keys meet on one rank, so the local joins
together are the join of the whole relations -- the partitioning of Alg. 2
applied across GPUs (Sec. 3.1).  Pairs stay on the rank that found them (rids
are the tuples' own rids, so they name global rows if the caller's rids do);
the count and both checksums are summed over the ranks with one all-reduce
(checksums modulo 2^64, as everywhere in the library).

This module only moves tensors between the library and the collective library
(NCCL for CUDA tensors); every step of the join itself is a libhj call.  The
split and join steps can be given as functions, which is how the exchange logic
is tested on the CPU with gloo.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist

from . import hj

_M64 = (1 << 64) - 1


def _to_i64(x: int) -> int:
    """An unsigned 64-bit value as the signed value with the same bits."""
    return x - (1 << 64) if x >= 1 << 63 else x


@dataclass
class ShardResult:
    count: int                 # pairs over all ranks
    checksum: tuple            # (c0, c1) over all ranks, modulo 2^64
    local_count: int           # pairs this rank found
    local: object              # what the join step returned on this rank (an hj.Result by default)
    sent: tuple                # tuples of R and of S this rank sent away (to other ranks)
    received: tuple            # tuples of R and of S this rank joined


def _exchange(grouped: torch.Tensor, offs: list, group) -> torch.Tensor:
    """All-to-all of the groups of one relation: rows [offs[g], offs[g+1]) go to
    rank g; returns what this rank receives, in rank order."""
    ws = dist.get_world_size(group)
    send = [offs[g + 1] - offs[g] for g in range(ws)]
    cnt_out = torch.tensor(send, dtype=torch.int64, device=grouped.device)
    cnt_in = torch.empty_like(cnt_out)
    dist.all_to_all_single(cnt_in, cnt_out, group=group)
    recv = [int(x) for x in cnt_in.tolist()]
    out = torch.empty((sum(recv), 2), dtype=grouped.dtype, device=grouped.device)
    dist.all_to_all_single(out, grouped, output_split_sizes=recv, input_split_sizes=send, group=group)
    return out


def shard_join(ctx, R: torch.Tensor, S: torch.Tensor, group=None, mode: int = hj.HJ_MATERIALIZE,
               checksum: bool = True, split=None, join=None, **join_kw) -> ShardResult:
    """Join R and S, whose rows are spread over the ranks of `group`, with one
    exchange step.  Every rank calls it with its own slices (any sizes, possibly
    empty).  `split(rel, nparts) -> (grouped, offsets)` and
    `join(R, S) -> (result, count, (c0, c1))` default to the library's hj_split and
    hj_join on `ctx`'s device."""
    ws = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    if split is None:
        def split(rel, nparts):
            return hj.hj_split(ctx, rel, nparts)
    if join is None:
        def join(Rl, Sl):
            res = hj.hj_join(ctx, Rl, Sl, mode=mode, checksum=checksum, **join_kw)
            return res, res.count, res.checksum
    if ws == 1:
        Rl, Sl, sent = R, S, (0, 0)
    else:
        rank = dist.get_rank(group)
        Rg, ro = split(R, ws)
        Sg, so = split(S, ws)
        sent = (ro[-1] - (ro[rank + 1] - ro[rank]), so[-1] - (so[rank + 1] - so[rank]))
        Rl = _exchange(Rg, ro, group)
        Sl = _exchange(Sg, so, group)
        del Rg, Sg
    local, cnt, (c0, c1) = join(Rl, Sl)
    received = (int(Rl.shape[0]), int(Sl.shape[0]))
    if ws == 1:
        return ShardResult(cnt, (c0, c1), cnt, local, sent, received)
    tot = torch.tensor([cnt, _to_i64(c0), _to_i64(c1)], dtype=torch.int64, device=R.device)
    dist.all_reduce(tot, group=group)
    t = [int(x) & _M64 for x in tot.tolist()]
    return ShardResult(t[0], (t[1], t[2]), cnt, local, sent, received)
