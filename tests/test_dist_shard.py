"""The exchange logic of the sharded join (paper_1307_1955_gb300.dist.shard_join) on
the CPU: two and three gloo ranks, each holding an uneven slice of R and S.  The
device steps are stood in for by the oracle -- the split groups tuples by the
library's sharding hash (the SplitMix64 finaliser's high 32 bits scaled to the
number of ranks, computed with the oracle's pinned finaliser) and the local join is
the oracle's hash join -- so what is tested is everything between them: group
sizes, the all-to-all of R and of S, and the all-reduce of the count and the
64-bit checksums.  The union of the ranks' pairs must equal the oracle's join of
the whole relations, and the all-reduced count and checksums its aggregate."""
import os
import pickle
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _relations(width: int):
    dt = np.uint32 if width == 4 else np.uint64
    rng = np.random.default_rng(17 + width)
    top = np.iinfo(dt).max
    rk = rng.integers(0, 2500, 4000).astype(dt)           # duplicates in R
    rk[:3] = top                                           # extreme keys
    sk = rng.integers(0, 5000, 9001).astype(dt)
    sk[:5] = top
    R = np.stack([rk, np.arange(len(rk), dtype=dt)], 1)
    S = np.stack([sk, np.arange(len(sk), dtype=dt) + 7], 1)
    return R, S


def _slices(n: int, ws: int):
    # uneven slices; the last rank of three gets nothing of R when n is small
    cuts = [0, n // 3, n // 3 + n // 2, n][: ws] + [n]
    return [(cuts[r], cuts[r + 1]) for r in range(ws)]


def _rank(rank, ws, port, width, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1307_1955_gb300 import dist as D
    from paper_1307_1955_gb300 import workload as W

    tdt = torch.int32 if width == 4 else torch.int64
    ndt = np.int32 if width == 4 else np.int64

    def split(rel, nparts):
        a = W.to_numpy_u(rel)
        g = np.array([((oracle.mix_a(int(k)) >> 32) * nparts) >> 32 for k in a[:, 0]], dtype=np.int64)
        order = np.argsort(g, kind="stable")
        offs = [0] + np.cumsum(np.bincount(g, minlength=nparts)).tolist()
        return torch.from_numpy(np.ascontiguousarray(a[order]).view(ndt)), offs

    def join(Rl, Sl):
        r, s = W.to_numpy_u(Rl), W.to_numpy_u(Sl)
        rr, ss = oracle.hash_join(r, s)
        cnt, c0, c1 = oracle.join_aggregate(r, s)
        return oracle.sorted_pairs(rr, ss), cnt, (c0, c1)

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        R, S = _relations(width)
        (ra, rb), (sa, sb) = _slices(len(R), ws)[rank], _slices(len(S), ws)[rank]
        Rt = torch.from_numpy(np.ascontiguousarray(R[ra:rb]).view(ndt))
        St = torch.from_numpy(np.ascontiguousarray(S[sa:sb]).view(ndt))
        assert Rt.dtype == tdt
        res = D.shard_join(None, Rt, St, split=split, join=join)
        with open(os.path.join(out_dir, f"rank{rank}.pkl"), "wb") as f:
            pickle.dump({"count": res.count, "checksum": res.checksum, "local_count": res.local_count,
                         "pairs": res.local, "received": res.received, "sent": res.sent}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,width", [(2, 4), (2, 8), (3, 4)])
def test_sharded_join_equals_the_whole_join(tmp_path, ws, width):
    import oracle

    mp.start_processes(_rank, args=(ws, _free_port(), width, str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    out = [pickle.load(open(tmp_path / f"rank{r}.pkl", "rb")) for r in range(ws)]
    R, S = _relations(width)
    want = oracle.sorted_pairs(*oracle.hash_join(R, S))
    cnt, c0, c1 = oracle.join_aggregate(R, S)
    got = np.concatenate([o["pairs"] for o in out])
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    assert np.array_equal(got, want)
    for o in out:
        assert o["count"] == cnt == len(want)
        assert o["checksum"] == (c0, c1)
    assert sum(o["local_count"] for o in out) == cnt
    # every tuple was received by exactly one rank
    assert sum(o["received"][0] for o in out) == len(R)
    assert sum(o["received"][1] for o in out) == len(S)
    assert all(o["sent"][0] + o["sent"][1] > 0 for o in out if o["received"] != (0, 0))


def test_one_rank_joins_its_relations_without_an_exchange():
    sys.path.insert(0, ROOT)
    import torch

    import oracle
    from paper_1307_1955_gb300 import dist as D
    from paper_1307_1955_gb300 import workload as W

    R, S = _relations(4)
    calls = []

    def join(Rl, Sl):
        calls.append((len(Rl), len(Sl)))
        r, s = W.to_numpy_u(Rl), W.to_numpy_u(Sl)
        return None, *(lambda a: (a[0], (a[1], a[2])))(oracle.join_aggregate(r, s))

    res = D.shard_join(None, torch.from_numpy(R.view(np.int32)), torch.from_numpy(S.view(np.int32)),
                       split=lambda *a: pytest.fail("no split with one rank"), join=join)
    assert calls == [(len(R), len(S))] and res.sent == (0, 0)
    assert (res.count, *res.checksum) == oracle.join_aggregate(R, S)
