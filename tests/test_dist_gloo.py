"""The multi-rank path of the bench on CPU: two gloo ranks, each joining its own
seeded relations (independent problems, no exchange of tuples), combined by the
bench's max-over-ranks time and whole-job throughput."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1307_1955_gb300 import workload as W

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = dict(nr=3000, ns=12000, dom=6000)
        R, S = bench.make_inputs(wl, rank, "cpu")  # the bench's own per-rank inputs
        rr, ss = oracle.hash_join(W.to_numpy_u(R), W.to_numpy_u(S))
        local_ms = 1.0 + rank  # rank r takes r + 1 ms per step
        ms = bench.ranks_max(local_ms, ws)
        value = bench.weak_value(wl["nr"] + wl["ns"], 4, ws, ms)
        counts = [None] * ws
        dist.all_gather_object(counts, (len(rr), int(R[:, 0].sum()), int(S[:, 0].sum())))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "value": value, "counts": counts}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_joins(tmp_path):
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["ms"] == 2.0  # the slowest rank's time
        assert r["value"] == pytest.approx((3000 + 12000) * 4 * ws / 2e-3)
    counts = res[0]["counts"]
    assert counts == res[1]["counts"]
    # each rank drew its own relations: different keys, each a valid join
    assert counts[0][1:] != counts[1][1:]
    for c in counts:
        assert 0 < c[0] <= 12000


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.ranks_max(3.5, 1) == 3.5
    assert bench.weak_value(100, 10, 1, 1000.0) == 1000.0
