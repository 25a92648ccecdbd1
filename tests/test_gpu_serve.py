"""hj_server: continuous batching of join requests.  Requests of different sizes
arrive from a client thread while others run; each served result must equal the
oracle's and be byte-identical to what hj_join returns for the same request
alone (the tolerance is zero: all join arithmetic is integer)."""
import random
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1307_1955_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hjm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1307_1955_gb300 import hj

    return hj


@pytest.fixture(scope="module")
def ctx(hjm):
    c = hjm.Context(0)
    yield c
    c.close()


def _sorted_pairs(res):
    p = res.pairs_numpy().astype(np.uint64)
    return p[np.lexsort((p[:, 1], p[:, 0]))] if len(p) else p.reshape(0, 2)


def _requests(n, seed, lo=6.0, hi=16.0):
    """Serving-shaped requests (|S| between |R| and 16 |R|, half of S matching),
    scaled down: one seeded relation pair per request."""
    specs = W.serving_specs(n, seed, 1.0, lo_log2=lo, hi_log2=hi)
    specs += [W.JoinSpec(0, 50, 10), W.JoinSpec(40, 0, 80), W.JoinSpec(1, 1, 2)]
    R, S, rs, ss = W.batched_relations(specs, seed, DEV, ids=(5,))
    return [(R[rs[j]:rs[j] + sp.n_r], S[ss[j]:ss[j] + sp.n_s]) for j, sp in enumerate(specs)]


def _alone(hjm, ctx, reqs, mode):
    out = []
    for R, S in reqs:
        res = hjm.hj_join(ctx, R, S, mode=mode, checksum=mode == hjm.HJ_MATERIALIZE)
        pairs = _sorted_pairs(res) if mode == hjm.HJ_MATERIALIZE else None
        out.append((res.count, res.checksum if mode != hjm.HJ_COUNT else None, pairs))
        res.free()
    return out


def _serve(srv, reqs, mode, seed, max_gap_s=0.002):
    """Submit from a client thread in bursts of 1 to 16 requests with random gaps
    between bursts (so that some requests queue behind running waves); collect on
    this thread."""
    ids = [None] * len(reqs)
    ready = [threading.Event() for _ in reqs]

    def client():
        rng = random.Random(seed)
        burst = 0
        for i, (R, S) in enumerate(reqs):
            ids[i] = srv.submit(R, S, mode)
            ready[i].set()
            if burst == 0:
                time.sleep(rng.random() * max_gap_s)
                burst = rng.randint(1, 16)
            burst -= 1

    th = threading.Thread(target=client)
    th.start()
    got = []
    for i in range(len(reqs)):
        ready[i].wait(60)
        r = srv.wait(ids[i], 120.0)
        assert r is not None, f"request {i} did not finish"
        res, t = r
        assert t.submit <= t.admit <= t.start <= t.done
        got.append(res)
    th.join()
    return got


def test_served_equals_alone_and_oracle(hjm, ctx):
    reqs = _requests(48, 0x5E1)
    want = _alone(hjm, ctx, reqs, hjm.HJ_MATERIALIZE)
    with hjm.Server(ctx, workers=3, max_wave=8) as srv:
        got = _serve(srv, reqs, hjm.HJ_MATERIALIZE, 1)
        for i, res in enumerate(got):
            cnt, _, pairs = want[i]
            assert res.count == cnt, i
            assert np.array_equal(_sorted_pairs(res), pairs), i
            res.free()
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["waves"] >= 2 and st["wave_max"] >= 2
        assert st["in_use"] == 0
    # the oracle on a seeded sample of the requests
    for i in random.Random(7).sample(range(len(reqs)), 8):
        R, S = reqs[i]
        rr, ss = oracle.hash_join(W.to_numpy_u(R), W.to_numpy_u(S))
        assert np.array_equal(oracle.sorted_pairs(rr, ss), want[i][2]), i


@pytest.mark.parametrize("mode", ["count", "checksum"])
def test_served_count_modes_and_graph_waves(hjm, ctx, mode):
    m = hjm.HJ_COUNT if mode == "count" else hjm.HJ_COUNT_CHECKSUM
    reqs = _requests(40, 0x5E2)
    want = _alone(hjm, ctx, reqs, m)
    with hjm.Server(ctx, workers=2, max_wave=16, graph=True) as srv:
        got = _serve(srv, reqs, m, 2, max_gap_s=0.0005)
        for i, res in enumerate(got):
            assert res.count == want[i][0], i
            if m == hjm.HJ_COUNT_CHECKSUM:
                assert res.checksum == want[i][1], i
            assert res.pairs_ptr == 0
    for i in (0, 5, 17):
        R, S = reqs[i]
        cnt, c0, c1 = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
        assert want[i][0] == cnt
        if m == hjm.HJ_COUNT_CHECKSUM:
            assert want[i][1] == (c0, c1)


def test_mixed_widths_and_modes_keep_fifo(hjm, ctx):
    small = _requests(12, 0x5E3, lo=5.0, hi=12.0)
    R64, S64 = W.zipf_pair(3000, 20000, 0.75, 0.5, 1 << 12, W.DEFAULT_SEED, DEV, ids=(9,))
    reqs = [(R, S, hjm.HJ_MATERIALIZE) for R, S in small[:6]] + [(R64, S64, hjm.HJ_COUNT_CHECKSUM)] + \
           [(R, S, hjm.HJ_COUNT) for R, S in small[6:]]
    with hjm.Server(ctx, workers=2) as srv:
        ids = [srv.submit(R, S, m) for R, S, m in reqs]
        for (R, S, m), rid in zip(reqs, ids):
            res, _ = srv.wait(rid, 120.0)
            alone = hjm.hj_join(ctx, R, S, mode=m)
            assert (res.count, res.checksum if m == hjm.HJ_COUNT_CHECKSUM else 0) == \
                   (alone.count, alone.checksum if m == hjm.HJ_COUNT_CHECKSUM else 0)
            if m == hjm.HJ_MATERIALIZE:
                assert np.array_equal(_sorted_pairs(res), _sorted_pairs(alone))
            alone.free()
            res.free()


def test_budget_bounds_admission(hjm, ctx):
    reqs = _requests(16, 0x5E4, lo=12.0, hi=14.0)
    tb = 8
    need = max((R.shape[0] + S.shape[0]) * tb * 11 // 10 + (16 << 20) + (S.shape[0] + 65536) * tb
               for R, S in reqs)
    budget = need + need // 2  # room for one request at a time
    with hjm.Server(ctx, budget=budget, workers=3) as srv:
        ids = [srv.submit(R, S) for R, S in reqs]
        for (R, S), rid in zip(reqs, ids):
            res, _ = srv.wait(rid, 120.0)
            alone = hjm.hj_join(ctx, R, S)
            assert res.count == alone.count
            alone.free()
            res.free()
        st = srv.stats()
        assert st["peak_in_use"] <= budget
        # a request larger than the whole budget is refused at once
        big = torch.zeros((budget // 8, 2), dtype=torch.int32, device=DEV)
        with pytest.raises(hjm.HJError) as e:
            srv.submit(big, big)
        assert e.value.status == hjm.HJ_E_NOMEM


def test_poll_pending_and_destroy_drains(hjm, ctx):
    reqs = _requests(20, 0x5E5)
    srv = hjm.Server(ctx, workers=2)
    ids = [srv.submit(R, S) for R, S in reqs]
    r = srv.poll(ids[-1])  # most likely still queued or running: None, or a finished result
    if r is not None:
        r[0].free()
    res, _ = srv.wait(ids[0], 120.0)
    res.free()
    with pytest.raises(hjm.HJError):
        srv.poll(ids[0])  # collected already
    srv.close()  # the rest are run to completion and released
    torch.cuda.synchronize()
