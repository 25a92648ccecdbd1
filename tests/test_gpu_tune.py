"""hj_tune: the model's cheapest plans timed on the device; the fastest is cached
for the size class and hj_join with HJ_ALGO_AUTO then runs it.  Whatever plan runs,
the result is the oracle's (bit-exact)."""
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


def test_tuned_plan_is_used_and_exact(hjm):
    R, S = W.unique_and_uniform(1 << 18, 1 << 20, 1 << 19, W.DEFAULT_SEED, DEV, ids=(31,))
    want = oracle.sorted_pairs(*oracle.hash_join(W.to_numpy_u(R), W.to_numpy_u(S)))
    with hjm.Context(0) as ctx:
        model = hjm.hj_plan(ctx, R, S)
        tuned = hjm.hj_tune(ctx, R, S, top_k=4)
        assert tuned["measured_ms"] > 0 and tuned["predicted_ms"] > 0
        res = hjm.hj_join(ctx, R, S)
        assert (res.algo, res.radix_bits, res.passes) == (tuned["algo"], tuned["radix_bits"], tuned["passes"])
        got = res.pairs_numpy().astype(np.uint64)
        res.free()
        assert np.array_equal(oracle.sorted_pairs(got[:, 0], got[:, 1]), want)
        assert hjm.hj_plan(ctx, R, S)["algo"] == tuned["algo"]
        # another size class is untouched; clearing the cache restores the model's plan
        hjm.hj_tune_clear(ctx)
        assert hjm.hj_plan(ctx, R, S)["algo"] == model["algo"]


def test_every_candidate_plan_gives_the_same_result(hjm):
    R, S = W.unique_and_uniform(40000, 300000, 60000, W.DEFAULT_SEED, DEV, ids=(32,))
    cnt, c0, c1 = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
    with hjm.Context(0) as ctx:
        for algo, bits, passes in ((1, 0, 0), (2, 1, 1), (2, 3, 1), (2, 8, 2), (2, 12, 1), (2, 13, 2)):
            r = hjm.hj_join(ctx, R, S, algo=algo, radix_bits=bits, passes=passes, mode=hjm.HJ_COUNT_CHECKSUM)
            assert (r.count, *r.checksum) == (cnt, c0, c1), (algo, bits, passes)


def test_profiling_one_kernel_brackets_only_its_launches(hjm):
    # hj_prof_only: event timing restricted to one kernel name; every launch is
    # still counted, and the result is unchanged.
    R, S = W.unique_and_uniform(1 << 16, 1 << 18, 1 << 17, W.DEFAULT_SEED, DEV, ids=(32,))
    cnt, c0, c1 = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
    with hjm.Context(0) as ctx:
        hjm.prof_reset(ctx)
        hjm.prof_enable(ctx, True)
        r = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=6, mode=hjm.HJ_COUNT_CHECKSUM)
        every = hjm.prof_read(ctx)
        assert "partition_join" in every and "partition_scatter" in every and len(every) > 2
        hjm.prof_reset(ctx)
        hjm.prof_only(ctx, "partition_join")
        n0 = hjm.launch_count(ctx)
        r2 = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=6, mode=hjm.HJ_COUNT_CHECKSUM)
        one = hjm.prof_read(ctx)
        assert set(one) == {"partition_join"} and one["partition_join"][0] == every["partition_join"][0]
        assert one["partition_join"][1] > 0
        assert hjm.launch_count(ctx) - n0 == sum(v[0] for v in every.values())
        hjm.prof_only(ctx, None)
        hjm.prof_enable(ctx, False)
        assert (r.count, *r.checksum) == (r2.count, *r2.checksum) == (cnt, c0, c1)
