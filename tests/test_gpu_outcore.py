"""hj_join_host_large: relations in host memory joined through a device budget far
smaller than they are (the paper's larger-than-buffer join, App. A).  The result
must be the oracle's (bit-exact), whatever the number of top-level partitions and
S groups the budget forces."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_1955_gb300 import workload as W

pytestmark = pytest.mark.gpu


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


def _sorted(p):
    p = np.asarray(p, np.uint64)
    return p[np.lexsort((p[:, 1], p[:, 0]))] if len(p) else p.reshape(0, 2)


@pytest.mark.parametrize("budget_mb", [160, 240, 4096])
def test_large_join_through_a_small_budget_matches_oracle(hjm, ctx, budget_mb):
    R, S = W.unique_and_uniform(1 << 20, 1 << 23, 1 << 21, W.DEFAULT_SEED, "cpu", ids=(40,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    want = oracle.sorted_pairs(*oracle.hash_join(r, s))
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    out = torch.empty((len(want) + 16, 2), dtype=torch.int32)
    res = hjm.hj_join_host_large(ctx, R, S, out, device_bytes=budget_mb << 20, checksum=True)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    got = out[:res.count].numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(_sorted(got), want)
    if budget_mb < 4096:
        assert res.radix_bits >= 1  # the top-level split ran
    cr = hjm.hj_join_host_large(ctx, R, S, None, device_bytes=budget_mb << 20, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (cr.count, *cr.checksum) == (cnt, c0, c1)


def test_large_join_skewed_u64_groups_of_s(hjm, ctx):
    # A hot S key makes one partition's S side far larger than the budget allows next
    # to its R partition: it is joined in S groups.
    # (|S| = 2^25 with S theta 1.2: the top key alone is about 6e6 tuples, more than
    # the 192 MB budget holds next to its R partition.)
    R, S = W.zipf_pair(1 << 16, 1 << 25, 0.5, 1.2, 1 << 14, W.DEFAULT_SEED, "cpu", ids=(41,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    res = hjm.hj_join_host_large(ctx, R, S, None, device_bytes=192 << 20, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    assert res.radix_bits >= 4


def test_large_join_overflow_reports_the_count(hjm, ctx):
    R, S = W.unique_and_uniform(1 << 18, 1 << 21, 1 << 18, W.DEFAULT_SEED, "cpu", ids=(42,))
    out = torch.empty((1000, 2), dtype=torch.int32)
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join_host_large(ctx, R, S, out, device_bytes=160 << 20)
    assert e.value.status == hjm.HJ_E_OVERFLOW
    # a budget below the fixed workspace of one join is refused up front
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join_host_large(ctx, R, S, out, device_bytes=32 << 20)
    assert e.value.status == hjm.HJ_E_INVALID
