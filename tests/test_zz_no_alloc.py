"""hj_join_static, the simple hash join that allocates nothing.

It serves callers that may not allocate device memory (for example a host process
whose device memory is owned by another allocator, or a loop that forbids
allocation after start-up): its scratch is one fixed device array inside the
library and the caller brings the pair buffer.  Here it is called through the C ABI
twice in a row, on different inputs, and each result must equal both what the
ordinary entry point (hj_join with the SHJ algorithm) returns and what the CPU
oracle computes: same pair multiset, count and checksums -- join results are
integers, so the comparison is exact.  The oracle shares no code with either CUDA
path, so a fault in the table code the two entry points share cannot cancel out.
The second call also checks that nothing left in the shared scratch by the first
call leaks into it.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
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


def _sorted(p: np.ndarray) -> np.ndarray:
    p = p.astype(np.uint64)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def _reference(hjm, R, S):
    with hjm.Context(0) as ctx:
        res = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_SHJ, checksum=True)
        out = (_sorted(res.pairs_numpy()), res.count, res.checksum)
        res.free()
    return out


def _oracle(R, S):
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    rr, ss = oracle.hash_join(r, s)
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    return oracle.sorted_pairs(rr, ss), cnt, (c0, c1)


def _static(hjm, R, S, cap, stream=None):
    dt = R.dtype
    pairs = torch.empty((cap, 2), dtype=dt, device=DEV)
    count, chk = hjm.hj_join_static(R, S, pairs, stream=stream)
    got = pairs[:count].cpu().numpy().view(np.uint32 if dt == torch.int32 else np.uint64)
    return _sorted(got), count, chk


def test_static_join_matches_hj_join_on_two_calls_in_a_row(hjm):
    # first call: unique R keys, half of S matching; second call: a 64-bit skewed
    # join with duplicates on both sides, smaller than the first, so that stale
    # table entries or counters from call one would show up in call two
    R1, S1 = W.unique_and_uniform(300_001, 1_000_003, 600_000, W.DEFAULT_SEED, DEV, ids=(20,))
    R2, S2 = W.zipf_pair(20_000, 90_000, 0.75, 0.5, 1 << 12, W.DEFAULT_SEED, DEV, ids=(21,))
    for R, S in ((R1, S1), (R2, S2)):
        want = _reference(hjm, R, S)
        ora = _oracle(R, S)
        got = _static(hjm, R, S, want[1] + 64)
        assert got[1] == want[1] == ora[1]
        assert got[2] == want[2] == ora[2]
        assert np.array_equal(got[0], want[0])
        assert np.array_equal(got[0], ora[0])


def test_static_join_follows_the_stream_that_made_its_inputs(hjm):
    # inputs made on a side torch stream and the join issued on that stream as the
    # current one: the default stream argument orders the join after the generation
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        R, S = W.unique_and_uniform(200_000, 800_000, 200_000, W.DEFAULT_SEED, DEV, ids=(23,))
        got = _static(hjm, R, S, 800_064)
    side.synchronize()
    ora = _oracle(R, S)
    assert got[1] == 800_000 == ora[1]          # every S key is an R key, R keys unique
    assert got[2] == ora[2]
    assert np.array_equal(got[0], ora[0])


def test_static_join_reports_overflow_and_size_limit(hjm):
    R, S = W.unique_and_uniform(5000, 20000, 5000, W.DEFAULT_SEED, DEV, ids=(22,))
    small = torch.empty((10, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join_static(R, S, small)
    assert e.value.status == hjm.HJ_E_OVERFLOW and e.value.count == 20000
    big = torch.zeros((2_097_152, 2), dtype=torch.int32, device=DEV)  # one tuple over the limit
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join_static(big, S, small)
    assert e.value.status == hjm.HJ_E_NOMEM
