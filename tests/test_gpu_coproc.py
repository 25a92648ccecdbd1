"""hj_join_coproc: the PHJ with its join step divided between the GPU and host
threads (the paper's data dividing applied to the join step).  For every CPU share
-- none, 10 %, half, all -- the result must be exactly the oracle's: sorted pair
multisets, counts and both checksums (join results are integers)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_1955_gb300 import workload as W

pytestmark = pytest.mark.gpu

SEED = W.DEFAULT_SEED
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


def _check(hjm, ctx, R, S, share, **kw):
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    want = oracle.sorted_pairs(*oracle.hash_join(r, s))
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    res, t = hjm.hj_join_coproc(ctx, R, S, share, checksum=True, **kw)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    got = res.pairs_numpy().astype(np.uint64)
    res.free()
    assert np.array_equal(oracle.sorted_pairs(got[:, 0], got[:, 1]), want)
    for mode in (hjm.HJ_COUNT, hjm.HJ_COUNT_CHECKSUM):
        r2, _ = hjm.hj_join_coproc(ctx, R, S, share, mode=mode, **kw)
        assert r2.count == cnt and r2.pairs_ptr == 0
        if mode == hjm.HJ_COUNT_CHECKSUM:
            assert r2.checksum == (c0, c1)
    return t


@pytest.mark.parametrize("share", [0.0, 0.1, 0.5, 1.0])
def test_coproc_u32_half_match(hjm, ctx, share):
    R, S = W.unique_and_uniform((1 << 18) + 3, (1 << 21) + 5, 1 << 19, SEED, DEV, ids=(60,))
    t = _check(hjm, ctx, R, S, share, radix_bits=9)
    assert t["partition_gpu"] > 0 and t["total"] > 0
    if share > 0:
        assert t["join_cpu"] > 0 and t["copy_to_host"] > 0
    else:
        assert t["join_cpu"] == 0


@pytest.mark.parametrize("share,threads", [(0.1, 1), (0.5, 3)])
def test_coproc_u64_skewed_duplicates(hjm, ctx, share, threads):
    R, S = W.zipf_pair(30_000, 200_000, 0.75, 0.5, 1 << 12, SEED, DEV, ids=(61,))
    _check(hjm, ctx, R, S, share, cpu_threads=threads, radix_bits=6)


def test_coproc_two_passes_and_a_heavy_key(hjm, ctx):
    # a key repeated 30000 times in R (its partition overflows shared memory on the
    # GPU side, and is a long rid list on the CPU side), two partition passes
    rng = np.random.default_rng(62)
    rk = np.concatenate([np.full(30000, 7, np.uint32), rng.integers(8, 1 << 20, 20000).astype(np.uint32)])
    R = np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1)
    sk = rng.integers(1, 1 << 20, 40000).astype(np.uint32)
    sk[:3] = 7
    S = np.stack([sk, np.arange(len(sk), dtype=np.uint32)], 1)
    Rg = torch.from_numpy(R.view(np.int32)).to(DEV)
    Sg = torch.from_numpy(S.view(np.int32)).to(DEV)
    for share in (0.3, 0.8):
        _check(hjm, ctx, Rg, Sg, share, radix_bits=8, passes=2)


def test_coproc_rejects_bad_arguments(hjm, ctx):
    R, S = W.unique_and_uniform(100, 100, 100, SEED, DEV, ids=(63,))
    for share in (-0.1, 1.5, float("nan")):
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_join_coproc(ctx, R, S, share)
        assert e.value.status == hjm.HJ_E_INVALID
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join_coproc(ctx, R, S, 0.5, cpu_threads=-1)
    assert e.value.status == hjm.HJ_E_INVALID
