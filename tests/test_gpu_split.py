"""hj_split, the local step of the sharded join, on the GPU: group offsets and group
membership exact against the sharding hash computed with the oracle's SplitMix64
finaliser, the output a permutation of the input, and -- the property the sharded
join rests on -- joining group g of R with group g of S for every g gives exactly
the oracle's join of R and S (pairs, count, checksums).  The groups here are
joined on one GPU, one after the other: no collective is involved."""
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


def _groups(keys: np.ndarray, nparts: int) -> np.ndarray:
    return np.array([((oracle.mix_a(int(k)) >> 32) * nparts) >> 32 for k in keys], dtype=np.int64)


def _rows(a: np.ndarray) -> np.ndarray:
    return a[np.lexsort((a[:, 1], a[:, 0]))]


@pytest.mark.parametrize("width", [4, 8])
@pytest.mark.parametrize("n,nparts", [(0, 4), (1, 3), (100_003, 1), (100_003, 2), (250_001, 8), (70_001, 4096)])
def test_split_groups_exactly(hjm, ctx, width, n, nparts):
    if width == 4:
        rel, _ = W.unique_and_uniform(n, 0, 1, SEED, DEV, ids=(50, n))
    else:
        rel, _ = W.zipf_pair(n, 0, 0.75, 0.5, 1 << 14, SEED, DEV, ids=(50, n))
    out, offs = hjm.hj_split(ctx, rel, nparts)
    a, b = W.to_numpy_u(rel), W.to_numpy_u(out)
    g = _groups(a[:, 0], nparts)
    want = [0] + np.cumsum(np.bincount(g, minlength=nparts)).tolist()
    assert offs == want
    assert np.array_equal(_rows(a), _rows(b))               # a permutation of the input
    gb = _groups(b[:, 0], nparts)
    for p in range(nparts):                                 # every row in its group's range
        assert (gb[offs[p]:offs[p + 1]] == p).all()


@pytest.mark.parametrize("width,nparts", [(4, 4), (4, 3), (8, 4)])
def test_groupwise_joins_make_the_whole_join(hjm, ctx, width, nparts):
    if width == 4:
        R, S = W.unique_and_uniform(300_001, 1_200_007, 600_000, SEED, DEV, ids=(51,))
    else:
        R, S = W.zipf_pair(40_000, 200_000, 0.75, 0.5, 1 << 13, SEED, DEV, ids=(51,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    want = oracle.sorted_pairs(*oracle.hash_join(r, s))
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    Rg, ro = hjm.hj_split(ctx, R, nparts)
    Sg, so = hjm.hj_split(ctx, S, nparts)
    pairs, tot, t0, t1 = [], 0, 0, 0
    for p in range(nparts):
        # (a group can start at an odd row: cloned, so that it starts on 16 bytes)
        res = hjm.hj_join(ctx, Rg[ro[p]:ro[p + 1]].clone(), Sg[so[p]:so[p + 1]].clone(), checksum=True)
        pairs.append(res.pairs_numpy().astype(np.uint64))
        tot += res.count
        t0 = (t0 + res.checksum[0]) & ((1 << 64) - 1)
        t1 = (t1 + res.checksum[1]) & ((1 << 64) - 1)
        res.free()
    got = np.concatenate(pairs)
    assert np.array_equal(oracle.sorted_pairs(got[:, 0], got[:, 1]), want)
    assert (tot, t0, t1) == (cnt, c0, c1)


def test_shard_join_on_one_gpu_is_the_join(hjm, ctx):
    from paper_1307_1955_gb300 import dist as D

    R, S = W.unique_and_uniform(50_000, 400_000, 100_000, SEED, DEV, ids=(52,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    res = D.shard_join(ctx, R, S)
    assert (res.count, *res.checksum) == oracle.join_aggregate(r, s)
    got = res.local.pairs_numpy().astype(np.uint64)
    res.local.free()
    assert np.array_equal(oracle.sorted_pairs(got[:, 0], got[:, 1]), oracle.sorted_pairs(*oracle.hash_join(r, s)))


def test_split_rejects_bad_arguments(hjm, ctx):
    R, _ = W.unique_and_uniform(100, 0, 1, SEED, DEV, ids=(53,))
    for nparts in (0, 4097):
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_split(ctx, R, nparts)
        assert e.value.status == hjm.HJ_E_INVALID
