"""Build relations with heavily repeated keys (the paper's skewed data sets,
Sec. 5.1: a fraction s of R's tuples share one key).  Such a key's partition does
not fit shared memory and a pair table would hold it as one long run, so these
joins go through the key-list table (one entry per distinct key with its rid list)
and the grid-wide expansion of long lists.  Results must be the oracle's,
bit-exact: sorted pair multisets, counts and both checksums."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_1955_gb300 import workload as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SEED = W.DEFAULT_SEED


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


def _want(R, S):
    Rn, Sn = W.to_numpy_u(R), W.to_numpy_u(S)
    rr, ss = oracle.hash_join(Rn, Sn)
    return oracle.sorted_pairs(rr, ss), oracle.join_aggregate(Rn, Sn)


def _check(hjm, ctx, R, S, want, agg, **kw):
    res = hjm.hj_join(ctx, R, S, checksum=True, **kw)
    assert (res.count, *res.checksum) == agg
    p = res.pairs_numpy().astype(np.uint64)
    res.free()
    assert np.array_equal(oracle.sorted_pairs(p[:, 0], p[:, 1]), want)
    r2 = hjm.hj_join(ctx, R, S, mode=hjm.HJ_COUNT_CHECKSUM, **kw)
    assert (r2.count, *r2.checksum) == agg


@pytest.mark.parametrize("s", [0.10, 0.25])
def test_heavy_hitter_phj(hjm, ctx, s):
    # |R| = 2^18 with s |R| copies of one key, |S| = 2^20 uniform over R's distinct
    # keys: the heavy partition goes to the key-list fallback, and the few S tuples
    # that meet the heavy key each expand to 26K-66K pairs (grid-wide expansion)
    R, S = W.heavy_hitter(1 << 18, 1 << 20, s, SEED, DEV, ids=(61, int(s * 100)))
    want, agg = _want(R, S)
    assert agg[0] > (1 << 20)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_PHJ, radix_bits=6)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_PHJ, radix_bits=10, passes=2)


@pytest.mark.parametrize("width", [4, 8])
@pytest.mark.parametrize("heavy", [0, 100_000])
def test_keylist_first_table_is_given_up_or_kept(hjm, ctx, width, heavy):
    # One radix bit: both partitions (about 2^18 R rows each) go to the key-list
    # fallback, whose first table is sized for a 32nd as many distinct keys as rows.
    # Distinct keys fill it past half: it is given up and built again at full size.
    # With 100000 copies of one key the distinct keys fit and it is kept.
    dt = np.uint32 if width == 4 else np.uint64
    rng = np.random.default_rng(75 + width)
    nr = 1 << 19
    rk = np.concatenate([np.full(heavy, 7), np.arange(100, 100 + nr - heavy)]).astype(dt)
    rk = rk[rng.permutation(len(rk))]
    sk = np.concatenate([np.full(5, 7), rng.integers(100, 100 + 2 * nr, (1 << 20) - 5)]).astype(dt)
    sk = sk[rng.permutation(len(sk))]
    view = np.int32 if width == 4 else np.int64
    Rg = torch.from_numpy(np.stack([rk, np.arange(nr, dtype=dt)], 1).view(view)).to(DEV)
    Sg = torch.from_numpy(np.stack([sk, np.arange(len(sk), dtype=dt)], 1).view(view)).to(DEV)
    want, agg = _want(Rg, Sg)
    _check(hjm, ctx, Rg, Sg, want, agg, algo=hjm.HJ_ALGO_PHJ, radix_bits=1)


@pytest.mark.parametrize("width", [4, 8])
def test_heavy_key_pairs_past_the_first_capacity(hjm, ctx, width):
    # One key held 40000 times by R and 200 times by S: its partition goes to the
    # key-list fallback, whose 8e6 pairs pass the first pair buffer (|S| plus a chunk
    # per warp) while the partition join's own pairs fit.  The buffer then grows to
    # the exact count and only the fallback runs again (its capacity is the count).
    dt = np.uint32 if width == 4 else np.uint64
    rng = np.random.default_rng(66 + width)
    heavy = 7
    rk = np.concatenate([np.full(40_000, heavy), rng.permutation(np.arange(100, 20_100))]).astype(dt)
    rk = rk[rng.permutation(len(rk))]
    sk = np.concatenate([np.full(200, heavy), rng.integers(100, 40_100, 100_003)]).astype(dt)
    sk = sk[rng.permutation(len(sk))]
    R = np.stack([rk, np.arange(len(rk), dtype=dt)], 1)
    S = np.stack([sk, np.arange(len(sk), dtype=dt)], 1)
    view = np.int32 if width == 4 else np.int64
    Rg = torch.from_numpy(R.view(view)).to(DEV)
    Sg = torch.from_numpy(S.view(view)).to(DEV)
    want, agg = _want(Rg, Sg)
    assert agg[0] > 8_000_000
    res = hjm.hj_join(ctx, Rg, Sg, checksum=True, algo=hjm.HJ_ALGO_PHJ, radix_bits=6)
    assert (res.count, *res.checksum) == agg
    assert res.pairs_cap == res.count  # grown to the exact count, not re-run whole
    p = res.pairs_numpy().astype(np.uint64)
    res.free()
    assert np.array_equal(oracle.sorted_pairs(p[:, 0], p[:, 1]), want)


@pytest.mark.parametrize("s", [0.10, 0.25])
def test_heavy_hitter_shj_and_build_probe(hjm, ctx, s):
    # SHJ: the pair table's build meets a run of repeated keys and the join takes a
    # key-list table instead; hj_build does the same within the call
    R, S = W.heavy_hitter(1 << 17, 1 << 19, s, SEED, DEV, ids=(62, int(s * 100)))
    want, agg = _want(R, S)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_SHJ)
    t = hjm.hj_build(ctx, R)
    try:
        res = hjm.hj_probe(ctx, t, S, checksum=True)
        assert (res.count, *res.checksum) == agg
        p = res.pairs_numpy().astype(np.uint64)
        res.free()
        assert np.array_equal(oracle.sorted_pairs(p[:, 0], p[:, 1]), want)
    finally:
        hjm.hj_table_free(ctx, t)


def test_heavy_all_ones_key_u64(hjm, ctx):
    # the heavy key is all ones (the aggregate table's empty marker): its rids live
    # at the end of the rid array
    R, S = W.heavy_hitter(1 << 16, 1 << 18, 0.2, SEED, DEV, width=8, ids=(63,), heavy_key=(1 << 64) - 1)
    want, agg = _want(R, S)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_PHJ, radix_bits=5)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_SHJ)


def test_moderate_duplicates_warp_lists(hjm, ctx):
    # 200 keys with 3000 copies each (lists the whole warp emits) plus 2^16 unique
    # keys; S uniform over every key, several S tuples per repeated key
    rng = np.random.default_rng(64)
    rep = np.repeat(np.arange(1, 201, dtype=np.uint32), 3000)
    uniq = np.arange(1000, 1000 + (1 << 16), dtype=np.uint32)
    keys = np.concatenate([rep, uniq])
    rng.shuffle(keys)
    Rn = np.stack([keys, np.arange(len(keys), dtype=np.uint32)], 1)
    dom = np.concatenate([np.arange(1, 201, dtype=np.uint32), uniq])
    sk = dom[rng.integers(0, len(dom), 1 << 18)]
    Sn = np.stack([sk, np.arange(len(sk), dtype=np.uint32)], 1)
    R = torch.from_numpy(Rn.view(np.int32)).to(DEV)
    S = torch.from_numpy(Sn.view(np.int32)).to(DEV)
    want, agg = _want(R, S)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_SHJ)
    _check(hjm, ctx, R, S, want, agg, algo=hjm.HJ_ALGO_PHJ, radix_bits=4)


def test_heavy_hitter_full_size_count(hjm, ctx):
    # the paper's default size, 2^24 x 2^24, both skews, through the planner:
    # counts and checksums against the oracle's per-key aggregation
    for s in (0.10, 0.25):
        R, S = W.heavy_hitter(1 << 24, 1 << 24, s, SEED, DEV, ids=(65, int(s * 100)))
        agg = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
        r = hjm.hj_join(ctx, R, S, mode=hjm.HJ_COUNT_CHECKSUM)
        assert (r.count, *r.checksum) == agg
        m = hjm.hj_join(ctx, R, S, checksum=True, algo=hjm.HJ_ALGO_PHJ)
        assert (m.count, *m.checksum) == agg
        m.free()
