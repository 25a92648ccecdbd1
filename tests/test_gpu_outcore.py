"""Joins of relations in host memory.  hj_join_host_large joins them through a
device budget far smaller than they are (the paper's larger-than-buffer join,
App. A); hj_join_host streams a large S through the device in chunks whose copies
overlap the joins.  The result must be the oracle's (bit-exact), whatever the
number of top-level partitions, S groups or chunks."""
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


@pytest.fixture(scope="module")
def lib(hjm):
    return hjm.load_library()


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("budget_mb", [160, 240, 4096])
def test_large_join_through_a_small_budget_matches_oracle(hjm, lib, budget_mb, split):
    # 160 MB: R does not fit beside two S chunks and their pair buffers, so the
    # relations are split (App. A); 240 MB: R stays on the device and S streams past
    # it in 2^20-row chunks, unless the split is forced; 4096 MB: one join.  The
    # device bytes the context holds never pass the budget.
    R, S = W.unique_and_uniform(1 << 20, 1 << 23, 1 << 21, W.DEFAULT_SEED, "cpu", ids=(40,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    want = oracle.sorted_pairs(*oracle.hash_join(r, s))
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    out = torch.empty((len(want) + 16, 2), dtype=torch.int32)
    with hjm.Context(0) as c:
        assert lib.hj_debug_outcore(c.handle, hjm.HJ_OUTCORE_SPLIT if split else hjm.HJ_OUTCORE_AUTO) == hjm.HJ_OK
        lib.hj_debug_peak_bytes(c.handle, 1)
        res = hjm.hj_join_host_large(c, R, S, out, device_bytes=budget_mb << 20, checksum=True)
        peak = lib.hj_debug_peak_bytes(c.handle, 1)
        assert (res.count, *res.checksum) == (cnt, c0, c1)
        got = out[:res.count].numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(_sorted(got), want)
        if budget_mb == 240 and not split:
            assert res.passes == 1  # R resident, S streamed
        elif budget_mb < 4096:
            assert res.passes == 0 and res.radix_bits >= 1  # the top-level split ran
        assert peak <= budget_mb << 20, (peak, budget_mb)
        cr = hjm.hj_join_host_large(c, R, S, None, device_bytes=budget_mb << 20, mode=hjm.HJ_COUNT_CHECKSUM)
        assert (cr.count, *cr.checksum) == (cnt, c0, c1)
        assert lib.hj_debug_peak_bytes(c.handle, 0) <= budget_mb << 20


def test_outcore_hook_rejects_bad_modes(hjm, lib):
    with hjm.Context(0) as c:
        for m in (-1, 2):
            assert lib.hj_debug_outcore(c.handle, m) == 1  # HJ_E_INVALID
    assert lib.hj_debug_outcore(None, 0) == 1


@pytest.mark.parametrize("split", [True, False])
def test_large_join_skewed_u64_groups_of_s(hjm, lib, split):
    # Split: a hot S key makes one partition's S side far larger than the budget
    # allows next to its R partition, so it is joined in S groups.  (|S| = 2^25 with
    # S theta 1.2: the top key alone is about 6e6 tuples, more than the 192 MB budget
    # holds next to its R partition.)  Not split: R stays on the device and the hot
    # key's tuples pass in S chunks.
    R, S = W.zipf_pair(1 << 16, 1 << 25, 0.5, 1.2, 1 << 14, W.DEFAULT_SEED, "cpu", ids=(41,))
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    with hjm.Context(0) as c:
        assert lib.hj_debug_outcore(c.handle, hjm.HJ_OUTCORE_SPLIT if split else hjm.HJ_OUTCORE_AUTO) == hjm.HJ_OK
        res = hjm.hj_join_host_large(c, R, S, None, device_bytes=192 << 20, mode=hjm.HJ_COUNT_CHECKSUM)
        assert (res.count, *res.checksum) == (cnt, c0, c1)
        if split:
            assert res.passes == 0 and res.radix_bits >= 4
        else:
            assert res.passes == 1


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


def _pairs_u64(t):
    return _sorted(t.numpy().view(np.uint32 if t.dtype == torch.int32 else np.uint64).astype(np.uint64))


def test_host_join_in_chunks_equals_device_join(hjm, ctx):
    # hj_join_host on a large S runs chunk by chunk, copies overlapping the joins
    # (several chunks, the last ragged); its pair multiset is the device join's and
    # its count and checksums the oracle's.
    R, S = W.unique_and_uniform(1 << 21, (1 << 25) + 12345, 1 << 22, W.DEFAULT_SEED, "cpu", ids=(43,))
    cnt, c0, c1 = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
    Rh, Sh = R.pin_memory(), S.pin_memory()
    out = torch.empty((cnt + 16, 2), dtype=torch.int32).pin_memory()
    res = hjm.hj_join_host(ctx, Rh, Sh, out, checksum=True)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    dev = hjm.hj_join(ctx, R.cuda(), S.cuda())
    assert np.array_equal(_pairs_u64(out[:res.count]), _sorted(dev.pairs_numpy()))
    dev.free()
    cm = hjm.hj_join_host(ctx, Rh, Sh, None, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (cm.count, *cm.checksum) == (cnt, c0, c1)


def test_host_join_in_chunks_u64_all_modes(hjm, ctx):
    # 8-byte tuples through the chunked host join: counts and checksums in every
    # mode are the oracle's, and every materialised pair joins equal keys.
    R, S = W.unique_and_uniform(1 << 20, (1 << 25) + 777, 1 << 21, W.DEFAULT_SEED, "cpu", width=8, ids=(44,))
    Ru, Su = W.to_numpy_u(R), W.to_numpy_u(S)
    cnt, c0, c1 = oracle.join_aggregate(Ru, Su)
    Rh, Sh = R.pin_memory(), S.pin_memory()
    assert hjm.hj_join_host(ctx, Rh, Sh, None, mode=hjm.HJ_COUNT).count == cnt
    cm = hjm.hj_join_host(ctx, Rh, Sh, None, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (cm.count, *cm.checksum) == (cnt, c0, c1)
    out = torch.empty((cnt + 16, 2), dtype=torch.int64).pin_memory()
    res = hjm.hj_join_host(ctx, Rh, Sh, out, checksum=True)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    got = out[:res.count].numpy().view(np.uint64)
    assert np.array_equal(Ru[got[:, 0].astype(np.int64), 0], Su[got[:, 1].astype(np.int64), 0])


def test_host_join_chunk_overflowing_its_buffer_is_rejoined(hjm, ctx):
    # The first chunk of S matches twice per tuple (R holds every key of its range
    # twice): more pairs than that chunk's buffer, so it is joined again on its own.
    n = 1 << 20
    keys = np.concatenate([np.arange(1, n + 1), np.arange(1, (n >> 2) + 1)]).astype(np.uint32)
    R = torch.from_numpy(np.stack([keys, np.arange(len(keys), dtype=np.uint32)], 1).view(np.int32))
    ns = (1 << 25) + 99
    rng = np.random.default_rng(5)
    sk = rng.integers(1, n + 1, ns).astype(np.uint32)
    sk[:1 << 24] = rng.integers(1, (n >> 2) + 1, 1 << 24).astype(np.uint32)
    S = torch.from_numpy(np.stack([sk, np.arange(ns, dtype=np.uint32)], 1).view(np.int32))
    cnt, c0, c1 = oracle.join_aggregate(W.to_numpy_u(R), W.to_numpy_u(S))
    assert cnt > (1 << 24) * 2
    out = torch.empty((cnt + 16, 2), dtype=torch.int32).pin_memory()
    res = hjm.hj_join_host(ctx, R.pin_memory(), S.pin_memory(), out, checksum=True)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    got = out[:res.count].numpy().view(np.uint32)
    # every pair joins equal keys, and no pair appears twice
    assert np.array_equal(keys[got[:, 0]], sk[got[:, 1]])
    code = np.sort(got[:, 0].astype(np.uint64) << np.uint64(32) | got[:, 1].astype(np.uint64))
    assert not np.any(code[1:] == code[:-1])
