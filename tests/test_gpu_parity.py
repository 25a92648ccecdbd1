"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle on
the same seeded inputs.  All join work is integer: results must be bit-exact
(sorted pair multisets, counts and both checksums identical)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1307_1955_gb300 import workload as W

pytestmark = pytest.mark.gpu

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


DEV = "cuda:0"


def _np(t):
    return W.to_numpy_u(t)


def _gpu(a: np.ndarray) -> torch.Tensor:
    dt = torch.int32 if a.dtype == np.uint32 else torch.int64
    return torch.from_numpy(a.view(np.int32 if a.dtype == np.uint32 else np.int64).copy()).to(DEV)


def _oracle(R, S):
    rr, ss = oracle.hash_join(_np(R), _np(S))
    return oracle.sorted_pairs(rr, ss)


def _got(res):
    p = res.pairs_numpy().astype(np.uint64)
    res.free()
    return oracle.sorted_pairs(p[:, 0], p[:, 1])


def _check_all_modes(hjm, ctx, R, S, **kw):
    """Materialised pairs, and both count modes, against the oracle."""
    want = _oracle(R, S)
    cnt, c0, c1 = oracle.join_aggregate(_np(R), _np(S))
    assert cnt == len(want)
    res = hjm.hj_join(ctx, R, S, mode=hjm.HJ_MATERIALIZE, checksum=True, **kw)
    assert res.count == len(want)
    assert res.checksum == (c0, c1)
    got = _got(res)
    assert np.array_equal(got, want)
    r1 = hjm.hj_join(ctx, R, S, mode=hjm.HJ_COUNT, **kw)
    assert r1.count == cnt and r1.pairs_ptr == 0
    r2 = hjm.hj_join(ctx, R, S, mode=hjm.HJ_COUNT_CHECKSUM, **kw)
    assert (r2.count, *r2.checksum) == (cnt, c0, c1)
    return res


# ----------------------------------------------------------------- configurations


def test_shj_unique_keys_full_size(hjm, ctx):
    # SHJ, |R| = |S| = 2^20, R keys a permutation, S keys drawn from R's keys.
    n = 1 << 20
    R, S = W.unique_and_uniform(n, n, n, SEED, DEV, ids=(1,))
    res = _check_all_modes(hjm, ctx, R, S, algo=hjm.HJ_ALGO_SHJ)
    assert res.algo == hjm.HJ_ALGO_SHJ


@pytest.mark.parametrize("bits,passes", [(1, 1), (5, 1), (8, 1), (11, 1), (12, 1), (2, 2), (9, 2), (12, 2), (13, 2),
                                         (14, 2), (21, 2), (22, 2)])
def test_phj_half_match_scaled(hjm, ctx, bits, passes):
    # (11 bits in one pass is the plan the tuner picks at full size, (12, 2) the
    # model's plan for twice that build side, and (21, 2) /
    # (22, 2) put 11-bit passes first / in both passes: the ring scatter at its
    # chunk and segment paths.)
    # PHJ on the |R| = 2^24, |S| = 2^28 workload scaled by 2^-8 (ragged sizes):
    # R unique, S keys uniform over twice R's key range (about half match).
    nr, ns = (1 << 16) + 37, (1 << 20) + 11
    R, S = W.unique_and_uniform(nr, ns, 2 * nr, SEED, DEV, ids=(2, bits, passes))
    res = _check_all_modes(hjm, ctx, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=bits, passes=passes)
    assert (res.algo, res.radix_bits, res.passes) == (hjm.HJ_ALGO_PHJ, bits, passes)


@pytest.mark.parametrize("theta_s", [0.5, 1.0])
def test_phj_zipf_u64_scaled(hjm, ctx, theta_s):
    # Skewed 64-bit workload scaled down: |R| = 2^14, |S| = 2^18, Zipf keys over 2^12
    # ranks (R theta 0.75); duplicates on both sides.
    R, S = W.zipf_pair(1 << 14, 1 << 18, 0.75, theta_s, 1 << 12, SEED, DEV, ids=(3, int(theta_s * 10)))
    cnt, c0, c1 = oracle.join_aggregate(_np(R), _np(S))
    for algo, bits in ((hjm.HJ_ALGO_PHJ, 6), (hjm.HJ_ALGO_SHJ, 0)):
        r = hjm.hj_join(ctx, R, S, algo=algo, radix_bits=bits, mode=hjm.HJ_COUNT_CHECKSUM)
        assert (r.count, *r.checksum) == (cnt, c0, c1)
    if theta_s == 0.5:
        want = _oracle(R, S)
        res = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=6)
        assert np.array_equal(_got(res), want)


@pytest.mark.parametrize("theta_s", [0.5, 1.0])
def test_phj_zipf_u64_count_full_size(hjm, ctx, theta_s):
    # The skewed 64-bit workload at full size (|R| = 2^22, |S| = 2^26, Zipf over 2^20
    # ranks; S theta 0.5 -- about 5e9 pairs -- and 1.0 -- about 3e11 pairs): count and
    # checksums only, against the oracle's per-key aggregation.  The plan is the one
    # the bench's tuner picks (PHJ with S slices for the heavy partitions).
    R, S = W.zipf_pair(1 << 22, 1 << 26, 0.75, theta_s, 1 << 20, SEED, DEV, ids=(3, int(theta_s * 10)))
    cnt, c0, c1 = oracle.join_aggregate(_np(R), _np(S))
    r = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (r.count, *r.checksum) == (cnt, c0, c1)
    assert cnt > (10 ** 11 if theta_s == 1.0 else 10 ** 9)


def _i64(v: int) -> int:
    return v - (1 << 64) if v >= 1 << 63 else v


def _fin_t(x: torch.Tensor) -> torch.Tensor:
    """SplitMix64 finaliser on int64 tensors (wrapping products, logical shifts);
    checked against the oracle's mixers below before use."""
    x = x ^ ((x >> 30) & ((1 << 34) - 1))
    x = x * _i64(0xBF58476D1CE4E5B9)
    x = x ^ ((x >> 27) & ((1 << 37) - 1))
    x = x * _i64(0x94D049BB133111EB)
    return x ^ ((x >> 31) & ((1 << 33) - 1))


def test_phj_zipf_u64_materialised_full_size(hjm, ctx):
    # The skewed 64-bit workload at theta 0.5 with every pair written: about 4.9e9
    # (rid_R, rid_S) pairs, 79 GB.  The count and the kernel's checksums against the
    # oracle's per-key aggregation; then the whole pair buffer, read back in 2 GB
    # pieces, checksummed on the GPU with torch arithmetic (independent of the join's
    # kernels) against the same oracle values -- a multiset check of all 4.9e9 pairs
    # -- and every pair checked to join equal keys.
    R, S = W.zipf_pair(1 << 22, 1 << 26, 0.75, 0.5, 1 << 20, SEED, DEV, ids=(3, 5))
    cnt, c0, c1 = oracle.join_aggregate(_np(R), _np(S))
    assert cnt > 4 * 10 ** 9
    res = hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, mode=hjm.HJ_MATERIALIZE, checksum=True,
                      out_capacity=cnt)
    try:
        assert (res.count, *res.checksum) == (cnt, c0, c1)
        probe = torch.tensor([0, 1, 12345, (1 << 40) + 7, (1 << 63) - 1], dtype=torch.int64, device=DEV)
        golden = _i64(0x9E3779B97F4A7C15)
        assert [v & ((1 << 64) - 1) for v in _fin_t(probe).tolist()] == [oracle.mix_a(v) for v in probe.tolist()]
        assert [v & ((1 << 64) - 1) for v in _fin_t(probe ^ golden).tolist()] == \
            [oracle.mix_b(v) for v in probe.tolist()]
        lib = hjm.load_library()
        piece = 1 << 27
        buf = torch.empty((piece, 2), dtype=torch.int64, device=DEV)
        m64 = (1 << 64) - 1
        t0 = t1 = 0
        for at in range(0, cnt, piece):
            n = min(piece, cnt - at)
            assert lib.hj_copy(ctx.handle, buf.data_ptr(), res.pairs_ptr + at * 16, n * 16) == hjm.HJ_OK
            a = _fin_t(buf[:n, 0])
            b = _fin_t(buf[:n, 1] ^ golden)
            t0 = (t0 + int((a * b).sum().item())) & m64
            t1 = (t1 + int(a.sum().item()) + int(b.sum().item())) & m64
            # every pair joins equal keys (rids are row numbers)
            assert torch.equal(R[buf[:n, 0], 0], S[buf[:n, 1], 0])
        assert (t0, t1) == (c0, c1)
    finally:
        res.free()


@pytest.mark.parametrize("algo", [1, 2])
def test_join_is_ordered_after_the_kernels_that_made_its_inputs(hjm, algo):
    # A default context orders its work on torch's current stream: a join queued
    # right after the (asynchronous) generation of its inputs sees them complete.
    # Every S key is an R key and R keys are unique, so the count is exactly |S|.
    with hjm.Context(0) as c:
        for _ in range(3):
            R, S = W.unique_and_uniform(1 << 22, 1 << 24, 1 << 22, SEED, DEV, ids=(7, algo))
            r = hjm.hj_join(c, R, S, algo=algo, mode=hjm.HJ_COUNT)
            assert r.count == 1 << 24


def test_phj_full_size_properties(hjm, ctx):
    # |R| = 2^24 unique keys, |S| = 2^28 keys uniform over [1, 2^25], the launch the
    # bench times (automatic plan).  Each S tuple whose key is <= 2^24 matches
    # exactly one R tuple, so: count = #{s : key <= 2^24}; every pair joins equal
    # keys; no S rid appears twice; a sample of S rows is found with its R row.
    nr, ns = 1 << 24, 1 << 28
    R, S = W.unique_and_uniform(nr, ns, 2 * nr, SEED, DEV, ids=(2,))
    skeys = S[:, 0].to(torch.int64) & 0xFFFFFFFF
    expect = int((skeys <= nr).sum())
    res = hjm.hj_join(ctx, R, S)
    assert res.algo == hjm.HJ_ALGO_PHJ
    assert res.count == expect
    pairs = torch.empty((res.count, 2), dtype=torch.int32, device=DEV)
    hjm.load_library().hj_copy(ctx.handle, pairs.data_ptr(), res.pairs_ptr, pairs.numel() * 4)
    res.free()
    rr = pairs[:, 0].to(torch.int64) & 0xFFFFFFFF
    ss = pairs[:, 1].to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(R[rr, 0], S[ss, 0])                      # every pair joins equal keys
    assert int(torch.unique(ss).numel()) == res.count            # no S row twice
    g = torch.Generator(device="cpu").manual_seed(7)
    rows = torch.randint(0, ns, (4096,), generator=g)
    hit = rows[(skeys[rows.to(DEV)] <= nr).cpu()]
    found = torch.isin(hit.to(DEV), ss)
    assert bool(found.all())


# --------------------------------------------------------------------- edge cases


@pytest.mark.parametrize("algo,bits", [(1, 0), (2, 3), (2, 10), (2, 11)])
@pytest.mark.parametrize("nr,ns", [(0, 0), (0, 100), (100, 0), (1, 1), (3, 7), (1025, 4097), (8191, 8193),
                                   (40_001, 123_457)])
def test_empty_and_ragged(hjm, ctx, algo, bits, nr, ns):
    R, S = W.unique_and_uniform(nr, ns, max(nr, 1), SEED, DEV, ids=(5, nr, ns))
    _check_all_modes(hjm, ctx, R, S, algo=algo, radix_bits=bits)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("algo,bits", [(1, 0), (2, 4)])
def test_extreme_keys_and_all_ones_tuples(hjm, ctx, dtype, algo, bits):
    top = np.iinfo(dtype).max
    rng = np.random.default_rng(3)
    keys = np.array([0, 1, top, top - 1], dtype)
    rk = rng.choice(keys, 301)
    rr = rng.choice(np.array([0, 5, top], dtype), 301)
    rk[:5] = top
    rr[:5] = top            # five tuples equal to the all-ones bit pattern
    sk = rng.choice(keys, 517)
    sr = np.arange(517, dtype=dtype)
    sr[3] = top
    R = _gpu(np.stack([rk, rr], 1))
    S = _gpu(np.stack([sk, sr], 1))
    _check_all_modes(hjm, ctx, R, S, algo=algo, radix_bits=bits)


@pytest.mark.parametrize("algo,bits", [(1, 0), (2, 5)])
def test_all_keys_equal_cross_product(hjm, ctx, algo, bits):
    R = _gpu(np.stack([np.full(37, 9, np.uint32), np.arange(37, dtype=np.uint32)], 1))
    S = _gpu(np.stack([np.full(53, 9, np.uint32), np.arange(53, dtype=np.uint32) + 100], 1))
    res = _check_all_modes(hjm, ctx, R, S, algo=algo, radix_bits=bits)
    assert res.count == 37 * 53


@pytest.mark.parametrize("mode", [2, 1])
def test_oversize_partition_takes_the_global_fallback(hjm, ctx, mode):
    # One key repeated 30000 times in R fills its partition beyond any shared-memory
    # table; the join must still be exact.
    rng = np.random.default_rng(11)
    rk = np.concatenate([np.full(30000, 7, np.uint32), rng.integers(8, 1 << 20, 20000).astype(np.uint32)])
    R = np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1)
    sk = rng.integers(1, 1 << 20, 40000).astype(np.uint32)
    sk[:3] = 7
    S = np.stack([sk, np.arange(len(sk), dtype=np.uint32)], 1)
    Rg, Sg = _gpu(R), _gpu(S)
    if mode == 2:
        want = _oracle(Rg, Sg)
        res = hjm.hj_join(ctx, Rg, Sg, algo=hjm.HJ_ALGO_PHJ, radix_bits=6)
        assert res.count == len(want)
        assert np.array_equal(_got(res), want)
    else:
        cnt, c0, c1 = oracle.join_aggregate(R, S)
        r = hjm.hj_join(ctx, Rg, Sg, algo=hjm.HJ_ALGO_PHJ, radix_bits=6, mode=1)
        assert (r.count, *r.checksum) == (cnt, c0, c1)


@pytest.mark.parametrize("width", [4, 8])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_many_oversize_partitions_fall_back_together(hjm, ctx, width, mode):
    # 60 keys repeated 2000-4000 times in R, spread over the 256 partitions of an
    # 8-bit plan, make most of those partitions' tables overflow shared memory; S
    # holds every heavy key a few times, in skewed amounts (large partitions are
    # probed in several slices).  The fallback gathers all of them into one table
    # per join; pairs, count and checksums must equal the oracle's.
    dt = np.uint32 if width == 4 else np.uint64
    rng = np.random.default_rng(12 + width)
    heavy = rng.choice(np.arange(10, 1 << 20), 60, replace=False).astype(dt)
    reps = rng.integers(2000, 4000, 60)
    rk = np.concatenate([np.repeat(heavy, reps), rng.integers(1 << 20, 1 << 21, 30000).astype(dt)])
    rk = rk[rng.permutation(len(rk))]
    R = np.stack([rk, np.arange(len(rk), dtype=dt)], 1)
    sk = np.concatenate([np.repeat(heavy, rng.integers(1, 40, 60)), rng.integers(1, 1 << 21, 300000).astype(dt)])
    sk = sk[rng.permutation(len(sk))]
    S = np.stack([sk, np.arange(len(sk), dtype=dt) + 3], 1)
    view = np.int32 if width == 4 else np.int64
    Rg = torch.from_numpy(np.ascontiguousarray(R).view(view)).to(DEV)
    Sg = torch.from_numpy(np.ascontiguousarray(S).view(view)).to(DEV)
    cnt, c0, c1 = oracle.join_aggregate(R, S)
    r = hjm.hj_join(ctx, Rg, Sg, algo=hjm.HJ_ALGO_PHJ, radix_bits=8, mode=mode, checksum=True)
    assert r.count == cnt
    if mode != 0:
        assert r.checksum == (c0, c1)
    if mode == 2:
        want = oracle.sorted_pairs(*oracle.hash_join(R, S))
        assert np.array_equal(_got(r), want)


@pytest.mark.parametrize("algo,bits", [(1, 0), (2, 6)])
def test_output_capacity_overflow_reruns_exactly(hjm, ctx, algo, bits):
    R, S = W.unique_and_uniform(5000, 30000, 5000, SEED, DEV, ids=(6,))
    want = _oracle(R, S)
    res = hjm.hj_join(ctx, R, S, algo=algo, radix_bits=bits, out_capacity=17)
    assert res.count == len(want) and res.pairs_cap >= res.count
    assert np.array_equal(_got(res), want)


# ----------------------------------------------------------------- build / probe


@pytest.mark.parametrize("width", [4, 8])
def test_build_then_probe(hjm, ctx, width):
    if width == 4:
        R, S = W.unique_and_uniform(40000, 90000, 60000, SEED, DEV, ids=(7,))
    else:
        R, S = W.zipf_pair(20000, 90000, 0.75, 0.5, 1 << 13, SEED, DEV, ids=(7,))
    want = _oracle(R, S)
    cnt, c0, c1 = oracle.join_aggregate(_np(R), _np(S))
    t = hjm.hj_build(ctx, R, mode=hjm.HJ_MATERIALIZE)
    res = hjm.hj_probe(ctx, t, S, checksum=True)
    assert res.checksum == (c0, c1)
    assert np.array_equal(_got(res), want)
    # the same table serves a second probe
    res2 = hjm.hj_probe(ctx, t, S[: len(S) // 2].contiguous())
    assert res2.count == len(_oracle(R, S[: len(S) // 2]))
    res2.free()
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_probe(ctx, t, S, mode=hjm.HJ_COUNT)
    assert e.value.status == hjm.HJ_E_INVALID
    t.free()
    ta = hjm.hj_build(ctx, R, mode=hjm.HJ_COUNT_CHECKSUM)
    r = hjm.hj_probe(ctx, ta, S, mode=hjm.HJ_COUNT_CHECKSUM)
    assert (r.count, *r.checksum) == (cnt, c0, c1)
    ta.free()


# ------------------------------------------------------------------ partitioning


@pytest.mark.parametrize("width,b1,b2,n", [(4, 1, 0, 1), (4, 6, 0, 100003), (4, 12, 0, 300001), (4, 5, 4, 200001),
                                           (8, 8, 0, 70001), (8, 3, 6, 90001), (4, 9, 0, 0)])
def test_partition_matches_oracle(hjm, ctx, width, b1, b2, n):
    if width == 4:
        rel, _ = W.unique_and_uniform(n, 0, 1, SEED, DEV, ids=(8, n))
    else:
        rel, _ = W.zipf_pair(n, 0, 0.75, 0.5, 1 << 14, SEED, DEV, ids=(8, n))
    want, woff = oracle.radix_partition(_np(rel), b1, b2)
    got, goff = hjm.hj_partition(ctx, rel, b1, b2)
    assert np.array_equal(goff, woff)                     # partition boundaries exact
    for p in range(len(woff) - 1):                         # same multiset in each partition
        a, b = int(woff[p]), int(woff[p + 1])
        if b - a > 1:
            x = got[a:b][np.lexsort((got[a:b, 1], got[a:b, 0]))]
            y = want[a:b][np.lexsort((want[a:b, 1], want[a:b, 0]))]
            assert np.array_equal(x, y), p
        else:
            assert np.array_equal(got[a:b], want[a:b])


# ------------------------------------------------------------------ error paths


def test_invalid_arguments(hjm, ctx):
    R, S = W.unique_and_uniform(100, 100, 100, SEED, DEV, ids=(9,))
    misaligned = R.view(-1)[2:].view(-1, 2)     # starts 8 bytes in: not 16-byte aligned
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join(ctx, misaligned, S)
    assert e.value.status == hjm.HJ_E_INVALID
    S64, _ = W.zipf_pair(10, 0, 0.5, 0.5, 16, SEED, DEV)
    with pytest.raises(hjm.HJError) as e:
        hjm.hj_join(ctx, R, S64)
    assert e.value.status == hjm.HJ_E_INVALID
    with pytest.raises(hjm.HJError):
        hjm.hj_join(ctx, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=13, passes=1)
    # 2^32 - 1 rows or more, either width: refused before any device memory is read
    lib = hjm.load_library()
    for width in (4, 8):
        big = hjm.hj_rel(R.data_ptr(), (1 << 32) - 1, width, 0)
        small = hjm.hj_rel(R.data_ptr(), 10, width, 0)
        res = hjm.hj_result()
        o = hjm._opts()
        assert lib.hj_join(ctx.handle, ctypes.byref(big), ctypes.byref(small), ctypes.byref(o),
                           ctypes.byref(res)) == hjm.HJ_E_INVALID
        assert lib.hj_join(ctx.handle, ctypes.byref(small), ctypes.byref(big), ctypes.byref(o),
                           ctypes.byref(res)) == hjm.HJ_E_INVALID


def test_injected_allocation_failure_leaks_nothing(hjm):
    lib = hjm.load_library()
    R, S = W.unique_and_uniform(3000, 9000, 3000, SEED, DEV, ids=(10,))
    with hjm.Context(0) as c:
        base = lib.hj_debug_bytes_in_use(c.handle)
        for k in range(6):
            lib.hj_debug_fail_alloc(c.handle, k)
            with pytest.raises(hjm.HJError) as e:
                hjm.hj_join(c, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=4)
            assert e.value.status == hjm.HJ_E_NOMEM
        lib.hj_debug_fail_alloc(c.handle, -1)
        assert lib.hj_debug_bytes_in_use(c.handle) == base   # every failed call released its buffers
        res = hjm.hj_join(c, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=4)
        assert np.array_equal(_got(res), _oracle(R, S))
        assert lib.hj_debug_bytes_in_use(c.handle) == base


def test_hbm_budget_is_enforced(hjm):
    R, S = W.unique_and_uniform(1 << 16, 1 << 18, 1 << 17, SEED, DEV, ids=(11,))
    with hjm.Context(0, budget=1 << 20) as c:
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_join(c, R, S)
        assert e.value.status == hjm.HJ_E_NOMEM
