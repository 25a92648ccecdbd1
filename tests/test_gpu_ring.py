"""The ring scatter -- the partition scatter that 4-byte joins take at 2^11 digits
(the plan the tuner picks for the 2^24 x 2^28 join) and 2^10, and 8-byte joins at
2^9 .. 2^11 -- against the CPU oracle,
element by element, on inputs that drive each of its paths: rings that overflow to
the far end of their run (keys crowded into two digits), duplicate build keys, a
batch whose group partitions on 11 bits (the per-segment input path), and its
bounded wait made to run out on purpose (a short limit; the kernel returns and the
host reports HJ_E_TIMEOUT, no GPU fault).  hj_debug_scatter forces the ring or the
region scatter, and both kernels are checked at every width and fan-out the ring
is built for, on ragged sizes and on crowded digits; the region scatter is also
checked at the low fan-outs where it keeps up to 256 slots per digit.  Join results are integers: every comparison is
exact."""
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


def _gpu(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(DEV)


def _sorted_got(res):
    p = res.pairs_numpy().astype(np.uint64)
    res.free()
    return oracle.sorted_pairs(p[:, 0], p[:, 1])


def _check(hjm, ctx, R, S, **kw):
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    want = oracle.sorted_pairs(*oracle.hash_join(r, s))
    cnt, c0, c1 = oracle.join_aggregate(r, s)
    res = hjm.hj_join(ctx, R, S, mode=hjm.HJ_MATERIALIZE, checksum=True, **kw)
    assert (res.count, *res.checksum) == (cnt, c0, c1)
    assert np.array_equal(_sorted_got(res), want)
    for mode in (hjm.HJ_COUNT, hjm.HJ_COUNT_CHECKSUM):
        r2 = hjm.hj_join(ctx, R, S, mode=mode, **kw)
        assert r2.count == cnt
        if mode == hjm.HJ_COUNT_CHECKSUM:
            assert r2.checksum == (c0, c1)


def _keys_of_digits(digits, n_keys: int, bits: int = 11, dtype=np.uint32) -> np.ndarray:
    """Keys among 1..n_keys whose pass-one digit at `bits` is in `digits`, found
    with the oracle's own partitioner (MurmurHash2 pinned by SMHasher's values)."""
    keys = np.arange(1, n_keys + 1, dtype=dtype)
    rel = np.stack([keys, keys], 1)
    out, off = oracle.radix_partition(rel, bits)
    return np.concatenate([out[int(off[d]):int(off[d + 1]), 0] for d in digits])


def _view(a: np.ndarray) -> torch.Tensor:
    dt = np.int32 if a.dtype == np.uint32 else np.int64
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(DEV)


RING_FANOUTS = [(4, 9), (4, 10), (4, 11), (8, 9), (8, 10), (8, 11)]


@pytest.mark.parametrize("kind", ["region", "ring"])
@pytest.mark.parametrize("width,bits", RING_FANOUTS)
def test_both_scatters_at_every_ring_fanout(hjm, width, bits, kind):
    # ragged sizes spread over every SM's chunk; 4-byte: unique R keys, S over twice
    # their range; 8-byte: Zipf keys on both sides (duplicate build keys)
    forced = hjm.HJ_SCATTER_REGION if kind == "region" else hjm.HJ_SCATTER_RING
    if width == 4:
        R, S = W.unique_and_uniform(300_007, 2_000_003, 600_014, SEED, DEV, ids=(45, bits))
    else:
        R, S = W.zipf_pair(120_011, 900_007, 0.75, 0.5, 1 << 16, SEED, DEV, ids=(45, bits))
    lib = hjm.load_library()
    with hjm.Context(0) as c:
        assert lib.hj_debug_scatter(c.handle, forced) == hjm.HJ_OK
        _check(hjm, c, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=bits, passes=1)


@pytest.mark.parametrize("width,bits", RING_FANOUTS)
def test_ring_with_crowded_digits_at_every_fanout(hjm, width, bits):
    # every tuple in digit 3 or in the last digit: two rings overflow at once and
    # most tuples take the far-end path; R holds each key once or twice
    dt = np.uint32 if width == 4 else np.uint64
    keys = _keys_of_digits((3, (1 << bits) - 1), 1 << 20, bits, dt)
    assert len(keys) > 500
    rng = np.random.default_rng(46 + bits)
    rk = np.concatenate([keys, keys[: len(keys) // 3]])
    rk = rk[rng.permutation(len(rk))]
    R = np.stack([rk, np.arange(len(rk), dtype=dt)], 1)
    sk = rng.choice(keys, 400_009).astype(dt)
    sk[::5] = np.setdiff1d(np.arange(1, 200, dtype=dt), keys)[0]  # a key R does not hold
    S = np.stack([sk, np.arange(len(sk), dtype=dt)], 1)
    lib = hjm.load_library()
    with hjm.Context(0) as c:
        assert lib.hj_debug_scatter(c.handle, hjm.HJ_SCATTER_RING) == hjm.HJ_OK
        _check(hjm, c, _view(R), _view(S), algo=hjm.HJ_ALGO_PHJ, radix_bits=bits, passes=1)


REGION_FANOUTS = [(4, 5), (4, 6), (4, 7), (4, 8), (8, 5), (8, 6), (8, 7)]


@pytest.mark.parametrize("crowded", [False, True])
@pytest.mark.parametrize("width,bits", REGION_FANOUTS)
def test_region_scatter_at_low_fanouts(hjm, ctx, width, bits, crowded):
    # the region scatter where its slots per digit are many (up to 256): ragged
    # uniform keys, whose digits mostly fit their slots, and keys of two digits,
    # which overflow them on every tile (far-end path); padded passes only run
    # inside joins, so the join result is what is compared
    dt = np.uint32 if width == 4 else np.uint64
    rng = np.random.default_rng(47 + bits + width)
    if crowded:
        keys = _keys_of_digits((0, (1 << bits) - 2), 1 << 18, bits, dt)
        assert len(keys) > 1000
        rk = rng.permutation(keys)[: min(len(keys), 20_000)]
        sk = rng.choice(keys, 300_007).astype(dt)
    else:
        rk = rng.permutation(np.arange(1, 100_004, dtype=dt))
        sk = rng.integers(1, 200_008, 600_011).astype(dt)
    R = np.stack([rk, np.arange(len(rk), dtype=dt)], 1)
    S = np.stack([sk, np.arange(len(sk), dtype=dt)], 1)
    _check(hjm, ctx, _view(R), _view(S), algo=hjm.HJ_ALGO_PHJ, radix_bits=bits, passes=1)


@pytest.mark.parametrize("ns", [200_003, 1_000_001])
def test_keys_crowded_into_two_digits_overflow_the_rings(hjm, ctx, ns):
    # Every tuple of every chunk lands in digit 5 or 1900: those two rings fill at
    # once and most tuples take the far-end path of their run; every other digit's
    # run is empty (padding only).  R holds each crowded key twice (duplicates).
    keys = _keys_of_digits((5, 1900), 1 << 22)
    assert len(keys) > 3000
    rng = np.random.default_rng(41)
    rk = np.concatenate([keys, keys[: len(keys) // 2]])
    rk = rk[rng.permutation(len(rk))]
    R = np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1)
    sk = rng.choice(keys, ns).astype(np.uint32)
    sk[::7] = np.setdiff1d(np.arange(1, 100, dtype=np.uint32), keys)[0]  # a key R does not hold
    S = np.stack([sk, np.arange(ns, dtype=np.uint32)], 1)
    _check(hjm, ctx, _gpu(R), _gpu(S), algo=hjm.HJ_ALGO_PHJ, radix_bits=11, passes=1)


def test_duplicate_build_keys_at_eleven_bits(hjm, ctx):
    # R: 150 001 tuples over 60 000 keys (each key 1-5 times), S uniform over twice
    # that key range: multi-match walks in the shared-memory tables after the ring
    # scatter.
    rng = np.random.default_rng(42)
    rk = rng.integers(1, 60_001, 150_001).astype(np.uint32)
    R = np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1)
    sk = rng.integers(1, 120_001, 700_001).astype(np.uint32)
    S = np.stack([sk, np.arange(len(sk), dtype=np.uint32)], 1)
    _check(hjm, ctx, _gpu(R), _gpu(S), algo=hjm.HJ_ALGO_PHJ, radix_bits=11, passes=1)


def test_batch_group_on_eleven_bits(hjm, ctx):
    # Two joins with |R| > 2^23 make a batch group that partitions on 11 bits (each
    # join one segment of the pass, read from its own array); a small join beside
    # them takes another group.  Every join's pairs, count and checksums against
    # the oracle.
    sizes = [((1 << 23) + 1030, (1 << 23) + 77), ((1 << 23) + 2049, (1 << 22) + 5), (5000, 20_001)]
    Rs, Ss = [], []
    for j, (nr, ns) in enumerate(sizes):
        r, s = W.unique_and_uniform(nr, ns, 2 * nr, SEED, DEV, ids=(43, j))
        Rs.append(r)
        Ss.append(s)
    res = hjm.hj_join_batch(ctx, Rs, Ss, checksum=True)
    assert res[0].radix_bits == 11 and res[1].radix_bits == 11
    for j in range(len(sizes)):
        r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
        cnt, c0, c1 = oracle.join_aggregate(r, s)
        assert (res[j].count, *res[j].checksum) == (cnt, c0, c1), j
        want = oracle.sorted_pairs(*oracle.hash_join(r, s))
        assert np.array_equal(_sorted_got(res[j]), want), j


@pytest.mark.parametrize("width", [4, 8])
def test_tma_wait_runs_out_and_the_context_recovers(hjm, width):
    # A limit of one: the TMA-staged scatter of an unpadded pass (hj_partition)
    # polls its first tile's mbarrier zero times, gives up, waits for the copy in
    # flight to land and returns.  hj_partition reports HJ_E_TIMEOUT and releases its
    # buffers; with the default limit the next partition on the context is the
    # oracle's, element by element.
    lib = hjm.load_library()
    n = (1 << 20) + 7
    if width == 4:
        rel, _ = W.unique_and_uniform(n, 0, 1, SEED, DEV, ids=(48,))
    else:
        rel, _ = W.zipf_pair(n, 0, 0.75, 0.5, 1 << 16, SEED, DEV, ids=(48,))
    with hjm.Context(0) as c:
        base = lib.hj_debug_bytes_in_use(c.handle)
        assert lib.hj_debug_wait_limit(c.handle, 1) == hjm.HJ_OK
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_partition(c, rel, 8)
        assert e.value.status == hjm.HJ_E_TIMEOUT
        assert lib.hj_debug_bytes_in_use(c.handle) == base
        assert lib.hj_debug_wait_limit(c.handle, 0) == hjm.HJ_OK
        got, goff = hjm.hj_partition(c, rel, 8)
        want, woff = oracle.radix_partition(W.to_numpy_u(rel), 8)
        assert np.array_equal(goff, woff)  # partition boundaries exact, the same rows in each
        for p in range(len(woff) - 1):
            a, b = int(woff[p]), int(woff[p + 1])
            x = got[a:b][np.lexsort((got[a:b, 1], got[a:b, 0]))]
            y = want[a:b][np.lexsort((want[a:b, 1], want[a:b, 0]))]
            assert np.array_equal(x, y), p
        assert lib.hj_debug_bytes_in_use(c.handle) == base


def test_bounded_wait_runs_out_and_the_context_recovers(hjm):
    # A limit of one flush pass: the flush warps give up while the insert warps are
    # still streaming, set the fault bit and return (insert warps never wait, so
    # every CTA ends).  The join reports HJ_E_TIMEOUT, releases its buffers, and the
    # next join on the same context, with the default limit, is exact.
    lib = hjm.load_library()
    R, S = W.unique_and_uniform(1 << 18, 1 << 22, 1 << 19, SEED, DEV, ids=(44,))
    with hjm.Context(0) as c:
        base = lib.hj_debug_bytes_in_use(c.handle)
        assert lib.hj_debug_wait_limit(c.handle, 1) == hjm.HJ_OK
        with pytest.raises(hjm.HJError) as e:
            hjm.hj_join(c, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=11, passes=1, mode=hjm.HJ_COUNT)
        assert e.value.status == hjm.HJ_E_TIMEOUT
        assert lib.hj_debug_bytes_in_use(c.handle) == base
        assert lib.hj_debug_wait_limit(c.handle, 0) == hjm.HJ_OK
        _check(hjm, c, R, S, algo=hjm.HJ_ALGO_PHJ, radix_bits=11, passes=1)
        assert lib.hj_debug_bytes_in_use(c.handle) == base
