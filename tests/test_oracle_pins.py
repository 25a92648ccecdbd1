"""Pins for the CPU oracle: each oracle function is checked against something other
than itself -- published test vectors, a hand-derived worked example, closed forms
of special inputs, brute force on tiny inputs, and independent routes to the same
number.  CPU only."""
import os

import numpy as np
import pytest

import oracle
from paper_1307_1955_gb300 import workload as W


def _np(rel):
    return W.to_numpy_u(rel)


def _rel(keys, rids, dtype):
    return np.stack([np.asarray(keys, dtype), np.asarray(rids, dtype)], axis=1)


# ------------------------------------------------------------------ published vectors


def _smhasher_verification(fn, nbytes):
    """SMHasher's verification value: hash keys {}, {0}, {0,1}, ... {0..254} with seed
    256 - len, concatenate the hashes, hash that with seed 0, take the low 32 bits."""
    key = bytearray(256)
    hashes = bytearray(nbytes * 256)
    for i in range(256):
        key[i] = i
        hashes[i * nbytes:(i + 1) * nbytes] = fn(bytes(key[:i]), 256 - i).to_bytes(nbytes, "little")
    return fn(bytes(hashes), 0) & 0xFFFFFFFF


def test_murmur2_32_matches_smhasher_verification():
    # MurmurHash 2.0 is the paper's hash function (Sec. 5.1); SMHasher publishes
    # 0x27864C1E as the verification value of the 32-bit variant.
    assert _smhasher_verification(oracle.murmur2_32, 4) == 0x27864C1E


def test_murmur64a_matches_smhasher_verification():
    # ... and 0x1F0D3804 for the 64-bit variant (MurmurHash64A).
    assert _smhasher_verification(oracle.murmur64a, 8) == 0x1F0D3804


def test_key_hash_is_murmur_of_key_bytes():
    for k in (0, 1, 0xDEADBEEF, 0xFFFFFFFF):
        assert oracle.key_hash(k, 4, 0) == oracle.murmur2_32(k.to_bytes(4, "little"), 0)
    for k in (0, 1, 0x0123456789ABCDEF, (1 << 64) - 1):
        assert oracle.key_hash(k, 8, 0) == oracle.murmur64a(k.to_bytes(8, "little"), 0)


def test_mix_a_is_splitmix64_finaliser():
    # SplitMix64 seeded with 0 returns fin(1*G), fin(2*G), fin(3*G), ... with
    # G = 0x9E3779B97F4A7C15; its published first outputs:
    g = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for i, e in enumerate(expect, start=1):
        assert oracle.mix_a((i * g) & ((1 << 64) - 1)) == e


def test_mix_b_is_mix_a_of_shifted_input():
    for x in (0, 1, 12345, (1 << 64) - 1):
        assert oracle.mix_b(x) == oracle.mix_a(x ^ 0x9E3779B97F4A7C15)
    # both mixers are bijections: no collisions on a block of inputs
    assert len({oracle.mix_a(x) for x in range(4096)}) == 4096
    assert len({oracle.mix_b(x) for x in range(4096)}) == 4096


# --------------------------------------------------------------------- worked example


def _load_golden(path):
    sec, data = None, {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                sec = line.strip("[]")
                data[sec] = []
                continue
            data[sec].append([int(x) for x in line.split()])
    return data


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_worked_example(golden_dir, dtype):
    g = _load_golden(os.path.join(golden_dir, "join_worked_example.txt"))
    R = np.array(g["R"], dtype)
    S = np.array(g["S"], dtype)
    want = np.array(sorted(map(tuple, g["pairs"])), np.uint64)
    for fn in (oracle.hash_join, oracle.nested_loop_join):
        got = oracle.sorted_pairs(*fn(R, S))
        assert np.array_equal(got, want)
    assert oracle.count_sortmerge(R, S) == len(want)
    cnt, c0, c1 = oracle.join_aggregate(R, S)
    assert cnt == len(want)
    assert (c0, c1) == oracle.checksum_pairs(want[:, 0], want[:, 1])
    # the checksum restated by hand from its definition, in Python integers
    m = (1 << 64) - 1
    e0 = sum(oracle.mix_a(int(a)) * oracle.mix_b(int(b)) for a, b in want) & m
    e1 = sum(oracle.mix_a(int(a)) + oracle.mix_b(int(b)) for a, b in want) & m
    assert (c0, c1) == (e0, e1)


# ------------------------------------------------------------------------ closed forms


def test_unique_build_keys_each_probe_matches_its_row():
    # |R| = |S| = n, R keys a permutation of 1..n, S keys drawn from R's keys:
    # exactly n pairs, and S row j pairs with the unique R row holding S.key[j].
    n = 1 << 14
    R, S = W.unique_and_uniform(n, n, n, 11, "cpu")
    R, S = _np(R), _np(S)
    rr, ss = oracle.hash_join(R, S)
    assert len(rr) == n
    row_of_key = np.empty(n + 1, np.int64)
    row_of_key[R[:, 0]] = np.arange(n)
    got = oracle.sorted_pairs(rr, ss)
    want = oracle.sorted_pairs(R[row_of_key[S[:, 0]], 1], S[:, 1])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_all_keys_equal_gives_cross_product(dtype):
    nr, ns = 37, 53
    top = np.iinfo(dtype).max
    R = _rel(np.full(nr, top), np.arange(nr), dtype)
    S = _rel(np.full(ns, top), np.arange(100, 100 + ns), dtype)
    rr, ss = oracle.hash_join(R, S)
    assert len(rr) == nr * ns
    want = np.array([(i, 100 + j) for i in range(nr) for j in range(ns)], np.uint64)
    assert np.array_equal(oracle.sorted_pairs(rr, ss), want)
    assert oracle.count_sortmerge(R, S) == nr * ns
    assert oracle.join_aggregate(R, S)[0] == nr * ns


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_disjoint_and_empty_give_no_pairs(dtype):
    R = _rel(np.arange(0, 100), np.arange(100), dtype)
    S = _rel(np.arange(100, 300), np.arange(200), dtype)
    E = np.zeros((0, 2), dtype)
    for a, b in ((R, S), (R, E), (E, S), (E, E)):
        rr, ss = oracle.hash_join(a, b)
        assert len(rr) == 0
        assert oracle.count_sortmerge(a, b) == 0
        assert oracle.join_aggregate(a, b) == (0, 0, 0)


# ------------------------------------------------------------------------- brute force


def _small_cases():
    rng = np.random.default_rng(7)
    yield "uniform_u32", _rel(rng.integers(0, 64, 300), np.arange(300), np.uint32), \
        _rel(rng.integers(0, 64, 500), np.arange(500), np.uint32)
    yield "extremes_u32", _rel(rng.choice([0, 1, 0xFFFFFFFF, 0xFFFFFFFE], 200), rng.integers(0, 2**32, 200), np.uint32), \
        _rel(rng.choice([0, 2, 0xFFFFFFFF], 300), rng.integers(0, 2**32, 300), np.uint32)
    kr = np.array([0, 2**64 - 1, 2**63], np.uint64)
    ks = np.array([0, 2**64 - 1, 5], np.uint64)
    yield "extremes_u64", _rel(rng.choice(kr, 150), np.arange(150), np.uint64), \
        _rel(rng.choice(ks, 250), np.arange(250), np.uint64)
    R, S = W.unique_and_uniform(1500, 4000, 3000, 3, "cpu")
    yield "half_match", _np(R), _np(S)
    R, S = W.zipf_pair(1200, 2500, 0.75, 1.0, 1 << 10, 5, "cpu")
    yield "zipf_u64", _np(R), _np(S)


@pytest.mark.parametrize("name,R,S", list(_small_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_hash_join_equals_brute_force(name, R, S):
    want = oracle.sorted_pairs(*oracle.nested_loop_join(R, S))
    got = oracle.sorted_pairs(*oracle.hash_join(R, S))
    assert np.array_equal(got, want)
    assert oracle.count_sortmerge(R, S) == len(want)
    cnt, c0, c1 = oracle.join_aggregate(R, S)
    assert cnt == len(want)
    assert (c0, c1) == oracle.checksum_pairs(want[:, 0], want[:, 1])


def test_checksum_detects_a_changed_pair():
    rr = np.arange(10, dtype=np.uint64)
    ss = np.arange(10, 20, dtype=np.uint64)
    base = oracle.checksum_pairs(rr, ss)
    ss2 = ss.copy()
    ss2[3] += 1
    assert oracle.checksum_pairs(rr, ss2) != base
    # and is independent of order
    p = np.random.default_rng(1).permutation(10)
    assert oracle.checksum_pairs(rr[p], ss[p]) == base


# ------------------------------------------------------------------------- partitioning


def _partition_index(rel, b1, b2):
    w = rel.dtype.itemsize
    h = np.array([oracle.key_hash(int(k), w, 0) for k in rel[:, 0]], np.uint64)
    d1 = h & np.uint64((1 << b1) - 1)
    d2 = (h >> np.uint64(b1)) & np.uint64((1 << b2) - 1)
    return (d1 << np.uint64(b2)) | d2


@pytest.mark.parametrize("w,b1,b2", [(4, 5, 0), (4, 3, 4), (8, 6, 0), (8, 2, 3), (4, 0, 0)])
def test_radix_partition_is_stable_sort_on_hash_digits(w, b1, b2):
    n = 3000
    if w == 4:
        R, _ = W.unique_and_uniform(n, 0, 1, 9, "cpu")
    else:
        R, _ = W.zipf_pair(n, 0, 0.75, 0.5, 1 << 9, 9, "cpu")
    R = _np(R)
    out, offs = oracle.radix_partition(R, b1, b2)
    p = _partition_index(R, b1, b2)
    order = np.argsort(p, kind="stable")          # numpy's stable sort, an independent route
    assert np.array_equal(out, R[order])
    counts = np.bincount(p.astype(np.int64), minlength=1 << (b1 + b2))
    assert np.array_equal(offs, np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64))


def test_radix_partition_two_passes_nest_single_passes():
    # Partitioning on b1 bits, then each partition on the next b2 bits (Alg. 2, two
    # passes) equals one call with (b1, b2).
    R, _ = W.unique_and_uniform(5000, 0, 1, 21, "cpu")
    R = _np(R)
    b1, b2 = 3, 2
    out, offs = oracle.radix_partition(R, b1, b2)
    first, o1 = oracle.radix_partition(R, b1, 0)
    pieces = []
    for d1 in range(1 << b1):
        part = first[o1[d1]:o1[d1 + 1]]
        # the second pass looks at bits [b1, b1+b2): partition on b1+b2 low bits and
        # keep the sub-partitions of this d1 in d2 order
        sub, so = oracle.radix_partition(part, b1 + b2, 0)
        for d2 in range(1 << b2):
            q = d1 | (d2 << b1)
            pieces.append(sub[so[q]:so[q + 1]])
    assert np.array_equal(out, np.concatenate(pieces))


def test_radix_partition_is_balanced_on_unique_keys():
    # MurmurHash2's low bits spread unique keys evenly: every partition within
    # 6 standard deviations of n / P.
    n, b = 1 << 16, 6
    R, _ = W.unique_and_uniform(n, 0, 1, 2, "cpu")
    _, offs = oracle.radix_partition(_np(R), b, 0)
    cnt = np.diff(offs.astype(np.int64))
    mean = n / (1 << b)
    assert np.all(np.abs(cnt - mean) < 6 * np.sqrt(mean))
