"""hj_join_batch: many joins of uneven sizes in one persistent launch per wave.
Every join's result must equal the oracle's (sorted pairs, count, checksums) and
what hj_join returns for the same join alone -- the result of a join is the same
alone and in the mix (exact, integer results)."""
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


@pytest.fixture(scope="module")
def ctx(hjm):
    c = hjm.Context(0)
    yield c
    c.close()


def _sorted(p):
    p = np.asarray(p, np.uint64)
    return p[np.lexsort((p[:, 1], p[:, 0]))] if len(p) else p.reshape(0, 2)


def _batch(n, seed, lo=4.0, hi=15.0):
    specs = W.batched_specs(n, seed, lo_log2=lo, hi_log2=hi)
    specs += [W.JoinSpec(0, 100, 10), W.JoinSpec(100, 0, 100), W.JoinSpec(1, 1, 1), W.JoinSpec(3, 7, 2)]
    R, S, rs, ss = W.batched_relations(specs, seed, DEV)
    Rs = [R[rs[j]:rs[j] + sp.n_r] for j, sp in enumerate(specs)]
    Ss = [S[ss[j]:ss[j] + sp.n_s] for j, sp in enumerate(specs)]
    return specs, Rs, Ss


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle_per_join(hjm, ctx, graph):
    specs, Rs, Ss = _batch(60, 5)
    res = hjm.hj_join_batch(ctx, Rs, Ss, checksum=True, graph=graph)
    for j in range(len(specs)):
        r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
        want = oracle.sorted_pairs(*oracle.hash_join(r, s))
        cnt, c0, c1 = oracle.join_aggregate(r, s)
        got = res[j].pairs_numpy()
        res[j].free()
        assert res[j].count == len(want) == cnt, j
        assert res[j].checksum == (c0, c1), j
        assert np.array_equal(_sorted(got), want), j


def test_batch_count_mode_and_alone_vs_mix(hjm, ctx):
    specs, Rs, Ss = _batch(40, 6, lo=8.0, hi=17.0)
    res = hjm.hj_join_batch(ctx, Rs, Ss, mode=hjm.HJ_COUNT_CHECKSUM)
    for j in range(len(specs)):
        alone = hjm.hj_join(ctx, Rs[j], Ss[j], mode=hjm.HJ_COUNT_CHECKSUM)
        assert (res[j].count, res[j].checksum) == (alone.count, alone.checksum), j
        r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
        assert (res[j].count, *res[j].checksum) == oracle.join_aggregate(r, s), j


def test_batch_u64_skewed_joins(hjm, ctx):
    Rs, Ss = [], []
    for j, (nr, ns, th) in enumerate([(3000, 9000, 0.5), (20000, 50000, 1.0), (500, 4000, 0.75)]):
        r, s = W.zipf_pair(nr, ns, 0.75, th, 1 << 10, 7, DEV, ids=(30, j))
        Rs.append(r)
        Ss.append(s)
    res = hjm.hj_join_batch(ctx, Rs, Ss, checksum=True)
    for j in range(3):
        r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
        want = oracle.sorted_pairs(*oracle.hash_join(r, s))
        assert res[j].count == len(want)
        assert res[j].checksum == oracle.join_aggregate(r, s)[1:]
        assert np.array_equal(_sorted(res[j].pairs_numpy()), want)
        res[j].free()


def test_batch_oversize_partition_and_overflow(hjm, ctx):
    rng = np.random.default_rng(12)
    rk = np.concatenate([np.full(30000, 7, np.uint32), rng.integers(8, 1 << 20, 5000).astype(np.uint32)])
    R0 = torch.from_numpy(np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1).view(np.int32)).to(DEV)
    sk = rng.integers(1, 1 << 20, 20000).astype(np.uint32)
    sk[:3] = 7                      # 3 x 30000 pairs from one key: more than |S| pairs
    S0 = torch.from_numpy(np.stack([sk, np.arange(len(sk), dtype=np.uint32)], 1).view(np.int32)).to(DEV)
    specs, Rs, Ss = _batch(10, 8)
    Rs, Ss = [R0] + Rs, [S0] + Ss
    res = hjm.hj_join_batch(ctx, Rs, Ss, checksum=True)
    for j in range(len(Rs)):
        r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
        want = oracle.sorted_pairs(*oracle.hash_join(r, s))
        assert res[j].count == len(want), j
        assert np.array_equal(_sorted(res[j].pairs_numpy()), want), j
        res[j].free()


@pytest.mark.parametrize("mode", [1, 2])
def test_batch_many_joins_with_many_oversize_partitions(hjm, ctx, mode):
    # Four joins whose R holds 3-40 keys repeated 1500-3000 times (several
    # partitions per join overflow shared memory; one join has a single such
    # partition), beside a join with none: the fallback groups the overflowing
    # tasks by join and gathers each join's rows into its own table.
    rng = np.random.default_rng(31)
    Rs, Ss, host = [], [], []
    for j, nheavy in enumerate([40, 3, 1, 25, 0]):
        heavy = rng.choice(np.arange(10, 1 << 20), max(nheavy, 1), replace=False).astype(np.uint32)[:nheavy]
        rk = np.concatenate([np.repeat(heavy, rng.integers(1500, 3000, nheavy)),
                             rng.integers(1 << 20, 1 << 21, 20000).astype(np.uint32)])
        rk = rk[rng.permutation(len(rk))]
        sk = np.concatenate([np.repeat(heavy, rng.integers(1, 20, nheavy)),
                             rng.integers(1, 1 << 21, 100000).astype(np.uint32)])
        sk = sk[rng.permutation(len(sk))]
        R = np.stack([rk, np.arange(len(rk), dtype=np.uint32)], 1)
        S = np.stack([sk, np.arange(len(sk), dtype=np.uint32) + 5], 1)
        host.append((R, S))
        Rs.append(torch.from_numpy(np.ascontiguousarray(R).view(np.int32)).to(DEV))
        Ss.append(torch.from_numpy(np.ascontiguousarray(S).view(np.int32)).to(DEV))
    res = hjm.hj_join_batch(ctx, Rs, Ss, mode=mode, checksum=True)
    for j, (R, S) in enumerate(host):
        cnt, c0, c1 = oracle.join_aggregate(R, S)
        assert (res[j].count, *res[j].checksum) == (cnt, c0, c1), j
        if mode == 2:
            want = oracle.sorted_pairs(*oracle.hash_join(R, S))
            assert np.array_equal(_sorted(res[j].pairs_numpy()), want), j
            res[j].free()


def test_batch_full_size_counts_and_sampled_pairs(hjm, ctx):
    # The 4096-join batch at full size (|R| log-uniform in [2^10, 2^22], |S| = 4 |R|, about
    # 1.1e10 tuples), in the launch configuration the bench times (pairs materialised,
    # one CUDA graph per wave).  R keys are exactly 1..|R|, so an S tuple matches once
    # if its key is at most |R| and never otherwise: every join's count is checked
    # against that property, and sampled joins' pairs against the oracle.
    specs = W.batched_specs(4096, W.DEFAULT_SEED)
    R_all, S_all, rs, ss = W.batched_relations(specs, W.DEFAULT_SEED, DEV)
    n = len(specs)
    Rs = [R_all[rs[j]:rs[j] + sp.n_r] for j, sp in enumerate(specs)]
    Ss = [S_all[ss[j]:ss[j] + sp.n_s] for j, sp in enumerate(specs)]
    # expected counts, chunk by chunk over S_all (padding rows between joins are skipped)
    starts = torch.tensor(ss, dtype=torch.int64, device=DEV)
    ends = starts + torch.tensor([sp.n_s for sp in specs], dtype=torch.int64, device=DEV)
    nr = torch.tensor([sp.n_r for sp in specs], dtype=torch.int64, device=DEV)
    want = torch.zeros(n, dtype=torch.int64, device=DEV)
    step = 1 << 27
    for a in range(0, S_all.shape[0], step):
        row = torch.arange(a, min(a + step, S_all.shape[0]), dtype=torch.int64, device=DEV)
        j = torch.searchsorted(starts, row, right=True) - 1
        live = row < ends[j]
        key = S_all[a:a + len(row), 0].to(torch.int64) & 0xFFFFFFFF
        want.index_add_(0, j, (live & (key <= nr[j])).to(torch.int64))
    want = want.cpu().tolist()
    ra, sa = hjm.rel_array(Rs), hjm.rel_array(Ss)
    outs = hjm.hj_join_batch(ctx, ra, sa, graph=True, raw=True)
    try:
        for j in range(n):
            assert outs[j].count == want[j], j
        order = sorted(range(n), key=lambda j: specs[j].n_r)
        for j in order[:4] + order[n // 2:n // 2 + 1] + order[-1:]:
            res = hjm._result(ctx, outs[j])
            got = res.pairs_numpy().astype(np.uint64)
            r, s = W.to_numpy_u(Rs[j]), W.to_numpy_u(Ss[j])
            assert np.array_equal(_sorted(got), oracle.sorted_pairs(*oracle.hash_join(r, s))), j
    finally:
        hjm.hj_results_free(ctx, outs, n)
