"""The seeded input generators: determinism, exact agreement with a plain-Python
restatement of the counter stream, and the structural promises each workload makes
(unique R keys, S key range, Zipf ranks).  CPU only."""
import math

import numpy as np
import pytest
import torch

from paper_1307_1955_gb300 import workload as W

M = (1 << 64) - 1


def _fin(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_words_match_python_integers():
    st = W.stream_id(W.DEFAULT_SEED, 3, 9)
    w = W.words(st, 100, 64, "cpu").numpy().view(np.uint64)
    for i in range(64):
        assert int(w[i]) == _fin((st + (101 + i) * W.GAMMA) & M)


def test_uniform_below_range_and_exact_formula():
    st = W.stream_id(1, 2)
    for n in (1, 7, 1000, 1 << 25, 1 << 31):
        v = W.uniform_below(n, st, 4096, "cpu").numpy()
        assert v.min() >= 0 and v.max() < n
        raw = W.words(st, 0, 8, "cpu").numpy().view(np.uint64)
        for i in range(8):
            assert int(v[i]) == ((int(raw[i]) >> 32) * n) >> 32


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1000, 4096, 70001])
def test_permutation_is_a_bijection(n):
    p = W.permutation(n, W.stream_id(5, n), "cpu").numpy()
    assert np.array_equal(np.sort(p), np.arange(n))
    # chunked evaluation gives the same entries
    if n > 10:
        part = W.permutation(n, W.stream_id(5, n), "cpu", start=3, count=7).numpy()
        assert np.array_equal(part, p[3:10])


def test_unique_and_uniform_structure():
    n_r, n_s, dom = 5000, 20000, 10000
    R, S = W.unique_and_uniform(n_r, n_s, dom, 7, "cpu")
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    assert r.dtype == np.uint32 and r.shape == (n_r, 2)
    assert np.array_equal(np.sort(r[:, 0]), np.arange(1, n_r + 1, dtype=np.uint32))
    assert np.array_equal(r[:, 1], np.arange(n_r, dtype=np.uint32))
    assert s[:, 0].min() >= 1 and s[:, 0].max() <= dom
    assert np.array_equal(s[:, 1], np.arange(n_s, dtype=np.uint32))
    # about half the S keys fall inside R's key range
    frac = np.mean(s[:, 0] <= n_r)
    assert abs(frac - 0.5) < 0.02
    # deterministic
    R2, S2 = W.unique_and_uniform(n_r, n_s, dom, 7, "cpu")
    assert torch.equal(R, R2) and torch.equal(S, S2)


@pytest.mark.parametrize("width,hk", [(4, 1), (4, 0xFFFFFFFF), (8, (1 << 64) - 1)])
def test_heavy_hitter_structure(width, hk):
    # round(s |R|) R tuples share the heavy key, the rest are distinct, S keys are
    # uniform over R's distinct keys (the heavy key among them)
    n_r, n_s, s = 4000, 30000, 0.25
    R, S = W.heavy_hitter(n_r, n_s, s, 9, "cpu", width=width, heavy_key=hk)
    r, q = W.to_numpy_u(R), W.to_numpy_u(S)
    nh = int(round(s * n_r))
    heavy = r[:, 0] == np.array(hk, dtype=r.dtype)
    assert heavy.sum() == nh
    others = np.sort(r[~heavy, 0])
    assert np.array_equal(others, np.arange(2, n_r - nh + 2, dtype=r.dtype))
    assert np.array_equal(r[:, 1], np.arange(n_r, dtype=r.dtype))
    assert np.isin(q[:, 0], r[:, 0]).all()
    # the heavy key gets its share 1 / (n_r - nh + 1) of S
    frac = np.mean(q[:, 0] == np.array(hk, dtype=q.dtype))
    assert abs(frac - 1.0 / (n_r - nh + 1)) < 0.002
    R2, S2 = W.heavy_hitter(n_r, n_s, s, 9, "cpu", width=width, heavy_key=hk)
    assert torch.equal(R, R2) and torch.equal(S, S2)


def test_u64_relation_bit_patterns():
    keys = torch.tensor([0, -1, 1 << 40], dtype=torch.int64)
    rel = W.make_relation(keys, torch.arange(3), 8)
    u = W.to_numpy_u(rel)
    assert u.dtype == np.uint64
    assert list(u[:, 0]) == [0, (1 << 64) - 1, 1 << 40]


def test_u32_relation_high_bit_values():
    keys = torch.tensor([0, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF], dtype=torch.int64)
    u = W.to_numpy_u(W.make_relation(keys, keys, 4))
    assert list(u[:, 0]) == [0, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF]


def test_zipf_ranks_follow_the_pmf():
    theta, nr = 1.0, 64
    st = W.stream_id(3, 1)
    cdf = W.zipf_cdf(nr, theta)
    u = W.unit_doubles(st, 200000, "cpu")
    rank = (torch.searchsorted(cdf, u, right=True) + 1).numpy()
    assert rank.min() >= 1 and rank.max() <= nr
    pmf = np.arange(1, nr + 1, dtype=np.float64) ** -theta
    pmf /= pmf.sum()
    freq = np.bincount(rank, minlength=nr + 1)[1:] / len(rank)
    assert np.all(np.abs(freq - pmf) < 5 * np.sqrt(pmf / len(rank)) + 1e-4)


def test_zipf_pair_shares_key_domain():
    R, S = W.zipf_pair(3000, 6000, 0.75, 0.5, 1 << 8, 4, "cpu")
    r, s = W.to_numpy_u(R), W.to_numpy_u(S)
    assert len(np.unique(r[:, 0])) <= 256
    assert set(np.unique(s[:, 0])) <= set(np.unique(np.concatenate([r[:, 0], s[:, 0]])))
    assert len(set(np.unique(s[:, 0])) & set(np.unique(r[:, 0]))) > 100


def test_batched_specs_ranges():
    specs = W.batched_specs(512, W.DEFAULT_SEED)
    for sp in specs:
        assert 1 << 10 <= sp.n_r <= 1 << 22
        assert sp.n_s == 4 * sp.n_r
        assert sp.s_domain == math.ceil(sp.n_r / 0.75)
    lg = np.log2([sp.n_r for sp in specs])
    assert abs(lg.mean() - 16.0) < 0.5


def test_serving_specs_ranges():
    specs = W.serving_specs(1000, W.DEFAULT_SEED, rate_per_s=100.0)
    t = [sp.arrival_s for sp in specs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert abs(t[-1] / 1000 - 0.01) < 0.002
    for sp in specs:
        assert 1 << 12 <= sp.n_r <= 1 << 24
        assert sp.n_r <= sp.n_s <= 16 * sp.n_r


def test_batched_relations_equal_per_join_generation():
    specs = W.batched_specs(40, 3, lo_log2=1, hi_log2=12)
    specs[3] = W.JoinSpec(1, 4, 2)
    specs[4] = W.JoinSpec(0, 0, 1)
    R, S, rs, ss = W.batched_relations(specs, 3, "cpu", chunk=1000)
    for j, sp in enumerate(specs):
        r1, s1 = W.unique_and_uniform(sp.n_r, sp.n_s, sp.s_domain, 3, "cpu", ids=(4, j))
        assert torch.equal(R[rs[j]:rs[j] + sp.n_r], r1)
        assert torch.equal(S[ss[j]:ss[j] + sp.n_s], s1)
        assert rs[j] % 2 == 0 and ss[j] % 2 == 0       # 16-byte aligned segments
