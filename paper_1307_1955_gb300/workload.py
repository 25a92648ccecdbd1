"""Seeded synthetic relations for the hash-join workloads.

This module generates inputs only: it holds none of the join's arithmetic, and
both the CUDA path's tests/bench and the CPU oracle's tests draw their inputs
from it.  Every value is a pure function of (seed, stream ids, row index), so the
same call gives identical bytes on a CPU tensor and on a CUDA tensor.

Relations are tensors of shape (n, 2): column 0 the key, column 1 the rid
(payload), stored as int32 (bit pattern of the unsigned 32-bit value) or int64
(bit pattern of the unsigned 64-bit value).  The paper's data sets are two
four-byte integer attributes per tuple, generated synthetically (Sec. 5.1).

Random words come from a counter-based SplitMix64 stream (Steele, Lea, Flood,
OOPSLA 2014): word i of stream s is the SplitMix64 finaliser of
s + (i + 1) * 0x9E3779B97F4A7C15, computed with wrapping int64 arithmetic and
logical shifts.  Permutations are a keyed bijection on [0, 2^k) (odd multiplier,
xorshift and key XOR rounds) restricted to [0, n) by cycle walking.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
DEFAULT_SEED = 0x5EED


def _s64(v: int) -> int:
    """Unsigned 64-bit value -> the int64 with the same bit pattern."""
    v &= M64
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _fin(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def _fin_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream_id(seed: int, *ids: int) -> int:
    """Derive a stream word from the seed and a tuple of small ids (pure Python)."""
    s = _fin_int(seed)
    for i in ids:
        s = _fin_int(s ^ _fin_int(i + 0x632BE59BD9B4E019))
    return s


def words(stream: int, start: int, count: int, device) -> torch.Tensor:
    """SplitMix64 words start .. start+count-1 of a stream, as int64 bit patterns."""
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _fin(i * _s64(GAMMA) + _s64(stream))


def uniform_below(n: int, stream: int, count: int, device, start: int = 0) -> torch.Tensor:
    """Integers uniform on [0, n), n <= 2^31 (multiply-shift on the high 32 bits)."""
    if not 1 <= n <= (1 << 31):
        raise ValueError("n must be in [1, 2^31]")
    hi = _srl(words(stream, start, count, device), 32)
    return (hi * n) >> 32


def unit_doubles(stream: int, count: int, device) -> torch.Tensor:
    """Doubles uniform on [0, 1): the top 53 bits of each word times 2^-53 (exact)."""
    return _srl(words(stream, 0, count, device), 11).to(torch.float64) * (2.0 ** -53)


def _bijection(x: torch.Tensor, k: int, keys: list[int]) -> torch.Tensor:
    mask = (1 << k) - 1
    s = max(1, (k + 1) // 2)
    for r, key in enumerate(keys):
        mult = (0xD1B54A32D192ED03 + 2 * r * 0x2545F4914F6CDD1D) | 1
        x = (x * _s64(mult)) & mask
        x = x ^ (x >> s)
        x = x ^ (key & mask)
    return x


def permutation(n: int, stream: int, device, start: int = 0, count: int | None = None) -> torch.Tensor:
    """Entries start .. start+count-1 of a seeded permutation of [0, n)."""
    count = n - start if count is None else count
    x = torch.arange(start, start + count, dtype=torch.int64, device=device)
    if n <= 1:
        return x
    k = max(2, math.ceil(math.log2(n)))
    keys = [_fin_int(stream + r + 1) for r in range(4)]
    y = _bijection(x, k, keys)
    while True:
        bad = y >= n
        if not bool(bad.any()):
            return y
        y = torch.where(bad, _bijection(y, k, keys), y)


def _u32_bits(v: torch.Tensor) -> torch.Tensor:
    """Unsigned 32-bit values held in int64 -> int32 with the same bit pattern."""
    v = v & 0xFFFFFFFF
    return (v - ((v >> 31) << 32)).to(torch.int32)


def make_relation(keys: torch.Tensor, rids: torch.Tensor, width: int) -> torch.Tensor:
    """Pack key and rid columns (int64 holding unsigned values) into an (n, 2) AoS tensor."""
    if width == 4:
        return torch.stack([_u32_bits(keys), _u32_bits(rids)], dim=1).contiguous()
    if width == 8:
        return torch.stack([keys, rids], dim=1).contiguous()
    raise ValueError("width must be 4 or 8")


# --------------------------------------------------------------------------- workloads


def unique_and_uniform(n_r: int, n_s: int, s_domain: int, seed: int, device, width: int = 4,
                       ids: tuple = ()):
    """R keys: a seeded permutation of 1..|R| (unique); R rid = row index.
    S keys: uniform on [1, s_domain]; S rid = row index.

    With s_domain = |R| every S tuple matches exactly one R tuple; with
    s_domain = |R| / m a fraction m of S matches (once each)."""
    pr = stream_id(seed, *ids, 1)
    ps = stream_id(seed, *ids, 2)
    rk = permutation(n_r, pr, device) + 1
    rr = torch.arange(n_r, dtype=torch.int64, device=device)
    sk = uniform_below(s_domain, ps, n_s, device) + 1 if n_s else torch.zeros(0, dtype=torch.int64, device=device)
    sr = torch.arange(n_s, dtype=torch.int64, device=device)
    return make_relation(rk, rr, width), make_relation(sk, sr, width)


def heavy_hitter(n_r: int, n_s: int, s: float, seed: int, device, width: int = 4, ids: tuple = (),
                 heavy_key: int = 1):
    """The paper's skewed data sets (Sec. 5.1: a fraction s of the tuples share one
    duplicated key value), read as: round(s |R|) R tuples carry one key, the heavy
    hitter (`heavy_key`, an unsigned value; 1 by default), and the other R tuples
    the distinct keys 2 .. |R| - round(s |R|) + 1, in a seeded order.  S keys are
    uniform over R's distinct keys, so a few S tuples meet the heavy hitter and
    every other S tuple exactly one R tuple.  rids are row indices."""
    nh = int(round(s * n_r))
    if not 0 < nh <= n_r:
        raise ValueError("s * |R| must round to between 1 and |R| tuples")
    pr = stream_id(seed, *ids, 1)
    ps = stream_id(seed, *ids, 2)
    p = permutation(n_r, pr, device)
    hk = torch.full_like(p, _s64(heavy_key))
    rk = torch.where(p < nh, hk, p - nh + 2)
    nd = n_r - nh + 1  # distinct R keys: the heavy hitter (drawn as 1) and 2 .. n_r - nh + 1
    if n_s:
        sk = uniform_below(nd, ps, n_s, device) + 1
        sk = torch.where(sk == 1, torch.full_like(sk, _s64(heavy_key)), sk)
    else:
        sk = torch.zeros(0, dtype=torch.int64, device=device)
    rr = torch.arange(n_r, dtype=torch.int64, device=device)
    sr = torch.arange(n_s, dtype=torch.int64, device=device)
    return make_relation(rk, rr, width), make_relation(sk, sr, width)


def zipf_cdf(n_ranks: int, theta: float) -> torch.Tensor:
    """CPU float64 CDF of P(rank = k) proportional to k^-theta, k = 1..n_ranks (last entry 1.0)."""
    k = torch.arange(1, n_ranks + 1, dtype=torch.float64)
    c = torch.cumsum(k.pow(-theta), 0)
    c = c / c[-1]
    c[-1] = 1.0
    return c


def zipf_keys(n: int, theta: float, n_ranks: int, stream: int, key_stream: int, device) -> torch.Tensor:
    """n keys whose ranks are Zipf(theta) over n_ranks values, drawn by inverse CDF;
    rank k maps to the 64-bit key SplitMix64-finaliser(k + key_stream) (a bijection,
    so distinct ranks give distinct keys spread over all 64 bits)."""
    cdf = zipf_cdf(n_ranks, theta).to(device)
    u = unit_doubles(stream, n, device)
    rank = torch.searchsorted(cdf, u, right=True) + 1
    return _fin(rank + _s64(key_stream))


def zipf_pair(n_r: int, n_s: int, theta_r: float, theta_s: float, n_ranks: int, seed: int, device,
              ids: tuple = ()):
    """Skewed 64-bit workload: R and S keys Zipf over the same n_ranks distinct keys,
    payload = row index, width 8."""
    ks = stream_id(seed, *ids, 0)
    rk = zipf_keys(n_r, theta_r, n_ranks, stream_id(seed, *ids, 1), ks, device)
    sk = zipf_keys(n_s, theta_s, n_ranks, stream_id(seed, *ids, 2), ks, device)
    rr = torch.arange(n_r, dtype=torch.int64, device=device)
    sr = torch.arange(n_s, dtype=torch.int64, device=device)
    return make_relation(rk, rr, 8), make_relation(sk, sr, 8)


@dataclass(frozen=True)
class JoinSpec:
    """Sizes of one join of a batch or of a served request."""
    n_r: int
    n_s: int
    s_domain: int
    arrival_s: float = 0.0


def batched_specs(n_joins: int, seed: int, lo_log2: float = 10.0, hi_log2: float = 22.0,
                  s_factor: int = 4, match_rate: float = 0.75) -> list[JoinSpec]:
    """|R| = floor(2^U), U ~ Uniform[lo, hi]; |S| = s_factor * |R|;
    S keys uniform over [1, ceil(|R| / match_rate)] (computed on the CPU)."""
    u = unit_doubles(stream_id(seed, 4, 0), n_joins, "cpu").tolist()
    out = []
    for x in u:
        n_r = int(math.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * x)))
        out.append(JoinSpec(n_r, s_factor * n_r, int(math.ceil(n_r / match_rate))))
    return out


def serving_specs(n_req: int, seed: int, rate_per_s: float, lo_log2: float = 12.0, hi_log2: float = 24.0,
                  max_s_factor_log16: float = 1.0, match_rate: float = 0.5) -> list[JoinSpec]:
    """Poisson arrivals at rate_per_s; |R| = 2^U, U ~ U[lo, hi] (rounded down);
    |S| = |R| * 16^V, V ~ U[0, 1]; S keys uniform over [1, ceil(|R| / match_rate)]."""
    u = unit_doubles(stream_id(seed, 5, 0), 3 * n_req, "cpu").tolist()
    t = 0.0
    out = []
    for i in range(n_req):
        ua, ur, us = u[3 * i], u[3 * i + 1], u[3 * i + 2]
        t += -math.log(1.0 - ua) / rate_per_s
        n_r = int(math.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * ur)))
        n_s = int(math.floor(n_r * 16.0 ** (max_s_factor_log16 * us)))
        out.append(JoinSpec(n_r, n_s, int(math.ceil(n_r / match_rate)), t))
    return out


def to_numpy_u(rel: torch.Tensor):
    """(n, 2) int32/int64 tensor -> numpy uint32/uint64 view of the same bytes (CPU copy)."""
    import numpy as np

    a = rel.detach().cpu().contiguous().numpy()
    return a.view(np.uint32 if a.dtype == np.int32 else np.uint64)


# ------------------------------------------------------------------ batched relations


def _bijection_vec(x: torch.Tensor, kbits: torch.Tensor, keys: torch.Tensor) -> torch.Tensor:
    """_bijection with a per-element bit width and per-element round keys [rounds, n]."""
    mask = (torch.ones_like(kbits) << kbits) - 1
    s = torch.clamp((kbits + 1) // 2, min=1)
    for r in range(keys.shape[0]):
        mult = (0xD1B54A32D192ED03 + 2 * r * 0x2545F4914F6CDD1D) | 1
        x = (x * _s64(mult)) & mask
        x = x ^ (x >> s)
        x = x ^ (keys[r] & mask)
    return x


def _segments(sizes: list[int]) -> list[int]:
    """Start rows of consecutive segments, each starting on an even row (16-byte
    aligned for 4-byte tuples); the last entry is the total row count."""
    out, at = [], 0
    for n in sizes:
        out.append(at)
        at += n + (n & 1)
    out.append(at)
    return out


def batched_relations(specs: list, seed: int, device, ids: tuple = (4,), chunk: int = 1 << 26):
    """All joins of a batch in two big int32 tensors: join j's R is rows
    [r_start[j], r_start[j] + n_r) of R_all (likewise S), byte-identical to
    unique_and_uniform(n_r, n_s, s_domain, seed, ids=ids + (j,)).  Returns
    (R_all, S_all, r_start, s_start)."""
    nj = len(specs)
    rs = _segments([sp.n_r for sp in specs])
    ss = _segments([sp.n_s for sp in specs])
    R = torch.zeros((rs[-1], 2), dtype=torch.int32, device=device)
    S = torch.zeros((ss[-1], 2), dtype=torch.int32, device=device)
    # per-join parameters (CPU), gathered per element on the device
    pr = [stream_id(seed, *ids, j, 1) for j in range(nj)]
    ps = [stream_id(seed, *ids, j, 2) for j in range(nj)]
    kb = [max(2, math.ceil(math.log2(sp.n_r))) if sp.n_r > 1 else 0 for sp in specs]
    rkeys = torch.tensor([[_s64(_fin_int(pr[j] + r + 1)) for j in range(nj)] for r in range(4)], dtype=torch.int64,
                         device=device)
    t_nr = torch.tensor([sp.n_r for sp in specs], dtype=torch.int64, device=device)
    t_dom = torch.tensor([sp.s_domain for sp in specs], dtype=torch.int64, device=device)
    t_kb = torch.tensor(kb, dtype=torch.int64, device=device)
    t_ps = torch.tensor([_s64(x) for x in ps], dtype=torch.int64, device=device)
    t_rs = torch.tensor(rs, dtype=torch.int64, device=device)
    t_ss = torch.tensor(ss, dtype=torch.int64, device=device)
    t_ns = torch.tensor([sp.n_s for sp in specs], dtype=torch.int64, device=device)
    for a in range(0, rs[-1], chunk):
        row = torch.arange(a, min(a + chunk, rs[-1]), dtype=torch.int64, device=device)
        j = torch.searchsorted(t_rs, row, right=True) - 1
        local = row - t_rs[j]
        live = local < t_nr[j]
        nr = t_nr[j]
        x = local.clone()
        big = live & (nr > 1)
        kj = t_kb[j]
        keys = rkeys[:, j]
        y = _bijection_vec(x, kj, keys)
        while True:
            bad = big & (y >= nr)
            if not bool(bad.any()):
                break
            y = torch.where(bad, _bijection_vec(y, kj, keys), y)
        key = torch.where(big, y, local) + 1
        blk = torch.stack([_u32_bits(key), _u32_bits(local)], dim=1)
        R[a:a + len(row)] = torch.where(live[:, None], blk, torch.zeros_like(blk))
    for a in range(0, ss[-1], chunk):
        row = torch.arange(a, min(a + chunk, ss[-1]), dtype=torch.int64, device=device)
        j = torch.searchsorted(t_ss, row, right=True) - 1
        local = row - t_ss[j]
        live = local < t_ns[j]
        w = _fin((local + 1) * _s64(GAMMA) + t_ps[j])
        key = ((_srl(w, 32) * t_dom[j]) >> 32) + 1
        blk = torch.stack([_u32_bits(key), _u32_bits(local)], dim=1)
        S[a:a + len(row)] = torch.where(live[:, None], blk, torch.zeros_like(blk))
    return R, S, rs[:-1], ss[:-1]
