// join.cu -- build and probe kernels (Alg. 1 steps b1-b4 and p1-p4).
//
//   * table_* : the simple hash join's table in global memory (SHJ), shared by all
//     CTAs (Sec. 3.3: one shared table rather than one per processor).
//   * partition_join : Alg. 2's per-partition SHJ with the table in shared memory,
//     one CTA per partition pair.
//
// Output placement for the pairs (Sec. 3.3's block allocator, GPU form): a CTA
// probes a tile of S, counts the matches of each thread, scans the counts across
// the block, reserves the tile's whole range with ONE atomicAdd on the global
// cursor, and threads write their pairs densely into it.  The common case of one
// match per tuple keeps the build rid from the first walk; only tuples with
// several matches walk their bucket run a second time.
#include "common.cuh"
#include "engine.cuh"

namespace hj {

// ------------------------------------------------------------------ tuple loads
// Tuples of a range are visited by 16-byte vectors: vector v holds tuples
// v*PV .. v*PV+PV-1.  The last vector of a 4-byte relation with an odd number of
// tuples is read with one 8-byte load so no read passes the array end.
template <int W>
__device__ __forceinline__ void load_vec(const void *base, uint64_t v, uint64_t n_total, typename Tup<W>::U *k,
                                         typename Tup<W>::U *r) {
    if constexpr (W == 8) {
        ulonglong2 x = ld_stream((const ulonglong2 *)base + v);
        k[0] = x.x;
        r[0] = x.y;
    } else {
        if (2 * v + 1 < n_total) {
            uint4 x = ld_stream((const uint4 *)base + v);
            k[0] = x.x;
            r[0] = x.y;
            k[1] = x.z;
            r[1] = x.w;
        } else {
            uint2 x = ((const uint2 *)base)[2 * v];
            k[0] = x.x;
            r[0] = x.y;
            k[1] = 0;
            r[1] = 0;
        }
    }
}

template <int W> struct PairOut;
template <> struct PairOut<4> {
    static __device__ __forceinline__ void put(void *p, uint64_t i, uint32_t a, uint32_t b) {
        ((uint2 *)p)[i] = make_uint2(a, b);
    }
};
template <> struct PairOut<8> {
    static __device__ __forceinline__ void put(void *p, uint64_t i, uint64_t a, uint64_t b) {
        ((ulonglong2 *)p)[i] = make_ulonglong2(a, b);
    }
};

// ----------------------------------------------------------------- table views
template <int W> struct PairView {
    using U = typename Tup<W>::U;
    const typename PairSlot<W>::S *slots;
    uint64_t cap;
    unsigned long long n_allones;
    template <class F> __device__ __forceinline__ void lookup(U k, uint64_t h, F &&f) const {
        pair_lookup<W>(slots, cap, n_allones, k, h, f);
    }
};
template <int W> struct AggView {
    using U = typename Tup<W>::U;
    const AggSlot<W> *slots;
    uint64_t cap;
    const TableSide *side;
    __device__ __forceinline__ void lookup(U k, uint64_t h, uint64_t *cnt, uint64_t *suma) const {
        agg_lookup<W>(slots, cap, side, k, h, cnt, suma);
    }
};

// Shared scratch for the tile emission (block scan + reserved base).
struct EmitShared {
    unsigned long long scan[33];
    unsigned long long base;
};

// Probe IT tuples per thread against a pair table and place their pairs.
// All threads of the block must call this (it contains barriers).
template <int W, int IT, class View>
__device__ __forceinline__ void probe_tile_pairs(const View &tab, const typename Tup<W>::U *k,
                                                 const typename Tup<W>::U *r, const bool *valid, void *pairs,
                                                 uint64_t pcap, hj_counters *ctr, bool chk, uint64_t &c0,
                                                 uint64_t &c1, EmitShared &es) {
    using U = typename Tup<W>::U;
    uint32_t cnt[IT];
    U first[IT];
    uint64_t mine = 0;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        cnt[i] = 0;
        first[i] = 0;
        if (valid[i]) {
            uint64_t h = key_hash<W>(k[i]);
            uint64_t bs = chk ? mix_b(r[i]) : 0;
            uint32_t c = 0;
            U f = 0;
            tab.lookup(k[i], h, [&](U rid) {
                if (c == 0) f = rid;
                ++c;
                if (chk) {
                    uint64_t a = mix_a(rid);
                    c0 += a * bs;
                    c1 += a + bs;
                }
            });
            cnt[i] = c;
            first[i] = f;
            mine += c;
        }
    }
    unsigned long long total;
    unsigned long long off = block_exclusive_scan<unsigned long long>(mine, es.scan, &total);
    if (threadIdx.x == 0) es.base = total ? atomicAdd(&ctr->count, total) : 0ull;
    __syncthreads();
    uint64_t pos = es.base + off;
    __syncthreads();
    if (mine) {
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            if (cnt[i] == 1) {
                if (pos < pcap) PairOut<W>::put(pairs, pos, first[i], r[i]);
                ++pos;
            } else if (cnt[i] > 1) {
                uint64_t h = key_hash<W>(k[i]);
                U s = r[i];
                tab.lookup(k[i], h, [&](U rid) {
                    if (pos < pcap) PairOut<W>::put(pairs, pos, rid, s);
                    ++pos;
                });
            }
        }
    }
}

// Probe IT tuples per thread against an aggregate table (count modes).
template <int W, int IT>
__device__ __forceinline__ void probe_tile_agg(const AggView<W> &tab, const typename Tup<W>::U *k,
                                               const typename Tup<W>::U *r, const bool *valid, bool chk,
                                               uint64_t &cnt, uint64_t &c0, uint64_t &c1) {
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        if (!valid[i]) continue;
        uint64_t n, sa;
        tab.lookup(k[i], key_hash<W>(k[i]), &n, &sa);
        cnt += n;
        if (chk && n) {
            uint64_t b = mix_b(r[i]);
            c0 += sa * b;
            c1 += sa + n * b;
        }
    }
}

__device__ __forceinline__ void flush_sums(hj_counters *ctr, uint64_t cnt, uint64_t c0, uint64_t c1, bool with_cnt) {
    cnt = warp_sum(cnt);
    c0 = warp_sum(c0);
    c1 = warp_sum(c1);
    if ((threadIdx.x & 31) == 0) {
        if (with_cnt && cnt) atomicAdd(&ctr->count, (unsigned long long)cnt);
        if (c0) atomicAdd(&ctr->c0, (unsigned long long)c0);
        if (c1) atomicAdd(&ctr->c1, (unsigned long long)c1);
    }
}

// ============================================================ global table (SHJ)

template <int W>
__global__ void agg_table_init(AggSlot<W> *slots, uint64_t cap) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x) {
        AggSlot<W> s;
        s.key = Tup<W>::kAllOnes;
        s.cnt = 0;
        s.suma = 0;
        if constexpr (W == 8) s.pad = 0;
        slots[i] = s;
    }
}

template <int W, bool AGG>
__global__ void __launch_bounds__(256) table_build_kernel(const void *R, uint64_t lo, uint64_t hi, uint64_t n_total,
                                                          void *slots, uint64_t cap, TableSide *side,
                                                          hj_counters *ctr) {
    using U = typename Tup<W>::U;
    constexpr int PV = Tup<W>::kPerVec;
    uint64_t va = lo / PV, vb = (hi + PV - 1) / PV;
    for (uint64_t v = va + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < vb;
         v += (uint64_t)gridDim.x * blockDim.x) {
        U k[2], r[2];
        load_vec<W>(R, v, n_total, k, r);
#pragma unroll
        for (int e = 0; e < PV; ++e) {
            uint64_t t = v * PV + e;
            if (t < lo || t >= hi) continue;
            uint64_t h = key_hash<W>(k[e]);
            bool ok = AGG ? agg_insert<W>((AggSlot<W> *)slots, cap, side, k[e], mix_a(r[e]), h)
                          : pair_insert<W>((typename PairSlot<W>::S *)slots, cap, side, k[e], r[e], h);
            if (!ok) atomicOr(&ctr->status, (unsigned long long)kStatusTableFull);
        }
    }
}

// Tuples per thread per tile: 4 (two 16-byte vectors of 4-byte tuples, or four
// vectors of 8-byte tuples).
template <int W> struct ProbeShape {
    static constexpr int PV = Tup<W>::kPerVec;
    static constexpr int VPT = 4 / PV;
    static constexpr int IT = 4;
};

template <int W, bool AGG>
__global__ void __launch_bounds__(512) table_probe_kernel(const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                                                          const void *slots, uint64_t cap, const TableSide *side,
                                                          void *pairs, uint64_t pcap, hj_counters *ctr, int chk) {
    using U = typename Tup<W>::U;
    using PSh = ProbeShape<W>;
    constexpr int PV = PSh::PV, VPT = PSh::VPT, IT = PSh::IT;
    __shared__ EmitShared es;
    uint64_t va = lo / PV, vb = (hi + PV - 1) / PV;
    uint64_t tile_vecs = (uint64_t)blockDim.x * VPT;
    uint64_t ntiles = (vb - va + tile_vecs - 1) / tile_vecs;
    uint64_t cnt = 0, c0 = 0, c1 = 0;
    PairView<W> pv{(const typename PairSlot<W>::S *)slots, cap, AGG ? 0ull : side->n_allones};
    AggView<W> av{(const AggSlot<W> *)slots, cap, side};
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        U k[IT], r[IT];
        bool valid[IT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            uint64_t v = va + tile * tile_vecs + (uint64_t)j * blockDim.x + threadIdx.x;
            U kk[2] = {0, 0}, rr[2] = {0, 0};
            if (v < vb) load_vec<W>(S, v, n_total, kk, rr);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                k[j * PV + e] = kk[e];
                r[j * PV + e] = rr[e];
                valid[j * PV + e] = v < vb && t >= lo && t < hi;
            }
        }
        if constexpr (AGG) {
            probe_tile_agg<W, IT>(av, k, r, valid, chk != 0, cnt, c0, c1);
        } else {
            probe_tile_pairs<W, IT>(pv, k, r, valid, pairs, pcap, ctr, chk != 0, c0, c1, es);
        }
    }
    flush_sums(ctr, cnt, c0, c1, AGG);
}

hj_status table_create(hj_ctx *c, int width, int agg, uint64_t n_build, hj_table **out) {
    *out = nullptr;
    hj_table *t = new hj_table();
    t->width = width;
    t->agg = agg;
    // Capacity: a power of two at least twice the build size (load factor <= 0.5).
    uint64_t cap = 64;
    while (cap < 2 * n_build + 1) cap <<= 1;
    t->cap = cap;
    uint64_t slot_bytes = agg ? (width == 4 ? sizeof(AggSlot<4>) : sizeof(AggSlot<8>)) : 2ull * width;
    hj_status st;
    t->slots = dalloc(c, cap * slot_bytes, &st);
    if (st != HJ_OK) {
        delete t;
        return st;
    }
    t->side = dalloc(c, sizeof(TableSide), &st);
    if (st != HJ_OK) {
        dfree(c, t->slots);
        delete t;
        return st;
    }
    cudaMemsetAsync(t->side, 0, sizeof(TableSide), c->stream);
    int grid = num_sms(c) * 4;
    if (!agg) {
        HJ_CUDA(c, cudaMemsetAsync(t->slots, 0xFF, cap * slot_bytes, c->stream));
    } else if (width == 4) {
        HJ_LAUNCH(c, "agg_table_init", agg_table_init<4>, grid, 256, 0, (AggSlot<4> *)t->slots, cap);
    } else {
        HJ_LAUNCH(c, "agg_table_init", agg_table_init<8>, grid, 256, 0, (AggSlot<8> *)t->slots, cap);
    }
    *out = t;
    return HJ_OK;
}

void table_destroy(hj_ctx *c, hj_table *t) {
    if (!t) return;
    dfree(c, t->slots);
    dfree(c, t->side);
    delete t;
}

hj_status table_build(hj_ctx *c, hj_table *t, const void *R, uint64_t lo, uint64_t hi, uint64_t n_total) {
    if (hi <= lo) return HJ_OK;
    uint64_t nvec = (hi - lo) / (t->width == 4 ? 2 : 1) + 2;
    uint64_t want = (nvec + 255) / 256;
    int grid = (int)(want < (uint64_t)num_sms(c) * 8 ? (want ? want : 1) : (uint64_t)num_sms(c) * 8);
    TableSide *side = (TableSide *)t->side;
    if (t->width == 4) {
        if (t->agg)
            HJ_LAUNCH(c, "table_build", (table_build_kernel<4, true>), grid, 256, 0, R, lo, hi, n_total, t->slots, t->cap, side, c->d_ctr);
        else
            HJ_LAUNCH(c, "table_build", (table_build_kernel<4, false>), grid, 256, 0, R, lo, hi, n_total, t->slots, t->cap, side, c->d_ctr);
    } else {
        if (t->agg)
            HJ_LAUNCH(c, "table_build", (table_build_kernel<8, true>), grid, 256, 0, R, lo, hi, n_total, t->slots, t->cap, side, c->d_ctr);
        else
            HJ_LAUNCH(c, "table_build", (table_build_kernel<8, false>), grid, 256, 0, R, lo, hi, n_total, t->slots, t->cap, side, c->d_ctr);
    }
    return HJ_OK;
}

hj_status table_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                      void *pairs, uint64_t pcap, int checksum) {
    if (hi <= lo) return HJ_OK;
    const int block = 512;
    uint64_t tile_tuples = (uint64_t)block * 4;
    uint64_t want = (hi - lo + tile_tuples - 1) / tile_tuples + 1;
    uint64_t maxg = (uint64_t)num_sms(c) * 4;
    int grid = (int)(want < maxg ? want : maxg);
    const TableSide *side = (const TableSide *)t->side;
    if (t->width == 4) {
        if (t->agg)
            HJ_LAUNCH(c, "table_probe", (table_probe_kernel<4, true>), grid, block, 0, S, lo, hi, n_total, t->slots, t->cap, side, pairs, pcap, c->d_ctr, checksum);
        else
            HJ_LAUNCH(c, "table_probe", (table_probe_kernel<4, false>), grid, block, 0, S, lo, hi, n_total, t->slots, t->cap, side, pairs, pcap, c->d_ctr, checksum);
    } else {
        if (t->agg)
            HJ_LAUNCH(c, "table_probe", (table_probe_kernel<8, true>), grid, block, 0, S, lo, hi, n_total, t->slots, t->cap, side, pairs, pcap, c->d_ctr, checksum);
        else
            HJ_LAUNCH(c, "table_probe", (table_probe_kernel<8, false>), grid, block, 0, S, lo, hi, n_total, t->slots, t->cap, side, pairs, pcap, c->d_ctr, checksum);
    }
    return HJ_OK;
}

// ================================================== per-partition join (PHJ)
//
// CTA p joins partition pair (R_p, S_p): it builds a table over R_p in shared
// memory (capacity about twice |R_p|, multiply-shift buckets so any capacity
// works), then streams S_p tile by tile.  A partition whose table cannot fit
// (|R_p| too large for a pair table, or more distinct keys than slots for an
// aggregate table) is handed to the global-table fallback.

template <int W, bool AGG>
__global__ void __launch_bounds__(512) partition_join_kernel(const void *Rp, const uint64_t *roff, uint64_t nR_total,
                                                             const void *Sp, const uint64_t *soff, uint64_t nS_total,
                                                             uint64_t cap_max, void *pairs, uint64_t pcap,
                                                             hj_counters *ctr, uint32_t *oversize, int chk) {
    using U = typename Tup<W>::U;
    using PSh = ProbeShape<W>;
    constexpr int PV = PSh::PV, VPT = PSh::VPT, IT = PSh::IT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EmitShared es;
    __shared__ TableSide side;
    __shared__ int s_full;

    const uint32_t p = blockIdx.x;
    const uint64_t r0 = roff[p], r1 = roff[p + 1], s0 = soff[p], s1 = soff[p + 1];
    const uint64_t nr = r1 - r0;
    if (s1 <= s0 || nr == 0) return;  // no probe tuples or no build tuples: no pairs

    uint64_t cap;
    if (AGG) {
        cap = 2 * nr + 32;
        cap = cap < cap_max ? cap : cap_max;
    } else {
        cap = ((2 * nr + 31) / 32) * 32;
        if (cap > cap_max) cap = cap_max;
        if (nr >= cap - cap / 4) {  // load factor above 3/4: leave to the fallback
            if (threadIdx.x == 0) oversize[atomicAdd(&ctr->n_oversize, 1ull)] = p;
            return;
        }
    }
    // initialise the table
    if (AGG) {
        AggSlot<W> *sl = (AggSlot<W> *)smem;
        for (uint64_t i = threadIdx.x; i < cap; i += blockDim.x) {
            sl[i].key = Tup<W>::kAllOnes;
            sl[i].cnt = 0;
            sl[i].suma = 0;
        }
    } else {
        using S = typename PairSlot<W>::S;
        S *sl = (S *)smem;
        for (uint64_t i = threadIdx.x; i < cap; i += blockDim.x) sl[i] = PairSlot<W>::empty();
    }
    if (threadIdx.x == 0) {
        side.n_allones = side.agg_cnt = side.agg_suma = side.full = 0;
        s_full = 0;
    }
    __syncthreads();
    // build over R_p
    {
        uint64_t va = r0 / PV, vb = (r1 + PV - 1) / PV;
        for (uint64_t v = va + threadIdx.x; v < vb; v += blockDim.x) {
            U k[2], r[2];
            load_vec<W>(Rp, v, nR_total, k, r);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                if (t < r0 || t >= r1) continue;
                uint64_t h = key_hash<W>(k[e]);
                bool ok = AGG ? agg_insert<W>((AggSlot<W> *)smem, cap, &side, k[e], mix_a(r[e]), h)
                              : pair_insert<W>((typename PairSlot<W>::S *)smem, cap, &side, k[e], r[e], h);
                if (!ok) s_full = 1;
            }
        }
    }
    __syncthreads();
    if (s_full) {
        if (threadIdx.x == 0) oversize[atomicAdd(&ctr->n_oversize, 1ull)] = p;
        return;
    }
    // probe S_p
    PairView<W> pv{(const typename PairSlot<W>::S *)smem, cap, side.n_allones};
    AggView<W> av{(const AggSlot<W> *)smem, cap, &side};
    uint64_t cnt = 0, c0 = 0, c1 = 0;
    uint64_t va = s0 / PV, vb = (s1 + PV - 1) / PV;
    uint64_t tile_vecs = (uint64_t)blockDim.x * VPT;
    for (uint64_t base = va; base < vb; base += tile_vecs) {
        U k[IT], r[IT];
        bool valid[IT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            uint64_t v = base + (uint64_t)j * blockDim.x + threadIdx.x;
            U kk[2] = {0, 0}, rr[2] = {0, 0};
            if (v < vb) load_vec<W>(Sp, v, nS_total, kk, rr);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                k[j * PV + e] = kk[e];
                r[j * PV + e] = rr[e];
                valid[j * PV + e] = v < vb && t >= s0 && t < s1;
            }
        }
        if constexpr (AGG) {
            probe_tile_agg<W, IT>(av, k, r, valid, chk != 0, cnt, c0, c1);
        } else {
            probe_tile_pairs<W, IT>(pv, k, r, valid, pairs, pcap, ctr, chk != 0, c0, c1, es);
        }
    }
    flush_sums(ctr, cnt, c0, c1, AGG);
}

hj_status partition_join(hj_ctx *c, int width, int agg, const void *Rp, const uint64_t *roff, uint64_t nR_total,
                         const void *Sp, const uint64_t *soff, uint64_t nS_total, uint64_t nparts,
                         uint64_t expect_r, void *pairs, uint64_t pcap, int checksum, uint32_t *oversize) {
    if (nparts == 0) return HJ_OK;
    uint64_t slot_bytes = agg ? (width == 4 ? sizeof(AggSlot<4>) : sizeof(AggSlot<8>)) : 2ull * width;
    // Table capacity for the launch: room for a partition of the expected size
    // plus six standard deviations, at load factor 1/2; at most 160 KiB.
    double mean = (double)expect_r;
    uint64_t want = (uint64_t)(2.0 * (mean + 6.0 * __builtin_sqrt(mean + 1.0) + 64.0));
    want = ((want + 31) / 32) * 32;
    uint64_t max_slots = (160ull << 10) / slot_bytes;
    uint64_t cap_max = want < max_slots ? want : max_slots;
    if (cap_max < 64) cap_max = 64;
    size_t smem = (size_t)(cap_max * slot_bytes);
    const int block = 512;
    unsigned grid = (unsigned)nparts;
#define HJ_PJ(WW, AA)                                                                                       \
    do {                                                                                                    \
        auto kern = partition_join_kernel<WW, AA>;                                                          \
        HJ_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));     \
        HJ_LAUNCH(c, "partition_join", kern, grid, block, smem, Rp, roff, nR_total, Sp, soff, nS_total,     \
                  cap_max, pairs, pcap, c->d_ctr, oversize, checksum);                                      \
    } while (0)
    if (width == 4) {
        if (agg) HJ_PJ(4, true); else HJ_PJ(4, false);
    } else {
        if (agg) HJ_PJ(8, true); else HJ_PJ(8, false);
    }
#undef HJ_PJ
    return HJ_OK;
}

}  // namespace hj
