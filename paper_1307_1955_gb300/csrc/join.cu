// join.cu -- build and probe kernels (Alg. 1 steps b1-b4 and p1-p4).
//
//   * table_* : the simple hash join's table in global memory (SHJ), one table
//     shared by all CTAs (Sec. 3.3 prefers one shared table to one per processor).
//   * partition_join : Alg. 2's "apply SHJ on each partition pair" with the table
//     in shared memory; persistent CTAs take partition pairs from a work counter.
//
// Probing is warp-level: each warp streams its share of S in groups of 16-byte
// vectors (the next group is loaded before the current one is probed), looks
// every tuple up, and appends pairs through emit.cuh (no block barrier in the
// probe loop).  A probe key with several build matches (duplicate R keys) is
// walked by the whole warp, 32 consecutive slots at a time -- the GPU answer to
// the divergence that skew causes in steps b3/p3 (Sec. 3.3, workload divergence).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "emit.cuh"
#include "engine.cuh"

namespace hj {

// ------------------------------------------------------------------ tuple loads
// Vector v of a tuple array holds tuples v*PV .. v*PV+PV-1.  The last vector of a
// 4-byte relation with an odd number of tuples is read with one 8-byte load so
// that no read passes the array end.
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

// A warp's group: U vectors per lane, lane-interleaved (vector g + u*32 + lane).
template <int W, int U> struct Group {
    static constexpr int PV = Tup<W>::kPerVec;
    static constexpr int IT = U * PV;
    typename Tup<W>::U k[IT], r[IT];
    bool valid[IT];
    __device__ __forceinline__ void load(const void *S, uint64_t g, uint64_t lo, uint64_t hi, uint64_t vb,
                                         uint64_t n_total) {
        const unsigned lane = threadIdx.x & 31;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint64_t v = g + (uint64_t)u * 32 + lane;
            typename Tup<W>::U kk[2] = {0, 0}, rr[2] = {0, 0};
            if (v < vb) load_vec<W>(S, v, n_total, kk, rr);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                k[u * PV + e] = kk[e];
                r[u * PV + e] = rr[e];
                valid[u * PV + e] = v < vb && t >= lo && t < hi;
            }
        }
    }
};

// ----------------------------------------------------------------- table views
// Pair table: slots in shared or global memory (generic addressing).
// A key's probe run starts at its home slot, bucket_of(h, cap / group) * group:
// group 1 for the global table, a bucket of `group` slots read together for the
// shared-memory tables.  Runs continue linearly (with wrap) to the first empty slot.
template <int W> struct PairTab {
    using U = typename Tup<W>::U;
    using PS = PairSlot<W>;
    const typename PS::S *slots;
    uint64_t cap;
    unsigned long long n_allones;
    uint32_t group;

    template <class F> __device__ __forceinline__ void lookup(U k, uint64_t h, F &&f) const {
        pair_lookup<W>(slots, cap, n_allones, k, h, group, f);
    }
    // The whole warp emits every build match of probe key kk (probe rid ss).
    __device__ __forceinline__ void coop_emit(U kk, U ss, OutState &st, const OutCtx &oc) const {
        const unsigned lane = threadIdx.x & 31;
        const uint64_t b = bucket_of<W>(key_hash<W>(kk), cap / group) * group;
        for (uint64_t off = 0; off < cap; off += 32) {
            const bool inr = off + lane < cap;
            uint64_t idx = b + off + lane;
            if (idx >= cap) idx -= cap;
            typename PS::S s = inr ? slots[idx] : PS::empty();
            const unsigned emp = __ballot_sync(0xffffffffu, !inr || PS::is_empty(s));
            const unsigned before = emp ? ((emp & (0u - emp)) - 1u) : 0xffffffffu;
            const bool m = ((before >> lane) & 1u) && PS::key(s) == kk;
            warp_append<W>(st, oc, m, PS::rid(s), ss);
            if (emp) break;
        }
        if (kk == Tup<W>::kAllOnes)
            for (unsigned long long i = 0; i < n_allones; i += 32)
                warp_append<W>(st, oc, i + lane < n_allones, Tup<W>::kAllOnes, ss);
    }
};

template <int W> struct AggTab {
    using U = typename Tup<W>::U;
    const AggSlot<W> *slots;
    uint64_t cap;
    const TableSide *side;
    __device__ __forceinline__ void lookup(U k, uint64_t h, uint64_t *cnt, uint64_t *suma) const {
        agg_lookup<W>(slots, cap, side, k, h, cnt, suma);
    }
};

// Per-lane accumulators of a probing warp.
struct ProbeAcc {
    unsigned long long cnt = 0, c0 = 0, c1 = 0;
};

// Probe one group against a pair table and append its pairs.
template <int W, int U>
__device__ __forceinline__ void probe_group_pairs(const PairTab<W> &tab, const Group<W, U> &g, const PartFilter &pf,
                                                  bool chk, OutState &st, const OutCtx &oc, ProbeAcc &acc) {
    using T = typename Tup<W>::U;
    constexpr int IT = Group<W, U>::IT;
    uint32_t cnt[IT];
    T first[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        uint32_t c = 0;
        T f = 0;
        const uint64_t h = key_hash<W>(g.k[i]);
        if (g.valid[i] && pf.keep(h)) {
            const uint64_t bs = chk ? mix_b(g.r[i]) : 0;
            tab.lookup(g.k[i], h, [&](T rid) {
                if (c == 0) f = rid;
                ++c;
                if (chk) {
                    uint64_t a = mix_a(rid);
                    acc.c0 += a * bs;
                    acc.c1 += a + bs;
                }
            });
        }
        cnt[i] = c;
        first[i] = f;
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) warp_append<W>(st, oc, cnt[i] == 1, first[i], g.r[i]);
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        unsigned multi = __ballot_sync(0xffffffffu, cnt[i] > 1);
        while (multi) {
            const int L = __ffs(multi) - 1;
            multi &= multi - 1;
            T kk = __shfl_sync(0xffffffffu, g.k[i], L);
            T ss = __shfl_sync(0xffffffffu, g.r[i], L);
            tab.coop_emit(kk, ss, st, oc);
        }
    }
}

template <int W, int U>
__device__ __forceinline__ void probe_group_agg(const AggTab<W> &tab, const Group<W, U> &g, const PartFilter &pf,
                                                bool chk, ProbeAcc &acc) {
    constexpr int IT = Group<W, U>::IT;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const uint64_t h = key_hash<W>(g.k[i]);
        if (!g.valid[i] || !pf.keep(h)) continue;
        uint64_t n, sa;
        tab.lookup(g.k[i], h, &n, &sa);
        acc.cnt += n;
        if (chk && n) {
            const uint64_t b = mix_b(g.r[i]);
            acc.c0 += sa * b;
            acc.c1 += sa + n * b;
        }
    }
}

// Stream S rows [lo, hi) through one warp: groups g = g0, g0 + gstride, ...
template <int W, int U, bool AGG, class Tab>
__device__ __forceinline__ void warp_probe(const Tab &tab, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                                           uint64_t g0, uint64_t gstride, const PartFilter &pf, bool chk,
                                           OutState &st, const OutCtx &oc, ProbeAcc &acc) {
    constexpr int PV = Tup<W>::kPerVec;
    const uint64_t vb = (hi + PV - 1) / PV;
    if (g0 >= vb) return;
    Group<W, U> cur, nxt;
    cur.load(S, g0, lo, hi, vb, n_total);
    for (uint64_t g = g0; g < vb; g += gstride) {
        const uint64_t gn = g + gstride;
        if (gn < vb) nxt.load(S, gn, lo, hi, vb, n_total);
        if constexpr (AGG) probe_group_agg<W, U>(tab, cur, pf, chk, acc);
        else probe_group_pairs<W, U>(tab, cur, pf, chk, st, oc, acc);
        cur = nxt;
    }
}

__device__ __forceinline__ void flush_acc(hj_counters *ctr, ProbeAcc acc, bool with_cnt) {
    acc.cnt = warp_sum(acc.cnt);
    acc.c0 = warp_sum(acc.c0);
    acc.c1 = warp_sum(acc.c1);
    if ((threadIdx.x & 31) == 0) {
        if (with_cnt && acc.cnt) atomicAdd(&ctr->count, acc.cnt);
        if (acc.c0) atomicAdd(&ctr->c0, acc.c0);
        if (acc.c1) atomicAdd(&ctr->c1, acc.c1);
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
                                                          hj_counters *ctr, PartFilter pf) {
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
            if (!pf.keep(h)) continue;
            bool ok = AGG ? agg_insert<W>((AggSlot<W> *)slots, cap, side, k[e], mix_a(r[e]), h)
                          : pair_insert<W>((typename PairSlot<W>::S *)slots, cap, side, k[e], r[e], h);
            if (!ok) atomicOr(&ctr->status, (unsigned long long)(AGG || cap <= kMaxPairWalk ? kStatusTableFull
                                                                                         : kStatusLongRun));
        }
    }
}

// Vectors per lane per probe group.
template <int W> struct ProbeU {
    static constexpr int value = 2;
};

// Pairs per warp in the probe's shared-memory staging buffer (exact output mode).
constexpr unsigned kProbeStage = 256;

template <int W, bool AGG>
__global__ void __launch_bounds__(256) table_probe_kernel(const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                                                          const void *slots, uint64_t cap, const TableSide *side,
                                                          void *pairs, uint64_t pcap, RecArea ra, hj_counters *ctr,
                                                          int chk, PartFilter pf, int dense) {
    constexpr int PV = Tup<W>::kPerVec, U = ProbeU<W>::value;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t va = lo / PV;
    OutState st;
    OutCtx oc{pairs, pcap, ctr, 0u, dense == 1};
    extern __shared__ __align__(16) unsigned char tp_stage[];
    if (dense == 2) {  // this warp's staging buffer
        oc.stage = tp_stage + (size_t)(threadIdx.x >> 5) * kProbeStage * 2 * W;
        oc.scap = kProbeStage;
        st.used = 0;
    }
    ProbeAcc acc;
    if constexpr (AGG) {
        AggTab<W> tab{(const AggSlot<W> *)slots, cap, side};
        warp_probe<W, U, true>(tab, S, lo, hi, n_total, va + (uint64_t)warp * 32 * U, (uint64_t)nwarps * 32 * U,
                               pf, chk != 0, st, oc, acc);
    } else {
        PairTab<W> tab{(const typename PairSlot<W>::S *)slots, cap, side->n_allones, 1u};
        warp_probe<W, U, false>(tab, S, lo, hi, n_total, va + (uint64_t)warp * 32 * U, (uint64_t)nwarps * 32 * U,
                                pf, chk != 0, st, oc, acc);
        if (oc.stage) warp_stage_flush<W>(st, oc);
        warp_finish(st, oc, ra);
    }
    flush_acc(ctr, acc, AGG);
}

hj_status table_create(hj_ctx *c, int width, int agg, uint64_t n_build, hj_table **out) {
    *out = nullptr;
    // Capacity: a power of two at least twice the build size (load factor <= 0.5).
    uint64_t cap = 64;
    while (cap < 2 * n_build + 1) cap <<= 1;
    uint64_t slot_bytes = agg ? (width == 4 ? sizeof(AggSlot<4>) : sizeof(AggSlot<8>)) : 2ull * width;
    DevBuf slots(c), side(c);
    HJ_TRY(slots.alloc(cap * slot_bytes));
    HJ_TRY(side.alloc(sizeof(TableSide)));
    HJ_CUDA(c, cudaMemsetAsync(side.p, 0, sizeof(TableSide), c->stream));
    int grid = num_sms(c) * 4;
    if (!agg) {
        HJ_CUDA(c, cudaMemsetAsync(slots.p, 0xFF, cap * slot_bytes, c->stream));
    } else if (width == 4) {
        HJ_LAUNCH(c, "agg_table_init", agg_table_init<4>, grid, 256, 0, slots.as<AggSlot<4>>(), cap);
    } else {
        HJ_LAUNCH(c, "agg_table_init", agg_table_init<8>, grid, 256, 0, slots.as<AggSlot<8>>(), cap);
    }
    hj_table *t = new hj_table();
    t->width = width;
    t->agg = agg;
    t->cap = cap;
    t->slots = slots.release();
    t->side = side.release();
    *out = t;
    return HJ_OK;
}

void table_destroy(hj_ctx *c, hj_table *t) {
    if (!t) return;
    dfree(c, t->slots);
    dfree(c, t->side);
    dfree(c, t->rids);
    delete t;
}

hj_status table_build(hj_ctx *c, hj_table *t, const void *R, uint64_t lo, uint64_t hi, uint64_t n_total,
                      PartFilter pf) {
    if (hi <= lo) return HJ_OK;
    uint64_t nvec = (hi - lo) / (t->width == 4 ? 2 : 1) + 2;
    uint64_t want = (nvec + 255) / 256;
    int grid = (int)(want < (uint64_t)num_sms(c) * 8 ? (want ? want : 1) : (uint64_t)num_sms(c) * 8);
    TableSide *side = (TableSide *)t->side;
#define HJ_TB(WW, AA) HJ_LAUNCH(c, "table_build", (table_build_kernel<WW, AA>), grid, 256, 0, R, lo, hi, n_total, t->slots, t->cap, side, c->d_ctr, pf)
    if (t->width == 4) {
        if (t->agg) HJ_TB(4, true); else HJ_TB(4, false);
    } else {
        if (t->agg) HJ_TB(8, true); else HJ_TB(8, false);
    }
#undef HJ_TB
    return HJ_OK;
}

uint64_t table_probe_warps(hj_ctx *c, uint64_t n) {
    const uint64_t per_cta_tuples = 8 * 32 * 8;  // 8 warps, 32 lanes, 8 tuples per lane group
    uint64_t want = (n + per_cta_tuples - 1) / per_cta_tuples;
    uint64_t maxg = (uint64_t)num_sms(c) * 8;
    uint64_t grid = want < maxg ? (want ? want : 1) : maxg;
    return grid * 8;
}

hj_status table_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                      void *pairs, uint64_t pcap, int checksum, RecArea ra, PartFilter pf, hj_counters *ctr, int dense) {
    if (hi <= lo) return HJ_OK;
    if (!ctr) ctr = c->d_ctr;
    const unsigned grid = (unsigned)(table_probe_warps(c, hi - lo) / 8);
    const TableSide *side = (const TableSide *)t->side;
    const size_t smem = dense == 2 && !t->agg ? (size_t)8 * kProbeStage * 2 * t->width : 0;
#define HJ_TP(WW, AA) HJ_LAUNCH(c, "table_probe", (table_probe_kernel<WW, AA>), grid, 256, smem, S, lo, hi, n_total, t->slots, t->cap, side, pairs, pcap, ra, ctr, checksum, pf, dense)
    if (t->width == 4) {
        if (t->agg) HJ_TP(4, true); else HJ_TP(4, false);
    } else {
        if (t->agg) HJ_TP(8, true); else HJ_TP(8, false);
    }
#undef HJ_TP
    return HJ_OK;
}

// ================================================== per-partition join (PHJ)
//
// Persistent CTAs take partition tasks (R_p with a slice of S_p) from ctr->work.
// For each, the CTA builds a table over R_p in shared memory (about three slots
// per build row, multiply-shift buckets so any capacity works), then its warps
// stream the S slice.  Partitions come from the padded partitioner: every
// partition starts and ends on a 32-byte sector, so whole 16-byte vectors can be
// loaded without bounds checks on tuples, and padding tuples (keys of another
// partition) match nothing.  A partition whose table cannot fit (|R_p| too large
// for a pair table, more distinct keys than slots for an aggregate table, or an
// insert walking past kMaxSmemWalk buckets: a heavily repeated key) goes to the
// host's fallback list, joined there with a global key-list table (pairs) or
// aggregate table (counts).

template <int W> struct HashT { using type = uint32_t; };
template <> struct HashT<8> { using type = uint64_t; };

// Bucket of a key inside a partition's shared-memory table: Fibonacci
// multiply-shift of the key.  Keys of one partition already share their
// MurmurHash2 partition digit, so a cheap hash that spreads them is enough here.
template <int W> __device__ __forceinline__ uint32_t part_bucket(typename Tup<W>::U k, uint32_t nb);
template <> __device__ __forceinline__ uint32_t part_bucket<4>(uint32_t k, uint32_t nb) {
    return __umulhi(k * 0x9E3779B1u, nb);
}
template <> __device__ __forceinline__ uint32_t part_bucket<8>(uint64_t k, uint32_t nb) {
    return __umulhi((uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 32), nb);
}

// Bucket hash of a partition's shared-memory aggregate table (the value that
// bucket_of<W> scales to the table): a Fibonacci multiply of the key, for the same
// reason as part_bucket.
template <int W> __device__ __forceinline__ uint64_t part_agg_hash(typename Tup<W>::U k);
template <> __device__ __forceinline__ uint64_t part_agg_hash<4>(uint32_t k) { return (uint32_t)(k * 0x9E3779B1u); }
template <> __device__ __forceinline__ uint64_t part_agg_hash<8>(uint64_t k) { return k * 0x9E3779B97F4A7C15ull; }

template <int W>
__device__ __forceinline__ typename HashT<W>::type hashw(typename Tup<W>::U k) {
    if constexpr (W == 4) return murmur2_u32(k);
    else return murmur2_u64(k);
}

// ----------------------------------------------------------- shared-memory table
// Bucketised open addressing in shared memory for one partition pair.  Bucket b is
// G slots (G = 4 for 4-byte tuples, 2 for 8-byte): its G keys are 16 bytes of the
// key region and its G rids 16 bytes of the rid region (separate regions, so that
// the key loads of random buckets spread over all shared-memory banks).
// Every real key of partition p hashes to p, so a key that hashes to another
// partition can never be stored or probed: it marks empty slots (no value of the
// key domain needs reserving).  A key's run starts at its home bucket and moves
// linearly over buckets; a bucket's overflow bit records that some insert moved
// past it, so a lookup stops at the first bucket that has an empty slot or no
// overflow bit.
template <int W> struct SoaTab {
    using T = typename Tup<W>::U;
    static constexpr uint32_t G = 16 / W;
    uint32_t nb;     // buckets
    T empty;
    const uint32_t *ovf;

    __device__ __forceinline__ bool overflowed(uint32_t b) const { return (ovf[b >> 5] >> (b & 31)) & 1u; }
    // keys (half 0) or rids (half 1) of bucket b.  Plain loads through the
    // shared-memory pointers: the compiler orders them with the barriers and may
    // overlap the independent lookups of a thread's items.
    const T *kptr;   // key region: G keys (16 bytes) per bucket
    const T *rptr;   // rid region, same shape
    __device__ __forceinline__ void ld(uint32_t b, uint32_t half, T *v) const {
        const T *p = (half ? rptr : kptr) + b * G;
        if constexpr (W == 4) {
            const uint4 x = *(const uint4 *)p;
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else {
            const ulonglong2 x = *(const ulonglong2 *)p;
            v[0] = x.x; v[1] = x.y;
        }
    }
    __device__ __forceinline__ T ld1(uint32_t b, uint32_t half, uint32_t q) const {
        return (half ? rptr : kptr)[b * G + q];
    }
};

// Lookup of key k: number of build matches and the rid of the first one.
template <int W>
__device__ __forceinline__ uint32_t soa_lookup(const SoaTab<W> &t, typename Tup<W>::U k, uint32_t home,
                                               typename Tup<W>::U *first) {
    using T = typename Tup<W>::U;
    constexpr uint32_t G = SoaTab<W>::G;
    uint32_t c = 0, bkt = home;
    for (uint32_t it = 0; it < t.nb; ++it) {
        T key[G];
        t.ld(bkt, 0, key);
        uint32_t m = 0;
        bool e = false;
#pragma unroll
        for (uint32_t q = 0; q < G; ++q) {
            m |= (uint32_t)(key[q] == k) << q;
            e |= key[q] == t.empty;
        }
        if (m) {
            T rid[G];
            t.ld(bkt, 1, rid);
            if (c == 0) {
                T f = rid[G - 1];
#pragma unroll
                for (int q = (int)G - 2; q >= 0; --q)
                    if ((m >> q) & 1u) f = rid[q];
                *first = f;
            }
            c += __popc(m);
        }
        if (e || !t.overflowed(bkt)) break;
        bkt = bkt + 1 == t.nb ? 0 : bkt + 1;
    }
    return c;
}

// Visit every build rid of key k (slow path for checksums).
template <int W, class F>
__device__ __forceinline__ void soa_visit(const SoaTab<W> &t, typename Tup<W>::U k, uint32_t home, F &&f) {
    using T = typename Tup<W>::U;
    constexpr uint32_t G = SoaTab<W>::G;
    uint32_t bkt = home;
    for (uint32_t it = 0; it < t.nb; ++it) {
        T key[G], rid[G];
        t.ld(bkt, 0, key);
        t.ld(bkt, 1, rid);
        bool e = false;
#pragma unroll
        for (uint32_t q = 0; q < G; ++q) {
            if (key[q] == k) f(rid[q]);
            e |= key[q] == t.empty;
        }
        if (e || !t.overflowed(bkt)) break;
        bkt = bkt + 1 == t.nb ? 0 : bkt + 1;
    }
}

// The whole warp emits every build match of key kk (probe rid ss): a window of
// 32 slots (32 / G buckets) per step, up to the first bucket that ends the run.
template <int W, class Sink>
__device__ __forceinline__ void soa_coop_emit(const SoaTab<W> &t, typename Tup<W>::U kk, typename Tup<W>::U ss,
                                              uint32_t home, Sink &sink) {
    using T = typename Tup<W>::U;
    constexpr uint32_t G = SoaTab<W>::G, BPW = 32 / G;
    const unsigned lane = threadIdx.x & 31, jb = lane / G, q = lane % G;
    for (uint32_t off = 0; off < t.nb; off += BPW) {
        const bool inr = off + jb < t.nb;
        uint32_t b = home + off + jb;
        if (b >= t.nb) b -= t.nb;
        const T key = inr ? t.ld1(b, 0, q) : t.empty;
        const T rid = inr ? t.ld1(b, 1, q) : T(0);
        const unsigned emp = __ballot_sync(0xffffffffu, key == t.empty);
        const bool bucket_empty_slot = ((emp >> (jb * G)) & ((1u << G) - 1u)) != 0;
        const bool bucket_end = !inr || bucket_empty_slot || !t.overflowed(b);
        const unsigned endm = __ballot_sync(0xffffffffu, bucket_end && q == 0);
        const unsigned last_lane = endm ? (unsigned)(__ffs(endm) - 1) + G - 1 : 31u;
        const bool m = inr && lane <= last_lane && key == kk;
        sink.append(m, rid, ss);
        if (endm) break;
    }
}

// ------------------------------------------------------------------ output sinks
// How a CTA's warps place the pairs of its partition tasks.
//
// ChunkSink: every warp takes whole chunks of the join's pair buffer (emit.cuh);
// partly used chunks are recorded and compacted on the device afterwards.  Used
// for a single join: no extra traffic, a small fix-up at the end.
//
// WarpStageSink (below): every warp stages its pairs in a private buffer and
// claims exact rows of the join's buffer per buffer-full.  Used for batches of
// joins, where per-warp chunks would leave a partly used chunk per warp per join.
// The join's pair count is the claim cursor (ctr->count).
template <int W> struct ChunkSink {
    using T = typename Tup<W>::U;
    OutState st;
    OutCtx oc;
    unsigned join = ~0u;
    const JoinSlot *slots;
    RecArea ra;
    __device__ __forceinline__ void begin_task(unsigned j) {
        if (j == join) return;
        if (join != ~0u) warp_finish(st, oc, ra);
        st = OutState();
        oc = OutCtx{slots[j].pairs, slots[j].pcap, slots[j].ctr, j, false};
        join = j;
    }
    __device__ __forceinline__ void append(bool has, T a, T b) { warp_append<W>(st, oc, has, a, b); }
    // one append for all single-match items of a group
    template <int IT>
    __device__ __forceinline__ void append_group(const uint32_t *cnt, const T *first, const T *r) {
        const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
        unsigned m[IT], tot = 0;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            m[i] = __ballot_sync(0xffffffffu, cnt[i] == 1);
            tot += __popc(m[i]);
        }
        if (!tot) return;
        const unsigned room = kChunkPairs - st.used;
        unsigned long long nbase = 0;
        if (tot > room) {
            if (lane == 0) nbase = atomicAdd(&oc.ctr->cursor, (unsigned long long)kChunkPairs);
            nbase = __shfl_sync(0xffffffffu, nbase, 0);
        }
        unsigned run = 0;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            if (cnt[i] == 1) {
                const unsigned rank = run + __popc(m[i] & lt);
                const unsigned long long pos = rank < room ? st.base + st.used + rank : nbase + (rank - room);
                if (pos < oc.pcap) PairOut<W>::put(oc.pairs, pos, first[i], r[i]);
            }
            run += __popc(m[i]);
        }
        if (tot > room) {
            st.base = nbase;
            st.used = tot - room;
            st.claimed = true;
        } else {
            st.used += tot;
        }
        st.pairs += tot;
    }
    // one append for all single-match items of a group (at most 32 * IT pairs, so
    // at most one new chunk): item-major positions, so that each store instruction
    // writes consecutive slots; capacity tested once per group
    template <int IT>
    __device__ __forceinline__ void append_runs(const uint32_t *cnt, const T *first, const T *r) {
        const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
        unsigned m[IT], tot = 0;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            m[i] = __ballot_sync(0xffffffffu, cnt[i] == 1);
            tot += __popc(m[i]);
        }
        if (!tot) return;
        const unsigned room = kChunkPairs - st.used;
        unsigned long long nb = 0;
        if (tot > room) {
            if (lane == 0) nb = atomicAdd(&oc.ctr->cursor, (unsigned long long)kChunkPairs);
            nb = __shfl_sync(0xffffffffu, nb, 0);
        }
        const unsigned long long c0 = st.base + st.used;
        const bool safe = c0 + (tot < room ? tot : room) <= oc.pcap && (tot <= room || nb + (tot - room) <= oc.pcap);
        unsigned run = 0;
        if (safe) {  // (warp-uniform) every position is inside the buffer
            // pair idx of the group goes to c0 + idx in the open chunk, else to
            // nb + (idx - room) in the new one: one base address per item (the
            // second base is only used for idx >= room, so its wrap is harmless)
            using P = typename std::conditional<W == 4, uint2, ulonglong2>::type;
            const uint64_t a0 = (uint64_t)oc.pairs + c0 * sizeof(P);
            const uint64_t a1 = (uint64_t)oc.pairs + (nb - room) * sizeof(P);
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const unsigned idx = run + __popc(m[i] & lt);
                P *dst = (P *)((idx < room ? a0 : a1) + (uint64_t)idx * sizeof(P));
                if (cnt[i] == 1) {
                    if constexpr (W == 4) *dst = make_uint2(first[i], r[i]);
                    else *dst = make_ulonglong2(first[i], r[i]);
                }
                run += __popc(m[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const unsigned idx = run + __popc(m[i] & lt);
                const unsigned long long pos = idx < room ? c0 + idx : nb + (idx - room);
                if (cnt[i] == 1 && pos < oc.pcap) PairOut<W>::put(oc.pairs, pos, first[i], r[i]);
                run += __popc(m[i]);
            }
        }
        if (tot > room) {
            st.base = nb;
            st.used = tot - room;
            st.claimed = true;
        } else {
            st.used += tot;
        }
        st.pairs += tot;
    }
    __device__ __forceinline__ hj_counters *ctr() const { return oc.ctr; }
    __device__ __forceinline__ void end_task() {}
    __device__ __forceinline__ void finish() {
        if (join != ~0u) warp_finish(st, oc, ra);
    }
};

// Per-warp staged exact output (batches of joins, whose many joins per launch
// would leave a partly filled chunk per warp and join): each warp collects its
// pairs in a private buffer of scap pairs in global memory (a few KB per warp,
// L2-resident) and, when the buffer fills or the warp moves on to another join,
// claims exactly that many rows of the join's buffer with one atomic add and
// copies them out with coalesced stores.  Output is dense as written (no
// compaction) and the sink needs no CTA barrier.  scap >= 32 x the items of a
// group, so one flush always makes room.
template <int W> struct WarpStageSink {
    using T = typename Tup<W>::U;
    using P = typename std::conditional<W == 4, uint2, ulonglong2>::type;
    P *stage = nullptr;  // this warp's buffer
    uint32_t scap = 0;
    const JoinSlot *slots = nullptr;
    unsigned join = ~0u;
    uint32_t used = 0;  // warp-uniform
    __device__ __forceinline__ static P mk(T a, T b) {
        if constexpr (W == 4) return make_uint2(a, b);
        else return make_ulonglong2(a, b);
    }
    // all 32 lanes: the staged pairs to exact rows of the join's buffer (pairs past
    // its capacity are dropped; the count stays exact)
    __device__ __forceinline__ void flush() {
        if (!used) return;
        __syncwarp();  // the buffer's stores are visible to every lane
        const unsigned lane = threadIdx.x & 31;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&slots[join].ctr->count, (unsigned long long)used);
        b = __shfl_sync(0xffffffffu, b, 0);
        P *out = (P *)slots[join].pairs;
        const unsigned long long pc = slots[join].pcap;
        for (uint32_t i = lane; i < used; i += 32)
            if (b + i < pc) out[b + i] = stage[i];
        __syncwarp();  // read before the buffer is refilled
        used = 0;
    }
    __device__ __forceinline__ void begin_task(unsigned j) {
        if (j == join) return;
        flush();
        join = j;
    }
    __device__ __forceinline__ void append(bool has, T a, T b) {
        const unsigned mask = __ballot_sync(0xffffffffu, has);
        if (!mask) return;
        const unsigned lane = threadIdx.x & 31, k = __popc(mask), rank = __popc(mask & ((1u << lane) - 1u));
        if (used + k > scap) flush();
        if (has) stage[used + rank] = mk(a, b);
        used += k;
    }
    template <int IT>
    __device__ __forceinline__ void append_group(const uint32_t *cnt, const T *first, const T *r) {
        const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
        unsigned m[IT], tot = 0;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            m[i] = __ballot_sync(0xffffffffu, cnt[i] == 1);
            tot += __popc(m[i]);
        }
        if (!tot) return;
        if (used + tot > scap) flush();
        unsigned run = used;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            if (cnt[i] == 1) stage[run + __popc(m[i] & lt)] = mk(first[i], r[i]);
            run += __popc(m[i]);
        }
        used += tot;
    }
    template <int IT>
    __device__ __forceinline__ void append_runs(const uint32_t *cnt, const T *first, const T *r) {
        append_group<IT>(cnt, first, r);
    }
    __device__ __forceinline__ hj_counters *ctr() const { return slots[join].ctr; }
    __device__ __forceinline__ void end_task() {}
    __device__ __forceinline__ void finish() { flush(); }
};

// One group of IT probe items against the table, in phases so that the items'
// shared-memory loads overlap: every item's home bucket (keys), then the match
// masks and the first match's rid (one indexed load).  cnt[i] and first[i] cover
// the home bucket only.  Inserts fill a bucket's slots in order and slots never
// empty again, and an insert moves past a bucket only while it is full, so a run
// goes on past the home bucket only if the bucket's last slot is taken AND its
// overflow bit is set: bit i of the returned mask marks such an item (with at
// most one home match; an item with several takes the whole-run walk instead).
// Items with live[i] false match nothing.
template <int W, int IT>
__device__ __forceinline__ uint32_t probe_items(const SoaTab<W> &tab, const typename Tup<W>::U *k, const bool *live,
                                                uint32_t *cnt, typename Tup<W>::U *first) {
    using T = typename Tup<W>::U;
    constexpr uint32_t G = SoaTab<W>::G;
    uint32_t home[IT];
    T kb[IT][G];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        home[i] = part_bucket<W>(k[i], tab.nb);  // < nb for any key: the load is in bounds
        tab.ld(home[i], 0, kb[i]);
    }
    uint32_t walk = 0;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        uint32_t m = 0;
#pragma unroll
        for (uint32_t q = 0; q < G; ++q) m |= (uint32_t)(kb[i][q] == k[i]) << q;
        if (!live[i]) m = 0;
        // the first match's rid, read without a branch (slot G - 1 when nothing matched)
        const T fr = tab.ld1(home[i], 1, (uint32_t)(__ffs(m | (1u << (G - 1))) - 1));
        first[i] = m ? fr : T(0);
        cnt[i] = __popc(m);
        walk |= (uint32_t)(live[i] && cnt[i] <= 1 && kb[i][G - 1] != tab.empty && tab.overflowed(home[i])) << i;
    }
    return walk;
}

// Longest walk (in buckets) of an insert into a partition's shared-memory table.
constexpr uint32_t kMaxSmemWalk = 64;

// Entries per warp of the queue of pending run walks (probe keys and rids whose
// run goes on past a full home bucket).
constexpr uint32_t kWalkQ = 64;

// Shared-memory layout of the join kernel: table slots (cap_max x slot bytes),
// the overflow bitmap, then each warp's walk queue (kWalkQ keys, kWalkQ rids).
__host__ __device__ constexpr uint32_t walkq_offset(uint32_t cap_max, uint32_t slot_bytes) {
    return (cap_max * slot_bytes + (cap_max / 2 / 32 + 1) * 4 + 16 + 15) / 16 * 16;
}

// The walks of n <= 32 queued items, one per lane: each lane follows its key's run
// from the bucket after its home and emits every match found there.  A walk is
// rare (a few per cent of probes), so walking them one lane at a time as they
// come would cost a whole warp pass each; batched, 32 walks cost about one.
template <int W, class Sink>
__device__ __forceinline__ void drain_walks(const SoaTab<W> &tab, const typename Tup<W>::U *qk,
                                            const typename Tup<W>::U *qr, uint32_t n, Sink &sink) {
    using T = typename Tup<W>::U;
    constexpr uint32_t G = SoaTab<W>::G;
    const unsigned lane = threadIdx.x & 31;
    bool active = lane < n;
    const T kk = active ? qk[lane] : tab.empty;
    const T rr = active ? qr[lane] : T(0);
    __syncwarp();  // entries read before the queue is refilled
    uint32_t b = 0;
    if (active) {
        const uint32_t h = part_bucket<W>(kk, tab.nb);
        b = h + 1 == tab.nb ? 0 : h + 1;
    }
    for (uint32_t it = 0; it < tab.nb; ++it) {
        if (!__any_sync(0xffffffffu, active)) break;
        uint32_t m = 0;
        bool e = false;
        if (active) {
            T key[G];
            tab.ld(b, 0, key);
#pragma unroll
            for (uint32_t q = 0; q < G; ++q) {
                m |= (uint32_t)(key[q] == kk) << q;
                e |= key[q] == tab.empty;
            }
        }
        // the matches of this bucket, one append per round (several only for
        // duplicate build keys)
        for (uint32_t q = 0; q < G; ++q) {
            const bool hm = m != 0;
            if (!__any_sync(0xffffffffu, hm)) break;
            T v = 0;
            if (hm) {
                v = tab.ld1(b, 1, (uint32_t)(__ffs(m) - 1));
                m &= m - 1;
            }
            sink.append(hm, v, rr);
        }
        active = active && !e && tab.overflowed(b);
        b = b + 1 == tab.nb ? 0 : b + 1;
    }
}

template <int W, int U, class Sink>
__device__ __forceinline__ void probe_fast(const SoaTab<W> &tab, const typename Tup<W>::Vec *Sv, uint32_t nsv,
                                           Sink &sink, unsigned warp, unsigned nwarps, unsigned lane,
                                           typename Tup<W>::U *wqk, typename Tup<W>::U *wqr) {
    using T = typename Tup<W>::U;
    using Vec = typename Tup<W>::Vec;
    constexpr int PV = Tup<W>::kPerVec, IT = U * PV;
    // runs that go on past a full home bucket are queued and walked 32 at a time
    constexpr bool kQueue = true;
    const uint32_t gstride = nwarps * 32u * U;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t g = warp * 32u * U;
    uint32_t qn = 0;  // queued walks (warp-uniform)
    Vec cur[U], nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t rel = g + u * 32u + lane;
        if (rel < nsv) cur[u] = ld_stream(Sv + rel);
    }
    for (; g < nsv; g += gstride) {
        const uint32_t gn = g + gstride;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t rel = gn + u * 32u + lane;
            if (rel < nsv) nxt[u] = ld_stream(Sv + rel);
        }
        T k[IT], r[IT];
        bool live[IT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = g + (uint32_t)u * 32u + lane < nsv;
            if constexpr (W == 4) {
                k[2 * u] = cur[u].x; r[2 * u] = cur[u].y; k[2 * u + 1] = cur[u].z; r[2 * u + 1] = cur[u].w;
                live[2 * u] = in;
                live[2 * u + 1] = in;
            } else {
                k[u] = cur[u].x; r[u] = cur[u].y;
                live[u] = in;
            }
        }
        uint32_t cnt[IT];
        T first[IT];
        const uint32_t walk = probe_items<W, IT>(tab, k, live, cnt, first);
        if constexpr (!kQueue) {
            // walked at once: the run's further matches join the item's count (and
            // an item with several then takes the whole-run walk below)
            if (walk) {
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    if (!((walk >> i) & 1u)) continue;
                    const uint32_t h = part_bucket<W>(k[i], tab.nb);
                    T f2 = 0;
                    const uint32_t c2 = soa_lookup<W>(tab, k[i], h + 1 == tab.nb ? 0 : h + 1, &f2);
                    if (cnt[i] == 0) first[i] = f2;
                    cnt[i] += c2;
                }
            }
        }
        sink.template append_runs<IT>(cnt, first, r);
        // several home matches (duplicate build keys): the whole warp walks each such run
        bool multi_any = false;
#pragma unroll
        for (int i = 0; i < IT; ++i) multi_any |= cnt[i] > 1;
        if (__any_sync(0xffffffffu, multi_any)) {
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                unsigned multi = __ballot_sync(0xffffffffu, cnt[i] > 1);
                while (multi) {
                    const int L = __ffs(multi) - 1;
                    multi &= multi - 1;
                    const T kk = __shfl_sync(0xffffffffu, k[i], L);
                    const T ss = __shfl_sync(0xffffffffu, r[i], L);
                    soa_coop_emit<W>(tab, kk, ss, part_bucket<W>(kk, tab.nb), sink);
                }
            }
        }
        // runs that go on past the home bucket: queued, walked 32 at a time
        if (kQueue && __any_sync(0xffffffffu, walk != 0)) {
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                const bool w = (walk >> i) & 1u;
                const unsigned wm = __ballot_sync(0xffffffffu, w);
                if (!wm) continue;
                if (w) {
                    const uint32_t pos = qn + (uint32_t)__popc(wm & lt);
                    wqk[pos] = k[i];
                    wqr[pos] = r[i];
                }
                qn += (uint32_t)__popc(wm);
                if (qn >= 32) {
                    __syncwarp();
                    drain_walks<W>(tab, wqk + (qn - 32), wqr + (qn - 32), 32, sink);
                    qn -= 32;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
    if (kQueue && qn) {
        __syncwarp();
        drain_walks<W>(tab, wqk, wqr, qn, sink);
    }
}

// Bytes per slot of a partition's shared-memory aggregate table: the key, the
// number of build tuples with that key and, with checksums, the sum of A(rid) over
// them.
__host__ __device__ constexpr uint32_t agg_slot_bytes(int width, int chk) {
    return (uint32_t)width + 4u + (chk ? 8u : 0u);
}

// Aggregate table of one partition in shared memory (Sec. 3.1's key list with each
// rid list folded into a count and a sum): the bucket layout of SoaTab -- G keys
// per 16-byte bucket, a key that hashes to another partition as the empty marker,
// runs that move linearly over buckets with overflow bits -- but one slot per
// distinct key, so a lookup finds at most one slot.  Regions: keys (cap x W
// bytes), sums (cap x 8, with checksums only), counts (cap x 4).
template <int W> struct AggSoa {
    using T = typename Tup<W>::U;
    static constexpr uint32_t G = 16 / W;
    uint32_t nb;
    T empty;
    uint32_t *ovf;
    T *keys;
    unsigned long long *suma;  // null without checksums
    uint32_t *cnt;

    __device__ static AggSoa at(unsigned char *base, uint32_t cap, T empty, uint32_t *ovf, bool chk) {
        AggSoa t;
        t.nb = cap / G;
        t.empty = empty;
        t.ovf = ovf;
        t.keys = (T *)base;
        t.suma = chk ? (unsigned long long *)(base + (size_t)cap * W) : nullptr;
        t.cnt = (uint32_t *)(base + (size_t)cap * (W + (chk ? 8 : 0)));
        return t;
    }
    __device__ __forceinline__ bool overflowed(uint32_t b) const { return (ovf[b >> 5] >> (b & 31)) & 1u; }
    __device__ __forceinline__ void ld(uint32_t b, T *v) const {
        if constexpr (W == 4) {
            const uint4 x = *(const uint4 *)(keys + b * G);
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        } else {
            const ulonglong2 x = *(const ulonglong2 *)(keys + b * G);
            v[0] = x.x; v[1] = x.y;
        }
    }
    // Add m build tuples of key k (a = the sum of their A(rid), used with
    // checksums).  The slot of k is the first slot of its run that holds k, else
    // the first empty one, claimed by CAS: slots only ever go from empty to a key,
    // so two inserts of the same key always meet in one slot.  False if every
    // bucket is full.
    __device__ __forceinline__ bool insert(T k, uint32_t m, uint64_t a) const {
        uint32_t b = part_bucket<W>(k, nb);
        for (uint32_t it = 0; it < nb; ++it) {
            volatile T *kb = keys + b * G;
            // each failed CAS follows one more slot of the bucket being filled
            for (uint32_t tries = 0; tries <= G; ++tries) {
                int hit = -1, emp = -1;
#pragma unroll
                for (uint32_t q = 0; q < G; ++q) {
                    const T x = kb[q];
                    if (x == k && hit < 0) hit = (int)q;
                    if (x == empty && emp < 0) emp = (int)q;
                }
                if (hit < 0 && emp >= 0) {
                    const T old = cas_key<W>(keys + b * G + emp, empty, k);
                    if (old != empty && old != k) continue;
                    hit = emp;
                }
                if (hit < 0) break;  // full bucket without k
                atomicAdd(&cnt[b * G + hit], m);
                if (suma) atomicAdd(&suma[b * G + hit], (unsigned long long)a);
                return true;
            }
            atomicOr(&ovf[b >> 5], 1u << (b & 31));
            b = b + 1 == nb ? 0 : b + 1;
        }
        return false;
    }
    // Slot of key k from bucket b on (the run's continuation), or ~0u.
    __device__ __forceinline__ uint32_t find_from(T k, uint32_t b) const {
        for (uint32_t it = 0; it < nb; ++it) {
            T key[G];
            ld(b, key);
            uint32_t m = 0;
            bool e = false;
#pragma unroll
            for (uint32_t q = 0; q < G; ++q) {
                m |= (uint32_t)(key[q] == k) << q;
                e |= key[q] == empty;
            }
            if (m) return b * G + (uint32_t)(__ffs(m) - 1);
            if (e || !overflowed(b)) return ~0u;
            b = b + 1 == nb ? 0 : b + 1;
        }
        return ~0u;
    }
};

template <int W, bool AGG, int NT, class Sink, bool FAST>
__global__ void __launch_bounds__(NT, 2048 / NT / 2) partition_join_kernel(
    const PartTask *tasks, uint64_t ntasks, const JoinSlot *slots, hj_counters *work, uint32_t cap_max, RecArea ra,
    uint32_t *oversize, int chk, void *stage_base, uint32_t scap) {
    using T = typename Tup<W>::U;
    using Vec = typename Tup<W>::Vec;
    constexpr int PV = Tup<W>::kPerVec, U = 2, IT = U * PV;
    constexpr uint32_t G = SoaTab<W>::G;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TableSide side;
    __shared__ int s_full;
    __shared__ unsigned long long s_p;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    Sink sink;
    if constexpr (std::is_same<Sink, ChunkSink<W>>::value) {
        sink.slots = slots;
        sink.ra = ra;
    } else {
        sink.stage = (typename WarpStageSink<W>::P *)stage_base + ((size_t)blockIdx.x * nwarps + warp) * scap;
        sink.scap = scap;
        sink.slots = slots;
    }
    for (;;) {
        if (threadIdx.x == 0) s_p = atomicAdd(&work->work, 1ull);
        __syncthreads();
        const uint64_t ti = s_p;
        if (ti >= ntasks) break;
        const PartTask tk = tasks[ti];
        const uint32_t nrv = tk.nr / PV, nsv = tk.ns / PV;
        const Vec *Rv = (const Vec *)tk.R;
        const Vec *Sv = (const Vec *)tk.S;
        const uint64_t nr = tk.nr;  // build rows, padding included
        const PartFilter pf{tk.p, (int)tk.b1, (int)tk.b2, 1};
        hj_counters *jc = slots[tk.join].ctr;
        sink.begin_task(tk.join);
        ProbeAcc acc;
        bool work_p = nsv > 0 && nrv > 0;
        uint32_t cap = 0;
        if (work_p) {
            if (AGG) {
                // about three slots per build row, whole buckets; with duplicate
                // keys fewer slots than rows may do, so no early fallback
                const uint64_t want = (3 * nr + 127) / 128 * 128;
                cap = want < cap_max ? (uint32_t)want : cap_max;
            } else {
                // about three slots per build row (load factor 1/3), whole buckets
                const uint64_t want = (3 * nr + 127) / 128 * 128;
                cap = want < cap_max ? (uint32_t)want : cap_max;
                if (nr >= cap - cap / 4) {  // load factor above 3/4: leave to the fallback
                    if (threadIdx.x == 0) oversize[atomicAdd(&work->n_oversize, 1ull)] = (uint32_t)ti;
                    work_p = false;
                }
            }
        }
        uint32_t *ovf = (uint32_t *)(smem + (size_t)cap_max * (AGG ? agg_slot_bytes(W, chk) : 2 * W));
        const T top = Tup<W>::kAllOnes;
        const T empty = pf.keep(hashw<W>(top)) ? (T)tk.ek1 : top;
        const SoaTab<W> tab{cap / G, empty, ovf, (const T *)smem, (const T *)smem + cap};
        const AggSoa<W> at = AggSoa<W>::at(smem, cap, empty, ovf, chk != 0);
        if (work_p) {
            T *kv = (T *)smem;  // key region: cap keys; the rid (or sum and count) regions follow
            for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) kv[i] = empty;
            for (uint32_t i = threadIdx.x; i < (cap / G + 31) / 32; i += blockDim.x) ovf[i] = 0;
            if (AGG) {
                for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) {
                    at.cnt[i] = 0;
                    if (chk) at.suma[i] = 0;
                }
            }
            if (threadIdx.x == 0) {
                side.n_allones = side.agg_cnt = side.agg_suma = side.full = 0;
                s_full = 0;
            }
            __syncthreads();
            // build over R_p
            if constexpr (AGG) {
                // lanes of a warp holding the same key insert once, their count and
                // A(rid) sum together (a repeated key's slot takes one atomic per warp
                // group instead of one per tuple); the loop is warp-uniform
                for (uint32_t v0 = threadIdx.x & ~31u; v0 < nrv; v0 += blockDim.x) {
                    const uint32_t v = v0 + lane;
                    T k[2] = {0, 0}, r[2] = {0, 0};
                    if (v < nrv) {
                        const Vec x = ld_stream(Rv + v);
                        if constexpr (W == 4) {
                            k[0] = x.x; r[0] = x.y; k[1] = x.z; r[1] = x.w;
                        } else {
                            k[0] = x.x; r[0] = x.y;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < PV; ++e) {
                        // a padding row carries 0 or a pass's second sentinel: only
                        // such keys are hashed to see whether the row is the partition's
                        const bool in = v < nrv && !((k[e] == T(0) || k[e] == (T)tk.pk1 || k[e] == (T)tk.pk2) &&
                                                     !pf.keep(hashw<W>(k[e])));
                        const unsigned g = __match_any_sync(0xffffffffu, k[e]) & __ballot_sync(0xffffffffu, in);
                        const uint64_t a = chk && in ? mix_a(r[e]) : 0;
                        uint64_t asum = a;
                        if (chk && __any_sync(0xffffffffu, in && __popc(g) > 1)) {
                            // the group's sum of A(rid): every lane's value, kept by
                            // the lanes of its group (whole-warp shuffles)
                            asum = 0;
#pragma unroll 8
                            for (int q = 0; q < 32; ++q) {
                                const uint64_t y = __shfl_sync(0xffffffffu, a, q);
                                if ((g >> q) & 1u) asum += y;
                            }
                        }
                        if (!in || (g & ((1u << lane) - 1u))) continue;  // the group's lowest lane inserts
                        if (!at.insert(k[e], (uint32_t)__popc(g), asum)) s_full = 1;
                    }
                }
            } else
            for (uint32_t v = threadIdx.x; v < nrv; v += blockDim.x) {
                const Vec x = ld_stream(Rv + v);
                T k[2], r[2];
                if constexpr (W == 4) {
                    k[0] = x.x; r[0] = x.y; k[1] = x.z; r[1] = x.w;
                } else {
                    k[0] = x.x; r[0] = x.y;
                }
#pragma unroll
                for (int e = 0; e < PV; ++e) {
                    // a padding row carries 0 or a pass's second sentinel: only
                    // such keys are hashed to see whether the row is the partition's
                    if ((k[e] == T(0) || k[e] == (T)tk.pk1 || k[e] == (T)tk.pk2) && !pf.keep(hashw<W>(k[e]))) continue;
                    bool ok = false;
                    {
                        T *kv = (T *)smem;
                        uint32_t bkt = part_bucket<W>(k[e], tab.nb);
                        // a walk past kMaxSmemWalk buckets means a heavily repeated
                        // key: the partition goes to the key-list fallback
                        const uint32_t lim = tab.nb < kMaxSmemWalk ? tab.nb : kMaxSmemWalk;
                        for (uint32_t it = 0; it < lim && !ok; ++it) {
                            for (uint32_t q = 0; q < G; ++q) {
                                T *slot = &kv[bkt * G + q];
                                if (cas_key<W>(slot, empty, k[e]) == empty) {
                                    slot[cap] = r[e];  // the same slot of the rid region
                                    ok = true;
                                    break;
                                }
                            }
                            if (!ok) {  // moving past a full bucket: mark it
                                atomicOr(&ovf[bkt >> 5], 1u << (bkt & 31));
                                bkt = bkt + 1 == tab.nb ? 0 : bkt + 1;
                            }
                        }
                    }
                    if (!ok) s_full = 1;
                }
            }
            __syncthreads();
            if (s_full) {
                if (threadIdx.x == 0) oversize[atomicAdd(&work->n_oversize, 1ull)] = (uint32_t)ti;
            } else {
                if constexpr (FAST) {  // no aggregate, no checksum
                    // one vector per thread and group (two 4-byte tuples, one 8-byte):
                    // fewer live registers than U, which leaves the batched walks room
                    constexpr int FU = 1;
                    T *wq = (T *)(smem + walkq_offset(cap_max, 2 * W)) + (size_t)warp * 2 * kWalkQ;
                    probe_fast<W, FU>(tab, Sv, nsv, sink, warp, nwarps, lane, wq, wq + kWalkQ);
                } else {
                const uint32_t gstride = nwarps * 32 * U;
                Vec cur[U], nxt[U];
                uint32_t g = warp * 32 * U;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t rel = g + u * 32 + lane;
                    if (rel < nsv) cur[u] = ld_stream(Sv + rel);
                }
                for (; g < nsv; g += gstride) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const uint32_t rel = g + gstride + u * 32 + lane;
                        if (rel < nsv) nxt[u] = ld_stream(Sv + rel);
                    }
                    T k[IT], r[IT];
                    bool val[IT];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const bool in = g + u * 32 + lane < nsv;
                        if constexpr (W == 4) {
                            k[2 * u] = cur[u].x; r[2 * u] = cur[u].y; k[2 * u + 1] = cur[u].z; r[2 * u + 1] = cur[u].w;
                            val[2 * u] = in;
                            val[2 * u + 1] = in;
                        } else {
                            k[u] = cur[u].x; r[u] = cur[u].y;
                            val[u] = in;
                        }
                    }
                    if constexpr (AGG) {
                        // home buckets of all items first; no partition filter: a padding
                        // tuple's key hashes to another partition, so it matches no slot
                        uint32_t home[IT];
                        T kb[IT][G];
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            home[i] = part_bucket<W>(k[i], at.nb);
#pragma unroll
                            for (uint32_t q = 0; q < G; ++q) kb[i][q] = at.empty;
                            if (val[i]) at.ld(home[i], kb[i]);
                        }
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            uint32_t mm = 0;
                            bool e = false;
#pragma unroll
                            for (uint32_t q = 0; q < G; ++q) {
                                mm |= (uint32_t)(kb[i][q] == k[i]) << q;
                                e |= kb[i][q] == at.empty;
                            }
                            // (a lane past the slice's end holds a stale key: no slot)
                            uint32_t sl = val[i] && mm ? home[i] * G + (uint32_t)(__ffs(mm) - 1) : ~0u;
                            if (val[i] && !mm && !e && at.overflowed(home[i]))  // the run continues (rare)
                                sl = at.find_from(k[i], home[i] + 1 == at.nb ? 0 : home[i] + 1);
                            if (sl != ~0u) {
                                const uint64_t n = at.cnt[sl];
                                acc.cnt += n;
                                if (chk) {
                                    const uint64_t sa = at.suma[sl], bb = mix_b(r[i]);
                                    acc.c0 += sa * bb;
                                    acc.c1 += sa + n * bb;
                                }
                            }
                        }
                    } else {
                        uint32_t cnt[IT], home[IT];
                        T first[IT];
                        bool live[IT];
                        T kb[IT][G];
                        // Home buckets of all items, key halves loaded together.  Padding
                        // tuples need no filtering here: their keys hash to another
                        // partition, so they equal neither a stored key nor the marker.
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            home[i] = part_bucket<W>(k[i], tab.nb);
                            live[i] = val[i];
#pragma unroll
                            for (uint32_t q = 0; q < G; ++q) kb[i][q] = tab.empty;
                            if (live[i]) tab.ld(home[i], 0, kb[i]);
                        }
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            uint32_t mm = 0;
                            bool e = false;
#pragma unroll
                            for (uint32_t q = 0; q < G; ++q) {
                                mm |= (uint32_t)(kb[i][q] == k[i]) << q;
                                e |= kb[i][q] == tab.empty;
                            }
                            uint32_t c = 0;
                            T f = 0;
                            if (live[i] && mm) {
                                T rid[G];
                                tab.ld(home[i], 1, rid);
                                f = rid[G - 1];
#pragma unroll
                                for (int q = (int)G - 2; q >= 0; --q)
                                    if ((mm >> q) & 1u) f = rid[q];
                                c = __popc(mm);
                            }
                            if (live[i] && !e && tab.overflowed(home[i])) {  // the run continues (rare)
                                const uint32_t nx = home[i] + 1 == tab.nb ? 0 : home[i] + 1;
                                T f2 = 0;
                                const uint32_t c2 = soa_lookup<W>(tab, k[i], nx, &f2);
                                if (c == 0) f = f2;
                                c += c2;
                            }
                            if (chk && c) {
                                const uint64_t bs = mix_b(r[i]);
                                soa_visit<W>(tab, k[i], home[i], [&](T rid) {
                                    const uint64_t a = mix_a(rid);
                                    acc.c0 += a * bs;
                                    acc.c1 += a + bs;
                                });
                            }
                            cnt[i] = c;
                            first[i] = f;
                        }
                        sink.template append_group<IT>(cnt, first, r);
                        // several matches: the whole warp walks each such key's run
#pragma unroll
                        for (int i = 0; i < IT; ++i) {
                            unsigned multi = __ballot_sync(0xffffffffu, cnt[i] > 1);
                            while (multi) {
                                const int L = __ffs(multi) - 1;
                                multi &= multi - 1;
                                const T kk = __shfl_sync(0xffffffffu, k[i], L);
                                const T ss = __shfl_sync(0xffffffffu, r[i], L);
                                const uint32_t hh = __shfl_sync(0xffffffffu, home[i], L);
                                soa_coop_emit<W>(tab, kk, ss, hh, sink);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) cur[u] = nxt[u];
                }
                }
            }
        }
        flush_acc(jc, acc, AGG);
        if constexpr (!AGG) sink.end_task();
        __syncthreads();  // every warp is done with this table and with s_p
    }
    if constexpr (!AGG) sink.finish();
}

// Tasks of one join partitioned into NP padded partitions: task p covers rows
// [roff[p], roff[p+1]) of Rp and [soff[p], soff[p+1]) of Sp.
// Tasks of one join partitioned into NP padded partitions.  Partition p covers
// rows [roff[p], roff[p+1]) of Rp and [soff[p], soff[p+1]) of Sp.  Its S rows are
// cut into slices of at most `slice` rows (a multiple of the sector's tuples, so
// every slice starts on a sector), one task per slice, all with the whole R_p: a
// partition that skew made large is probed by several CTAs at once, each building
// its own copy of the (small) R_p table.  Task p is the first slice of partition
// p; further slices take indices from NP on, handed out by a counter (*next,
// zero at launch; their order does not matter).
__global__ void make_tasks_kernel(const void *Rp, const uint64_t *roff, const void *Sp, const uint64_t *soff,
                                  uint64_t NP, uint64_t slice, uint64_t tail_from, unsigned long long *next,
                                  uint32_t join, int b1, int b2, uint64_t ek1, uint64_t pk1, uint64_t pk2, int tb,
                                  PartTask *tasks) {
    const uint64_t sv = 32 / (uint64_t)tb;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < NP; p += (uint64_t)gridDim.x * blockDim.x) {
        PartTask t;
        t.R = (const char *)Rp + roff[p] * tb;
        t.nr = (uint32_t)(roff[p + 1] - roff[p]);
        t.join = join;
        t.p = (uint32_t)p;
        t.b1 = (uint16_t)b1;
        t.b2 = (uint16_t)b2;
        t.pad = 0;
        t.ek1 = ek1;
        t.pk1 = pk1;
        t.pk2 = pk2;
        const uint64_t s0 = soff[p], ns = soff[p + 1] - s0;
        // the partitions of the persistent join's last, partly filled round are
        // probed in two halves, so that the round's idle CTAs take the other halves
        uint64_t sl = slice;
        if (p >= tail_from && ns >= 2 * sv) {
            const uint64_t h = ((ns + 1) / 2 + sv - 1) / sv * sv;
            if (h < sl) sl = h;
        }
        const uint64_t extra = ns > sl ? (ns + sl - 1) / sl - 1 : 0;
        const uint64_t base = extra ? NP + atomicAdd(next, (unsigned long long)extra) : 0;
        for (uint64_t i = 0, at = 0; i == 0 || at < ns; ++i, at += sl) {
            t.S = (const char *)Sp + (s0 + at) * tb;
            t.ns = (uint32_t)(ns - at < sl ? ns - at : sl);
            tasks[i == 0 ? p : base + i - 1] = t;
        }
    }
}

uint64_t task_slice_rows(int width, uint64_t n_s, uint64_t NP) {
    // four times the mean partition, at least 2^16 rows, whole sectors
    const uint64_t sv = 32 / tuple_bytes(width);
    uint64_t sl = 4 * ((n_s + NP - 1) / (NP ? NP : 1));
    if (sl < (1ull << 16)) sl = 1ull << 16;
    return (sl + sv - 1) / sv * sv;
}

uint64_t max_tasks(uint64_t NP, uint64_t s_rows, uint64_t slice) { return NP + s_rows / slice + 1; }

uint64_t tail_split_from(hj_ctx *c, int width, int agg, uint64_t NP, uint64_t expect_r) {
    const uint64_t grid = partition_join_ctas(c, width, agg, expect_r), r = grid ? NP % grid : 0;
    return NP < grid || r == 0 ? NP : NP - r;
}

hj_status make_tasks(hj_ctx *c, const void *Rp, const uint64_t *roff, const void *Sp, const uint64_t *soff,
                     uint64_t NP, uint32_t join, int b1, int b2, int width, uint64_t slice, uint64_t ntasks,
                     PartTask *tasks, uint64_t tail_from) {
    const unsigned grid = (unsigned)((NP + 255) / 256);
    // unused task slots stay empty (no rows; the join skips them), and the slice
    // counter just past the array starts at zero
    HJ_CUDA(c, cudaMemsetAsync(tasks, 0, ntasks * sizeof(PartTask) + 8, c->stream));
    HJ_LAUNCH(c, "make_tasks", make_tasks_kernel, grid ? grid : 1, 256, 0, Rp, roff, Sp, soff, NP, slice, tail_from,
              (unsigned long long *)(tasks + ntasks), join, b1, b2, empty_key2(width, b1, b2),
              pass_pad_key(width, 0, b1), b2 ? pass_pad_key(width, b1, b2) : 0ull, (int)tuple_bytes(width), tasks);
    return HJ_OK;
}

// Second empty-marker candidate for pass bits (b1, b2): the first key below the top
// of the key domain whose partition differs from the top key's.  Padding keys of
// the partitioner come from the bottom of the domain (0, 1, 2, ...), so a probe key
// never equals a marker.
uint64_t empty_key2(int width, int b1, int b2) {
    auto pidx = [&](uint64_t k) {
        uint64_t h = width == 4 ? (uint64_t)murmur2_u32((uint32_t)k) : murmur2_u64(k);
        uint64_t d1 = h & ((1ull << b1) - 1), d2 = b2 ? (h >> b1) & ((1ull << b2) - 1) : 0;
        return (d1 << b2) | d2;
    };
    const uint64_t top = width == 4 ? 0xFFFFFFFFull : ~0ull;
    uint64_t k = top - 1;
    while (pidx(k) == pidx(top)) --k;
    return k;
}

// Join launch shape: two 512-thread CTAs per SM with tables up to 100 KiB, or one
// 1024-thread CTA per SM with up to 200 KiB when the expected build partition
// needs the room (load factor about 1/3 either way).
struct JoinCfg {
    int nt;
    uint64_t smem_limit;
};
static uint64_t join_slot_bytes(int width, int agg, int checksum) {
    return agg ? agg_slot_bytes(width, checksum) : 2ull * width;
}
static JoinCfg join_cfg(int width, int agg, int checksum, uint64_t expect_r) {
    const uint64_t slot = join_slot_bytes(width, agg, checksum);
    const uint64_t need = 3 * (expect_r + 6 * (uint64_t)__builtin_sqrt((double)expect_r + 1.0) + 64) * slot;
    if (need <= (100ull << 10)) return JoinCfg{512, 100ull << 10};
    return JoinCfg{1024, 200ull << 10};
}

uint64_t partition_join_warps(hj_ctx *c) { return (uint64_t)num_sms(c) * 32; }
uint64_t partition_join_ctas(hj_ctx *c, int width, int agg, uint64_t expect_r) {
    return (uint64_t)num_sms(c) * (2048 / join_cfg(width, agg, 1, expect_r).nt / 2);
}

hj_status partition_join(hj_ctx *c, int width, int agg, const PartTask *tasks, uint64_t ntasks, const JoinSlot *slots,
                         uint64_t expect_r, int checksum, uint32_t *oversize, RecArea ra, void *stage,
                         uint32_t scap) {
    if (ntasks == 0) return HJ_OK;
    const uint64_t slot_bytes = join_slot_bytes(width, agg, checksum);
    const JoinCfg cfg = join_cfg(width, agg, checksum, expect_r);
    // Capacity: room for a partition of the expected size plus six standard
    // deviations at load factor 1/3 (whole buckets), within the shape's budget.
    const double mean = (double)expect_r;
    uint64_t want = (uint64_t)(3.0 * (mean + 6.0 * __builtin_sqrt(mean + 1.0) + 64.0));
    want = (want + 127) / 128 * 128;
    const uint64_t bitmap_bytes = 4096;
    // the fast probe (no aggregate, no checksum) into the chunk sink adds each
    // warp's walk queue, within what the shape's CTAs per SM can have (two
    // 512-thread CTAs share an SM)
    const uint64_t qbytes = (!agg && !checksum) ? (uint64_t)(cfg.nt / 32) * kWalkQ * 2 * width : 0;
    const uint64_t total_max = cfg.nt == 512 ? (112ull << 10) : (222ull << 10);
    const uint64_t budget = std::min<uint64_t>(cfg.smem_limit + qbytes, total_max) - qbytes;
    uint64_t max_slots = (budget - bitmap_bytes) / slot_bytes / 128 * 128;
    uint64_t cap_max = want < max_slots ? want : max_slots;
    if (cap_max < 128) cap_max = 128;
    const size_t smem = (size_t)walkq_offset((uint32_t)cap_max, (uint32_t)slot_bytes) + (size_t)qbytes;
    unsigned grid = (unsigned)num_sms(c) * (2048 / cfg.nt / 2);
    if (grid > ntasks) grid = (unsigned)ntasks;
#define HJ_PJ(WW, AA, NT, SK, FF)                                                                               \
    do {                                                                                                        \
        auto kern = partition_join_kernel<WW, AA, NT, SK<WW>, FF>;                                              \
        HJ_TRY(allow_max_smem(c, (const void *)kern));                                                         \
        HJ_LAUNCH(c, "partition_join", kern, grid, NT, smem, tasks, ntasks, slots, c->d_ctr, (uint32_t)cap_max, \
                  ra, oversize, checksum, stage, scap);                                                         \
    } while (0)
#define HJ_PJ_NT(WW, AA, SK, FF)                                \
    do {                                                        \
        if (cfg.nt == 512) HJ_PJ(WW, AA, 512, SK, FF);           \
        else HJ_PJ(WW, AA, 1024, SK, FF);                        \
    } while (0)
#define HJ_PJ_F(WW, SK)                                         \
    do {                                                        \
        if (checksum) HJ_PJ_NT(WW, false, SK, false);            \
        else HJ_PJ_NT(WW, false, SK, true);                      \
    } while (0)
#define HJ_PJ_SK(WW)                                            \
    do {                                                        \
        if (stage) HJ_PJ_F(WW, WarpStageSink);                       \
        else HJ_PJ_F(WW, ChunkSink);                             \
    } while (0)
    if (width == 4) {
        if (agg) HJ_PJ_NT(4, true, ChunkSink, false); else HJ_PJ_SK(4);
    } else {
        if (agg) HJ_PJ_NT(8, true, ChunkSink, false); else HJ_PJ_SK(8);
    }
#undef HJ_PJ
#undef HJ_PJ_NT
#undef HJ_PJ_SK
#undef HJ_PJ_F
    return HJ_OK;
}

}  // namespace hj
