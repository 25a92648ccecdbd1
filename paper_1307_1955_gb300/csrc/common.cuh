// common.cuh -- device building blocks shared by the hash-join kernels:
// the key hash (MurmurHash2, Sec. 5.1), the checksum mixers, tuple types, the two
// hash-table layouts (one entry per build tuple, or one aggregate per distinct
// key) and a block-wide exclusive scan used to place output.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hj {

// ------------------------------------------------------------------ tuple types
// A tuple is <key, rid>, both W bytes (W = 4 or 8); tuples are read two (W = 4) or
// one (W = 8) per 16-byte vector load.
template <int W> struct Tup;
template <> struct Tup<4> {
    using U = uint32_t;
    using Vec = uint4;                 // one 16-byte load = 2 tuples
    static constexpr int kPerVec = 2;
    static constexpr U kAllOnes = 0xFFFFFFFFu;
};
template <> struct Tup<8> {
    using U = uint64_t;
    using Vec = ulonglong2;            // one 16-byte load = 1 tuple
    static constexpr int kPerVec = 1;
    static constexpr U kAllOnes = ~0ull;
};

// Load vector v (16 bytes) of a tuple array and unpack its tuples.
template <int W> struct VecIO;
template <> struct VecIO<4> {
    static __device__ __forceinline__ void unpack(const uint4 &v, uint32_t *k, uint32_t *r) {
        k[0] = v.x; r[0] = v.y; k[1] = v.z; r[1] = v.w;
    }
};
template <> struct VecIO<8> {
    static __device__ __forceinline__ void unpack(const ulonglong2 &v, uint64_t *k, uint64_t *r) {
        k[0] = v.x; r[0] = v.y;
    }
};

// Streaming 16-byte load that does not allocate in L1:
// every input tuple is read once per pass.
template <class V> __device__ __forceinline__ V ld_stream(const V *p);
template <> __device__ __forceinline__ uint4 ld_stream<uint4>(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
template <> __device__ __forceinline__ ulonglong2 ld_stream<ulonglong2>(const ulonglong2 *p) {
    ulonglong2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0,%1}, [%2];"
                 : "=l"(v.x), "=l"(v.y) : "l"(p));
    return v;
}

// ------------------------------------------------------------- MurmurHash2 (Sec. 5.1)
// MurmurHash2 (Appleby) of a key's little-endian bytes with seed 0: for a 4-byte
// key one block step (k *= m, k ^= k >> 24, k *= m, h = h*m ^ k) after
// h = seed ^ len, then the final avalanche (h ^= h >> 13, h *= m, h ^= h >> 15).
__host__ __device__ __forceinline__ uint32_t murmur2_u32(uint32_t key) {
    const uint32_t m = 0x5bd1e995u;
    uint32_t k = key * m;
    k ^= k >> 24;
    k *= m;
    uint32_t h = (0u ^ 4u) * m;
    h ^= k;
    h ^= h >> 13;
    h *= m;
    h ^= h >> 15;
    return h;
}
// MurmurHash64A of an 8-byte key, seed 0: h = seed ^ (8 * m); one block step
// (k *= m, k ^= k >> 47, k *= m, h ^= k, h *= m); final h ^= h >> 47, h *= m,
// h ^= h >> 47.
__host__ __device__ __forceinline__ uint64_t murmur2_u64(uint64_t key) {
    const uint64_t m = 0xc6a4a7935bd1e995ull;
    uint64_t h = 0ull ^ (8ull * m);
    uint64_t k = key * m;
    k ^= k >> 47;
    k *= m;
    h ^= k;
    h *= m;
    h ^= h >> 47;
    h *= m;
    h ^= h >> 47;
    return h;
}
template <int W> __device__ __forceinline__ uint64_t key_hash(typename Tup<W>::U k);
template <> __device__ __forceinline__ uint64_t key_hash<4>(uint32_t k) { return murmur2_u32(k); }
template <> __device__ __forceinline__ uint64_t key_hash<8>(uint64_t k) { return murmur2_u64(k); }

// Radix digit: `bits` bits of the hash starting at `shift` (low bits first, Alg. 2).
__device__ __forceinline__ uint32_t digit_of(uint64_t h, int shift, int bits) {
    return (uint32_t)(h >> shift) & ((1u << bits) - 1u);
}

// Membership of a hash in partition p of a PHJ with pass bits (b1, b2): the
// partition index is ((h mod 2^b1) << b2) | ((h >> b1) mod 2^b2) (Alg. 2's nested
// passes).  Inside the join, partitions may hold padding tuples whose key hashes
// elsewhere; build and probe drop every tuple this test rejects.
struct PartFilter {
    uint32_t p;
    int b1, b2, on;
    __device__ __forceinline__ bool keep(uint64_t h) const {
        if (!on) return true;
        const uint32_t h32 = (uint32_t)h, m1 = (1u << b1) - 1u, m2 = (1u << b2) - 1u;
        return (((h32 & m1) << b2) | ((h32 >> b1) & m2)) == p;
    }
};

// Table bucket in [0, cap): the high 32 bits of the hash scaled to cap
// (multiply-shift range reduction), independent of the low radix bits.
template <int W> __device__ __forceinline__ uint64_t bucket_of(uint64_t h, uint64_t cap);
template <> __device__ __forceinline__ uint64_t bucket_of<4>(uint64_t h, uint64_t cap) {
    return ((h & 0xFFFFFFFFull) * cap) >> 32;
}
template <> __device__ __forceinline__ uint64_t bucket_of<8>(uint64_t h, uint64_t cap) {
    return __umul64hi(h, cap);
}

// ------------------------------------------------------------- checksum mixers
// A(x) = SplitMix64 finaliser (Steele, Lea, Flood 2014); B(x) = A(x ^ golden).
__device__ __forceinline__ uint64_t sm64_fin(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t mix_a(uint64_t x) { return sm64_fin(x); }
__device__ __forceinline__ uint64_t mix_b(uint64_t x) { return sm64_fin(x ^ 0x9E3779B97F4A7C15ull); }

// ------------------------------------------------------------ 128-bit CAS
// Compare-and-swap of a 16-byte word (sm_90+): used to claim a table slot that
// holds a whole <key, rid> tuple of two 8-byte fields.
__device__ __forceinline__ ulonglong2 cas128(ulonglong2 *p, ulonglong2 cmp, ulonglong2 val) {
    ulonglong2 old;
    asm volatile(
        "{\n\t.reg .b128 c, v, o;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.cas.b128 o, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(old.x), "=l"(old.y)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
        : "memory");
    return old;
}

// ------------------------------------------------------------- pair table
// Open-addressing table with one slot per build tuple (Sec. 3.1's bucket headers
// plus rid lists, flattened: equal keys occupy separate slots of one probe run).
// A slot holds the tuple itself; the empty slot is all ones.  The one tuple whose
// bit pattern equals the empty marker (key and rid both all ones) is not stored:
// it is counted in `side` and re-emitted for probe keys equal to all ones.
// Slots are claimed with a CAS of the whole tuple; probing is linear with wrap.
template <int W> struct PairSlot;
template <> struct PairSlot<4> {
    using S = unsigned long long;
    static __device__ __forceinline__ S empty() { return ~0ull; }
    static __device__ __forceinline__ S pack(uint32_t k, uint32_t r) { return (S)k | ((S)r << 32); }
    static __device__ __forceinline__ bool is_empty(S s) { return s == ~0ull; }
    static __device__ __forceinline__ uint32_t key(S s) { return (uint32_t)s; }
    static __device__ __forceinline__ uint32_t rid(S s) { return (uint32_t)(s >> 32); }
    static __device__ __forceinline__ bool try_claim(S *p, S v) { return atomicCAS(p, ~0ull, v) == ~0ull; }
};
template <> struct PairSlot<8> {
    using S = ulonglong2;
    static __device__ __forceinline__ S empty() { return make_ulonglong2(~0ull, ~0ull); }
    static __device__ __forceinline__ S pack(uint64_t k, uint64_t r) { return make_ulonglong2(k, r); }
    static __device__ __forceinline__ bool is_empty(S s) { return (s.x & s.y) == ~0ull; }
    static __device__ __forceinline__ uint64_t key(S s) { return s.x; }
    static __device__ __forceinline__ uint64_t rid(S s) { return s.y; }
    static __device__ __forceinline__ bool try_claim(S *p, S v) {
        S o = cas128(p, empty(), v);
        return (o.x & o.y) == ~0ull;
    }
};

// ------------------------------------------------------------- aggregate table
// One slot per distinct build key (Sec. 3.1's key list with the rid list folded
// into a count and a sum): key, number of R tuples with that key, and the sum of
// A(rid) over them (mod 2^64).  The empty key is all ones; R tuples whose key is
// all ones are folded into a side aggregate instead.
template <int W> struct AggSlot;
template <> struct AggSlot<4> {
    uint32_t key;
    uint32_t cnt;
    unsigned long long suma;
};
template <> struct AggSlot<8> {
    unsigned long long key;
    unsigned long long cnt;
    unsigned long long suma;
    unsigned long long pad;
};

template <int W> __device__ __forceinline__ typename Tup<W>::U cas_key(typename Tup<W>::U *p,
                                                                       typename Tup<W>::U cmp,
                                                                       typename Tup<W>::U val);
template <> __device__ __forceinline__ uint32_t cas_key<4>(uint32_t *p, uint32_t c, uint32_t v) {
    return atomicCAS(p, c, v);
}
template <> __device__ __forceinline__ uint64_t cas_key<8>(uint64_t *p, uint64_t c, uint64_t v) {
    return atomicCAS((unsigned long long *)p, (unsigned long long)c, (unsigned long long)v);
}
__device__ __forceinline__ void add_cnt(uint32_t *p, uint32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_cnt(unsigned long long *p, unsigned long long v) { atomicAdd(p, v); }

// Side aggregates and counters that accompany a table.
struct TableSide {
    unsigned long long n_allones;   // pair table: R tuples equal to the empty marker
    unsigned long long agg_cnt;     // aggregate table: R tuples with the all-ones key
    unsigned long long agg_suma;
    unsigned long long full;        // set when an insert found no free slot
};

// Longest walk of a pair-table insert.  Unique keys at load factor <= 1/2 never
// come near it; a key with many copies does (every copy walks past the earlier
// ones), and the join then takes a key-list table instead.
constexpr uint64_t kMaxPairWalk = 1024;

// Insert one build tuple into a pair table of `cap` slots.  Returns false if
// the table had no free slot (cannot happen while cap > number of tuples) or
// the walk passed max_walk slots.
template <int W>
__device__ __forceinline__ bool pair_insert(typename PairSlot<W>::S *slots, uint64_t cap, TableSide *side,
                                            typename Tup<W>::U k, typename Tup<W>::U r, uint64_t h,
                                            uint64_t max_walk = kMaxPairWalk) {
    using PS = PairSlot<W>;
    if (k == Tup<W>::kAllOnes && r == Tup<W>::kAllOnes) {
        atomicAdd(&side->n_allones, 1ull);
        return true;
    }
    typename PS::S v = PS::pack(k, r);
    uint64_t b = bucket_of<W>(h, cap);
    const uint64_t lim = cap < max_walk ? cap : max_walk;
    for (uint64_t it = 0; it < lim; ++it) {
        if (PS::try_claim(&slots[b], v)) return true;
        if (++b == cap) b = 0;
    }
    return false;
}

// Visit every build rid whose key equals k: f(rid).  The key's run starts at its
// home slot bucket_of(h, cap / group) * group and ends at the first empty slot (a
// table always keeps at least one), after at most cap slots.
template <int W, class F>
__device__ __forceinline__ void pair_lookup(const typename PairSlot<W>::S *slots, uint64_t cap,
                                            unsigned long long n_allones, typename Tup<W>::U k, uint64_t h,
                                            uint32_t group, F &&f) {
    using PS = PairSlot<W>;
    uint64_t b = bucket_of<W>(h, cap / group) * group;
    for (uint64_t it = 0; it < cap; ++it) {
        typename PS::S s = slots[b];
        if (PS::is_empty(s)) break;
        if (PS::key(s) == k) f(PS::rid(s));
        if (++b == cap) b = 0;
    }
    if (k == Tup<W>::kAllOnes)
        for (unsigned long long i = 0; i < n_allones; ++i) f(Tup<W>::kAllOnes);
}

// Insert a build tuple into an aggregate table.  Returns false if the key is new
// and no free slot remains.
template <int W>
__device__ __forceinline__ bool agg_insert(AggSlot<W> *slots, uint64_t cap, TableSide *side,
                                           typename Tup<W>::U k, uint64_t a, uint64_t h) {
    if (k == Tup<W>::kAllOnes) {
        atomicAdd(&side->agg_cnt, 1ull);
        atomicAdd(&side->agg_suma, (unsigned long long)a);
        return true;
    }
    uint64_t b = bucket_of<W>(h, cap);
    for (uint64_t it = 0; it < cap; ++it) {
        typename Tup<W>::U old = cas_key<W>((typename Tup<W>::U *)&slots[b].key, Tup<W>::kAllOnes, k);
        if (old == Tup<W>::kAllOnes || old == k) {
            add_cnt(&slots[b].cnt, 1);
            atomicAdd(&slots[b].suma, (unsigned long long)a);
            return true;
        }
        if (++b == cap) b = 0;
    }
    return false;
}

// Look a probe key up in an aggregate table: (count, suma) of its build tuples.
template <int W>
__device__ __forceinline__ void agg_lookup(const AggSlot<W> *slots, uint64_t cap, const TableSide *side,
                                           typename Tup<W>::U k, uint64_t h, uint64_t *cnt, uint64_t *suma) {
    *cnt = 0;
    *suma = 0;
    if (k == Tup<W>::kAllOnes) {
        *cnt = side->agg_cnt;
        *suma = side->agg_suma;
        return;
    }
    uint64_t b = bucket_of<W>(h, cap);
    for (uint64_t it = 0; it < cap; ++it) {
        typename Tup<W>::U sk = slots[b].key;
        if (sk == k) {
            *cnt = slots[b].cnt;
            *suma = slots[b].suma;
            return;
        }
        if (sk == Tup<W>::kAllOnes) return;
        if (++b == cap) b = 0;
    }
}

// ------------------------------------------------------------- block scan
// Exclusive scan of one unsigned value per thread across the block; returns the
// thread's prefix and writes the block total to *total.  `scratch` holds 33
// entries.  All threads must call it.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *scratch, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < nw ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) scratch[lane] = s;       // inclusive warp totals
        if (lane == nw - 1) scratch[32] = s;
    }
    __syncthreads();
    T warp_base = warp ? scratch[warp - 1] : T(0);
    *total = scratch[32];
    T r = warp_base + x - v;
    __syncthreads();   // scratch may be reused by the caller
    return r;
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------- TMA bulk copies
// One-dimensional bulk copy global -> shared completed on an mbarrier (sm_90+).
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Order this thread's earlier generic-proxy shared accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for an mbarrier phase with an iteration limit; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Status bits written by kernels into the context's device status word.
enum : int {
    kStatusTableFull = 1,
    kStatusTimeout = 2,
    kStatusBadInput = 4,
    kStatusRecords = 8,    // a chunk-record area was too small
    kStatusCompact = 16,   // device compaction found holes and tail pairs of different sizes
    kStatusLongRun = 32,   // a pair-table insert walked past kMaxPairWalk slots (heavily repeated keys)
};

}  // namespace hj
