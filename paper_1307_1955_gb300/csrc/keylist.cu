// keylist.cu -- the hash table of Sec. 3.1 with key lists and rid lists, for
// build relations whose keys repeat heavily.
//
// Open addressing over (key, rid) slots stores each duplicate in a slot of its
// own: a key with a million copies becomes a run of a million slots that every
// probe landing in it has to walk.  The paper's table instead gives each
// distinct key one entry whose rid list holds all of its build tuples' rids.
// Here that is the aggregate table (one slot per distinct key with its count)
// plus one array of rids:
//   1. insert every kept key of R into the aggregate table with its count (the
//      first table sized for a 32nd as many distinct keys as rows, built again at
//      full size if it passes half full);
//   2. an exclusive scan of the counts gives each key the offset of its rid list;
//   3. a second pass over R places every rid in its key's list (a per-key fill
//      position claimed by atomicAdd; the order inside a list is free).
// In steps 1 and 3 the lanes of a warp holding one key act as one, and keys that
// fill several lanes are also gathered per CTA tile in shared memory: a heavy
// hitter's count and fill position take one global atomic per tile.
// A probe finds its key's one slot and emits the key's rid list with its own rid:
// lists of fewer than 32 pairs flattened across the warp (pair p of their
// concatenation written by lane p mod 32); a list of up to kCoopPairs by the
// whole warp, reading the list with coalesced loads; a longer list (a heavy
// hitter) is recorded and expanded afterwards by a grid-wide kernel in segments
// of kSegPairs pairs, so that the millions of pairs of one probe tuple are
// written by every SM.  The rows of a warp's step (the lists of its 32 probe
// tuples) are claimed with one atomic add on the join's count: one global atomic
// per 32 probes, not per 32 pairs.
// R tuples whose key is all ones (the aggregate table's empty marker) are
// counted on the table's side and keep their rids at the end of the array.
#include <algorithm>

#include "common.cuh"
#include "ctx.cuh"
#include "emit.cuh"
#include "engine.cuh"

namespace hj {

namespace {

constexpr unsigned kScanThreads = 1024;
constexpr uint64_t kScanBlock = 2 * kScanThreads;  // entries per scan block
constexpr uint64_t kCoopPairs = 4096;              // longest list one warp emits
constexpr uint64_t kSegPairs = 1ull << 13;         // pairs per expansion segment (one CTA's)

template <int W>
__device__ __forceinline__ void kl_load(const void *base, uint64_t v, uint64_t n_total, typename Tup<W>::U *k,
                                        typename Tup<W>::U *r) {
    if constexpr (W == 8) {
        const ulonglong2 x = ld_stream((const ulonglong2 *)base + v);
        k[0] = x.x;
        r[0] = x.y;
    } else if (2 * v + 1 < n_total) {
        const uint4 x = ld_stream((const uint4 *)base + v);
        k[0] = x.x; r[0] = x.y; k[1] = x.z; r[1] = x.w;
    } else {
        const uint2 x = ((const uint2 *)base)[2 * v];
        k[0] = x.x; r[0] = x.y; k[1] = 0; r[1] = 0;
    }
}

// Slot of key k (not all ones) in the aggregate table, or cap if absent.
template <int W>
__device__ __forceinline__ uint64_t kl_find(const AggSlot<W> *slots, uint64_t cap, typename Tup<W>::U k, uint64_t h) {
    uint64_t b = bucket_of<W>(h, cap);
    for (uint64_t it = 0; it < cap; ++it) {
        const typename Tup<W>::U sk = slots[b].key;
        if (sk == k) return b;
        if (sk == Tup<W>::kAllOnes) return cap;
        if (++b == cap) b = 0;
    }
    return cap;
}

// ------------------------------------------------------------------ scans
// Exclusive scans of per-entry counts, in three launches (block sums, a scan of
// the block sums by one block, per-block scans); Src::get(i) is entry i's count,
// Dst::put(i, off) stores its offset, and bsum[nb] receives the total.

struct AggCnt4 {
    AggSlot<4> *s;
    __device__ uint64_t get(uint64_t i) const { return s[i].cnt; }
    // offset in the low half of the 64-bit field, the list's fill position (0) in the high half
    __device__ void put(uint64_t i, uint64_t off) const { s[i].suma = (uint32_t)off; }
};
struct AggCnt8 {
    AggSlot<8> *s;
    __device__ uint64_t get(uint64_t i) const { return s[i].cnt; }
    __device__ void put(uint64_t i, uint64_t off) const {
        s[i].suma = off;
        s[i].pad = 0;
    }
};
struct Big {
    unsigned long long off, cnt, s;
};
struct SegCnt {
    const Big *b;
    unsigned long long *pref;
    __device__ uint64_t get(uint64_t i) const { return (b[i].cnt + kSegPairs - 1) / kSegPairs; }
    __device__ void put(uint64_t i, uint64_t off) const { pref[i] = off; }
};

// Exclusive block-wide scan of one value per thread (kScanThreads threads).
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *total) {
    __shared__ unsigned long long ws[32];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= (unsigned)d) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const uint64_t before = (warp ? ws[warp - 1] : 0) + x - v;
    *total = ws[31];
    __syncthreads();  // ws is reused by the next call
    return before;
}

template <class Src>
__global__ void __launch_bounds__(kScanThreads) kl_block_sums(Src src, uint64_t n, unsigned long long *bsum) {
    const uint64_t i0 = blockIdx.x * kScanBlock + 2 * threadIdx.x;
    const uint64_t v = (i0 < n ? src.get(i0) : 0) + (i0 + 1 < n ? src.get(i0 + 1) : 0);
    uint64_t tot;
    block_excl_scan(v, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) kl_scan_sums(unsigned long long *bsum, uint64_t nb) {
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const uint64_t i = b0 + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        uint64_t tot;
        const uint64_t x = block_excl_scan(v, &tot);
        if (i < nb) bsum[i] = carry + x;
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <class Src, class Dst>
__global__ void __launch_bounds__(kScanThreads) kl_apply(Src src, Dst dst, uint64_t n, const unsigned long long *bsum) {
    const uint64_t i0 = blockIdx.x * kScanBlock + 2 * threadIdx.x;
    const uint64_t a = i0 < n ? src.get(i0) : 0, b = i0 + 1 < n ? src.get(i0 + 1) : 0;
    uint64_t tot;
    const uint64_t x = bsum[blockIdx.x] + block_excl_scan(a + b, &tot);
    if (i0 < n) dst.put(i0, x);
    if (i0 + 1 < n) dst.put(i0 + 1, x + a);
}

template <class Src, class Dst>
hj_status scan_entries(hj_ctx *c, Src src, Dst dst, uint64_t n, uint64_t *total_host) {
    const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    DevBuf bsum(c);
    HJ_TRY(bsum.alloc((nb + 1) * 8));
    if (nb) {
        HJ_LAUNCH(c, "keylist_scan", kl_block_sums<Src>, (unsigned)nb, kScanThreads, 0, src, n,
                  bsum.as<unsigned long long>());
        HJ_LAUNCH(c, "keylist_scan", kl_scan_sums, 1, kScanThreads, 0, bsum.as<unsigned long long>(), nb);
        HJ_LAUNCH(c, "keylist_scan", (kl_apply<Src, Dst>), (unsigned)nb, kScanThreads, 0, src, dst, n,
                  bsum.as<unsigned long long>());
    } else {
        HJ_CUDA(c, cudaMemsetAsync(bsum.p, 0, 8, c->stream));
    }
    if (total_host) {
        HJ_CUDA(c, cudaMemcpyAsync(total_host, bsum.as<unsigned long long>() + nb, 8, cudaMemcpyDeviceToHost,
                                   c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HJ_OK;
}

// --------------------------------------------------------------- build
// Lanes of a warp holding the same kept key act as one: the lowest takes the
// group's count in one atomic (a heavy hitter has many copies in every warp, and
// one atomic per copy on one address would serialise the build).
__device__ __forceinline__ unsigned lanes_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

constexpr uint64_t kGuessWalk = 64;
// Keys that fill several lanes of a warp group (the heavy hitters that make a
// partition need a key-list table) are also gathered per tile of a CTA: up to
// kHot of them in shared memory, each then taking one global atomic per tile
// instead of one per warp group.
constexpr int kHot = 8;

// Entry of key k among the tile's gathered keys (a free one taken), or -1.
template <int W> __device__ __forceinline__ int hot_entry(typename Tup<W>::U *hk, typename Tup<W>::U k) {
    using U = typename Tup<W>::U;
#pragma unroll 1
    for (int j = 0; j < kHot; ++j) {
        const U cur = ((volatile U *)hk)[j];
        if (cur == k) return j;
        if (cur == Tup<W>::kAllOnes) {
            const U old = cas_key<W>(&hk[j], Tup<W>::kAllOnes, k);
            if (old == Tup<W>::kAllOnes || old == k) return j;
        }
    }
    return -1;
}

// Adds m to key k's count, inserting the key (CAS on the key); returns 1 if this
// call inserted it.  A walk that ends without a slot gives up a first table
// (guess: *nkeys is pushed past any limit) or flags a full one.
template <int W>
__device__ __forceinline__ unsigned kl_add(AggSlot<W> *slots, uint64_t cap, typename Tup<W>::U k, uint64_t h,
                                           unsigned m, bool guess, unsigned long long *nkeys, hj_counters *ctr) {
    using U = typename Tup<W>::U;
    const uint64_t walk = guess && cap > kGuessWalk ? kGuessWalk : cap;
    uint64_t b = bucket_of<W>(h, cap);
    for (uint64_t it = 0; it < walk; ++it) {
        const U old = cas_key<W>((U *)&slots[b].key, Tup<W>::kAllOnes, k);
        if (old == Tup<W>::kAllOnes || old == k) {
            add_cnt(&slots[b].cnt, (decltype(slots[b].cnt))m);
            return old == Tup<W>::kAllOnes;
        }
        if (++b == cap) b = 0;
    }
    if (guess) atomicAdd(nkeys, (unsigned long long)cap);
    else atomicOr(&ctr->status, (unsigned long long)kStatusTableFull);
    return 0;
}

// Step 1: every kept key in the table, its count added.  Each key inserted counts
// in *nkeys; with a first table sized for fewer distinct keys than rows
// (key_limit = half its slots) the CTAs stop once they pass the limit, walks end
// after kGuessWalk slots (at load <= 1/2 a longer one gives the table up too),
// and the host builds again at full size.
template <int W>
__global__ void __launch_bounds__(256) kl_count(const void *R, uint64_t n, AggSlot<W> *slots, uint64_t cap,
                                                TableSide *side, hj_counters *ctr, PartFilter pf,
                                                unsigned long long *nkeys, uint64_t key_limit) {
    using U = typename Tup<W>::U;
    constexpr int PV = Tup<W>::kPerVec;
    __shared__ U hk[kHot];        // the tile's gathered keys (all ones: free)
    __shared__ unsigned hc[kHot];  // and their counts
    __shared__ int stop;
    const unsigned lane = threadIdx.x & 31;
    const bool guess = key_limit != ~0ull;
    const uint64_t nv = (n + PV - 1) / PV;
    const uint64_t tiles = (nv + blockDim.x - 1) / blockDim.x;
    if (threadIdx.x < kHot) {
        hk[threadIdx.x] = Tup<W>::kAllOnes;
        hc[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) stop = 0;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {  // block-uniform
        const uint64_t v = tile * blockDim.x + threadIdx.x;
        U k[2] = {0, 0}, r[2] = {0, 0};
        if (v < nv) kl_load<W>(R, v, n, k, r);
        unsigned fresh = 0;  // keys this lane inserted (first table only)
#pragma unroll
        for (int e = 0; e < PV; ++e) {
            const uint64_t h = key_hash<W>(k[e]);
            const bool ok = v < nv && v * PV + e < n && pf.keep(h);
            const unsigned g = __match_any_sync(0xffffffffu, k[e]) & __ballot_sync(0xffffffffu, ok);
            if (!ok || (g & lanes_lt())) continue;  // the group's lowest lane counts for it
            const unsigned m = __popc(g);
            if (k[e] == Tup<W>::kAllOnes) {
                atomicAdd(&side->agg_cnt, (unsigned long long)m);
                continue;
            }
            if (guess && *(volatile unsigned long long *)nkeys > key_limit) continue;  // given up
            if (m > 1) {
                const int j = hot_entry<W>(hk, k[e]);
                if (j >= 0) {
                    atomicAdd(&hc[j], m);
                    continue;
                }
            }
            fresh += kl_add<W>(slots, cap, k[e], h, m, guess, nkeys, ctr);
        }
        if (guess) {  // (the warp is converged again here)
            const unsigned tot = __reduce_add_sync(0xffffffffu, fresh);
            if (lane == 0 && tot) atomicAdd(nkeys, (unsigned long long)tot);
        }
        __syncthreads();
        if (threadIdx.x < kHot) {  // the gathered keys: one add each
            const U hkey = hk[threadIdx.x];
            if (hkey != Tup<W>::kAllOnes) {
                if (kl_add<W>(slots, cap, hkey, key_hash<W>(hkey), hc[threadIdx.x], guess, nkeys, ctr) && guess)
                    atomicAdd(nkeys, 1ull);
                hk[threadIdx.x] = Tup<W>::kAllOnes;
                hc[threadIdx.x] = 0;
            }
        }
        if (threadIdx.x == 0) stop = guess && *(volatile unsigned long long *)nkeys > key_limit;
        __syncthreads();
        if (stop) break;
    }
}

// Step 3: every kept R tuple's rid into its key's list: a warp group's places
// [at, at + popc(g)) claimed by its leader on the key's fill position, a gathered
// key's places claimed once per tile.
template <int W>
__global__ void __launch_bounds__(256) kl_scatter(const void *R, uint64_t n, AggSlot<W> *slots, uint64_t cap,
                                                  TableSide *side, typename Tup<W>::U *rids, hj_counters *ctr,
                                                  PartFilter pf) {
    using U = typename Tup<W>::U;
    constexpr int PV = Tup<W>::kPerVec;
    __shared__ U hk[kHot];
    __shared__ unsigned hc[kHot];
    __shared__ unsigned long long hb[kHot];  // first place of a gathered key's tuples (~0: none)
    const unsigned lane = threadIdx.x & 31;
    const uint64_t nv = (n + PV - 1) / PV;
    const uint64_t tiles = (nv + blockDim.x - 1) / blockDim.x;
    if (threadIdx.x < kHot) {
        hk[threadIdx.x] = Tup<W>::kAllOnes;
        hc[threadIdx.x] = 0;
    }
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {  // block-uniform
        const uint64_t v = tile * blockDim.x + threadIdx.x;
        U k[2] = {0, 0}, r[2] = {0, 0};
        if (v < nv) kl_load<W>(R, v, n, k, r);
        int hj[2] = {-1, -1};      // gathered entry of item e
        unsigned hr[2] = {0, 0};   // and its place among the entry's tuples
#pragma unroll
        for (int e = 0; e < PV; ++e) {
            const uint64_t h = key_hash<W>(k[e]);
            const bool ok = v < nv && v * PV + e < n && pf.keep(h);
            const unsigned g = __match_any_sync(0xffffffffu, k[e]) & __ballot_sync(0xffffffffu, ok);
            const int leader = g ? __ffs(g) - 1 : 0;
            // the leader claims the group's places: [at, at + popc(g)) of the key's
            // list, or of the all-ones keys' list counted down from the array's end,
            // or of the key's gathered tuples in this tile
            uint64_t at = 0;
            bool fail = false;
            int j = -1;
            if (ok && lane == (unsigned)leader) {
                const uint64_t m = __popc(g);
                if (k[e] == Tup<W>::kAllOnes) {
                    at = atomicAdd(&side->n_allones, (unsigned long long)m);
                } else {
                    if (m > 1) j = hot_entry<W>(hk, k[e]);
                    if (j >= 0) {
                        at = atomicAdd(&hc[j], (unsigned)m);
                    } else {
                        const uint64_t b = kl_find<W>(slots, cap, k[e], h);
                        if (b == cap) {  // cannot happen: step 1 inserted every kept key
                            fail = true;
                        } else if constexpr (W == 4) {
                            unsigned *half = (unsigned *)&slots[b].suma;  // [0] offset, [1] fill position
                            at = half[0] + atomicAdd(&half[1], (unsigned)m);
                        } else {
                            at = slots[b].suma + atomicAdd(&slots[b].pad, (unsigned long long)m);
                        }
                    }
                }
                if (fail) atomicOr(&ctr->status, (unsigned long long)kStatusTableFull);
            }
            at = __shfl_sync(0xffffffffu, at, leader);
            fail = __shfl_sync(0xffffffffu, fail, leader);
            j = __shfl_sync(0xffffffffu, j, leader);
            if (!ok || fail) continue;
            const uint64_t rank = __popc(g & lanes_lt());
            if (j >= 0) {
                hj[e] = j;
                hr[e] = (unsigned)(at + rank);
            } else if (k[e] == Tup<W>::kAllOnes) {
                rids[n - 1 - (at + rank)] = r[e];
            } else {
                rids[at + rank] = r[e];
            }
        }
        __syncthreads();
        if (threadIdx.x < kHot) {  // the gathered keys: their places in one claim each
            const U hkey = hk[threadIdx.x];
            if (hkey != Tup<W>::kAllOnes) {
                const uint64_t b = kl_find<W>(slots, cap, hkey, key_hash<W>(hkey));
                const unsigned m = hc[threadIdx.x];
                if (b == cap) {
                    atomicOr(&ctr->status, (unsigned long long)kStatusTableFull);
                    hb[threadIdx.x] = ~0ull;
                } else if constexpr (W == 4) {
                    unsigned *half = (unsigned *)&slots[b].suma;
                    hb[threadIdx.x] = half[0] + atomicAdd(&half[1], m);
                } else {
                    hb[threadIdx.x] = slots[b].suma + atomicAdd(&slots[b].pad, (unsigned long long)m);
                }
                hk[threadIdx.x] = Tup<W>::kAllOnes;
                hc[threadIdx.x] = 0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PV; ++e)
            if (hj[e] >= 0 && hb[hj[e]] != ~0ull) rids[hb[hj[e]] + hr[e]] = r[e];
    }
}

// --------------------------------------------------------------- probe
template <int W>
__global__ void __launch_bounds__(256) kl_probe(const void *S, uint64_t ns, const AggSlot<W> *slots, uint64_t cap,
                                                const TableSide *side, const typename Tup<W>::U *rids, uint64_t nr,
                                                void *pairs, uint64_t pcap, hj_counters *ctr, int chk, PartFilter pf,
                                                Big *big, unsigned long long *nbig) {
    using U = typename Tup<W>::U;
    using P = typename PairVec<W>::T;
    constexpr int PV = Tup<W>::kPerVec;
    constexpr unsigned kUnroll = 4;  // pairs per lane and step of a list walk (loads in flight)
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nv = (ns + PV - 1) / PV;
    P *out = (P *)pairs;
    auto mk = [](U a, U b) -> P {
        if constexpr (W == 4) return make_uint2(a, b);
        else return make_ulonglong2(a, b);
    };
    unsigned long long c0 = 0, c1 = 0;
    const uint64_t allones = side->agg_cnt;
    for (uint64_t v0 = warp * 32; v0 < nv; v0 += nwarps * 32) {
        const uint64_t v = v0 + lane;
        U k[2] = {0, 0}, r[2] = {0, 0};
        if (v < nv) kl_load<W>(S, v, ns, k, r);
#pragma unroll
        for (int e = 0; e < PV; ++e) {
            uint64_t cnt = 0, off = 0;
            if (v < nv && v * PV + e < ns) {
                const uint64_t h = key_hash<W>(k[e]);
                if (pf.keep(h)) {
                    if (k[e] == Tup<W>::kAllOnes) {
                        cnt = allones;
                        off = nr - allones;
                    } else {
                        const uint64_t b = kl_find<W>(slots, cap, k[e], h);
                        if (b < cap) {
                            cnt = slots[b].cnt;
                            off = W == 4 ? (uint32_t)slots[b].suma : slots[b].suma;
                        }
                    }
                }
            }
            const U s = r[e];
            // a heavy hitter: expanded by the grid afterwards (it claims its own rows)
            if (cnt > kCoopPairs) {
                const unsigned long long i = atomicAdd(nbig, 1ull);
                big[i] = Big{off, cnt, (unsigned long long)s};  // at most one entry per probe tuple
            }
            // every other list of this step: one claim for the whole warp.  Lists
            // of fewer than 32 pairs first, flattened: pair p of their concatenation
            // (in lane order) is written by lane p mod 32 at base + p, its list found
            // by a search over the lanes' prefix sums; then each longer list by the
            // whole warp in turn, at base + (small pairs) + the prefix of the longer
            // lists before it.
            const uint64_t mine = cnt <= kCoopPairs ? cnt : 0;
            const uint64_t small = mine < 32 ? mine : 0, mid = mine - small;
            uint64_t incl = small | (mid << 32);  // (small sums stay below 2^10, mid sums below 2^18)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (unsigned)o) incl += y;
            }
            const uint64_t last = __shfl_sync(0xffffffffu, incl, 31);
            const uint64_t tot_s = last & 0xffffffffu, tot = tot_s + (last >> 32);
            if (!tot) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctr->count, (unsigned long long)tot);
            base = __shfl_sync(0xffffffffu, base, 0);
            const uint64_t incl_s = incl & 0xffffffffu, incl_m = incl >> 32;
            for (uint64_t p0 = 0; p0 < tot_s; p0 += 32) {
                const uint64_t p = p0 + lane;
                unsigned L = 0;  // first lane whose inclusive prefix passes p
#pragma unroll
                for (unsigned b = 16; b >= 1; b >>= 1) {
                    const uint64_t x = __shfl_sync(0xffffffffu, incl_s, L + b - 1);
                    if (x <= p) L += b;
                }
                const uint64_t first = __shfl_sync(0xffffffffu, incl_s - small, L & 31);
                const uint64_t o = __shfl_sync(0xffffffffu, off, L & 31);
                const U ss = __shfl_sync(0xffffffffu, s, L & 31);
                if (p < tot_s) {
                    const U a = rids[o + (p - first)];
                    if (base + p < pcap) out[base + p] = mk(a, ss);
                    if (chk) {
                        const uint64_t A = mix_a(a), B = mix_b(ss);
                        c0 += A * B;
                        c1 += A + B;
                    }
                }
            }
            const uint64_t at = base + tot_s + incl_m - mid;
            // a longer list: the whole warp, kUnroll x 32 pairs per step
            unsigned coop = __ballot_sync(0xffffffffu, mid > 0);
            while (coop) {
                const int L = __ffs(coop) - 1;
                coop &= coop - 1;
                const uint64_t o = __shfl_sync(0xffffffffu, off, L), n = __shfl_sync(0xffffffffu, mid, L);
                const uint64_t dst = __shfl_sync(0xffffffffu, at, L);
                const U ss = __shfl_sync(0xffffffffu, s, L);
                const uint64_t B = chk ? mix_b(ss) : 0;
                for (uint64_t j0 = 0; j0 < n; j0 += 32 * kUnroll) {
                    U ra[kUnroll];
#pragma unroll
                    for (unsigned u = 0; u < kUnroll; ++u) {
                        const uint64_t j = j0 + u * 32 + lane;
                        ra[u] = j < n ? rids[o + j] : U(0);
                    }
#pragma unroll
                    for (unsigned u = 0; u < kUnroll; ++u) {
                        const uint64_t j = j0 + u * 32 + lane;
                        if (j < n) {
                            if (dst + j < pcap) out[dst + j] = mk(ra[u], ss);
                            if (chk) {
                                const uint64_t A = mix_a(ra[u]);
                                c0 += A * B;
                                c1 += A + B;
                            }
                        }
                    }
                }
            }
        }
    }
    c0 = warp_sum(c0);
    c1 = warp_sum(c1);
    if (lane == 0) {
        if (c0) atomicAdd(&ctr->c0, c0);
        if (c1) atomicAdd(&ctr->c1, c1);
    }
}

// Segment g of the heavy hitters' pairs: its entry (the last with pref <= g), rows
// claimed from ctr->count by the CTA, pairs written by all its threads.
template <int W>
__global__ void __launch_bounds__(256) kl_expand(const Big *big, const unsigned long long *pref, uint64_t nbig,
                                                 uint64_t nseg, const typename Tup<W>::U *rids, void *pairs,
                                                 uint64_t pcap, hj_counters *ctr, int chk) {
    using U = typename Tup<W>::U;
    using P = typename PairVec<W>::T;
    __shared__ unsigned long long s_base;
    unsigned long long c0 = 0, c1 = 0;
    for (uint64_t g = blockIdx.x; g < nseg; g += gridDim.x) {
        uint64_t lo = 0, hi = nbig;  // pref[lo] <= g < pref[hi], with pref[nbig] read as nseg
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (pref[mid] <= g) lo = mid;
            else hi = mid;
        }
        const Big b = big[lo];
        const uint64_t j0 = (g - pref[lo]) * kSegPairs;
        const uint64_t len = b.cnt - j0 < kSegPairs ? b.cnt - j0 : kSegPairs;
        if (threadIdx.x == 0) s_base = atomicAdd(&ctr->count, (unsigned long long)len);
        __syncthreads();
        const unsigned long long base = s_base;
        const U s = (U)b.s;
        const uint64_t B = chk ? mix_b(s) : 0;
#pragma unroll 4
        for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) {
            const U a = rids[b.off + j0 + i];
            if (base + i < pcap) {
                if constexpr (W == 4) ((P *)pairs)[base + i] = make_uint2(a, s);
                else ((P *)pairs)[base + i] = make_ulonglong2(a, s);
            }
            if (chk) {
                const uint64_t A = mix_a(a);
                c0 += A * B;
                c1 += A + B;
            }
        }
        __syncthreads();  // s_base is rewritten for the next segment
    }
    c0 = warp_sum(c0);
    c1 = warp_sum(c1);
    if ((threadIdx.x & 31) == 0) {
        if (c0) atomicAdd(&ctr->c0, c0);
        if (c1) atomicAdd(&ctr->c1, c1);
    }
}

}  // namespace

// First table of a key-list build over more than kKeyGuessMin rows: sized for
// rows / kKeyGuessDiv distinct keys.  A relation whose repeated keys sent it here
// holds far fewer distinct keys than rows, and the scan of step 2 reads the
// whole table; one with more distinct keys stops early and is built again at
// full size.
constexpr uint64_t kKeyGuessMin = 1ull << 16;
constexpr uint64_t kKeyGuessDiv = 32;

hj_status keylist_build(hj_ctx *c, int width, const void *R, uint64_t n, PartFilter pf, hj_table **out) {
    *out = nullptr;
    DevBuf rids(c), nkeys(c);
    HJ_TRY(nkeys.alloc(8));
    hj_table *t = nullptr;
    struct Guard {
        hj_ctx *c;
        hj_table *t;
        ~Guard() {
            if (t) table_destroy(c, t);
        }
    } g{c, nullptr};
    for (uint64_t keys = n > kKeyGuessMin ? std::max(kKeyGuessMin, n / kKeyGuessDiv) : n;;) {
        HJ_TRY(table_create(c, width, 1, keys, &t));
        g.t = t;
        const uint64_t limit = keys < n ? t->cap / 2 : ~0ull;
        HJ_CUDA(c, cudaMemsetAsync(nkeys.p, 0, 8, c->stream));
        const uint64_t nv = (n + 1) / (width == 4 ? 2 : 1);
        const unsigned grid = (unsigned)std::min<uint64_t>((nv + 255) / 256 + 1, (uint64_t)num_sms(c) * 8);
        if (width == 4)
            HJ_LAUNCH(c, "keylist_count", kl_count<4>, grid, 256, 0, R, n, (AggSlot<4> *)t->slots, t->cap,
                      (TableSide *)t->side, c->d_ctr, pf, nkeys.as<unsigned long long>(), limit);
        else
            HJ_LAUNCH(c, "keylist_count", kl_count<8>, grid, 256, 0, R, n, (AggSlot<8> *)t->slots, t->cap,
                      (TableSide *)t->side, c->d_ctr, pf, nkeys.as<unsigned long long>(), limit);
        if (keys >= n) break;
        uint64_t got = 0;
        HJ_CUDA(c, cudaMemcpyAsync(&got, nkeys.p, 8, cudaMemcpyDeviceToHost, c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        if (got <= limit) break;
        // more distinct keys than the first table holds: full size
        table_destroy(c, t);
        g.t = t = nullptr;
        keys = n;
    }
    if (width == 4) HJ_TRY(scan_entries(c, AggCnt4{(AggSlot<4> *)t->slots}, AggCnt4{(AggSlot<4> *)t->slots}, t->cap, nullptr));
    else HJ_TRY(scan_entries(c, AggCnt8{(AggSlot<8> *)t->slots}, AggCnt8{(AggSlot<8> *)t->slots}, t->cap, nullptr));
    HJ_TRY(rids.alloc((n ? n : 1) * (uint64_t)width));
    const uint64_t nv = (n + 1) / (width == 4 ? 2 : 1);
    const unsigned grid = (unsigned)std::min<uint64_t>((nv + 255) / 256 + 1, (uint64_t)num_sms(c) * 8);
    if (width == 4)
        HJ_LAUNCH(c, "keylist_scatter", kl_scatter<4>, grid, 256, 0, R, n, (AggSlot<4> *)t->slots, t->cap,
                  (TableSide *)t->side, (uint32_t *)rids.p, c->d_ctr, pf);
    else
        HJ_LAUNCH(c, "keylist_scatter", kl_scatter<8>, grid, 256, 0, R, n, (AggSlot<8> *)t->slots, t->cap,
                  (TableSide *)t->side, (uint64_t *)rids.p, c->d_ctr, pf);
    t->agg = 0;  // a table for pairs, whatever its slots
    t->keylist = 1;
    t->rids = rids.release();
    t->nr = n;
    *out = t;
    g.t = nullptr;
    return HJ_OK;
}

hj_status keylist_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t ns, PartFilter pf, void *pairs,
                        uint64_t pcap, hj_counters *ctr, int chk) {
    if (!ns) return HJ_OK;
    const int W = t->width;
    const void *rids = t->rids;
    const uint64_t nr = t->nr;
    DevBuf big(c), nbig(c), pref(c);
    HJ_TRY(big.alloc(ns * sizeof(Big)));
    HJ_TRY(nbig.alloc(8));
    HJ_CUDA(c, cudaMemsetAsync(nbig.p, 0, 8, c->stream));
    const uint64_t nv = (ns + 1) / (W == 4 ? 2 : 1);
    const unsigned grid = (unsigned)std::min<uint64_t>((nv + 255) / 256 + 1, (uint64_t)num_sms(c) * 8);
    if (W == 4)
        HJ_LAUNCH(c, "keylist_probe", kl_probe<4>, grid, 256, 0, S, ns, (const AggSlot<4> *)t->slots, t->cap,
                  (const TableSide *)t->side, (const uint32_t *)rids, nr, pairs, pcap, ctr, chk, pf, big.as<Big>(),
                  nbig.as<unsigned long long>());
    else
        HJ_LAUNCH(c, "keylist_probe", kl_probe<8>, grid, 256, 0, S, ns, (const AggSlot<8> *)t->slots, t->cap,
                  (const TableSide *)t->side, (const uint64_t *)rids, nr, pairs, pcap, ctr, chk, pf, big.as<Big>(),
                  nbig.as<unsigned long long>());
    uint64_t nb = 0;
    HJ_CUDA(c, cudaMemcpyAsync(&nb, nbig.p, 8, cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!nb) return HJ_OK;
    // heavy hitters: segments of kSegPairs pairs over the whole grid
    HJ_TRY(pref.alloc((nb + 1) * 8));
    uint64_t nseg = 0;
    HJ_TRY(scan_entries(c, SegCnt{big.as<Big>(), pref.as<unsigned long long>()},
                        SegCnt{big.as<Big>(), pref.as<unsigned long long>()}, nb, &nseg));
    const unsigned eg = (unsigned)std::min<uint64_t>(nseg, (uint64_t)num_sms(c) * 8);
    if (W == 4)
        HJ_LAUNCH(c, "keylist_expand", kl_expand<4>, eg, 256, 0, big.as<Big>(), pref.as<unsigned long long>(), nb,
                  nseg, (const uint32_t *)rids, pairs, pcap, ctr, chk);
    else
        HJ_LAUNCH(c, "keylist_expand", kl_expand<8>, eg, 256, 0, big.as<Big>(), pref.as<unsigned long long>(), nb,
                  nseg, (const uint64_t *)rids, pairs, pcap, ctr, chk);
    return HJ_OK;  // the buffers are freed in stream order after the expansion
}

}  // namespace hj
