// emit.cuh -- dense output of join pairs with few global atomics.
//
// GPU form of the block allocator of Sec. 3.3 (a work group takes a block from a
// global pointer, its threads sub-allocate from the block): here every WARP takes
// a chunk of kChunkPairs output slots from the global cursor with one atomicAdd
// and appends the pairs its lanes find with ballot/popc offsets -- no block-wide
// barrier, one global atomic per kChunkPairs pairs.  A warp's last chunk is
// usually partly filled; the warp records (base, used) so that a small device-side
// move of pairs from the tail into those holes makes pairs[0, count) dense.
#pragma once

#include "common.cuh"
#include "ctx.cuh"

namespace hj {

constexpr unsigned kChunkPairs = 1024;

struct ChunkRec {
    unsigned long long base;
    unsigned int used;
    unsigned int join;
};

// Where the warps of one launch record their partly filled chunks.
struct RecArea {
    unsigned long long *n;  // number of records written
    ChunkRec *rec;
    unsigned long long cap;
};

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

// Output context of a launch: the pair buffer of one join and its counters.  With
// `dense`, every append claims exactly its pairs from ctr->count (no chunks, no
// holes).  With `stage` (this warp's shared-memory buffer of `scap` pairs), a warp
// collects its pairs there and claims exactly as many rows of ctr->count when the
// buffer fills or the warp is done, then copies them out with coalesced stores:
// no holes either, one atomic per buffer.  Otherwise warps take whole chunks from
// ctr->cursor.
struct OutCtx {
    void *pairs;
    uint64_t pcap;
    hj_counters *ctr;
    unsigned int join = 0;
    bool dense = false;
    void *stage = nullptr;
    unsigned scap = 0;
};

// Warp-uniform state of a warp's current chunk.
struct OutState {
    unsigned long long base = 0;
    unsigned used = kChunkPairs;  // no chunk open yet
    bool claimed = false;
    unsigned long long pairs = 0;
};

template <int W> struct PairVec { using T = uint2; };
template <> struct PairVec<8> { using T = ulonglong2; };

// Staged output: claim rows for the st.used pairs in the warp's buffer and copy
// them out (pairs past the capacity are dropped; the count stays exact).  All 32
// lanes must call.
template <int W> __device__ __forceinline__ void warp_stage_flush(OutState &st, const OutCtx &oc) {
    using P = typename PairVec<W>::T;
    const unsigned n = st.used;
    if (!n) return;
    __syncwarp();  // the buffer's stores are visible to every lane
    const unsigned lane = threadIdx.x & 31;
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(&oc.ctr->count, (unsigned long long)n);
    b = __shfl_sync(0xffffffffu, b, 0);
    const P *sp = (const P *)oc.stage;
    P *out = (P *)oc.pairs;
    for (unsigned i = lane; i < n; i += 32)
        if (b + i < oc.pcap) out[b + i] = sp[i];
    __syncwarp();  // read before the buffer is refilled
    st.used = 0;
}

// Append one pair per lane whose `has` is set.  All 32 lanes must call.
template <int W>
__device__ __forceinline__ void warp_append(OutState &st, const OutCtx &oc, bool has, typename Tup<W>::U a,
                                            typename Tup<W>::U b_) {
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (!mask) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned k = __popc(mask);
    const unsigned rank = __popc(mask & ((1u << lane) - 1u));
    if (oc.stage) {  // (k <= 32 <= scap: one flush makes room)
        if (st.used + k > oc.scap) warp_stage_flush<W>(st, oc);
        using P = typename PairVec<W>::T;
        if (has) {
            if constexpr (W == 4) ((P *)oc.stage)[st.used + rank] = make_uint2(a, b_);
            else ((P *)oc.stage)[st.used + rank] = make_ulonglong2(a, b_);
        }
        st.used += k;
        return;
    }
    if (oc.dense) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&oc.ctr->count, (unsigned long long)k);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (has && b + rank < oc.pcap) PairOut<W>::put(oc.pairs, b + rank, a, b_);
        return;
    }
    const unsigned room = kChunkPairs - st.used;
    unsigned long long nb = 0;
    if (k > room) {
        if (lane == 0) nb = atomicAdd(&oc.ctr->cursor, (unsigned long long)kChunkPairs);
        nb = __shfl_sync(0xffffffffu, nb, 0);
    }
    if (has) {
        unsigned long long pos = rank < room ? st.base + st.used + rank : nb + (rank - room);
        if (pos < oc.pcap) PairOut<W>::put(oc.pairs, pos, a, b_);
    }
    if (k > room) {
        st.base = nb;
        st.used = k - room;
        st.claimed = true;
    } else {
        st.used += k;
    }
    st.pairs += k;
}

// Record the warp's partly filled chunk and add its pair count.  All lanes call.
__device__ __forceinline__ void warp_finish(const OutState &st, const OutCtx &oc, const RecArea &ra) {
    if ((threadIdx.x & 31) != 0) return;
    if (oc.dense || oc.stage) return;  // exact claims count themselves and leave no holes
    if (st.claimed && st.used < kChunkPairs) {
        unsigned long long i = atomicAdd(ra.n, 1ull);
        if (i < ra.cap) {
            ra.rec[i].base = st.base;
            ra.rec[i].used = st.used;
            ra.rec[i].join = oc.join;
        } else {
            atomicOr(&oc.ctr->status, (unsigned long long)kStatusRecords);
        }
    }
    if (st.pairs) atomicAdd(&oc.ctr->count, st.pairs);
}

}  // namespace hj
