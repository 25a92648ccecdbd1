// output.cu -- the pair buffer of a materialising join and its final compaction.
//
// Warps fill whole chunks of kChunkPairs slots (emit.cuh); each warp's last chunk
// is usually partly used.  After the join kernels finish, two small kernels make
// pairs[0, count) dense without a round trip to the host: one CTA reads the
// recorded partial chunks, lists the holes below `count` and the valid runs at or
// above `count` with prefix sums over both lists, and a warp per hole then moves
// the matching tail pairs into it.  The moved volume is at most one chunk per
// warp.  Both kernels read count and cursor from the device counters, and leave
// the buffer untouched when the cursor ran past the capacity (the caller then runs
// the join again with a larger buffer).
#include <memory>
#include <vector>

#include "emit.cuh"
#include "engine.cuh"

namespace hj {

// Scratch of the device-side compaction, after the records of an area:
// [plan][tail_used: cap + 2][dst_start, dst_pref: cap + 1 each][src_start, src_pref: cap + 3 each]
struct CompactPlan {
    unsigned long long ndst, nsrc, total, pad;
};

static uint64_t area_bytes(uint64_t warps) {
    return 16 + warps * sizeof(ChunkRec) + sizeof(CompactPlan) + (warps + 2) * 4 + 8 /*align*/ +
           2 * (warps + 1) * 8 + 2 * (warps + 3) * 8;
}

struct PlanView {
    CompactPlan *plan;
    uint32_t *tail_used;
    unsigned long long *dst_start, *dst_pref, *src_start, *src_pref;
};

__host__ __device__ inline PlanView plan_view(void *area, uint64_t warps) {
    char *p = (char *)area + 16 + warps * sizeof(ChunkRec);
    PlanView v;
    v.plan = (CompactPlan *)p;
    p += sizeof(CompactPlan);
    v.tail_used = (uint32_t *)p;
    p += ((warps + 2) * 4 + 7) / 8 * 8;
    v.dst_start = (unsigned long long *)p;
    v.dst_pref = v.dst_start + (warps + 1);
    v.src_start = v.dst_pref + (warps + 1);
    v.src_pref = v.src_start + (warps + 3);
    return v;
}

// Block-wide exclusive scan of 64-bit values (1024 threads at most); *total gets the sum.
__device__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *sh, unsigned long long *total) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        if (lane < nw) sh[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const unsigned long long before = warp ? sh[warp - 1] : 0ull;
    *total = sh[nw - 1];
    __syncthreads();
    return before + x - v;
}

// Records (or tail chunks) per thread and step of the plan: each thread loads its
// kPlanPer entries at once, so a list of up to 1024 * kPlanPer entries takes one
// block scan.
constexpr int kPlanPer = 4;

__global__ void __launch_bounds__(1024) compact_plan_kernel(const unsigned long long *nrec_p, const ChunkRec *rec,
                                                            uint64_t cap, hj_counters *ctr, uint64_t pcap,
                                                            PlanView pv) {
    __shared__ unsigned long long sh[32];
    const unsigned long long count = ctr->count, cursor = ctr->cursor;
    if (cursor > pcap || count >= cursor) {
        if (threadIdx.x == 0) pv.plan->ndst = pv.plan->total = 0;
        return;
    }
    const uint64_t n = *nrec_p < cap ? *nrec_p : cap;
    const uint64_t tb = count / kChunkPairs, nt = (cursor + kChunkPairs - 1) / kChunkPairs - tb;  // nt <= n + 2
    for (uint64_t t = threadIdx.x; t < nt; t += blockDim.x) pv.tail_used[t] = kChunkPairs;
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t ci = rec[i].base / kChunkPairs;
        if (ci >= tb && ci < tb + nt) pv.tail_used[ci - tb] = rec[i].used;
    }
    __syncthreads();
    const uint64_t step = (uint64_t)blockDim.x * kPlanPer;
    // holes below count, in record order (thread t holds records t*kPlanPer ...)
    unsigned long long nd = 0, dp = 0;
    for (uint64_t b = 0; b < n; b += step) {
        unsigned long long s0[kPlanPer], len[kPlanPer], f = 0, l = 0;
#pragma unroll
        for (int q = 0; q < kPlanPer; ++q) {
            const uint64_t i = b + (uint64_t)threadIdx.x * kPlanPer + q;
            s0[q] = len[q] = 0;
            if (i < n) {
                const ChunkRec r = rec[i];
                s0[q] = r.base + r.used;
                const unsigned long long e = r.base + kChunkPairs < count ? r.base + kChunkPairs : count;
                len[q] = s0[q] < e ? e - s0[q] : 0ull;
            }
            f += len[q] ? 1ull : 0ull;
            l += len[q];
        }
        unsigned long long tf, tl;
        unsigned long long xf = block_scan_u64(f, sh, &tf);
        unsigned long long xl = block_scan_u64(l, sh, &tl);
#pragma unroll
        for (int q = 0; q < kPlanPer; ++q) {
            if (len[q]) {
                pv.dst_start[nd + xf] = s0[q];
                pv.dst_pref[nd + xf] = dp + xl;
                ++xf;
                xl += len[q];
            }
        }
        nd += tf;
        dp += tl;
    }
    // valid runs of the tail chunks, in address order
    unsigned long long ns = 0, sp = 0;
    for (uint64_t b = 0; b < nt; b += step) {
        unsigned long long a[kPlanPer], len[kPlanPer], f = 0, l = 0;
#pragma unroll
        for (int q = 0; q < kPlanPer; ++q) {
            const uint64_t t = b + (uint64_t)threadIdx.x * kPlanPer + q;
            a[q] = len[q] = 0;
            if (t < nt) {
                const unsigned long long cb = (tb + t) * kChunkPairs, ce = cb + pv.tail_used[t];
                a[q] = cb > count ? cb : count;
                const unsigned long long e = ce < cursor ? ce : cursor;
                len[q] = a[q] < e ? e - a[q] : 0ull;
            }
            f += len[q] ? 1ull : 0ull;
            l += len[q];
        }
        unsigned long long tf, tl;
        unsigned long long xf = block_scan_u64(f, sh, &tf);
        unsigned long long xl = block_scan_u64(l, sh, &tl);
#pragma unroll
        for (int q = 0; q < kPlanPer; ++q) {
            if (len[q]) {
                pv.src_start[ns + xf] = a[q];
                pv.src_pref[ns + xf] = sp + xl;
                ++xf;
                xl += len[q];
            }
        }
        ns += tf;
        sp += tl;
    }
    if (threadIdx.x == 0) {
        pv.dst_pref[nd] = dp;
        pv.src_pref[ns] = sp;
        if (dp != sp) {  // the holes must take exactly the tail's pairs
            atomicOr(&ctr->status, (unsigned long long)kStatusCompact);
            nd = 0;
        }
        pv.plan->ndst = nd;
        pv.plan->nsrc = ns;
        pv.plan->total = dp;
    }
}

// Pairs moved by a warp per step of its copy loop, per lane.
constexpr unsigned kMoveUnroll = 4;

template <class P>
__global__ void compact_move_kernel(P *pairs, PlanView pv) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t nd = pv.plan->ndst, ns = pv.plan->nsrc;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = w0; i < nd; i += nw) {
        const unsigned long long ds = pv.dst_start[i], m0 = pv.dst_pref[i], m1 = pv.dst_pref[i + 1];
        // the source run holding move index m0: the last t with src_pref[t] <= m0
        // (src_pref is strictly increasing, src_pref[ns] = the total > m0).  Each
        // round the lanes test 32 evenly spaced pivots strictly inside (lo, hi):
        // the largest with src_pref <= m0 becomes lo, the smallest above m0 becomes
        // hi.  Lane 31's pivot lo + floor(32 (hi - lo) / 33) is inside whenever
        // hi - lo >= 2, so every round shrinks the interval (about 33x).
        uint64_t lo = 0, hi = ns;
        for (int it = 0; it < 64 && hi - lo > 1; ++it) {
            const uint64_t piv = lo + ((hi - lo) * (lane + 1)) / 33;
            const bool in = piv > lo && piv < hi;
            const bool le = in && pv.src_pref[piv] <= m0;
            const unsigned ml = __ballot_sync(0xffffffffu, le), mg = __ballot_sync(0xffffffffu, in && !le);
            const uint64_t nlo = ml ? __shfl_sync(0xffffffffu, piv, 31 - __clz(ml)) : lo;
            const uint64_t nhi = mg ? __shfl_sync(0xffffffffu, piv, __ffs(mg) - 1) : hi;
            lo = nlo;
            hi = nhi;
        }
        unsigned long long m = m0;
        for (uint64_t t = lo; m < m1 && t < ns; ++t) {
            const unsigned long long o = m - pv.src_pref[t], avail = pv.src_pref[t + 1] - m;
            const unsigned long long k = avail < m1 - m ? avail : m1 - m;
            const unsigned long long src = pv.src_start[t] + o, dst = ds + (m - m0);
            for (unsigned long long j = lane; j < k; j += 32 * kMoveUnroll) {
                P v[kMoveUnroll];
#pragma unroll
                for (unsigned u = 0; u < kMoveUnroll; ++u)
                    if (j + 32 * u < k) v[u] = pairs[src + j + 32 * u];
#pragma unroll
                for (unsigned u = 0; u < kMoveUnroll; ++u)
                    if (j + 32 * u < k) pairs[dst + j + 32 * u] = v[u];
            }
            m += k;
        }
    }
}

hj_status PairSink::reset(uint64_t cap_pairs) {
    areas.clear();
    caps.clear();
    pcap = cap_pairs ? cap_pairs : 1;
    return pairs.alloc(pcap * 2ull * width);
}

hj_status PairSink::grow(uint64_t cap_pairs, uint64_t keep) {
    DevBuf nb(c);
    HJ_TRY(nb.alloc(cap_pairs * 2ull * width));
    if (keep)
        HJ_CUDA(c, cudaMemcpyAsync(nb.p, pairs.p, keep * 2ull * width, cudaMemcpyDeviceToDevice, c->stream));
    pairs.reset();
    pairs.p = nb.release();
    pcap = cap_pairs;
    return HJ_OK;
}

hj_status PairSink::new_area(uint64_t warps, RecArea *ra) {
    auto b = std::make_unique<DevBuf>(c);
    HJ_TRY(b->alloc(area_bytes(warps)));
    HJ_CUDA(c, cudaMemsetAsync(b->p, 0, 16, c->stream));
    ra->n = (unsigned long long *)b->p;
    ra->rec = (ChunkRec *)((char *)b->p + 16);
    ra->cap = warps;
    areas.push_back(std::move(b));
    caps.push_back(warps);
    return HJ_OK;
}

hj_status PairSink::finalize_device(hj_counters *ctr) {
    if (areas.size() != 1) return set_err(c, HJ_E_CUDA, "device compaction takes one record area");
    void *a = areas[0]->p;
    const uint64_t warps = caps[0];
    const PlanView pv = plan_view(a, warps);
    HJ_LAUNCH(c, "pairs_plan", compact_plan_kernel, 1, 1024, 0, (const unsigned long long *)a,
              (const ChunkRec *)((char *)a + 16), warps, ctr, pcap, pv);
    const unsigned grid = (unsigned)num_sms(c) * 4;
    if (width == 4)
        HJ_LAUNCH(c, "pairs_compact", compact_move_kernel<uint2>, grid, 256, 0, (uint2 *)pairs.p, pv);
    else
        HJ_LAUNCH(c, "pairs_compact", compact_move_kernel<ulonglong2>, grid, 256, 0, (ulonglong2 *)pairs.p, pv);
    return HJ_OK;
}

}  // namespace hj
