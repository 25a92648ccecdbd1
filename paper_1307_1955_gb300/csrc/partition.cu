// partition.cu -- radix partitioning, Alg. 2 steps n1-n3.
//
// One pass splits every segment of its input on `bits` bits of the key hash.
// GPU form of "compute partition number / visit partition header / insert into
// partition":
//   1. chunks : each segment is cut into chunks of `chunk` rows, one CTA each;
//   2. hist   : a CTA counts the digits of its chunk in shared memory (n1, n2) and
//               writes them to H in (segment, digit, chunk) order;
//   3. scan   : an exclusive scan of H gives every (segment, digit, chunk) its
//               first output row -- partitions come out contiguous;
//   4. scatter: a CTA re-reads its chunk tile by tile, sorts each tile by digit in
//               shared memory, and writes each digit's run to consecutive rows
//               (n3), so a warp's stores cover a few contiguous runs instead of
//               32 scattered rows.
// The order of tuples inside a partition is not specified.
#include <algorithm>

#include "common.cuh"
#include "engine.cuh"

namespace hj {

// -------------------------------------------------------------------- scan
// Exclusive scan of n uint32 counts into n + 1 uint64 offsets (out[n] = total),
// in three launches: per-block sums, a scan of the sums, per-block scans.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr uint64_t kScanBlock = (uint64_t)kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *in, uint64_t n,
                                                                   unsigned long long *partial) {
    __shared__ unsigned long long sc[33];
    uint64_t base = blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    unsigned long long tot;
    block_exclusive_scan<unsigned long long>(s, sc, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(unsigned long long *partial, uint64_t nb,
                                                                     unsigned long long *total_out) {
    __shared__ unsigned long long sc[33];
    unsigned long long carry = 0;
    for (uint64_t b = 0; b < nb; b += kScanThreads) {
        uint64_t i = b + threadIdx.x;
        unsigned long long v = i < nb ? partial[i] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan<unsigned long long>(v, sc, &tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *in, uint64_t n,
                                                                  const unsigned long long *partial,
                                                                  unsigned long long *out) {
    __shared__ unsigned long long sc[33];
    uint64_t base = blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan<unsigned long long>(s, sc, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
}

static hj_status scan_u32_u64(hj_ctx *c, const uint32_t *in, uint64_t n, unsigned long long *out) {
    uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) nb = 1;
    DevBuf partial(c);
    HJ_TRY(partial.alloc(nb * 8));
    auto *pp = partial.as<unsigned long long>();
    HJ_LAUNCH(c, "scan_reduce", scan_reduce_kernel, (unsigned)nb, kScanThreads, 0, in, n, pp);
    HJ_LAUNCH(c, "scan_partials", scan_partials_kernel, 1, kScanThreads, 0, pp, nb, out + n);
    HJ_LAUNCH(c, "scan_apply", scan_apply_kernel, (unsigned)nb, kScanThreads, 0, in, n, pp, out);
    return HJ_OK;
}

// ------------------------------------------------------------------ chunks
// Number of chunks of every segment (ceil(len / chunk)), scanned afterwards into
// chunk_base[nseg + 1].
__global__ void seg_chunks_kernel(const uint64_t *seg_off, uint64_t nseg, uint64_t chunk, uint32_t *nch) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nseg; s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t len = seg_off[s + 1] - seg_off[s];
        nch[s] = (uint32_t)((len + chunk - 1) / chunk);
    }
}

// Segment that owns global chunk g: the last s with chunk_base[s] <= g.
__device__ __forceinline__ uint64_t seg_of_chunk(const unsigned long long *cb, uint64_t nseg, uint64_t g) {
    uint64_t lo = 0, hi = nseg;  // invariant: cb[lo] <= g < cb[hi]
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (cb[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Warp-aggregated shared-memory increment: lanes with equal digits add once;
// returns this lane's rank among the tuples counted for `d` so far.
__device__ __forceinline__ uint32_t agg_rank(uint32_t *cnt, uint32_t d, bool active) {
    unsigned mask = __ballot_sync(0xffffffffu, active);
    uint32_t rank = 0;
    if (active) {
        unsigned peers = __match_any_sync(mask, d);
        int leader = __ffs(peers) - 1;
        int lane = threadIdx.x & 31;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&cnt[d], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        rank = base + __popc(peers & ((1u << lane) - 1u));
    }
    return rank;
}

template <int W> struct PartShape {
    static constexpr int PV = Tup<W>::kPerVec;
    static constexpr int VPT = 4;             // vectors per thread per tile
    static constexpr int IT = VPT * PV;       // tuples per thread per tile
};

template <int W> __device__ __forceinline__ void load_vec_p(const void *base, uint64_t v, uint64_t n_total,
                                                            typename Tup<W>::U *k, typename Tup<W>::U *r) {
    if constexpr (W == 8) {
        ulonglong2 x = ld_stream((const ulonglong2 *)base + v);
        k[0] = x.x;
        r[0] = x.y;
    } else {
        if (2 * v + 1 < n_total) {
            uint4 x = ld_stream((const uint4 *)base + v);
            k[0] = x.x; r[0] = x.y; k[1] = x.z; r[1] = x.w;
        } else {
            uint2 x = ((const uint2 *)base)[2 * v];
            k[0] = x.x; r[0] = x.y; k[1] = 0; r[1] = 0;
        }
    }
}

// ------------------------------------------------------------------- hist
template <int W>
__global__ void __launch_bounds__(512) hist_kernel(const void *in, uint64_t n_total, const uint64_t *seg_off,
                                                   uint64_t nseg, const unsigned long long *cb, uint64_t chunk,
                                                   int shift, int bits, uint32_t *H) {
    using U = typename Tup<W>::U;
    constexpr int PV = Tup<W>::kPerVec;
    extern __shared__ uint32_t hist[];
    const uint32_t P = 1u << bits;
    const uint64_t g = blockIdx.x;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) hist[d] = 0;
    const uint64_t total = cb[nseg];
    if (g >= total) {  // spare chunk id: its H row lies past every real row
        for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) H[g * P + d] = 0;
        return;
    }
    const uint64_t s = seg_of_chunk(cb, nseg, g);
    const uint64_t cidx = g - cb[s], nch = cb[s + 1] - cb[s];
    const uint64_t lo = seg_off[s] + cidx * chunk;
    const uint64_t hi = min(lo + chunk, (uint64_t)seg_off[s + 1]);
    __syncthreads();
    const uint64_t va = lo / PV, vb = (hi + PV - 1) / PV;
    constexpr int UNR = 4;
    for (uint64_t v0 = va; v0 < vb; v0 += (uint64_t)blockDim.x * UNR) {
        U k[UNR][2], r[UNR][2];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            uint64_t v = v0 + (uint64_t)u * blockDim.x + threadIdx.x;
            k[u][0] = k[u][1] = 0;
            if (v < vb) load_vec_p<W>(in, v, n_total, k[u], r[u]);
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            uint64_t v = v0 + (uint64_t)u * blockDim.x + threadIdx.x;
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                bool act = v < vb && t >= lo && t < hi;
                uint32_t d = digit_of(key_hash<W>(k[u][e]), shift, bits);
                agg_rank(hist, d, act);
            }
        }
    }
    __syncthreads();
    const uint64_t row = cb[s] * P;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) H[row + (uint64_t)d * nch + cidx] = hist[d];
}

__global__ void extract_offsets_kernel(const uint64_t *seg_off, uint64_t nseg, const unsigned long long *cb,
                                       const unsigned long long *Hs, int bits, uint64_t *part_off) {
    const uint64_t P = 1ull << bits, n = nseg * P;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i == n) {
            part_off[i] = seg_off[nseg];
            continue;
        }
        uint64_t s = i >> bits, d = i & (P - 1);
        uint64_t nch = cb[s + 1] - cb[s];
        part_off[i] = nch ? seg_off[0] + Hs[cb[s] * P + d * nch] : seg_off[s];
    }
}

// ----------------------------------------------------------------- scatter
template <int W> struct SortSlot { using T = unsigned long long; };
template <> struct SortSlot<8> { using T = ulonglong2; };

template <int W>
__global__ void __launch_bounds__(512) scatter_kernel(const void *in, uint64_t n_total, const uint64_t *seg_off,
                                                      uint64_t nseg, const unsigned long long *cb, uint64_t chunk,
                                                      int shift, int bits, const unsigned long long *Hs, void *out) {
    using U = typename Tup<W>::U;
    using PS = PartShape<W>;
    using Slot = typename SortSlot<W>::T;
    constexpr int PV = PS::PV, VPT = PS::VPT, IT = PS::IT;
    const uint32_t P = 1u << bits;
    const uint32_t T = blockDim.x * IT;
    extern __shared__ __align__(16) unsigned char smem[];
    Slot *buf = (Slot *)smem;                                        // T tuples
    unsigned long long *gcur = (unsigned long long *)(buf + T);      // P running output rows
    uint32_t *lcnt = (uint32_t *)(gcur + P);                         // P tile counts
    uint32_t *loff = lcnt + P;                                       // P + 1 tile offsets
    uint16_t *dig = (uint16_t *)(loff + P + 1);                      // T digits (sorted order)
    __shared__ uint32_t sc[33];

    const uint64_t g = blockIdx.x;
    if (g >= cb[nseg]) return;
    const uint64_t s = seg_of_chunk(cb, nseg, g);
    const uint64_t cidx = g - cb[s], nch = cb[s + 1] - cb[s];
    const uint64_t lo = seg_off[s] + cidx * chunk;
    const uint64_t hi = min(lo + chunk, (uint64_t)seg_off[s + 1]);
    const uint64_t row = cb[s] * P;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) {
        gcur[d] = seg_off[0] + Hs[row + (uint64_t)d * nch + cidx];
        lcnt[d] = 0;
    }
    __syncthreads();
    const uint32_t ept = (P + blockDim.x - 1) / blockDim.x;  // digits per thread in the tile scan
    const uint64_t va = lo / PV, vb = (hi + PV - 1) / PV;
    const uint64_t tile_vecs = (uint64_t)blockDim.x * VPT;
    for (uint64_t base = va; base < vb; base += tile_vecs) {
        U k[IT], r[IT];
        uint32_t d[IT], rk[IT];
        bool act[IT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            uint64_t v = base + (uint64_t)j * blockDim.x + threadIdx.x;
            U kk[2] = {0, 0}, rr[2] = {0, 0};
            if (v < vb) load_vec_p<W>(in, v, n_total, kk, rr);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                uint64_t t = v * PV + e;
                k[j * PV + e] = kk[e];
                r[j * PV + e] = rr[e];
                act[j * PV + e] = v < vb && t >= lo && t < hi;
            }
        }
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            d[i] = digit_of(key_hash<W>(k[i]), shift, bits);
            rk[i] = agg_rank(lcnt, d[i], act[i]);
        }
        __syncthreads();
        // exclusive scan of the tile's digit counts
        {
            uint32_t d0 = threadIdx.x * ept, sum = 0;
            for (uint32_t q = 0; q < ept; ++q)
                if (d0 + q < P) sum += lcnt[d0 + q];
            uint32_t tot;
            uint32_t ex = block_exclusive_scan<uint32_t>(sum, sc, &tot);
            for (uint32_t q = 0; q < ept; ++q)
                if (d0 + q < P) {
                    loff[d0 + q] = ex;
                    ex += lcnt[d0 + q];
                }
            if (threadIdx.x == 0) loff[P] = tot;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            if (!act[i]) continue;
            uint32_t p = loff[d[i]] + rk[i];
            if constexpr (W == 4) buf[p] = (unsigned long long)k[i] | ((unsigned long long)r[i] << 32);
            else buf[p] = make_ulonglong2(k[i], r[i]);
            dig[p] = (uint16_t)d[i];
        }
        __syncthreads();
        const uint32_t nv = loff[P];
        for (uint32_t p = threadIdx.x; p < nv; p += blockDim.x) {
            uint32_t dd = dig[p];
            uint64_t dst = gcur[dd] + (p - loff[dd]);
            ((Slot *)out)[dst] = buf[p];
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
            gcur[q] += lcnt[q];
            lcnt[q] = 0;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- driver

hj_status partition_pass(hj_ctx *c, int width, const void *in, uint64_t n_total, const uint64_t *seg_off,
                         uint64_t nseg, int shift, int bits, void *out, uint64_t *part_off) {
    if (bits < 1 || bits > 12) return set_err(c, HJ_E_INVALID, "partition pass bits %d outside [1, 12]", bits);
    const uint64_t P = 1ull << bits;
    const int block = 512;
    const uint64_t tile = (uint64_t)block * (width == 4 ? PartShape<4>::IT : PartShape<8>::IT);
    // Chunk size: about two chunks per SM over the whole input, a multiple of the
    // scatter tile, at least one tile.
    uint64_t target = (uint64_t)num_sms(c) * 2;
    uint64_t chunk = (n_total + target - 1) / (target ? target : 1);
    chunk = ((chunk + tile - 1) / tile) * tile;
    if (chunk < tile) chunk = tile;
    const uint64_t max_chunks = (n_total + chunk - 1) / chunk + nseg;

    DevBuf b_nch(c), b_cb(c), b_H(c), b_Hs(c);
    HJ_TRY(b_nch.alloc((nseg + 1) * 4));
    HJ_TRY(b_cb.alloc((nseg + 1) * 8));
    HJ_TRY(b_H.alloc(max_chunks * P * 4));
    HJ_TRY(b_Hs.alloc((max_chunks * P + 1) * 8));
    uint32_t *nch = b_nch.as<uint32_t>(), *H = b_H.as<uint32_t>();
    unsigned long long *cb = b_cb.as<unsigned long long>(), *Hs = b_Hs.as<unsigned long long>();

    int g1 = (int)std::min<uint64_t>((nseg + 255) / 256, 4096);
    HJ_LAUNCH(c, "seg_chunks", seg_chunks_kernel, g1 ? g1 : 1, 256, 0, seg_off, nseg, chunk, nch);
    HJ_TRY(scan_u32_u64(c, nch, nseg, cb));
    size_t hsmem = P * 4;
    if (width == 4)
        HJ_LAUNCH(c, "partition_hist", hist_kernel<4>, (unsigned)max_chunks, block, hsmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, H);
    else
        HJ_LAUNCH(c, "partition_hist", hist_kernel<8>, (unsigned)max_chunks, block, hsmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, H);
    HJ_TRY(scan_u32_u64(c, H, max_chunks * P, Hs));
    {
        uint64_t n = nseg * P + 1;
        int g = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms(c) * 8);
        HJ_LAUNCH(c, "partition_offsets", extract_offsets_kernel, g, 256, 0, seg_off, nseg, cb, Hs, bits, part_off);
    }
    size_t slot = width == 4 ? 8 : 16;
    size_t ssmem = tile * slot + P * 8 + P * 4 + (P + 1) * 4 + tile * 2;
    ssmem = (ssmem + 15) & ~size_t(15);
    if (width == 4) {
        HJ_CUDA(c, cudaFuncSetAttribute(scatter_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
        HJ_LAUNCH(c, "partition_scatter", scatter_kernel<4>, (unsigned)max_chunks, block, ssmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, Hs, out);
    } else {
        HJ_CUDA(c, cudaFuncSetAttribute(scatter_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
        HJ_LAUNCH(c, "partition_scatter", scatter_kernel<8>, (unsigned)max_chunks, block, ssmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, Hs, out);
    }
    return HJ_OK;
}

}  // namespace hj
