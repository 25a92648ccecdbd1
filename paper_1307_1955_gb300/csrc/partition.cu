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

hj_status scan_counts(hj_ctx *c, const uint32_t *in, uint64_t n, unsigned long long *out) {
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

// chunk_base of a single segment: {0, ceil(len / chunk)} in one launch.
__global__ void one_seg_chunks_kernel(const uint64_t *seg_off, uint64_t chunk, unsigned long long *cb) {
    cb[0] = 0;
    cb[1] = (seg_off[1] - seg_off[0] + chunk - 1) / chunk;
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

// Shared-memory increment of digit d's counter; returns this tuple's rank among
// the tuples of digit d counted so far (order among equal digits is free).
__device__ __forceinline__ uint32_t digit_rank(uint32_t *cnt, uint32_t d, bool active) {
    return active ? atomicAdd(&cnt[d], 1u) : 0u;
}

// Tuples of W-byte fields per 32-byte sector: the unit the scatter writes whole.
template <int W> struct Sector {
    static constexpr int kTuples = 32 / (2 * W);
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

// Chunk g of the pass: its segment, index within the segment, and row range.
struct ChunkPos {
    uint64_t s, cidx, nch, lo, hi;
};
__device__ __forceinline__ ChunkPos chunk_pos(const uint64_t *seg_off, uint64_t nseg, const unsigned long long *cb,
                                              uint64_t chunk, uint64_t g) {
    ChunkPos c;
    c.s = seg_of_chunk(cb, nseg, g);
    c.cidx = g - cb[c.s];
    c.nch = cb[c.s + 1] - cb[c.s];
    c.lo = seg_off[c.s] + c.cidx * chunk;
    c.hi = min(c.lo + chunk, (uint64_t)seg_off[c.s + 1]);
    return c;
}

// ------------------------------------------------------------------- hist
// Counts per (chunk, digit); with `pad` each count is rounded up to whole sectors
// so that every (chunk, digit) run of the scatter starts on a sector boundary.
constexpr int kHistThreads = 1024;
constexpr int kHistUnroll = 4;

template <int W>
__global__ void __launch_bounds__(kHistThreads) hist_kernel(const void *in, uint64_t n_total, const uint64_t *seg_off,
                                                            uint64_t nseg, const unsigned long long *cb,
                                                            uint64_t chunk, int shift, int bits, int pad,
                                                            uint32_t *H, const void *const *seg_ptrs) {
    using U = typename Tup<W>::U;
    constexpr int PV = Tup<W>::kPerVec, SV = Sector<W>::kTuples;
    extern __shared__ uint32_t hist[];
    const uint32_t P = 1u << bits;
    const uint64_t g = blockIdx.x;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) hist[d] = 0;
    if (g >= cb[nseg]) {  // spare chunk id: its H row lies past every real row
        for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) H[g * P + d] = 0;
        return;
    }
    const ChunkPos cp = chunk_pos(seg_off, nseg, cb, chunk, g);
    // tuples come from `in` (global row index), or from the segment's own array
    const void *src = seg_ptrs ? seg_ptrs[cp.s] : in;
    const uint64_t ioff = seg_ptrs ? seg_off[cp.s] : 0;
    const uint64_t lo = cp.lo - ioff, hi = cp.hi - ioff;
    __syncthreads();
    // whole vectors of the chunk: no per-tuple range tests, 32-bit indices
    const uint64_t va = (lo + PV - 1) / PV, vb = hi / PV;
    using Vec = typename Tup<W>::Vec;
    const Vec *vp = (const Vec *)src + va;
    const uint32_t nv = vb > va ? (uint32_t)(vb - va) : 0u;
    for (uint32_t v0 = 0; v0 < nv; v0 += blockDim.x * kHistUnroll) {
        Vec x[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const uint32_t v = v0 + (uint32_t)u * blockDim.x + threadIdx.x;
            if (v < nv) x[u] = ld_stream(vp + v);
        }
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const uint32_t v = v0 + (uint32_t)u * blockDim.x + threadIdx.x;
            if (v < nv) {
                if constexpr (W == 4) {
                    atomicAdd(&hist[digit_of(key_hash<W>(x[u].x), shift, bits)], 1u);
                    atomicAdd(&hist[digit_of(key_hash<W>(x[u].z), shift, bits)], 1u);
                } else {
                    atomicAdd(&hist[digit_of(key_hash<W>(x[u].x), shift, bits)], 1u);
                }
            }
        }
    }
    // rows of a 4-byte relation outside whole vectors: [lo, min(2 va, hi)) and
    // [2 max(va, vb), hi), at most one row each
    if constexpr (W == 4) {
        if (threadIdx.x == 0) {
            const uint32_t *t32 = (const uint32_t *)src;
            const uint64_t f1 = PV * va < hi ? PV * va : hi, b0 = PV * (va > vb ? va : vb);
            for (uint64_t t = lo; t < f1; ++t) atomicAdd(&hist[digit_of(key_hash<W>(t32[2 * t]), shift, bits)], 1u);
            for (uint64_t t = b0; t < hi; ++t) atomicAdd(&hist[digit_of(key_hash<W>(t32[2 * t]), shift, bits)], 1u);
        }
    }
    __syncthreads();
    const uint64_t row = cb[cp.s] * P;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) {
        uint32_t n = hist[d];
        if (pad) n = (n + SV - 1) / SV * SV;
        H[row + (uint64_t)d * cp.nch + cp.cidx] = n;
    }
}

__global__ void extract_offsets_kernel(const uint64_t *seg_off, uint64_t nseg, const unsigned long long *cb,
                                       const unsigned long long *Hs, int bits, uint64_t *part_off,
                                       uint64_t total_rows_plus_base) {
    const uint64_t P = 1ull << bits, n = nseg * P;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i == n) {
            part_off[i] = total_rows_plus_base ? seg_off[0] + Hs[cb[nseg] * P] : seg_off[nseg];
            continue;
        }
        uint64_t s = i >> bits, d = i & (P - 1);
        uint64_t nch = cb[s + 1] - cb[s];
        // an empty segment starts where the padded output of the segments before it ends
        part_off[i] = seg_off[0] + (nch ? Hs[cb[s] * P + d * nch] : Hs[cb[s] * P]);
    }
}

// ------------------------------------------------- run positions of a chunk
// Where a padded scatter CTA writes.  General form: the pass's segments, chunks and
// the exclusive scan Hs of the counts in (segment, digit, chunk) order.  Single-
// segment form (H1 set; the first pass of a join): rows [0, n1) in nch1 chunks;
// H1[g * P + d] is chunk g's padded count of digit d and base1[g * P + d] the row
// of its run among digit d's runs (taken with one atomic add on the digit's total
// T1[d] when the histogram was made, so runs of a digit follow in the order the
// chunks finished counting: the order of tuples inside a partition is free).
struct RunGeom {
    const uint64_t *seg_off;
    uint64_t nseg;
    const unsigned long long *cb, *Hs;
    const uint32_t *H1, *base1, *T1;
    uint64_t n1, nch1;
    uint64_t *part_off;  // single-segment form: partition offsets, written by chunk 0
};

// Chunk position and run bounds of scatter CTA g: run_lo[d] / run_hi[d] are the
// rows of its digit-d run relative to the returned output base.  False when g has
// no chunk (or, general form, the pass's output does not start on a sector).  All
// NT threads of the CTA call it (the single-segment form scans the digit totals).
template <uint32_t P, int NT>
__device__ __forceinline__ bool chunk_runs(const RunGeom &rg, uint64_t chunk, uint64_t g, uint32_t SV, ChunkPos *cp,
                                           uint64_t *obase, uint32_t *run_lo, uint32_t *run_hi,
                                           unsigned long long *fault) {
    if (!rg.H1) {
        if (g >= rg.cb[rg.nseg]) return false;
        // runs start on whole sectors only if the pass's first output row does (the
        // padded counts are whole sectors): otherwise the sector stores would be
        // misaligned, so refuse the input
        if (rg.seg_off[0] % SV) {
            if (threadIdx.x == 0) atomicOr(fault, (unsigned long long)kStatusBadInput);
            return false;
        }
        *cp = chunk_pos(rg.seg_off, rg.nseg, rg.cb, chunk, g);
        const uint64_t row = rg.cb[cp->s] * P;
        *obase = (rg.seg_off[0] + rg.Hs[row]) / SV * SV;
        for (uint32_t d = threadIdx.x; d < P; d += NT) {
            // the run of (this chunk, d) is [Hs[i], Hs[i + 1]): the scan is in
            // (digit, chunk) order, so the next entry starts the next run of the pass
            const uint64_t i = row + (uint64_t)d * cp->nch + cp->cidx;
            run_lo[d] = (uint32_t)(rg.seg_off[0] + rg.Hs[i] - *obase);
            run_hi[d] = (uint32_t)(rg.seg_off[0] + rg.Hs[i + 1] - *obase);
        }
        return true;
    }
    if (g >= rg.nch1) return false;
    cp->s = 0;
    cp->cidx = g;
    cp->nch = rg.nch1;
    cp->lo = g * chunk;
    cp->hi = min(cp->lo + chunk, rg.n1);
    *obase = 0;
    // digit d's partition starts at the sum of the padded totals of digits < d
    __shared__ unsigned long long sc[33];
    constexpr uint32_t PER = (P + NT - 1) / NT;  // digits per thread, consecutive
    unsigned long long v[PER], sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < PER; ++q) {
        const uint32_t d = threadIdx.x * PER + q;
        v[q] = d < P ? rg.T1[d] : 0u;
        sum += v[q];
    }
    unsigned long long tot;
    unsigned long long at = block_exclusive_scan<unsigned long long>(sum, sc, &tot);
#pragma unroll
    for (uint32_t q = 0; q < PER; ++q) {
        const uint32_t d = threadIdx.x * PER + q;
        if (d < P) {
            const uint64_t i = g * P + d;
            run_lo[d] = (uint32_t)(at + rg.base1[i]);
            run_hi[d] = run_lo[d] + rg.H1[i];
            if (g == 0) rg.part_off[d] = at;
        }
        at += v[q];
    }
    if (g == 0 && threadIdx.x == 0) rg.part_off[P] = tot;
    return true;
}

// Histogram of the single-segment form: chunk g of rows [0, n) counts its digits
// (pass one: the low `bits` bits of the hash), rounds each count up to whole
// sectors, writes it to H1[g * P + d] and takes the rows of its run among the
// digit's runs with one atomic add on the digit's total T1[d] (zero beforehand).
template <int W>
__global__ void __launch_bounds__(kHistThreads) hist1_kernel(const void *in, uint64_t n, uint64_t chunk, int bits,
                                                             uint32_t *H1, uint32_t *base1, uint32_t *T1) {
    using Vec = typename Tup<W>::Vec;
    constexpr int PV = Tup<W>::kPerVec, SV = Sector<W>::kTuples;
    extern __shared__ uint32_t hist[];
    const uint32_t P = 1u << bits;
    const uint64_t g = blockIdx.x, lo = g * chunk, hi = min(lo + chunk, n);
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    // chunks start on whole vectors; a 4-byte relation's odd last row is read alone
    const Vec *vp = (const Vec *)in + lo / PV;
    const uint32_t nv = (uint32_t)((hi - lo) / PV);
    for (uint32_t v0 = 0; v0 < nv; v0 += blockDim.x * kHistUnroll) {
        Vec x[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const uint32_t v = v0 + (uint32_t)u * blockDim.x + threadIdx.x;
            if (v < nv) x[u] = ld_stream(vp + v);
        }
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const uint32_t v = v0 + (uint32_t)u * blockDim.x + threadIdx.x;
            if (v < nv) {
                atomicAdd(&hist[digit_of(key_hash<W>(x[u].x), 0, bits)], 1u);
                if constexpr (W == 4) atomicAdd(&hist[digit_of(key_hash<W>(x[u].z), 0, bits)], 1u);
            }
        }
    }
    if constexpr (W == 4) {
        if (threadIdx.x == 0 && (hi - lo) % 2) {
            const uint32_t k = ((const uint32_t *)in)[2 * (hi - 1)];
            atomicAdd(&hist[digit_of(key_hash<W>(k), 0, bits)], 1u);
        }
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) {
        const uint32_t c = (hist[d] + SV - 1) / SV * SV;
        H1[g * P + d] = c;
        base1[g * P + d] = c ? atomicAdd(&T1[d], c) : 0u;
    }
}

// ----------------------------------------------------------------- scatter
// One CTA per chunk.  Tile by tile (the next tile's vectors are loaded before the
// current one is processed):
//   1. digit of every tuple, its rank within the digit (shared-memory atomics);
//   2. per digit: the tile count n, the carried count c (tuples of earlier tiles
//      short of a whole sector), and the rows [gcur, bnd) that now complete whole
//      sectors; one block scan gives both the tile offsets and a list of
//      "units" -- the 32-byte output sectors to write this tile;
//   3. tuples placed in a digit-sorted shared buffer;
//   4. one thread per unit gathers its sector (carry first, then tile tuples) and
//      writes it with a single 32-byte store;
//   5. tuples past the last whole sector become the digit's new carry.
// Every global write is therefore a whole sector written by one instruction,
// except the first sector of a run that starts unaligned.  With `pad`, runs start
// aligned and each run's last sector is completed with padding tuples whose key
// hashes to another digit, so all writes are whole sectors.
template <int W> struct SortSlot { using T = unsigned long long; };
template <> struct SortSlot<8> { using T = ulonglong2; };

// NT threads, VPT 16-byte vectors per thread per tile.
template <int W, int NT, int VPT_> struct ScatterShape {
    static constexpr int PV = Tup<W>::kPerVec;
    static constexpr int VPT = VPT_;
    static constexpr int IT = VPT * PV;           // tuples per thread per tile
    static constexpr int T = NT * IT;             // tuples per tile
    static constexpr int SV = Sector<W>::kTuples;
};

template <int W, int NT, int VPT>
__host__ __device__ inline size_t scatter_smem_bytes(uint32_t P) {
    using SS = ScatterShape<W, NT, VPT>;
    size_t slot = 2 * W;
    size_t b = (size_t)SS::T * slot                 // buf: the digit-sorted tile
               + (size_t)P * (SS::SV - 1) * slot    // carry: tuples short of a sector
               + (size_t)P * 4                      // gcur: next output row per digit (segment-relative)
               + (size_t)P * 4                      // lcnt: tile count per digit
               + (size_t)P * 4                      // oc: o | c_old << 16 per digit
               + ((size_t)P + 1) * 2                // loff: tile offset per digit
               + (size_t)P * 2                      // uoff: first unit per digit
               + ((size_t)SS::T / SS::SV + 2 * (size_t)P) * 2   // udig: digit of each unit
               + (size_t)P;                         // ccount: carried tuples per digit
    return (b + 15) & ~size_t(15);
}

// Whole-sector store: 32 bytes from one thread.
__device__ __forceinline__ void st_sector(void *p, const unsigned long long *t4) {
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(t4[0]), "l"(t4[1]), "l"(t4[2]),
                 "l"(t4[3])
                 : "memory");
}

template <int W, int NT, int VPT_>
__global__ void __launch_bounds__(NT) scatter_kernel(const void *in, uint64_t n_total,
                                                                  const uint64_t *seg_off, uint64_t nseg,
                                                                  const unsigned long long *cb, uint64_t chunk,
                                                                  int shift, int bits, const unsigned long long *Hs,
                                                                  void *out, int pad, uint64_t sent_k0,
                                                                  uint64_t sent_k1) {
    using U = typename Tup<W>::U;
    using SS = ScatterShape<W, NT, VPT_>;
    using Slot = typename SortSlot<W>::T;
    constexpr int PV = SS::PV, VPT = SS::VPT, IT = SS::IT, SV = SS::SV;
    const uint32_t P = 1u << bits;
    extern __shared__ __align__(16) unsigned char smem[];
    Slot *buf = (Slot *)smem;                                          // T
    Slot *carry = buf + SS::T;                                         // P * (SV - 1)
    uint32_t *gcur = (uint32_t *)(carry + (size_t)P * (SV - 1));       // P
    uint32_t *lcnt = gcur + P;                                         // P
    uint32_t *oc = lcnt + P;                                           // P
    uint16_t *loff = (uint16_t *)(oc + P);                             // P + 1
    uint16_t *uoff = loff + P + 1;                                     // P
    uint16_t *udig = uoff + P;                                         // T / SV + P
    uint8_t *ccount = (uint8_t *)(udig + SS::T / SV + 2 * P);          // P
    __shared__ uint32_t sc[33];
    __shared__ uint32_t s_nunits;

    const uint64_t g = blockIdx.x;
    if (g >= cb[nseg]) return;
    const ChunkPos cp = chunk_pos(seg_off, nseg, cb, chunk, g);
    const uint64_t row = cb[cp.s] * P;
    // Cursors are kept relative to `obase`, the segment's first output row rounded
    // down to a sector, so that sector boundaries are the same absolute and relative.
    const uint64_t seg_start = seg_off[0] + Hs[row];
    const uint64_t obase = seg_start / SV * SV;
    Slot *outp = (Slot *)out + obase;
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) {
        gcur[d] = (uint32_t)(seg_off[0] + Hs[row + (uint64_t)d * cp.nch + cp.cidx] - obase);
        lcnt[d] = 0;
        ccount[d] = 0;
    }
    __syncthreads();
    const uint32_t ept = (P + blockDim.x - 1) / blockDim.x;
    const uint64_t va = cp.lo / PV, vb = (cp.hi + PV - 1) / PV;
    const uint64_t tile_vecs = (uint64_t)blockDim.x * VPT;

    U k[IT], r[IT], nk[IT], nr[IT];
    auto load_tile = [&](uint64_t base, U *kk, U *rr) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            uint64_t v = base + (uint64_t)j * blockDim.x + threadIdx.x;
            U a[2] = {0, 0}, b[2] = {0, 0};
            if (v < vb) load_vec_p<W>(in, v, n_total, a, b);
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                kk[j * PV + e] = a[e];
                rr[j * PV + e] = b[e];
            }
        }
    };
    if (va < vb) load_tile(va, k, r);
    for (uint64_t base = va; base < vb; base += tile_vecs) {
        if (base + tile_vecs < vb) load_tile(base + tile_vecs, nk, nr);
        // 1. digits and ranks
        uint32_t d[IT], rk[IT];
        bool act[IT];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                const int i = j * PV + e;
                const uint64_t v = base + (uint64_t)j * blockDim.x + threadIdx.x;
                const uint64_t t = v * PV + e;
                act[i] = v < vb && t >= cp.lo && t < cp.hi;
                d[i] = digit_of(key_hash<W>(k[i]), shift, bits);
                rk[i] = act[i] ? atomicAdd(&lcnt[d[i]], 1u) : 0u;
            }
        }
        __syncthreads();
        // 2. tile offsets and output units (n in the low half, units in the high half)
        {
            const uint32_t d0 = threadIdx.x * ept;
            uint32_t sum = 0;
            for (uint32_t q = 0; q < ept; ++q) {
                const uint32_t dd = d0 + q;
                if (dd >= P) break;
                const uint32_t n = lcnt[dd], c = ccount[dd], gc = gcur[dd];
                const uint32_t bnd = (gc + c + n) / SV * SV;
                const uint32_t nu = bnd > gc ? bnd / SV - gc / SV : 0u;
                sum += n | (nu << 16);
            }
            uint32_t tot;
            uint32_t ex = block_exclusive_scan<uint32_t>(sum, sc, &tot);
            for (uint32_t q = 0; q < ept; ++q) {
                const uint32_t dd = d0 + q;
                if (dd >= P) break;
                const uint32_t n = lcnt[dd], c = ccount[dd], gc = gcur[dd];
                const uint32_t bnd = (gc + c + n) / SV * SV;
                const uint32_t o = bnd > gc ? bnd - gc : 0u;
                const uint32_t nu = o ? bnd / SV - gc / SV : 0u;
                loff[dd] = (uint16_t)(ex & 0xFFFFu);
                uoff[dd] = (uint16_t)(ex >> 16);
                for (uint32_t u = 0; u < nu; ++u) udig[(ex >> 16) + u] = (uint16_t)dd;
                oc[dd] = o | (c << 16);
                ex += n | (nu << 16);
            }
            if (threadIdx.x == 0) {
                loff[P] = (uint16_t)(tot & 0xFFFFu);
                s_nunits = tot >> 16;
            }
        }
        __syncthreads();
        // 3. digit-sorted tile
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            if (!act[i]) continue;
            const uint32_t p = loff[d[i]] + rk[i];
            if constexpr (W == 4) buf[p] = (unsigned long long)k[i] | ((unsigned long long)r[i] << 32);
            else buf[p] = make_ulonglong2(k[i], r[i]);
        }
        __syncthreads();
        // 4. one thread per output sector
        const uint32_t nunits = s_nunits;
        for (uint32_t ui = threadIdx.x; ui < nunits; ui += blockDim.x) {
            const uint32_t dd = udig[ui];
            const uint32_t ocv = oc[dd], c = ocv >> 16;
            const uint32_t gc = gcur[dd];
            const uint32_t sec = gc / SV + (ui - uoff[dd]);
            const uint32_t row0 = sec * SV > gc ? sec * SV : gc;
            const Slot *cy = carry + (size_t)dd * (SV - 1);
            const uint32_t lo_t = loff[dd];
            Slot tup[SV];
#pragma unroll
            for (int q = 0; q < SV; ++q) {
                const uint32_t rr = sec * SV + q;
                const uint32_t j = rr - gc;   // position in carry ++ tile run (valid when rr >= gc)
                if (rr >= row0) tup[q] = j < c ? cy[j] : buf[lo_t + j - c];
            }
            if (row0 == sec * SV) {
                st_sector(outp + (size_t)sec * SV, (const unsigned long long *)tup);
            } else {
                for (uint32_t q = row0 - sec * SV; q < (uint32_t)SV; ++q) outp[(size_t)sec * SV + q] = tup[q];
            }
        }
        __syncthreads();
        // 5. new carries, cursors
        for (uint32_t dd = threadIdx.x; dd < P; dd += blockDim.x) {
            const uint32_t ocv = oc[dd], o = ocv & 0xFFFFu, c = ocv >> 16, n = lcnt[dd];
            Slot *cy = carry + (size_t)dd * (SV - 1);
            for (uint32_t j = (o > c ? o : c); j < c + n; ++j) cy[j - o] = buf[loff[dd] + (j - c)];
            gcur[dd] += o;
            ccount[dd] = (uint8_t)(c + n - o);
            lcnt[dd] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            k[i] = nk[i];
            r[i] = nr[i];
        }
    }
    // final carries; with pad, padding tuples complete each run's last sector
    for (uint32_t dd = threadIdx.x; dd < P; dd += blockDim.x) {
        const uint32_t c = ccount[dd], gc = gcur[dd];
        const Slot *cy = carry + (size_t)dd * (SV - 1);
        if (pad) {
            if (c == 0) continue;
            const uint64_t sk = digit_of(key_hash<W>((U)sent_k0), shift, bits) != dd ? sent_k0 : sent_k1;
            Slot tup[SV];
#pragma unroll
            for (int q = 0; q < SV; ++q) {
                if ((uint32_t)q < c) tup[q] = cy[q];
                else if constexpr (W == 4) tup[q] = (unsigned long long)(uint32_t)sk;
                else tup[q] = make_ulonglong2(sk, 0ull);
            }
            st_sector(outp + gc, (const unsigned long long *)tup);
        } else {
            for (uint32_t j = 0; j < c; ++j) outp[gc + j] = cy[j];
        }
    }
}

// Scatter with the next tile staged by a TMA bulk copy.  Same phases as
// scatter_kernel; instead of registers, tile t + 1 travels global -> shared in one
// cp.async.bulk issued right after tile t's tuples have been read out of the
// staging buffer, so the copy overlaps phases 2-5 of tile t and only the current
// tile lives in registers (1024 threads per CTA).
constexpr int kTmaThreads = 1024;
constexpr uint32_t kWaitLimit = 1u << 26;  // mbarrier polls before giving up


template <int W> struct TmaShape {
    static constexpr int IT = W == 4 ? 8 : 4;    // tuples per thread per tile
    static constexpr int T = kTmaThreads * IT;
    static constexpr int SV = Sector<W>::kTuples;
};

// Per-digit state of the TMA scatter.  What the per-sector writer needs is one
// 8-byte record (a single shared load); the per-tuple fields -- the tile count
// bumped by every tuple and the tile offset read by every tuple -- live in dense
// arrays so that random digits spread over all shared-memory banks.
struct DigitMeta {
    uint32_t gcur;  // next output row (relative to the chunk's sector-aligned base)
    uint32_t oc;    // o (rows completed this tile) | carried count << 16
};

template <int W>
__host__ __device__ inline size_t scatter_tma_smem_bytes(uint32_t P) {
    using TS = TmaShape<W>;
    size_t slot = 2 * W;
    size_t b = ((size_t)TS::T + 4) * slot + (size_t)TS::T * slot  // stage (tile + alignment slack), buf
               + (size_t)P * (TS::SV - 1) * slot                  // carry
               + (size_t)P * sizeof(DigitMeta)                    // meta
               + (size_t)P * 4                                    // cnt
               + (size_t)P * 2 * 2                                // loff, uoff
               + ((size_t)TS::T / TS::SV + 2 * (size_t)P) * 2     // udig
               + (size_t)P;                                       // ccount
    return (b + 15) & ~size_t(15);
}

template <int W>
__global__ void __launch_bounds__(kTmaThreads, 1) scatter_tma_kernel(
    const void *in, uint64_t n_total, const uint64_t *seg_off, uint64_t nseg, const unsigned long long *cb,
    uint64_t chunk, int shift, int bits, const unsigned long long *Hs, void *out, int pad, uint64_t sent_k0,
    uint64_t sent_k1, unsigned long long *fault, const void *const *seg_ptrs, uint32_t wait_limit) {
    using U = typename Tup<W>::U;
    using TS = TmaShape<W>;
    using Slot = typename SortSlot<W>::T;
    constexpr int IT = TS::IT, SV = TS::SV, T = TS::T;
    constexpr int EPT = 2;  // digits per thread (fan-out <= 2 * kTmaThreads)
    const uint32_t P = 1u << bits;
    extern __shared__ __align__(16) unsigned char smem[];
    Slot *stage = (Slot *)smem;                                        // T + 4: an unaligned tile
    Slot *buf = stage + T + 4;                                         // T      spans T + 2 slots
    Slot *carry = buf + T;                                             // P * (SV - 1)
    DigitMeta *meta = (DigitMeta *)(carry + (size_t)P * (SV - 1));     // P
    uint32_t *cnt = (uint32_t *)(meta + P);                            // P
    uint16_t *loff = (uint16_t *)(cnt + P);                            // P
    uint16_t *uoff = loff + P;                                         // P
    uint16_t *udig = uoff + P;                                         // T / SV + 2P
    uint8_t *ccount = (uint8_t *)(udig + T / SV + 2 * P);              // P
    __shared__ uint32_t sc[33];
    __shared__ uint32_t s_nunits;
    __shared__ int s_abort;
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
    const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);

    const uint64_t g = blockIdx.x;
    if (g >= cb[nseg]) return;
    const ChunkPos cp = chunk_pos(seg_off, nseg, cb, chunk, g);
    const uint64_t row = cb[cp.s] * P;
    const uint64_t seg_start = seg_off[0] + Hs[row];
    const uint64_t obase = seg_start / SV * SV;
    Slot *outp = (Slot *)out + obase;
    const uint64_t tb = 2 * W;
    // tuples come from `in` (global row index), or from the segment's own array
    const void *src = seg_ptrs ? seg_ptrs[cp.s] : in;
    const uint64_t ioff = seg_ptrs ? seg_off[cp.s] : 0;
    const uint64_t nsrc = seg_ptrs ? seg_off[cp.s + 1] - seg_off[cp.s] : n_total;
    const uint64_t last16 = (nsrc * tb) / 16 * 16;  // bytes of `src` a 16-byte copy may touch
    for (uint32_t d = threadIdx.x; d < P; d += blockDim.x) {
        DigitMeta m;
        m.gcur = (uint32_t)(seg_off[0] + Hs[row + (uint64_t)d * cp.nch + cp.cidx] - obase);
        m.oc = 0;
        meta[d] = m;
        cnt[d] = 0;
        ccount[d] = 0;
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // byte range of src staged for the tile of global rows [t0, t1): 16-byte
    // aligned, inside the array
    auto stage_range = [&](uint64_t t0, uint64_t t1, uint64_t *b0, uint64_t *b1) {
        *b0 = ((t0 - ioff) * tb) / 16 * 16;
        uint64_t e = ((t1 - ioff) * tb + 15) / 16 * 16;
        *b1 = e < last16 ? e : last16;
    };
    auto issue = [&](uint64_t t0, uint64_t t1) {
        uint64_t b0, b1;
        stage_range(t0, t1, &b0, &b1);
        if (b1 > b0) {
            mbar_expect_tx(bar, (uint32_t)(b1 - b0));
            bulk_g2s(stage_s, (const char *)src + b0, (uint32_t)(b1 - b0), bar);
        } else {
            mbar_expect_tx(bar, 0);
        }
    };
    const uint32_t d0 = threadIdx.x * EPT;  // this thread's digits: d0, d0 + 1
    uint32_t parity = 0;
    if (threadIdx.x == 0 && cp.lo < cp.hi) issue(cp.lo, min(cp.lo + (uint64_t)T, cp.hi));
    for (uint64_t t0 = cp.lo; t0 < cp.hi; t0 += T) {
        const uint64_t t1 = min(t0 + (uint64_t)T, cp.hi);
        if (!mbar_wait_bounded(bar, parity, wait_limit)) s_abort = 1;
        parity ^= 1u;
        __syncthreads();
        if (s_abort) {  // a copy did not complete: report, let it drain, stop
            if (threadIdx.x == 0) {
                atomicOr(fault, (unsigned long long)kStatusTimeout);
                mbar_wait_bounded(bar, parity ^ 1u, kWaitLimit);
            }
            return;
        }
        // 1. tuples of this tile (staged, except an odd final tuple past the last 16 bytes)
        uint64_t b0, b1;
        stage_range(t0, t1, &b0, &b1);
        const uint32_t ntile = (uint32_t)(t1 - t0);
        const uint32_t skew = (uint32_t)(t0 - ioff - b0 / tb);            // 0 or 1 leading slots
        const uint32_t staged = b1 > b0 ? (uint32_t)((b1 - b0) / tb) : 0u;
        const uint32_t nstaged = staged > skew ? staged - skew : 0u;       // tuples of the tile in the stage
        U k[IT], r[IT];
        uint32_t d[IT], rk[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t t = (uint32_t)i * kTmaThreads + threadIdx.x;
            Slot sl;
            if (t < nstaged) sl = stage[t + skew];
            else if (t < ntile) sl = ((const Slot *)src)[t0 - ioff + t];
            else {
                if constexpr (W == 4) sl = 0ull;
                else sl = make_ulonglong2(0ull, 0ull);
            }
            if constexpr (W == 4) {
                k[i] = (uint32_t)sl;
                r[i] = (uint32_t)(sl >> 32);
            } else {
                k[i] = sl.x;
                r[i] = sl.y;
            }
            d[i] = digit_of(key_hash<W>(k[i]), shift, bits);
            rk[i] = t < ntile ? atomicAdd(&cnt[d[i]], 1u) : 0u;
        }
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && t1 < cp.hi) issue(t1, min(t1 + (uint64_t)T, cp.hi));
        // 2. tile offsets and output units (n in the low half, units in the high half)
        uint32_t n_[EPT], c_[EPT], gc_[EPT], o_[EPT], nu_[EPT];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const uint32_t dd = d0 + q;
            n_[q] = c_[q] = gc_[q] = o_[q] = nu_[q] = 0;
            if (dd < P) {
                n_[q] = cnt[dd];
                c_[q] = ccount[dd];
                gc_[q] = meta[dd].gcur;
                const uint32_t bnd = (gc_[q] + c_[q] + n_[q]) / SV * SV;
                o_[q] = bnd > gc_[q] ? bnd - gc_[q] : 0u;
                nu_[q] = o_[q] ? bnd / SV - gc_[q] / SV : 0u;
                sum += n_[q] | (nu_[q] << 16);
            }
        }
        {
            uint32_t tot;
            uint32_t ex = block_exclusive_scan<uint32_t>(sum, sc, &tot);
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const uint32_t dd = d0 + q;
                if (dd < P) {
                    meta[dd].oc = o_[q] | (c_[q] << 16);
                    loff[dd] = (uint16_t)(ex & 0xFFFFu);
                    uoff[dd] = (uint16_t)(ex >> 16);
                    for (uint32_t u = 0; u < nu_[q]; ++u) udig[(ex >> 16) + u] = (uint16_t)dd;
                    ex += n_[q] | (nu_[q] << 16);
                }
            }
            if (threadIdx.x == 0) s_nunits = tot >> 16;
        }
        __syncthreads();
        // 3. digit-sorted tile
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const uint32_t t = (uint32_t)i * kTmaThreads + threadIdx.x;
            if (t >= ntile) continue;
            const uint32_t p = loff[d[i]] + rk[i];
            if constexpr (W == 4) buf[p] = (unsigned long long)k[i] | ((unsigned long long)r[i] << 32);
            else buf[p] = make_ulonglong2(k[i], r[i]);
        }
        __syncthreads();
        // 4. one thread per output sector
        const uint32_t nunits = s_nunits;
        for (uint32_t ui = threadIdx.x; ui < nunits; ui += blockDim.x) {
            const uint32_t dd = udig[ui];
            const DigitMeta m = meta[dd];
            const uint32_t c = m.oc >> 16, gc = m.gcur, lo_t = loff[dd];
            const uint32_t sec = gc / SV + (ui - uoff[dd]);
            const uint32_t row0 = sec * SV > gc ? sec * SV : gc;
            const Slot *cy = carry + (size_t)dd * (SV - 1);
            Slot tup[SV];
#pragma unroll
            for (int q = 0; q < SV; ++q) {
                const uint32_t rr = sec * SV + q;
                const uint32_t j = rr - gc;
                if (rr >= row0) tup[q] = j < c ? cy[j] : buf[lo_t + j - c];
            }
            if (row0 == sec * SV) {
                st_sector(outp + (size_t)sec * SV, (const unsigned long long *)tup);
            } else {
#pragma unroll
                for (int q = 0; q < SV; ++q)
                    if (sec * SV + q >= row0) outp[(size_t)sec * SV + q] = tup[q];
            }
        }
        __syncthreads();
        // 5. new carries, cursors (this thread's digits, values from phase 2)
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const uint32_t dd = d0 + q;
            if (dd < P) {
                Slot *cy = carry + (size_t)dd * (SV - 1);
                const uint32_t lo_t = loff[dd];
                for (uint32_t j = (o_[q] > c_[q] ? o_[q] : c_[q]); j < c_[q] + n_[q]; ++j)
                    cy[j - o_[q]] = buf[lo_t + (j - c_[q])];
                meta[dd].gcur = gc_[q] + o_[q];
                cnt[dd] = 0;
                ccount[dd] = (uint8_t)(c_[q] + n_[q] - o_[q]);
            }
        }
        __syncthreads();
    }
    // final carries; with pad, padding tuples complete each run's last sector
    for (uint32_t dd = threadIdx.x; dd < P; dd += blockDim.x) {
        const uint32_t c = ccount[dd], gc = meta[dd].gcur;
        const Slot *cy = carry + (size_t)dd * (SV - 1);
        if (pad) {
            if (c == 0) continue;
            const uint64_t sk = digit_of(key_hash<W>((U)sent_k0), shift, bits) != dd ? sent_k0 : sent_k1;
            Slot tup[SV];
#pragma unroll
            for (int q = 0; q < SV; ++q) {
                if ((uint32_t)q < c) tup[q] = cy[q];
                else if constexpr (W == 4) tup[q] = (unsigned long long)(uint32_t)sk;
                else tup[q] = make_ulonglong2(sk, 0ull);
            }
            st_sector(outp + gc, (const unsigned long long *)tup);
        } else {
            for (uint32_t j = 0; j < c; ++j) outp[gc + j] = cy[j];
        }
    }
}


// --------------------------------------------------------- region scatter
// Scatter of a padded pass (every (chunk, digit) run starts on a sector) without a
// per-tile sort.  Shared memory holds, per digit, K slots laid out position-major
// (slot j of digit d at region[j * P + d], so that consecutive digits are
// consecutive words); P = 2^LOG2P is a compile-time constant so that every index
// is a shift and an or.  Tuples come straight from global memory into registers,
// the next tile's 16-byte vectors loaded while the current tile is processed.  Per
// tile:
//   1. insert: every tuple takes the next slot of its digit with one shared
//      atomicAdd; a tuple that finds its digit's K slots taken (rare for uniform
//      keys) is written at once to the far end of the digit's run instead, at a
//      row taken by a shared atomicSub on the run's tail cursor;
//   2. flush: one thread per digit writes every whole sector its slots hold with
//      one 32-byte store at the run's head cursor and moves the remaining (fewer
//      than a sector's) tuples to the front of its slots.
// After the last tile the gap between a run's head and tail -- its carried
// tuples plus the padding the histogram added -- is filled tuple by tuple
// (padding tuples hash to another digit; the join drops them).
constexpr int kRegionThreads = 1024;

template <int W, int LOG2P> struct RegionShape {
    static constexpr uint32_t P = 1u << LOG2P;
    static constexpr int SV = Sector<W>::kTuples;
    static constexpr int PV = Tup<W>::kPerVec;
    static constexpr int VPT = 4;                    // 16-byte vectors per thread per tile
    static constexpr int IT = VPT * PV;              // tuples per thread per tile
    static constexpr uint32_t T = kRegionThreads * IT;
    static constexpr size_t kBudget = 227u * 1024u - 1024u;  // dynamic shared memory
    static constexpr uint32_t K0 = (uint32_t)((kBudget - (size_t)P * 12) / ((size_t)P * 2 * W)) / SV * SV;
    // slots per digit: what shared memory holds, at most 256.  At 2^6 digits a tile
    // puts 128 tuples on a digit on average (4-byte tuples); with 64 slots half of
    // them took the far-end path and a 2^6-digit pass of 2^28 tuples ran 2.1 ms
    // instead of 1.4 (measured)
    static constexpr uint32_t K = K0 > 256 ? 256 : K0;
    static constexpr size_t kSmem = (size_t)K * P * 2 * W + (size_t)P * 12;
};

template <int W, int LOG2P>
__global__ void __launch_bounds__(kRegionThreads, 1) scatter_region_kernel(
    const void *in, uint64_t n_total, RunGeom rg, uint64_t chunk, int shift, void *out, uint64_t sent_k0,
    uint64_t sent_k1, const void *const *seg_ptrs, unsigned long long *fault) {
    using U = typename Tup<W>::U;
    using Vec = typename Tup<W>::Vec;
    using RS = RegionShape<W, LOG2P>;
    using Slot = typename SortSlot<W>::T;
    constexpr uint32_t P = RS::P, K = RS::K;
    constexpr int SV = RS::SV, PV = RS::PV, VPT = RS::VPT, NT = kRegionThreads;
    static_assert(K >= 2 * SV, "each digit needs room for a carried partial sector and a whole one");
    extern __shared__ __align__(16) unsigned char smem[];
    Slot *region = (Slot *)smem;                     // K * P
    uint32_t *fill = (uint32_t *)(region + K * P);  // P: slots taken (may pass K)
    uint32_t *head = fill + P;                       // P: next row of whole sectors
    uint32_t *tail = head + P;                       // P: rows at and above belong to overflow tuples

    const uint64_t g = blockIdx.x;
    ChunkPos cp;
    uint64_t obase;
    if (!chunk_runs<P, NT>(rg, chunk, g, SV, &cp, &obase, head, tail, fault)) return;
    Slot *outp = (Slot *)out + obase;
    // this chunk's tuples: rows [lo, hi) of src; lo is a whole number of vectors
    // (chunks, segments and arrays start on 16 bytes)
    const void *src = seg_ptrs ? seg_ptrs[cp.s] : in;
    const uint64_t ioff = seg_ptrs ? rg.seg_off[cp.s] : 0;
    const Vec *vsrc = (const Vec *)src + (cp.lo - ioff) / PV;
    const uint32_t nrows = (uint32_t)(cp.hi - cp.lo);
    for (uint32_t d = threadIdx.x; d < P; d += NT) fill[d] = 0;
    // vector j of the tile [t0, lim) for this thread; a last vector holding one
    // tuple of a 4-byte relation is read with an 8-byte load (nothing past the
    // array end)
    auto load = [&](uint32_t t0, uint32_t lim, Vec *v) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            const uint32_t r0 = t0 + ((uint32_t)j * NT + threadIdx.x) * PV;
            if (r0 + PV <= lim) v[j] = ld_stream(vsrc + r0 / PV);
            else if (r0 < lim) {
                if constexpr (W == 4) {
                    const uint2 x = ((const uint2 *)vsrc)[r0];
                    v[j] = make_uint4(x.x, x.y, 0u, 0u);
                }
            }
        }
    };
    auto tile_end = [&](uint32_t t0) { return t0 + RS::T < nrows ? t0 + RS::T : nrows; };
    Vec cur[VPT], nxt[VPT];
    if (nrows) load(0, tile_end(0), cur);
    __syncthreads();
    for (uint32_t t0 = 0, t1; t0 < nrows; t0 = t1) {
        t1 = tile_end(t0);
        if (t1 < nrows) load(t1, tile_end(t1), nxt);
        // 1. insert
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
#pragma unroll
            for (int e = 0; e < PV; ++e) {
                const uint32_t r = t0 + ((uint32_t)j * NT + threadIdx.x) * PV + e;
                if (r >= t1) continue;
                Slot sl;
                U k;
                if constexpr (W == 4) {
                    k = e ? cur[j].z : cur[j].x;
                    const uint32_t rid = e ? cur[j].w : cur[j].y;
                    sl = (unsigned long long)k | ((unsigned long long)rid << 32);
                } else {
                    k = cur[j].x;
                    sl = cur[j];
                }
                const uint32_t d = (uint32_t)(key_hash<W>(k) >> shift) & (P - 1u);
                const uint32_t pos = atomicAdd(&fill[d], 1u);
                if (pos < K) region[(pos << LOG2P) | d] = sl;
                else outp[atomicSub(&tail[d], 1u) - 1u] = sl;
            }
        }
        __syncthreads();
        // 2. flush whole sectors, keep the rest at the front
#pragma unroll
        for (uint32_t d0 = 0; d0 < (P + NT - 1) / NT * NT; d0 += NT) {
            const uint32_t d = d0 + threadIdx.x;
            if (P % NT && d >= P) break;
            const uint32_t f = fill[d];
            const uint32_t n = f < K ? f : K;
            if (n >= (uint32_t)SV) {
                const uint32_t whole = n / SV * SV;
                const uint32_t hd = head[d];
                for (uint32_t s0 = 0; s0 < whole; s0 += SV) {
                    Slot tup[SV];
#pragma unroll
                    for (int q = 0; q < SV; ++q) tup[q] = region[((s0 + q) << LOG2P) | d];
                    st_sector(outp + hd + s0, (const unsigned long long *)tup);
                }
                for (uint32_t q = whole; q < n; ++q) region[((q - whole) << LOG2P) | d] = region[(q << LOG2P) | d];
                head[d] = hd + whole;
                fill[d] = n - whole;
            } else if (f != n) {
                fill[d] = n;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < VPT; ++j) cur[j] = nxt[j];
    }
    // the gap [head, tail) of every run: its carried tuples, then padding
    for (uint32_t d = threadIdx.x; d < P; d += NT) {
        const uint32_t hd = head[d], tl = tail[d], c = fill[d];
        const uint64_t sk = ((uint32_t)(key_hash<W>((U)sent_k0) >> shift) & (P - 1u)) != d ? sent_k0 : sent_k1;
        Slot pt;
        if constexpr (W == 4) pt = (unsigned long long)(uint32_t)sk;
        else pt = make_ulonglong2(sk, 0ull);
        for (uint32_t r = hd; r < tl; ++r) outp[r] = r - hd < c ? region[((r - hd) << LOG2P) | d] : pt;
    }
}

template <int W, int LOG2P>
static hj_status launch_region(hj_ctx *c, unsigned grid, const void *in, uint64_t n_total, const RunGeom &rg,
                               uint64_t chunk, int shift, void *out, uint64_t k0, uint64_t k1,
                               const void *const *seg_ptrs) {
    auto kern = scatter_region_kernel<W, LOG2P>;
    const size_t smem = RegionShape<W, LOG2P>::kSmem;
    HJ_TRY(allow_max_smem(c, (const void *)kern));
    HJ_LAUNCH(c, "partition_scatter", kern, grid, kRegionThreads, smem, in, n_total, rg, chunk, shift, out, k0, k1,
              seg_ptrs, &c->d_ctr->fault);
    return HJ_OK;
}

// ------------------------------------------------------------- ring scatter
// Padded passes at a high fan-out (2^9 .. 2^11 digits): the insert and flush work
// of the region scatter split between warps that run at the same time, with no
// barrier after the set-up.  Digit d owns a ring of K slots (slot j at
// ring[j * P + d], a slot holding one tuple; empty slots hold a key of another
// digit) and one packed word, claimed | flushed << 16: positions claimed and
// positions flushed, both counted modulo M (a multiple of K and of the sector, so
// a position's slot is the same in every lap of the count).
//   * An insert warp streams its own blocks of the chunk.  A tuple reads its
//     digit's word once (acquire) and, while claimed - flushed < K, claims
//     position w with one CAS of the word and stores itself in slot w mod K; with
//     the ring full it is written from the run's far end, as in the region
//     scatter.  A 4-byte tuple is one 8-byte store; an 8-byte tuple stores its
//     rid, then its key with release semantics (a flush lane reads the key with
//     acquire, so a key it sees comes with its rid).
//   * A flush lane owns a set of digits (consecutive digits across a warp's lanes,
//     so its slot accesses do not conflict).  Once the claimed positions of one
//     sector at the flushed count all hold tuples, it writes them as one 32-byte
//     sector at the run's next row, empties the slots, then adds the sector to
//     the flushed half with a release add (inserts read the word with acquire, so
//     a slot is refilled only after it was emptied).  Only that lane writes the
//     flushed half.
//   * When every insert warp is done (release / acquire on a counter) the flush
//     lanes write what is left of each ring, then padding, into the run's gap.
// One packed word instead of two cursors saves an insert one shared load: the
// kernel is bound by the shared-memory data pipe, not by DRAM (measured).
// Every wait is bounded: a flush warp that passes `max_passes` (kRingMaxPasses, or
// the context's test setting) sets the timeout bit of the sticky fault word and
// returns; insert warps never wait, so the CTA still ends.
constexpr int kRingThreads = 1024;
constexpr uint32_t kRingMaxClaim = 64;             // CAS attempts before the far-end path
constexpr uint64_t kRingMaxPasses = 1ull << 22;    // flush passes before the timeout bit
constexpr int kRingVec = 4;                        // 16-byte vectors per lane in flight

template <int W, int LOG2P> struct RingShape {
    static constexpr uint32_t P = 1u << LOG2P;
    static constexpr uint32_t SV = (uint32_t)Sector<W>::kTuples;
    static constexpr size_t kSlot = 2 * W;
    static constexpr size_t kBudget = 227u * 1024u - 1024u;  // dynamic shared memory
    // slots per digit: whole sectors in what the ring may use (12 for 4-byte tuples
    // at 2^11 digits, 6 for 8-byte ones), at most 64
    static constexpr uint32_t K0 = (uint32_t)((kBudget - (size_t)P * 12 - 16) / ((size_t)P * kSlot)) / SV * SV;
    static constexpr uint32_t K = K0 > 64 ? 64 : K0;
    static constexpr uint32_t M = 65535u / K * K;  // positions modulo M: whole laps, in 16 bits
    static constexpr size_t kSmem = (size_t)K * P * kSlot + (size_t)P * 12 + 16;
    // flush warps of the 32 (measured): 4 for 4-byte tuples (2 fall behind, 6 or 8
    // slow the inserts); 8-byte tuples flush a sector per two tuples, twice as
    // often: 8 at 2^10 and 2^11 digits, 6 at 2^9
    static constexpr int FW = W == 4 ? 4 : (LOG2P == 9 ? 6 : 8);
    static_assert(K >= 2 * SV, "a ring holds at least two sectors");
    static_assert(M % SV == 0, "the flushed count wraps on a sector");
};

__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_cta_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.cta.shared.u64 %0, [%1];" : "=l"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.cta.shared.u64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_cta(uint32_t *p, uint32_t v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
}

template <int W, int LOG2P>
__global__ void __launch_bounds__(kRingThreads, 1) scatter_ring_kernel(
    const void *in, uint64_t n_total, RunGeom rg, uint64_t chunk, int shift, void *out, uint64_t sent_k0,
    uint64_t sent_k1, const void *const *seg_ptrs, unsigned long long *fault, uint64_t max_passes) {
    using U = typename Tup<W>::U;
    using Vec = typename Tup<W>::Vec;
    using RS = RingShape<W, LOG2P>;
    using Slot = typename SortSlot<W>::T;  // 8 bytes (key | rid << 32) or 16 (key, rid)
    constexpr uint32_t P = RS::P, K = RS::K, SV = RS::SV, M = RS::M;
    constexpr uint32_t PV = (uint32_t)Tup<W>::kPerVec;
    constexpr unsigned NI = kRingThreads / 32 - RS::FW, NFL = RS::FW * 32;
    extern __shared__ __align__(16) unsigned char smem[];
    Slot *ring = (Slot *)smem;                              // K * P, slot j of digit d at ring[j * P + d]
    uint32_t *word = (uint32_t *)(ring + (size_t)K * P);   // P: claimed | flushed << 16 (mod M)
    uint32_t *nxt = word + P;                               // P: next output row of the run
    uint32_t *tail = nxt + P;                               // P: rows at and above hold far-end tuples
    uint32_t *s_done = tail + P;                            // insert warps finished

    const uint64_t g = blockIdx.x;
    ChunkPos cp;
    uint64_t obase;
    if (!chunk_runs<P, kRingThreads>(rg, chunk, g, SV, &cp, &obase, nxt, tail, fault)) return;
    Slot *outp = (Slot *)out + obase;
    const void *src = seg_ptrs ? seg_ptrs[cp.s] : in;
    const uint64_t ioff = seg_ptrs ? rg.seg_off[cp.s] : 0;
    const Vec *vsrc = (const Vec *)src + (cp.lo - ioff) / PV;  // chunks start on whole vectors
    const uint32_t nrows = (uint32_t)(cp.hi - cp.lo);
    const uint32_t dk0 = (uint32_t)(key_hash<W>((U)sent_k0) >> shift) & (P - 1u);
    auto empty_key = [&](uint32_t d) -> U { return d != dk0 ? (U)sent_k0 : (U)sent_k1; };
    auto empty_slot = [&](uint32_t d) -> Slot {
        if constexpr (W == 4) return (unsigned long long)empty_key(d);
        else return make_ulonglong2(empty_key(d), 0ull);
    };
    for (uint32_t d = threadIdx.x; d < P; d += kRingThreads) word[d] = 0;
    for (uint32_t i = threadIdx.x; i < K * P; i += kRingThreads) ring[i] = empty_slot(i & (P - 1u));
    if (threadIdx.x == 0) *s_done = 0;
    __syncthreads();
    const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp < NI) {
        auto put = [&](U k, U rid) {
            const uint32_t d = (uint32_t)(key_hash<W>(k) >> shift) & (P - 1u);
            for (uint32_t it = 0; it < kRingMaxClaim; ++it) {
                const uint32_t v = ld_acquire_cta(&word[d]);
                const uint32_t w = v & 0xFFFFu, f = v >> 16;
                const uint32_t used = w >= f ? w - f : w + M - f;
                if (used >= K) break;
                const uint32_t w1 = w + 1u == M ? 0u : w + 1u;
                if (atomicCAS(&word[d], v, (v & 0xFFFF0000u) | w1) == v) {
                    Slot *s = &ring[(size_t)(w % K) * P + d];
                    if constexpr (W == 4) {
                        *s = (unsigned long long)k | ((unsigned long long)rid << 32);
                    } else {
                        s->y = rid;
                        st_release_cta_u64(&s->x, k);
                    }
                    return;
                }
            }
            Slot sl;
            if constexpr (W == 4) sl = (unsigned long long)k | ((unsigned long long)rid << 32);
            else sl = make_ulonglong2(k, rid);
            outp[atomicSub(&tail[d], 1u) - 1u] = sl;
        };
        const uint32_t nvec = (nrows + PV - 1u) / PV;
        for (uint32_t b = warp * (32u * kRingVec); b < nvec; b += NI * 32u * kRingVec) {
            Vec x[kRingVec];
#pragma unroll
            for (int j = 0; j < kRingVec; ++j) {
                const uint32_t v = b + (uint32_t)j * 32u + lane;
                if (v < nvec) {
                    if constexpr (W == 4) {
                        if (2u * v + 1u < nrows) {
                            x[j] = ld_stream(vsrc + v);
                        } else {  // the last tuple alone: nothing past the array end is read
                            const uint2 y = ((const uint2 *)vsrc)[2u * v];
                            x[j] = make_uint4(y.x, y.y, 0u, 0u);
                        }
                    } else {
                        x[j] = ld_stream(vsrc + v);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kRingVec; ++j) {
                const uint32_t v = b + (uint32_t)j * 32u + lane;
                if (v < nvec) {
                    if constexpr (W == 4) {
                        put(x[j].x, x[j].y);
                        if (2u * v + 1u < nrows) put(x[j].z, x[j].w);
                    } else {
                        put(x[j].x, x[j].y);
                    }
                }
            }
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) atomicAdd(s_done, 1u);
        return;
    }

    // ----------------------------------------------------------- flush warps
    const uint32_t fid = (warp - NI) * 32u + lane;
    uint64_t pass = 0;
    for (; pass < max_passes; ++pass) {
        const bool fin = ld_acquire_cta(s_done) == NI;
        bool any = false;
        for (uint32_t d = fid; d < P; d += NFL) {
            const uint32_t v = *(volatile uint32_t *)&word[d];
            const uint32_t w = v & 0xFFFFu, f = v >> 16;
            const uint32_t used = w >= f ? w - f : w + M - f;
            if (used < SV) continue;
            const uint32_t s0 = f % K;
            const U ek = empty_key(d);
            unsigned long long t[4];  // the sector: 4 x (key | rid << 32) or 2 x (key, rid)
            bool full = true;
#pragma unroll
            for (uint32_t q = 0; q < SV; ++q) {
                Slot *s = &ring[(size_t)(s0 + q) * P + d];
                if constexpr (W == 4) {
                    t[q] = *(volatile unsigned long long *)s;
                    full &= (uint32_t)t[q] != ek;
                } else {
                    t[2 * q] = ld_acquire_cta_u64(&s->x);
                    full &= t[2 * q] != ek;
                }
            }
            if (!full) continue;  // a claimed slot is not written yet
            if constexpr (W == 8) {
#pragma unroll
                for (uint32_t q = 0; q < SV; ++q) t[2 * q + 1] = *(volatile unsigned long long *)&ring[(size_t)(s0 + q) * P + d].y;
            }
            const uint32_t o = nxt[d];
            st_sector(outp + o, t);
#pragma unroll
            for (uint32_t q = 0; q < SV; ++q) {
                if constexpr (W == 4) ring[(size_t)(s0 + q) * P + d] = (unsigned long long)ek;
                else ring[(size_t)(s0 + q) * P + d].x = ek;
            }
            nxt[d] = o + SV;
            // the slots are empty before the flushed count says so (release)
            red_release_add_cta(&word[d], (f + SV == M ? SV - M : SV) << 16);
            any = true;
        }
        if (fin && !any) break;
        if (!any) __nanosleep(256);
    }
    if (pass == max_passes) {
        atomicOr(fault, (unsigned long long)kStatusTimeout);
        return;
    }
    // every insert warp is done and seen: the ring's remainder, then padding
    for (uint32_t d = fid; d < P; d += NFL) {
        const uint32_t v = word[d], w = v & 0xFFFFu, f = v >> 16;
        const uint32_t used = w >= f ? w - f : w + M - f;
        const uint32_t hd = nxt[d], tl = tail[d];
        const Slot pad = empty_slot(d);
        for (uint32_t r = hd; r < tl; ++r) {
            const uint32_t q = r - hd;
            outp[r] = q < used ? ring[(size_t)((f + q) % K) * P + d] : pad;
        }
    }
}

template <int W, int LOG2P>
static hj_status launch_ring(hj_ctx *c, unsigned grid, const void *in, uint64_t n_total, const RunGeom &rg,
                             uint64_t chunk, int shift, void *out, uint64_t k0, uint64_t k1,
                             const void *const *seg_ptrs) {
    auto kern = scatter_ring_kernel<W, LOG2P>;
    HJ_TRY(allow_max_smem(c, (const void *)kern));
    const uint64_t passes = c->wait_limit ? std::min<uint64_t>(c->wait_limit, kRingMaxPasses) : kRingMaxPasses;
    constexpr size_t smem = RingShape<W, LOG2P>::kSmem;
    HJ_LAUNCH(c, "partition_scatter", kern, grid, kRingThreads, smem, in, n_total, rg, chunk, shift, out, k0, k1,
              seg_ptrs, &c->d_ctr->fault, passes);
    return HJ_OK;
}

// Which padded-pass scatter runs at a fan-out: the ring where it measured faster
// than the region kernel (per launch at 2^23 x 2^27 uniform 4-byte tuples and the
// 2^22 x 2^26 Zipf 8-byte workload: 4-byte 0.34 / 0.35 ms against 0.40 / 0.40 at
// 2^11 / 2^10 digits, a tie at 2^9; 8-byte 0.33 / 0.32 / 0.37 against 0.39 / 0.48
// / 0.42 at 2^11 / 2^10 / 2^9), unless the context forces one (hj_debug_scatter).
static bool use_ring(const hj_ctx *c, int width, int bits) {
    if (bits < 9 || bits > 11) return false;
    if (c->scatter_kind == HJ_SCATTER_REGION) return false;
    if (c->scatter_kind == HJ_SCATTER_RING) return true;
    return width == 8 || bits >= 10;
}

template <int W>
static hj_status launch_region_bits(hj_ctx *c, int bits, unsigned grid, const void *in, uint64_t n_total,
                                    const RunGeom &rg, uint64_t chunk, int shift, void *out, uint64_t k0,
                                    uint64_t k1, const void *const *seg_ptrs) {
#define HJ_RG(B)                                                                                                 \
    case B:                                                                                                      \
        return launch_region<W, B>(c, grid, in, n_total, rg, chunk, shift, out, k0, k1, seg_ptrs)
#define HJ_RI(B)                                                                                                 \
    case B:                                                                                                      \
        return launch_ring<W, B>(c, grid, in, n_total, rg, chunk, shift, out, k0, k1, seg_ptrs)
    if (use_ring(c, W, bits)) {
        switch (bits) {
            HJ_RI(9); HJ_RI(10); HJ_RI(11);
            default: break;
        }
    }
    switch (bits) {
        HJ_RG(1); HJ_RG(2); HJ_RG(3); HJ_RG(4); HJ_RG(5); HJ_RG(6);
        HJ_RG(7); HJ_RG(8); HJ_RG(9); HJ_RG(10); HJ_RG(11);
        default: return set_err(c, HJ_E_INVALID, "region scatter takes 1..11 bits, not %d", bits);
    }
#undef HJ_RG
#undef HJ_RI
}

// ------------------------------------------------------------------- driver

// Scatter configuration (threads, vectors per thread) for a fan-out: 8192-tuple
// tiles of 4-byte tuples while the per-digit state leaves room, 4096 otherwise.
struct ScatterCfg {
    int nt, vpt;
    uint64_t tile;
    bool tma;
};
static ScatterCfg scatter_cfg(int width, int bits) {
    // up to 2^11 digits the TMA-staged kernel fits shared memory
    if (bits <= 11) return ScatterCfg{kTmaThreads, 0, (uint64_t)(width == 4 ? TmaShape<4>::T : TmaShape<8>::T), true};  // 2^bits <= 2 * kTmaThreads
    if (width == 4) return ScatterCfg{1024, 2, 4096, false};
    return ScatterCfg{1024, 2, 2048, false};
}

// Chunk size of a pass: about one chunk per SM over the whole input (one scatter
// CTA fits an SM at the largest fan-out), at most 2^21 rows so that many segments
// spread over the SMs, a multiple of the scatter tile.
static uint64_t pass_chunk(hj_ctx *c, int width, int bits, uint64_t n_total) {
    const uint64_t tile = scatter_cfg(width, bits).tile;
    const uint64_t target = (uint64_t)num_sms(c);
    uint64_t chunk = (n_total + target - 1) / target;
    if (chunk > (1ull << 21)) chunk = 1ull << 21;
    chunk = ((chunk + tile - 1) / tile) * tile;
    return chunk < tile ? tile : chunk;
}

uint64_t partition_out_rows(hj_ctx *c, int width, uint64_t n_total, uint64_t nseg, int bits, int pad) {
    if (!pad) return n_total;
    const uint64_t chunk = pass_chunk(c, width, bits, n_total);
    const uint64_t max_chunks = (n_total + chunk - 1) / chunk + nseg;
    const uint64_t sv = 32 / (2 * width);
    return n_total + max_chunks * (1ull << bits) * (sv - 1);
}

// Two sentinel keys for a pass: 0, and the first key whose digit differs from 0's.
static void sentinel_keys(int width, int shift, int bits, uint64_t *k0, uint64_t *k1);
uint64_t pass_pad_key(int width, int shift, int bits) {
    uint64_t k0, k1;
    sentinel_keys(width, shift, bits, &k0, &k1);
    return k1;
}
static void sentinel_keys(int width, int shift, int bits, uint64_t *k0, uint64_t *k1) {
    auto dg = [&](uint64_t k) {
        uint64_t h = width == 4 ? (uint64_t)murmur2_u32((uint32_t)k) : murmur2_u64(k);
        return (h >> shift) & ((1ull << bits) - 1);
    };
    *k0 = 0;
    uint64_t k = 1;
    while (dg(k) == dg(0)) ++k;
    *k1 = k;
}

hj_status partition_pass(hj_ctx *c, int width, const void *in, uint64_t n_total, const uint64_t *seg_off,
                         uint64_t nseg, int shift, int bits, void *out, uint64_t *part_off, int pad,
                         const void *const *seg_ptrs) {
    if (bits < 1 || bits > 12) return set_err(c, HJ_E_INVALID, "partition pass bits %d outside [1, 12]", bits);
    const uint64_t P = 1ull << bits;
    const ScatterCfg cfg = scatter_cfg(width, bits);
    if (seg_ptrs && !cfg.tma)
        return set_err(c, HJ_E_UNSUPPORTED, "per-segment inputs need a fan-out of at most 2^11");
    const uint64_t chunk = pass_chunk(c, width, bits, n_total);
    const uint64_t max_chunks = (n_total + chunk - 1) / chunk + nseg;

    DevBuf b_nch(c), b_cb(c), b_H(c), b_Hs(c);
    HJ_TRY(b_nch.alloc((nseg + 1) * 4));
    HJ_TRY(b_cb.alloc((nseg + 1) * 8));
    HJ_TRY(b_H.alloc(max_chunks * P * 4));
    HJ_TRY(b_Hs.alloc((max_chunks * P + 1) * 8));
    uint32_t *nch = b_nch.as<uint32_t>(), *H = b_H.as<uint32_t>();
    unsigned long long *cb = b_cb.as<unsigned long long>(), *Hs = b_Hs.as<unsigned long long>();

    int g1 = (int)std::min<uint64_t>((nseg + 255) / 256, 4096);
    if (nseg == 1) {
        HJ_LAUNCH(c, "seg_chunks", one_seg_chunks_kernel, 1, 1, 0, seg_off, chunk, cb);
    } else {
        HJ_LAUNCH(c, "seg_chunks", seg_chunks_kernel, g1 ? g1 : 1, 256, 0, seg_off, nseg, chunk, nch);
        HJ_TRY(scan_counts(c, nch, nseg, cb));
    }
    size_t hsmem = P * 4;
    if (width == 4)
        HJ_LAUNCH(c, "partition_hist", hist_kernel<4>, (unsigned)max_chunks, kHistThreads, hsmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, pad, H, seg_ptrs);
    else
        HJ_LAUNCH(c, "partition_hist", hist_kernel<8>, (unsigned)max_chunks, kHistThreads, hsmem, in, n_total, seg_off, nseg, cb, chunk, shift, bits, pad, H, seg_ptrs);
    HJ_TRY(scan_counts(c, H, max_chunks * P, Hs));
    {
        uint64_t n = nseg * P + 1;
        int g = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms(c) * 8);
        HJ_LAUNCH(c, "partition_offsets", extract_offsets_kernel, g, 256, 0, seg_off, nseg, cb, Hs, bits, part_off,
                  (uint64_t)pad);
    }
    uint64_t k0, k1;
    sentinel_keys(width, shift, bits, &k0, &k1);
#define HJ_SC(WW, NT, VPT)                                                                                    \
    do {                                                                                                      \
        auto kern = scatter_kernel<WW, NT, VPT>;                                                              \
        const size_t ssmem = scatter_smem_bytes<WW, NT, VPT>((uint32_t)P);                                    \
        HJ_TRY(allow_max_smem(c, (const void *)kern));                                                       \
        HJ_LAUNCH(c, "partition_scatter", kern, (unsigned)max_chunks, NT, ssmem, in, n_total, seg_off, nseg, cb, \
                  chunk, shift, bits, Hs, out, pad, k0, k1);                                                  \
    } while (0)
    const size_t tma_smem = width == 4 ? scatter_tma_smem_bytes<4>((uint32_t)P) : scatter_tma_smem_bytes<8>((uint32_t)P);
    if (cfg.tma && pad) {
        const RunGeom rg{seg_off, nseg, cb, Hs, nullptr, nullptr, nullptr, 0, 0, nullptr};
        if (width == 4)
            HJ_TRY(launch_region_bits<4>(c, bits, (unsigned)max_chunks, in, n_total, rg, chunk, shift, out, k0, k1,
                                         seg_ptrs));
        else
            HJ_TRY(launch_region_bits<8>(c, bits, (unsigned)max_chunks, in, n_total, rg, chunk, shift, out, k0, k1,
                                         seg_ptrs));
    } else if (cfg.tma) {
        // mbarrier polls per tile: the default, or n - 1 under a test limit of n (so
        // that n = 1 gives up at the first wait, however long the hardware suspends
        // a polling thread)
        const uint32_t polls = c->wait_limit ? (uint32_t)std::min<uint64_t>(c->wait_limit - 1, kWaitLimit) : kWaitLimit;
        if (width == 4) {
            HJ_TRY(allow_max_smem(c, (const void *)scatter_tma_kernel<4>));
            HJ_LAUNCH(c, "partition_scatter", scatter_tma_kernel<4>, (unsigned)max_chunks, kTmaThreads, tma_smem, in,
                      n_total, seg_off, nseg, cb, chunk, shift, bits, Hs, out, pad, k0, k1, &c->d_ctr->fault, seg_ptrs,
                      polls);
        } else {
            HJ_TRY(allow_max_smem(c, (const void *)scatter_tma_kernel<8>));
            HJ_LAUNCH(c, "partition_scatter", scatter_tma_kernel<8>, (unsigned)max_chunks, kTmaThreads, tma_smem, in,
                      n_total, seg_off, nseg, cb, chunk, shift, bits, Hs, out, pad, k0, k1, &c->d_ctr->fault, seg_ptrs,
                      polls);
        }
    } else if (width == 4) {
        if (cfg.nt == 512) HJ_SC(4, 512, 8); else HJ_SC(4, 1024, 2);
    } else {
        if (cfg.nt == 512) HJ_SC(8, 512, 4); else HJ_SC(8, 1024, 2);
    }
#undef HJ_SC
    return HJ_OK;
}

// One padded pass over a single segment of n rows at 2^bits <= 2^11 digits (the
// first pass of a join): hist1_kernel and the scatter, whose CTAs place their runs
// from the digit totals themselves -- two launches and a memset in place of the
// general pass's chunk, scan and offset launches.  Same output contract as
// partition_pass with pad: 2^bits partitions, each run padded to whole sectors,
// part_off[2^bits + 1].
hj_status partition_pass1(hj_ctx *c, int width, const void *in, uint64_t n, int bits, void *out, uint64_t *part_off) {
    if (bits < 1 || bits > 11) return set_err(c, HJ_E_INVALID, "single-segment pass bits %d outside [1, 11]", bits);
    const uint64_t P = 1ull << bits;
    if (n == 0) {
        HJ_CUDA(c, cudaMemsetAsync(part_off, 0, (P + 1) * 8, c->stream));
        return HJ_OK;
    }
    const uint64_t chunk = pass_chunk(c, width, bits, n);
    const uint64_t nch = (n + chunk - 1) / chunk;
    DevBuf H1(c), base1(c), T1(c);
    HJ_TRY(H1.alloc(nch * P * 4));
    HJ_TRY(base1.alloc(nch * P * 4));
    HJ_TRY(T1.alloc(P * 4));
    HJ_CUDA(c, cudaMemsetAsync(T1.p, 0, P * 4, c->stream));
    if (width == 4)
        HJ_LAUNCH(c, "partition_hist", hist1_kernel<4>, (unsigned)nch, kHistThreads, P * 4, in, n, chunk, bits,
                  H1.as<uint32_t>(), base1.as<uint32_t>(), T1.as<uint32_t>());
    else
        HJ_LAUNCH(c, "partition_hist", hist1_kernel<8>, (unsigned)nch, kHistThreads, P * 4, in, n, chunk, bits,
                  H1.as<uint32_t>(), base1.as<uint32_t>(), T1.as<uint32_t>());
    uint64_t k0, k1;
    sentinel_keys(width, 0, bits, &k0, &k1);
    const RunGeom rg{nullptr, 1, nullptr, nullptr, H1.as<uint32_t>(), base1.as<uint32_t>(), T1.as<uint32_t>(), n,
                     nch, part_off};
    if (width == 4)
        HJ_TRY(launch_region_bits<4>(c, bits, (unsigned)nch, in, n, rg, chunk, 0, out, k0, k1, nullptr));
    else
        HJ_TRY(launch_region_bits<8>(c, bits, (unsigned)nch, in, n, rg, chunk, 0, out, k0, k1, nullptr));
    return HJ_OK;
}

}  // namespace hj
