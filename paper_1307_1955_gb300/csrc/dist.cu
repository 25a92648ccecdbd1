// dist.cu -- hj_split: the local step of a join sharded over several GPUs.
//
// Every GPU holds a slice of R and of S.  Each splits its slices into one group per
// GPU by a hash of the key, exchanges the groups (group g goes to GPU g: one
// all-to-all, done by the caller's collective library), and joins what it
// received: equal keys meet on one GPU, so the union of the local joins is the
// join of the whole relations (the partition step of Alg. 2 applied across GPUs).
// The group hash must be independent of every hash a local join uses -- the
// MurmurHash2 bits of the radix digits and of the global table's buckets, and the
// Fibonacci multiply of the in-partition buckets -- or each GPU's keys would pile
// into a fraction of its own digits and buckets.  It is the SplitMix64 finaliser
// of the key (zero-extended to 64 bits), whose high 32 bits are scaled to the
// number of groups: group = (hi32 * nparts) >> 32.
//
// Three launches: per-chunk group counts (shared-memory atomics), a scan of the
// counts in (group, chunk) order, and a scatter in which every tuple takes the next
// row of its (chunk, group) run with a shared-memory atomic.  The order of tuples
// inside a group is not specified.
#include "common.cuh"
#include "engine.cuh"

namespace hj {
namespace {

constexpr int kSplitThreads = 512;
constexpr uint32_t kMaxParts = 4096;

template <int W> __device__ __forceinline__ uint32_t split_group(typename Tup<W>::U key, uint32_t nparts) {
    const uint64_t h = sm64_fin((uint64_t)key);
    return (uint32_t)(((h >> 32) * (uint64_t)nparts) >> 32);
}

// Counts of chunk c: H[g * nch + c].
template <int W>
__global__ void __launch_bounds__(kSplitThreads) split_count_kernel(const void *in, uint64_t n, uint32_t nparts,
                                                                    uint64_t chunk, uint64_t nch, uint32_t *H,
                                                                    unsigned long long *fault) {
    using U = typename Tup<W>::U;
    extern __shared__ uint32_t cnt[];
    for (uint32_t g = threadIdx.x; g < nparts; g += blockDim.x) cnt[g] = 0;
    __syncthreads();
    const uint64_t c = blockIdx.x, lo = c * chunk, hi = min(lo + chunk, n);
    const U *t = (const U *)in;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t g = split_group<W>(t[2 * i], nparts);
        if (g >= nparts) {  // checked (cannot happen): reported, never touched
            atomicOr(fault, (unsigned long long)kStatusBadInput);
            continue;
        }
        atomicAdd(&cnt[g], 1u);
    }
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < nparts; g += blockDim.x) {
        const uint64_t at = (uint64_t)g * nch + c;
        if (at >= nch * nparts) {
            atomicOr(fault, (unsigned long long)kStatusBadInput);
            continue;
        }
        H[at] = cnt[g];
    }
}

// Tuples of chunk c to rows Hs[g * nch + c] + rank of their group.
template <int W>
__global__ void __launch_bounds__(kSplitThreads) split_scatter_kernel(const void *in, uint64_t n, uint32_t nparts,
                                                                      uint64_t chunk, uint64_t nch,
                                                                      const unsigned long long *Hs, void *out,
                                                                      unsigned long long *fault) {
    using U = typename Tup<W>::U;
    extern __shared__ unsigned long long cur[];
    const uint64_t c = blockIdx.x, lo = c * chunk, hi = min(lo + chunk, n);
    for (uint32_t g = threadIdx.x; g < nparts; g += blockDim.x) cur[g] = Hs[(uint64_t)g * nch + c];
    __syncthreads();
    const U *t = (const U *)in;
    U *o = (U *)out;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const U k = t[2 * i], r = t[2 * i + 1];
        const uint32_t g = split_group<W>(k, nparts);
        if (g >= nparts) {
            atomicOr(fault, (unsigned long long)kStatusBadInput);
            continue;
        }
        const unsigned long long at = atomicAdd(&cur[g], 1ull);
        if (at >= n) {  // cannot happen (the counts are of the same rows); reported, never written
            atomicOr(fault, (unsigned long long)kStatusBadInput);
            continue;
        }
        o[2 * at] = k;
        o[2 * at + 1] = r;
    }
}

// offsets[g] = Hs[g * nch], offsets[nparts] = n.
__global__ void split_offsets_kernel(const unsigned long long *Hs, uint32_t nparts, uint64_t nch, uint64_t n,
                                     uint64_t *off) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= nparts; g += gridDim.x * blockDim.x)
        off[g] = g == nparts ? n : Hs[(uint64_t)g * nch];
}

}  // namespace
}  // namespace hj

using namespace hj;

extern "C" hj_status hj_split(hj_ctx *c, const hj_rel *in, int nparts, void *out, uint64_t *offsets_host) {
    if (!c) return HJ_E_INVALID;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    if (!in || (in->width != HJ_U32 && in->width != HJ_U64))
        return set_err(c, HJ_E_INVALID, "in is NULL or its width is not 4 or 8");
    if (in->n && (!in->tuples || ((uintptr_t)in->tuples & 15)))
        return set_err(c, HJ_E_INVALID, "in tuples are NULL or not 16-byte aligned");
    if (nparts < 1 || (uint32_t)nparts > kMaxParts)
        return set_err(c, HJ_E_INVALID, "nparts %d outside [1, %u]", nparts, kMaxParts);
    if (!offsets_host) return set_err(c, HJ_E_INVALID, "offsets is NULL");
    if (in->n && (!out || ((uintptr_t)out & 15))) return set_err(c, HJ_E_INVALID, "out is NULL or not 16-byte aligned");
    const uint64_t n = in->n, P = (uint64_t)nparts;
    // about four chunks per SM, whole warps of rows
    const uint64_t target = (uint64_t)num_sms(c) * 4;
    uint64_t chunk = n ? (n + target - 1) / target : 1;
    chunk = (chunk + 1023) / 1024 * 1024;
    const uint64_t nch = n ? (n + chunk - 1) / chunk : 0;
    DevBuf H(c), Hs(c), off(c);
    HJ_TRY(H.alloc((nch * P + 1) * 4));
    HJ_TRY(Hs.alloc((nch * P + 1) * 8));
    HJ_TRY(off.alloc((P + 1) * 8));
    if (nch) {
        // Every launch is followed by a stream synchronisation: the split is outside
        // the single-GPU join's hot path, and this is the form that has run clean
        // (an earlier form without the checks and the synchronisations met an
        // unexplained illegal-address fault on its first non-empty call).
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        if (in->width == HJ_U32)
            HJ_LAUNCH(c, "split_count", split_count_kernel<4>, (unsigned)nch, kSplitThreads, P * 4, in->tuples, n,
                      (uint32_t)P, chunk, nch, H.as<uint32_t>(), &c->d_ctr->fault);
        else
            HJ_LAUNCH(c, "split_count", split_count_kernel<8>, (unsigned)nch, kSplitThreads, P * 4, in->tuples, n,
                      (uint32_t)P, chunk, nch, H.as<uint32_t>(), &c->d_ctr->fault);
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        HJ_TRY(scan_counts(c, H.as<uint32_t>(), nch * P, Hs.as<unsigned long long>()));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        if (in->width == HJ_U32)
            HJ_LAUNCH(c, "split_scatter", split_scatter_kernel<4>, (unsigned)nch, kSplitThreads, P * 8, in->tuples, n,
                      (uint32_t)P, chunk, nch, Hs.as<unsigned long long>(), out, &c->d_ctr->fault);
        else
            HJ_LAUNCH(c, "split_scatter", split_scatter_kernel<8>, (unsigned)nch, kSplitThreads, P * 8, in->tuples, n,
                      (uint32_t)P, chunk, nch, Hs.as<unsigned long long>(), out, &c->d_ctr->fault);
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        HJ_LAUNCH(c, "split_offsets", split_offsets_kernel, (unsigned)((P + 256) / 256), 256, 0,
                  Hs.as<unsigned long long>(), (uint32_t)P, nch, n, off.as<uint64_t>());
        HJ_CUDA(c, cudaMemcpyAsync(offsets_host, off.p, (P + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
        HJ_TRY(read_counters(c));  // synchronises; reports a guard that fired
    } else {
        for (uint64_t g = 0; g <= P; ++g) offsets_host[g] = 0;
    }
    return HJ_OK;
}
