// static_join.cu -- hj_join_static: the simple hash join without any device
// allocation.  Its scratch (counters and the hash table) lives in one file-scope
// __device__ array; the caller provides the inputs and the pair buffer.
//
// The kernels are variants of the SHJ build and probe of join.cu: the same
// open-addressing pair table (common.cuh), but the probe places pairs densely with
// one warp-aggregated atomicAdd per group of matches, so no chunk bookkeeping or
// compaction (which needs extra buffers) is involved.
#include <mutex>

#include "common.cuh"
#include "ctx.cuh"

namespace {

using namespace hj;

constexpr uint64_t kScratchBytes = HJ_STATIC_SCRATCH_BYTES;
constexpr uint64_t kHeaderBytes = 256;  // counters and table side data

// The scratch.  In host code this name is a stand-in, not a device address: host
// code obtains the device address with cudaGetSymbolAddress (scratch_address).
__device__ __align__(256) unsigned char g_hj_static_scratch[kScratchBytes];

struct StaticHeader {
    hj_counters ctr;
    TableSide side;
};
static_assert(sizeof(StaticHeader) <= kHeaderBytes, "header does not fit");

constexpr uint64_t kStaticMaxWalk = 1ull << 16;  // longest insert walk of the static table

template <int W>
__global__ void static_build_kernel(const void *R, uint64_t n, void *slots, uint64_t cap, StaticHeader *hdr) {
    using U = typename Tup<W>::U;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const U k = ((const U *)R)[2 * t], r = ((const U *)R)[2 * t + 1];
        // (no key-list form here: a longer walk bound than the library's joins, so
        // that keys repeated some thousand times still work)
        if (!pair_insert<W>((typename PairSlot<W>::S *)slots, cap, &hdr->side, k, r, key_hash<W>(k), kStaticMaxWalk))
            atomicOr(&hdr->ctr.status,
                     (unsigned long long)(cap <= kStaticMaxWalk ? kStatusTableFull : kStatusLongRun));
    }
}

// Dense append of one pair per lane with `has` set: one atomicAdd per warp.
template <int W>
__device__ __forceinline__ void dense_append(StaticHeader *hdr, void *pairs, uint64_t pcap, bool has,
                                             typename Tup<W>::U a, typename Tup<W>::U b) {
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (!mask) return;
    const unsigned lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&hdr->ctr.count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) {
        const unsigned long long pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < pcap) {
            if constexpr (W == 4) ((uint2 *)pairs)[pos] = make_uint2(a, b);
            else ((ulonglong2 *)pairs)[pos] = make_ulonglong2(a, b);
        }
    }
}

template <int W>
__global__ void static_probe_kernel(const void *S, uint64_t n, const void *slots, uint64_t cap, StaticHeader *hdr,
                                    void *pairs, uint64_t pcap) {
    using U = typename Tup<W>::U;
    using PS = PairSlot<W>;
    const typename PS::S *sl = (const typename PS::S *)slots;
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long nall = hdr->side.n_allones;
    unsigned long long c0 = 0, c1 = 0;
    for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
        const uint64_t t = base + lane;
        const bool valid = t < n;
        const U k = valid ? ((const U *)S)[2 * t] : U(0), r = valid ? ((const U *)S)[2 * t + 1] : U(0);
        uint32_t cnt = 0;
        U first = 0;
        if (valid) {
            const uint64_t bs = mix_b(r);
            pair_lookup<W>(sl, cap, nall, k, key_hash<W>(k), 1u, [&](U rid) {
                if (cnt == 0) first = rid;
                ++cnt;
                const uint64_t a = mix_a(rid);
                c0 += a * bs;
                c1 += a + bs;
            });
        }
        dense_append<W>(hdr, pairs, pcap, cnt == 1, first, r);
        // keys with several build matches: the warp walks each one's run together
        unsigned multi = __ballot_sync(0xffffffffu, cnt > 1);
        while (multi) {
            const int L = __ffs(multi) - 1;
            multi &= multi - 1;
            const U kk = __shfl_sync(0xffffffffu, k, L), ss = __shfl_sync(0xffffffffu, r, L);
            const uint64_t b0 = bucket_of<W>(key_hash<W>(kk), cap);
            for (uint64_t off = 0; off < cap; off += 32) {
                const bool inr = off + lane < cap;
                uint64_t idx = b0 + off + lane;
                if (idx >= cap) idx -= cap;
                const typename PS::S s = inr ? sl[idx] : PS::empty();
                const unsigned emp = __ballot_sync(0xffffffffu, !inr || PS::is_empty(s));
                const unsigned before = emp ? ((emp & (0u - emp)) - 1u) : 0xffffffffu;
                dense_append<W>(hdr, pairs, pcap, ((before >> lane) & 1u) && PS::key(s) == kk, PS::rid(s), ss);
                if (emp) break;
            }
            if (kk == Tup<W>::kAllOnes)
                for (unsigned long long i = 0; i < nall; i += 32)
                    dense_append<W>(hdr, pairs, pcap, i + lane < nall, Tup<W>::kAllOnes, ss);
        }
    }
    c0 = warp_sum(c0);
    c1 = warp_sum(c1);
    if (lane == 0) {
        if (c0) atomicAdd(&hdr->ctr.c0, c0);
        if (c1) atomicAdd(&hdr->ctr.c1, c1);
    }
}

// Device address of the scratch array, looked up once per device with that device
// current.
std::mutex g_mu;
void *g_scratch_addr[256] = {};

hj_status scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= 256) return HJ_E_INVALID;
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_hj_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return HJ_E_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return HJ_OK;
}

bool bad_rel(const hj_rel *r) {
    if (!r || (r->width != HJ_U32 && r->width != HJ_U64)) return true;
    if (r->n && (!r->tuples || ((uintptr_t)r->tuples & 15))) return true;
    return false;
}

}  // namespace

extern "C" hj_status hj_join_static(const hj_rel *R, const hj_rel *S, void *cuda_stream, void *pairs,
                                    uint64_t pairs_cap, uint64_t *count, uint64_t *checksum) {
    if (bad_rel(R) || bad_rel(S) || R->width != S->width || !count) return HJ_E_INVALID;
    if (pairs_cap && !pairs) return HJ_E_INVALID;
    const int W = R->width;
    uint64_t cap = 64;
    while (cap < 2 * R->n + 1) cap <<= 1;
    const uint64_t table_bytes = cap * 2ull * (uint64_t)W;
    if (kHeaderBytes + table_bytes > kScratchBytes) return HJ_E_NOMEM;  // beyond the static maximum
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return HJ_E_CUDA;
    }
    void *base = nullptr;
    hj_status st = scratch_address(device, &base);
    if (st != HJ_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    StaticHeader *hdr = (StaticHeader *)base;
    void *slots = (char *)base + kHeaderBytes;
    // the array keeps the previous call's contents: clear the counters and the table
    cudaError_t e = cudaMemsetAsync(hdr, 0, kHeaderBytes, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(slots, 0xFF, table_bytes, stream);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms <= 0) sms = 1;
    const uint64_t bgrid = R->n ? (R->n + 255) / 256 : 1;
    const unsigned gb = (unsigned)(bgrid < (uint64_t)sms * 8 ? bgrid : (uint64_t)sms * 8);
    const unsigned gp = (unsigned)sms * 4;
    if (e == cudaSuccess) {
        if (W == 4) {
            if (R->n) static_build_kernel<4><<<gb, 256, 0, stream>>>(R->tuples, R->n, slots, cap, hdr);
            if (S->n) static_probe_kernel<4><<<gp, 256, 0, stream>>>(S->tuples, S->n, slots, cap, hdr, pairs, pairs_cap);
        } else {
            if (R->n) static_build_kernel<8><<<gb, 256, 0, stream>>>(R->tuples, R->n, slots, cap, hdr);
            if (S->n) static_probe_kernel<8><<<gp, 256, 0, stream>>>(S->tuples, S->n, slots, cap, hdr, pairs, pairs_cap);
        }
        e = cudaGetLastError();
    }
    hj_counters h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, &hdr->ctr, sizeof h, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HJ_E_CUDA;
    }
    if (h.status & kStatusTableFull) return HJ_E_CUDA;
    if (h.status & kStatusLongRun) return HJ_E_UNSUPPORTED;  // a key repeated too often for this table
    *count = h.count;
    if (checksum) {
        checksum[0] = h.c0;
        checksum[1] = h.c1;
    }
    return h.count > pairs_cap ? HJ_E_OVERFLOW : HJ_OK;
}
