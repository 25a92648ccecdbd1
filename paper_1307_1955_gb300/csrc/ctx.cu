// ctx.cu -- context lifetime, memory pool with HBM budget, errors, profiling.
#include <cstddef>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"
#include "ctx.cuh"

namespace hj {

hj_status set_err(hj_ctx *c, hj_status code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

hj_status cuda_err(hj_ctx *c, cudaError_t e, const char *what) {
    return set_err(c, HJ_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dalloc(hj_ctx *c, uint64_t bytes, hj_status *st) {
    *st = HJ_OK;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~uint64_t(255);
    if (c->fail_alloc_after == 0) {
        c->fail_alloc_after = -1;
        *st = set_err(c, HJ_E_NOMEM, "injected allocation failure (%llu bytes)", (unsigned long long)bytes);
        return nullptr;
    }
    if (c->fail_alloc_after > 0) c->fail_alloc_after--;
    if (c->budget && c->in_use + bytes > c->budget) {
        *st = set_err(c, HJ_E_NOMEM, "HBM budget exceeded: %llu in use + %llu requested > %llu",
                      (unsigned long long)c->in_use, (unsigned long long)bytes,
                      (unsigned long long)c->budget);
        return nullptr;
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        *st = set_err(c, HJ_E_NOMEM, "device allocation of %llu bytes failed: %s",
                      (unsigned long long)bytes, cudaGetErrorString(e));
        return nullptr;
    }
    c->allocs[p] = bytes;
    c->in_use += bytes;
    if (c->in_use > c->peak) c->peak = c->in_use;
    return p;
}

void dfree(hj_ctx *c, void *p) {
    if (!p) return;
    auto it = c->allocs.find(p);
    if (it == c->allocs.end()) return;
    c->in_use -= it->second;
    c->allocs.erase(it);
    cudaFreeAsync(p, c->stream);
}

static cudaEvent_t take_event(hj_ctx *c) {
    if (!c->spare_events.empty()) {
        cudaEvent_t e = c->spare_events.back();
        c->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(hj_ctx *c, const char *name) {
    c->launches++;
    c->prof_open = false;
    if (!c->prof) return;
    if (!c->prof_only.empty() && c->prof_only != name) return;
    c->prof_open = true;
    hj_ctx::Rec r;
    r.name = name;
    r.a = take_event(c);
    r.b = take_event(c);
    cudaEventRecord(r.a, c->stream);
    c->recs.push_back(r);
}

void prof_end(hj_ctx *c) {
    if (!c->prof_open || c->recs.empty()) return;
    c->prof_open = false;
    cudaEventRecord(c->recs.back().b, c->stream);
}

hj_status check_launch(hj_ctx *c, const char *name) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(c, HJ_E_CUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
    return HJ_OK;
}

static void prof_collect(hj_ctx *c) {
    for (auto &r : c->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &acc = c->prof_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        c->spare_events.push_back(r.a);
        c->spare_events.push_back(r.b);
    }
    c->recs.clear();
}

hj_status read_counters(hj_ctx *c) {
    HJ_CUDA(c, cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(hj_counters), cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    const unsigned long long fault = c->h_ctr->fault;
    if (fault) {  // reported once: the next call starts clean
        HJ_CUDA(c, cudaMemsetAsync(&c->d_ctr->fault, 0, sizeof(unsigned long long), c->stream));
        c->h_ctr->fault = 0;
    }
    const unsigned long long st = c->h_ctr->status | fault;
    if (st & kStatusTimeout) return set_err(c, HJ_E_TIMEOUT, "a bounded device wait expired");
    if (st & kStatusBadInput) return set_err(c, HJ_E_INVALID, "a kernel rejected its input");
    return HJ_OK;
}

hj_status zero_counters(hj_ctx *c) {
    // every field but the sticky fault word
    HJ_CUDA(c, cudaMemsetAsync(c->d_ctr, 0, offsetof(hj_counters, fault), c->stream));
    return HJ_OK;
}

hj_status allow_max_smem(hj_ctx *c, const void *func) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;  // (device, function) pairs already set
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({c->device, func})) return HJ_OK;
    int optin = 0;
    HJ_CUDA(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    cudaFuncAttributes fa;
    HJ_CUDA(c, cudaFuncGetAttributes(&fa, func));
    HJ_CUDA(c, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    done.insert({c->device, func});
    return HJ_OK;
}

hj_status copy_wide(hj_ctx *c, void *dst, const void *src, uint64_t bytes, cudaMemcpyKind kind) {
    constexpr int K = hj_ctx::kCopyStreams;
    if (bytes < (64ull << 20)) {
        HJ_CUDA(c, cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
        return HJ_OK;
    }
    if (!c->cstream[0]) {
        for (int i = 0; i < K; ++i) HJ_CUDA(c, cudaStreamCreateWithFlags(&c->cstream[i], cudaStreamNonBlocking));
        for (int i = 0; i <= K; ++i) HJ_CUDA(c, cudaEventCreateWithFlags(&c->cev[i], cudaEventDisableTiming));
    }
    HJ_CUDA(c, cudaEventRecord(c->cev[K], c->stream));
    const uint64_t piece = (bytes / K + 255) & ~uint64_t(255);
    for (int i = 0; i < K; ++i) {
        const uint64_t off = (uint64_t)i * piece;
        if (off >= bytes) break;
        const uint64_t len = bytes - off < piece ? bytes - off : piece;
        HJ_CUDA(c, cudaStreamWaitEvent(c->cstream[i], c->cev[K], 0));
        HJ_CUDA(c, cudaMemcpyAsync((char *)dst + off, (const char *)src + off, len, kind, c->cstream[i]));
        HJ_CUDA(c, cudaEventRecord(c->cev[i], c->cstream[i]));
        HJ_CUDA(c, cudaStreamWaitEvent(c->stream, c->cev[i], 0));
    }
    return HJ_OK;
}

int num_sms(hj_ctx *c) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device);
    return n > 0 ? n : 1;
}

}  // namespace hj

using namespace hj;

extern "C" {

hj_status hj_create(hj_ctx **out, int device, void *cuda_stream, uint64_t budget) {
    return hj::ctx_create(out, device, cuda_stream, budget, nullptr);
}

}  // extern "C"

namespace hj {

hj_status ctx_create(hj_ctx **out, int device, void *cuda_stream, uint64_t budget, cudaMemPool_t shared_pool) {
    if (!out) return HJ_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HJ_E_INVALID;
    }
    hj_ctx *c = new hj_ctx();
    c->device = device;
    c->budget = budget;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e == cudaSuccess && shared_pool) {
        c->pool = shared_pool;
        c->own_pool = false;
    } else if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&c->pool, &props);
    }
    if (e == cudaSuccess && c->own_pool) {
        uint64_t keep = ~0ull;  // keep freed blocks for reuse by later joins
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ctr, sizeof(hj_counters));
    if (e == cudaSuccess) e = cudaMemset(c->d_ctr, 0, sizeof(hj_counters));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_ctr, sizeof(hj_counters));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->d_ctr) cudaFree(c->d_ctr);
        if (c->pool && c->own_pool) cudaMemPoolDestroy(c->pool);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return HJ_E_CUDA;
    }
    *out = c;
    return HJ_OK;
}

}  // namespace hj

extern "C" {

hj_status hj_destroy(hj_ctx *c) {
    if (!c) return HJ_E_INVALID;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->allocs) cudaFreeAsync(kv.first, c->stream);
    cudaStreamSynchronize(c->stream);
    c->allocs.clear();
    for (auto &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->spare_events) cudaEventDestroy(e);
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    for (void *hb : c->host_buf)
        if (hb) cudaFreeHost(hb);
    if (c->pipe_in) cudaStreamDestroy(c->pipe_in);
    if (c->pipe_out) cudaStreamDestroy(c->pipe_out);
    for (auto &row : c->pipe_ev)
        for (cudaEvent_t e : row)
            if (e) cudaEventDestroy(e);
    if (c->pipe_h) cudaFreeHost(c->pipe_h);
    for (int i = 0; i < hj_ctx::kCopyStreams; ++i)
        if (c->cstream[i]) cudaStreamDestroy(c->cstream[i]);
    for (int i = 0; i <= hj_ctx::kCopyStreams; ++i)
        if (c->cev[i]) cudaEventDestroy(c->cev[i]);
    if (c->pool && c->own_pool) cudaMemPoolDestroy(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->cpu_pool) hj::cpu_pool_delete(c->cpu_pool);
    delete c;
    return HJ_OK;
}

const char *hj_last_error(const hj_ctx *c) { return c ? c->err.c_str() : "null context"; }

hj_status hj_sync(hj_ctx *c) {
    if (!c) return HJ_E_INVALID;
    cudaSetDevice(c->device);
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    return HJ_OK;
}

hj_status hj_prof_enable(hj_ctx *c, int on) {
    if (!c) return HJ_E_INVALID;
    c->prof = on != 0;
    return HJ_OK;
}

hj_status hj_prof_only(hj_ctx *c, const char *name) {
    if (!c) return HJ_E_INVALID;
    if (name && strlen(name) >= sizeof(hj_prof_entry{}.name)) return set_err(c, HJ_E_INVALID, "kernel name too long");
    c->prof_only = name ? name : "";
    return HJ_OK;
}

hj_status hj_prof_reset(hj_ctx *c) {
    if (!c) return HJ_E_INVALID;
    cudaStreamSynchronize(c->stream);
    prof_collect(c);
    c->prof_acc.clear();
    return HJ_OK;
}

hj_status hj_prof_read(hj_ctx *c, hj_prof_entry *ent, int cap, int *n_out) {
    if (!c || !n_out || (cap > 0 && !ent)) return HJ_E_INVALID;
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    prof_collect(c);
    int i = 0;
    for (auto &kv : c->prof_acc) {
        if (i < cap) {
            memset(ent[i].name, 0, sizeof ent[i].name);
            strncpy(ent[i].name, kv.first.c_str(), sizeof ent[i].name - 1);
            ent[i].launches = kv.second.first;
            ent[i].ms = kv.second.second;
        }
        i++;
    }
    *n_out = i;
    return HJ_OK;
}

uint64_t hj_launch_count(const hj_ctx *c) { return c ? c->launches : 0; }

/* Test hook: make the n-th device allocation from now fail with HJ_E_NOMEM
 * (n < 0 disarms).  Host-side fault injection; no GPU fault is involved. */
hj_status hj_debug_fail_alloc(hj_ctx *c, int64_t n) {
    if (!c) return HJ_E_INVALID;
    c->fail_alloc_after = n;
    return HJ_OK;
}

uint64_t hj_debug_bytes_in_use(const hj_ctx *c) { return c ? c->in_use : 0; }

/* Test hook: the most device bytes held at once since creation or the last reset;
 * a reset restarts the count from the bytes held now. */
uint64_t hj_debug_peak_bytes(hj_ctx *c, int reset) {
    if (!c) return 0;
    const uint64_t p = c->peak;
    if (reset) c->peak = c->in_use;
    return p;
}

/* Test and measurement hook: hj_join_host_large's plan (HJ_OUTCORE_*). */
hj_status hj_debug_outcore(hj_ctx *c, int mode) {
    if (!c || mode < HJ_OUTCORE_AUTO || mode > HJ_OUTCORE_SPLIT) return HJ_E_INVALID;
    c->outcore_mode = mode;
    return HJ_OK;
}

/* Test hook: limits of the bounded waits (ring scatter flush passes, n; TMA-staged
 * scatter mbarrier polls, n - 1) before a kernel gives up and the call reports
 * HJ_E_TIMEOUT; 0 restores the defaults. */
hj_status hj_debug_wait_limit(hj_ctx *c, uint64_t n) {
    if (!c) return HJ_E_INVALID;
    c->wait_limit = n;
    return HJ_OK;
}

/* Measurement hook: force the region or the ring scatter (HJ_SCATTER_*). */
hj_status hj_debug_scatter(hj_ctx *c, int kind) {
    if (!c || kind < HJ_SCATTER_AUTO || kind > HJ_SCATTER_RING) return HJ_E_INVALID;
    c->scatter_kind = kind;
    return HJ_OK;
}

}  // extern "C"
