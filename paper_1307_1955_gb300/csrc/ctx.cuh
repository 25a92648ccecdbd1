// ctx.cuh -- host-side engine state behind an hj_ctx: the device, the stream, a
// stream-ordered memory pool with an HBM budget, the last error text, a small
// device counter block, and optional per-kernel event timing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/hj.h"

// Counters every join kernel accumulates into (device, zeroed per join).
struct hj_counters {
    unsigned long long count;      // pairs found
    unsigned long long c0, c1;     // checksums
    unsigned long long n_oversize; // partitions left to the global-table fallback
    unsigned long long status;     // kStatus* bits
    unsigned long long cursor;     // output slots handed out in whole chunks (pairs + holes)
    unsigned long long work;       // next partition for the persistent join kernel
    // Sticky fault bits of partition passes (kStatus* bits; a bounded wait that
    // expired).  zero_counters leaves this word alone, so that a fault of a pass
    // queued before a join's counters are cleared still reaches the host;
    // read_counters reports and clears it.
    unsigned long long fault;
};

namespace hj {
// Device figures the plan cost model works from (defaults: GB300).
struct CostModel {
    int sms = 152;
    double sm_hz = 2.07e9;
    double hbm_bps = 8.18e12;   // nominal: 2 x memory clock x bus width
    double l2_bytes = 126e6;
};
struct TunedPlan {
    int algo, bits, passes;
};
struct CpuPool;
void cpu_pool_delete(CpuPool *p);
}  // namespace hj

struct hj_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t budget = 0;  // 0 = unlimited
    uint64_t in_use = 0;
    uint64_t peak = 0;
    std::unordered_map<void *, uint64_t> allocs;
    cudaMemPool_t pool = nullptr;
    bool own_pool = true;  // false: the pool belongs to a server that shares it among its workers
    std::string err;
    hj_counters *d_ctr = nullptr;      // device counters
    hj_counters *h_ctr = nullptr;      // pinned host mirror
    // profiling
    bool prof = false;
    bool prof_open = false;   // the last launch was bracketed (its end event is due)
    std::string prof_only;    // bracket only this kernel ("" = all)
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> spare_events;
    std::map<std::string, std::pair<uint64_t, double>> prof_acc;
    uint64_t launches = 0;
    // plan choice: cost model of the device, and plans measured by hj_tune per size class
    hj::CostModel model;
    bool model_ready = false;
    std::map<uint64_t, hj::TunedPlan> tuned;
    // side streams and events that split large host<->device copies over several
    // copy engines (created on first use)
    static constexpr int kCopyStreams = 4;
    cudaStream_t cstream[kCopyStreams] = {};
    cudaEvent_t cev[kCopyStreams + 1] = {};
    // pipelined host joins: copy-in and copy-out streams, per-buffer-set events
    // and page-locked counter copies (created on first use)
    cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
    cudaEvent_t pipe_ev[2][3] = {};
    void *pipe_h = nullptr;
    // page-locked host buffers kept for hj_join_host_large (R side, S side)
    void *host_buf[2] = {nullptr, nullptr};
    uint64_t host_cap[2] = {0, 0};
    // co-processing: host worker threads (created on first use)
    hj::CpuPool *cpu_pool = nullptr;
    // test hooks (host-side fault injection)
    int64_t fail_alloc_after = -1;  // fail the N-th allocation from now (0 = next)
    uint64_t wait_limit = 0;        // bounded device waits: passes / polls before giving up (0 = default)
    int scatter_kind = 0;           // HJ_SCATTER_*: padded-pass scatter at 2^9 .. 2^11 digits
    int outcore_mode = 0;           // HJ_OUTCORE_*: hj_join_host_large's plan
};

struct hj_table {
    int width = 4;
    int agg = 0;          // 1: aggregate table (count modes), 0: pairs (pair or key-list table)
    void *slots = nullptr;
    uint64_t cap = 0;
    void *side = nullptr; // hj::TableSide on the device
    int keylist = 0;      // 1: aggregate-table slots plus rid lists (heavily repeated build keys)
    void *rids = nullptr; // key-list table: every key's rids, contiguous
    uint64_t nr = 0;      // key-list table: build tuples (size of rids)
};

namespace hj {

hj_status set_err(hj_ctx *c, hj_status code, const char *fmt, ...);
hj_status cuda_err(hj_ctx *c, cudaError_t e, const char *what);
void *dalloc(hj_ctx *c, uint64_t bytes, hj_status *st);
void dfree(hj_ctx *c, void *p);

// Kernel launch bracketed by profiling events when enabled.
void prof_begin(hj_ctx *c, const char *name);
void prof_end(hj_ctx *c);
hj_status check_launch(hj_ctx *c, const char *name);

// Read the counter block back (synchronises the stream).
hj_status read_counters(hj_ctx *c);
hj_status zero_counters(hj_ctx *c);

int num_sms(hj_ctx *c);

// Let `func` take up to the device's opt-in maximum of dynamic shared memory.
// Always the same value per function, so concurrent callers on several threads
// (the server's workers) cannot undo each other's setting between set and launch.
hj_status allow_max_smem(hj_ctx *c, const void *func);

// cudaMemcpyAsync of a large host<->device range, ordered on the context's
// stream, split into pieces copied concurrently on side streams (several copy
// engines); small copies go straight to the context's stream.
hj_status copy_wide(hj_ctx *c, void *dst, const void *src, uint64_t bytes, cudaMemcpyKind kind);

// hj_create with an existing memory pool (not owned: hj_destroy leaves it alone).
hj_status ctx_create(hj_ctx **out, int device, void *cuda_stream, uint64_t budget, cudaMemPool_t shared_pool);

// A device buffer from the context's pool, released when the guard goes out of
// scope unless ownership is taken with release().
struct DevBuf {
    hj_ctx *c;
    void *p = nullptr;
    explicit DevBuf(hj_ctx *ctx) : c(ctx) {}
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    hj_status alloc(uint64_t bytes) {
        reset();
        hj_status st;
        p = dalloc(c, bytes, &st);
        return st;
    }
    void reset() {
        if (p) dfree(c, p);
        p = nullptr;
    }
    void *release() {
        void *q = p;
        p = nullptr;
        return q;
    }
    template <class T> T *as() const { return (T *)p; }
};

}  // namespace hj

#define HJ_LAUNCH(ctx, name, kernel, grid, block, smem, ...)                 \
    do {                                                                     \
        hj::prof_begin((ctx), (name));                                       \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);    \
        hj::prof_end(ctx);                                                   \
        hj_status _st = hj::check_launch((ctx), (name));                     \
        if (_st != HJ_OK) return _st;                                        \
    } while (0)

#define HJ_CUDA(ctx, call)                                                   \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return hj::cuda_err((ctx), _e, #call);       \
    } while (0)

#define HJ_TRY(expr)                                                         \
    do {                                                                     \
        hj_status _s = (expr);                                               \
        if (_s != HJ_OK) return _s;                                          \
    } while (0)
