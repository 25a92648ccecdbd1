// batch.cu -- many independent joins in a few launches (hj_join_batch).
//
// Joins are grouped by the radix bits their build size calls for (about 8192 build
// tuples per partition, at least one bit so that every partition is padded and
// filtered the same way).  Per group, one partition pass partitions every join's R
// (then every join's S) at once, reading each relation in place; then ONE
// persistent launch of the shared-memory join kernel runs every (join, partition)
// task of every group, taking tasks from a work counter so that joins of very
// different sizes share the GPU.  Pairs are placed by exact per-task claims into
// each join's own buffer (the staging sink), so no compaction is needed.  When the
// workspace of all joins would exceed the HBM budget, joins run in waves.  With
// HJ_FLAG_GRAPH the device work of a wave is captured into a CUDA graph and
// launched as one graph.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "common.cuh"
#include "emit.cuh"
#include "engine.cuh"

using namespace hj;

namespace {

constexpr uint32_t kStagePairs = 256;  // staging rows per warp (>= 32 x the items of a probe group)

int join_bits(uint64_t nR) {
    int b = 1;
    while (b < 11 && (nR >> b) > 8192) b++;
    return b;
}

__global__ void batch_tasks_kernel(const void *Rp, const uint64_t *roff, const void *Sp, const uint64_t *soff,
                                   const uint32_t *join_ids, uint64_t ngroup, int bits, uint64_t ek1, uint64_t pk1,
                                   int tb, PartTask *tasks) {
    const uint64_t P = 1ull << bits, n = ngroup * P;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t g = i >> bits, p = i & (P - 1);
        PartTask t;
        t.R = (const char *)Rp + roff[i] * tb;
        t.S = (const char *)Sp + soff[i] * tb;
        t.nr = (uint32_t)(roff[i + 1] - roff[i]);
        t.ns = (uint32_t)(soff[i + 1] - soff[i]);
        t.join = join_ids[g];
        t.p = (uint32_t)p;
        t.b1 = (uint16_t)bits;
        t.b2 = 0;
        t.pad = 0;
        t.ek1 = ek1;
        t.pk1 = pk1;
        t.pk2 = 0;
        tasks[i] = t;
    }
}

__global__ void batch_slots_kernel(JoinSlot *slots, void *const *pairs, const unsigned long long *caps,
                                   hj_counters *ctrs, uint64_t n) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        slots[j].pairs = pairs[j];
        slots[j].pcap = caps[j];
        slots[j].ctr = ctrs + j;
        slots[j].pad = 0;
    }
}

template <class T> hj_status upload(hj_ctx *c, const std::vector<T> &v, DevBuf &out) {
    HJ_TRY(out.alloc(std::max<size_t>(v.size(), 1) * sizeof(T)));
    if (!v.empty()) HJ_CUDA(c, cudaMemcpyAsync(out.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return HJ_OK;
}

struct Group {
    int bits;
    std::vector<uint32_t> joins;  // indices into the batch
};

// One wave: per group the device copies of the segment tables (prepared and
// uploaded before any capture), then the device work (partition passes, task
// list, join launch), which can be captured.
struct GroupDev {
    int bits;
    uint64_t ng, nr, ns;
    DevBuf ro, so, rp, sp, jid;
    explicit GroupDev(hj_ctx *c) : ro(c), so(c), rp(c), sp(c), jid(c) {}
};

struct Wave {
    std::vector<std::unique_ptr<GroupDev>> groups;
    std::vector<std::unique_ptr<DevBuf>> bufs;
    DevBuf *tasks = nullptr;
    uint64_t ntasks = 0;
    DevBuf *oversize = nullptr;
};

DevBuf *newbuf(hj_ctx *c, Wave &w) {
    w.bufs.push_back(std::make_unique<DevBuf>(c));
    return w.bufs.back().get();
}

hj_status prepare_wave(hj_ctx *c, const hj_rel *Rs, const hj_rel *Ss, const std::vector<Group> &groups, Wave &w) {
    for (auto &g : groups) {
        auto gd = std::make_unique<GroupDev>(c);
        const uint64_t ng = g.joins.size();
        std::vector<uint64_t> ro(ng + 1), so(ng + 1);
        std::vector<const void *> rp(ng), sp(ng);
        ro[0] = so[0] = 0;
        for (uint64_t i = 0; i < ng; ++i) {
            const uint32_t j = g.joins[i];
            ro[i + 1] = ro[i] + Rs[j].n;
            so[i + 1] = so[i] + Ss[j].n;
            rp[i] = Rs[j].tuples;
            sp[i] = Ss[j].tuples;
        }
        gd->bits = g.bits;
        gd->ng = ng;
        gd->nr = ro[ng];
        gd->ns = so[ng];
        HJ_TRY(upload(c, ro, gd->ro));
        HJ_TRY(upload(c, so, gd->so));
        HJ_TRY(upload(c, rp, gd->rp));
        HJ_TRY(upload(c, sp, gd->sp));
        HJ_TRY(upload(c, g.joins, gd->jid));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vectors end here
        w.groups.push_back(std::move(gd));
    }
    return HJ_OK;
}

hj_status launch_wave(hj_ctx *c, int W, const JoinSlot *slots, bool agg, bool chk, Wave &w, DevBuf &stage) {
    const uint64_t tb = tuple_bytes(W);
    uint64_t ntasks = 0;
    for (auto &g : w.groups) ntasks += g->ng << g->bits;
    w.tasks = newbuf(c, w);
    HJ_TRY(w.tasks->alloc(std::max<uint64_t>(ntasks, 1) * sizeof(PartTask)));
    uint64_t task_at = 0;
    for (auto &g : w.groups) {
        const uint64_t ng = g->ng, P = 1ull << g->bits;
        const uint64_t rrows = partition_out_rows(c, W, g->nr, ng, g->bits, 1);
        const uint64_t srows = partition_out_rows(c, W, g->ns, ng, g->bits, 1);
        DevBuf *Rp = newbuf(c, w), *Sp = newbuf(c, w), *roff = newbuf(c, w), *soff = newbuf(c, w);
        HJ_TRY(Rp->alloc(rrows * tb + 64));
        HJ_TRY(Sp->alloc(srows * tb + 64));
        HJ_TRY(roff->alloc((ng * P + 1) * 8));
        HJ_TRY(soff->alloc((ng * P + 1) * 8));
        HJ_TRY(partition_pass(c, W, nullptr, g->nr, g->ro.as<uint64_t>(), ng, 0, g->bits, Rp->p, roff->as<uint64_t>(), 1,
                              (const void *const *)g->rp.p));
        HJ_TRY(partition_pass(c, W, nullptr, g->ns, g->so.as<uint64_t>(), ng, 0, g->bits, Sp->p, soff->as<uint64_t>(), 1,
                              (const void *const *)g->sp.p));
        const uint64_t n = ng * P;
        const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms(c) * 8);
        HJ_LAUNCH(c, "batch_tasks", batch_tasks_kernel, grid ? grid : 1, 256, 0, Rp->p, roff->as<uint64_t>(), Sp->p,
                  soff->as<uint64_t>(), g->jid.as<uint32_t>(), ng, g->bits, empty_key2(W, g->bits, 0),
                  pass_pad_key(W, 0, g->bits), (int)tb,
                  w.tasks->as<PartTask>() + task_at);
        task_at += n;
    }
    w.ntasks = ntasks;
    w.oversize = newbuf(c, w);
    HJ_TRY(w.oversize->alloc(std::max<uint64_t>(ntasks, 1) * 4));
    RecArea ra{nullptr, nullptr, 0};
    HJ_TRY(partition_join(c, W, agg, w.tasks->as<PartTask>(), ntasks, slots, 8192, chk, w.oversize->as<uint32_t>(), ra,
                          agg ? nullptr : stage.p, kStagePairs));
    return HJ_OK;
}

bool is_agg(int mode) { return mode == HJ_COUNT || mode == HJ_COUNT_CHECKSUM; }

}  // namespace

extern "C" hj_status hj_join_batch(hj_ctx *c, int n, const hj_rel *Rs, const hj_rel *Ss, const hj_opts *opts,
                                   hj_result *outs) {
    if (!c) return HJ_E_INVALID;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    if (n < 0 || (n > 0 && (!Rs || !Ss || !outs))) return set_err(c, HJ_E_INVALID, "bad batch arguments");
    if (n == 0) return HJ_OK;
    hj_opts o{};
    o.mode = HJ_MATERIALIZE;
    if (opts) o = *opts;
    if (o.mode < HJ_COUNT || o.mode > HJ_MATERIALIZE) return set_err(c, HJ_E_INVALID, "bad mode %d", o.mode);
    const int W = Rs[0].width;
    for (int j = 0; j < n; ++j) {
        for (const hj_rel *r : {&Rs[j], &Ss[j]}) {
            if (r->width != W) return set_err(c, HJ_E_INVALID, "join %d: all relations of a batch share one width", j);
            if (r->n && (!r->tuples || ((uintptr_t)r->tuples & 15)))
                return set_err(c, HJ_E_INVALID, "join %d: tuples NULL or not 16-byte aligned", j);
            if (r->n >= 0xFFFFFFFFull) return set_err(c, HJ_E_INVALID, "join %d: relation too large for a batch", j);
        }
        outs[j] = hj_result{};
    }
    if (W != HJ_U32 && W != HJ_U64) return set_err(c, HJ_E_INVALID, "width %d is not 4 or 8", W);
    const bool agg = is_agg(o.mode), mat = o.mode == HJ_MATERIALIZE;
    const bool chk = o.mode == HJ_COUNT_CHECKSUM || (mat && (o.flags & HJ_FLAG_CHECKSUM));
    const bool graph = (o.flags & HJ_FLAG_GRAPH) != 0;
    const uint64_t tb = tuple_bytes(W);

    // per-join output buffers and counters
    std::vector<uint64_t> cap(n, 0);
    std::vector<void *> pairs(n, nullptr);
    auto release_pairs = [&]() {
        for (int j = 0; j < n; ++j) dfree(c, pairs[j]);
    };
    // workspace per join: partitioned copies of R and S, and the pair buffer
    auto need = [&](int j) {
        uint64_t ws = (Rs[j].n + Ss[j].n) * tb * 11 / 10 + 8192 * tb;
        if (mat) ws += (Ss[j].n + 64) * tb;
        return ws;
    };
    // free device memory plus what the context's pool holds reserved but unused
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    unsigned long long reserved = 0, used_pool = 0;  // the attributes are 64-bit
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &used_pool);
    const uint64_t avail = freeb + (reserved > used_pool ? reserved - used_pool : 0);
    uint64_t budget = (uint64_t)(avail * 0.7);
    if (c->budget) budget = std::min<uint64_t>(budget, c->budget > c->in_use ? (c->budget - c->in_use) * 9 / 10 : 0);

    // waves
    std::vector<std::vector<int>> waves;
    {
        std::vector<int> cur;
        uint64_t used = 0;
        for (int j = 0; j < n; ++j) {
            if (!Rs[j].n || !Ss[j].n) continue;  // empty joins have no pairs
            const uint64_t w = need(j);
            if (!cur.empty() && used + w > budget) {
                waves.push_back(cur);
                cur.clear();
                used = 0;
            }
            cur.push_back(j);
            used += w;
        }
        if (!cur.empty()) waves.push_back(cur);
    }
    DevBuf ctrs(c), slots(c), dpairs(c), dcaps(c), stage(c);
    if (!agg) HJ_TRY(stage.alloc(partition_join_warps(c) * kStagePairs * tb));
    HJ_TRY(ctrs.alloc((uint64_t)n * sizeof(hj_counters)));
    HJ_TRY(slots.alloc((uint64_t)n * sizeof(JoinSlot)));
    HJ_CUDA(c, cudaMemsetAsync(ctrs.p, 0, (uint64_t)n * sizeof(hj_counters), c->stream));
    std::vector<hj_counters> hc(n);
    for (auto &wj : waves) {
        // pair buffers of this wave's joins
        std::vector<unsigned long long> caps(n, 0);
        std::vector<void *> ptrs(n, nullptr);
        for (int j : wj) {
            if (mat) {
                cap[j] = (o.out_capacity ? o.out_capacity : Ss[j].n) + 64;
                hj_status st;
                pairs[j] = dalloc(c, cap[j] * tb, &st);
                if (st != HJ_OK) {
                    release_pairs();
                    return st;
                }
            }
            caps[j] = cap[j];
            ptrs[j] = pairs[j];
        }
        {
            hj_status st = upload(c, ptrs, dpairs);
            if (st == HJ_OK) st = upload(c, caps, dcaps);
            if (st != HJ_OK) {
                release_pairs();
                return st;
            }
        }
        const unsigned sg = (unsigned)std::min<uint64_t>(((uint64_t)n + 255) / 256, 1024);
        HJ_LAUNCH(c, "batch_slots", batch_slots_kernel, sg, 256, 0, slots.as<JoinSlot>(), (void *const *)dpairs.p,
                  dcaps.as<unsigned long long>(), ctrs.as<hj_counters>(), (uint64_t)n);
        // groups by radix bits
        std::vector<Group> groups;
        for (int b = 1; b <= 11; ++b) {
            Group g{b, {}};
            for (int j : wj)
                if (join_bits(Rs[j].n) == b) g.joins.push_back((uint32_t)j);
            if (!g.joins.empty()) groups.push_back(g);
        }
        HJ_TRY(zero_counters(c));  // the work counter of the join launch
        Wave w;
        hj_status st = prepare_wave(c, Rs, Ss, groups, w);
        if (st != HJ_OK) {
            release_pairs();
            return st;
        }
        if (graph) {
            // The wave is captured on a private stream (the context's stream may be
            // the legacy default stream, which cannot be captured) and the graph is
            // launched on the context's stream, after the work already queued there.
            const bool prof = c->prof;
            c->prof = false;
            cudaGraph_t g = nullptr;
            cudaStream_t orig = c->stream, cap = nullptr;
            HJ_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            c->stream = cap;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = launch_wave(c, W, slots.as<JoinSlot>(), agg, chk, w, stage);
                e = cudaStreamEndCapture(cap, &g);
            }
            c->stream = orig;
            cudaStreamDestroy(cap);
            c->prof = prof;
            if (st == HJ_OK && e != cudaSuccess) st = cuda_err(c, e, "wave capture");
            cudaGraphExec_t ge = nullptr;
            if (st == HJ_OK) {
                e = cudaGraphInstantiate(&ge, g, 0);
                if (e != cudaSuccess) st = cuda_err(c, e, "cudaGraphInstantiate");
            }
            if (st == HJ_OK) {
                e = cudaGraphLaunch(ge, c->stream);  // its kernels were counted at capture
                if (e != cudaSuccess) st = cuda_err(c, e, "cudaGraphLaunch");
            }
            if (st == HJ_OK) {
                e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) st = cuda_err(c, e, "graph execution");
            }
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
        } else {
            st = launch_wave(c, W, slots.as<JoinSlot>(), agg, chk, w, stage);
        }
        if (st == HJ_OK) st = read_counters(c);
        if (st == HJ_OK && c->h_ctr->n_oversize) {
            std::vector<JoinSlot> sh(n);
            for (int j = 0; j < n; ++j)
                sh[j] = JoinSlot{pairs[j], cap[j], ctrs.as<hj_counters>() + j, 0};
            st = oversize_fallback(c, W, agg, chk, w.tasks->as<PartTask>(), w.oversize->as<uint32_t>(),
                                   c->h_ctr->n_oversize, sh);
            if (st == HJ_OK) st = read_counters(c);
        }
        if (st == HJ_OK && (c->h_ctr->status & (kStatusTableFull | kStatusTimeout)))
            st = set_err(c, HJ_E_CUDA, "a batch kernel reported status %llu", (unsigned long long)c->h_ctr->status);
        if (st != HJ_OK) {
            release_pairs();
            return st;
        }
    }
    HJ_CUDA(c, cudaMemcpyAsync(hc.data(), ctrs.p, (uint64_t)n * sizeof(hj_counters), cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int j = 0; j < n; ++j) {
        hj_result &r = outs[j];
        r.count = hc[j].count;
        r.checksum[0] = hc[j].c0;
        r.checksum[1] = hc[j].c1;
        r.width = W;
        r.algo = HJ_ALGO_PHJ;
        r.radix_bits = join_bits(Rs[j].n);
        r.passes = 1;
        r.pairs = mat ? pairs[j] : nullptr;
        r.pairs_cap = mat ? cap[j] : 0;
        if (!mat && pairs[j]) dfree(c, pairs[j]);
    }
    // joins with more pairs than their buffer: run again alone at the exact size
    if (mat) {
        for (int j = 0; j < n; ++j) {
            if (outs[j].count <= cap[j] || !Rs[j].n || !Ss[j].n) continue;
            dfree(c, outs[j].pairs);
            outs[j] = hj_result{};
            hj_opts oj = o;
            oj.algo = HJ_ALGO_AUTO;
            oj.flags &= ~(uint64_t)HJ_FLAG_GRAPH;
            oj.out_capacity = hc[j].count;
            hj_status st = hj_join(c, &Rs[j], &Ss[j], &oj, &outs[j]);
            if (st != HJ_OK) {
                for (int i = 0; i < n; ++i) hj_result_free(c, &outs[i]);
                return st;
            }
        }
    }
    return HJ_OK;
}
