// api.cu -- the C ABI of include/hj.h: argument checks, plan choice, and the
// SHJ / PHJ drivers that sequence the kernels of join.cu and partition.cu.
#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cmath>
#include <memory>
#include <thread>
#include <vector>

#include "common.cuh"
#include "emit.cuh"
#include "engine.cuh"

using namespace hj;

namespace hj {

// A global table released when it goes out of scope.
struct TableHold {
    hj_ctx *c;
    hj_table *t = nullptr;
    ~TableHold() { table_destroy(c, t); }
};

// Partitions whose table did not fit in shared memory (a heavily repeated key, or
// more build rows than the table holds): per join, the R rows of every such
// partition and the S rows of every such task are gathered into two compact
// arrays (rows of another partition -- the padding -- dropped by their hash), and
// one global table over the gathered R serves all of them: partitions are
// disjoint in key, so one table per join is the union of the per-partition
// tables.  Pairs come from a key-list table (one entry per distinct key, its rids
// in one list; Sec. 3.1's layout), count modes use the aggregate table.  A fixed
// number of launches per join, however many partitions fall back; a join with a
// single such partition uses its rows in place, with the partition filter.
namespace fallback {

struct GatherRange {
    const void *ptr;
    uint64_t n;
    uint32_t p;
    uint16_t b1, b2;
};

__global__ void pick_tasks_kernel(const PartTask *tasks, const uint32_t *list, uint64_t n, PartTask *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = tasks[list[i]];
}

// Rows of the listed ranges whose key falls in the range's partition, appended to
// `out` (cap rows) at positions taken by one atomic add per warp and step.
template <int W>
__global__ void __launch_bounds__(256) gather_rows_kernel(const GatherRange *rg, uint64_t nrg, void *out, uint64_t cap,
                                                          unsigned long long *count, unsigned long long *fault) {
    using U = typename Tup<W>::U;
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    U *o = (U *)out;
    for (uint64_t r = blockIdx.x; r < nrg; r += gridDim.x) {
        const GatherRange g = rg[r];
        const PartFilter pf{g.p, (int)g.b1, (int)g.b2, 1};
        const U *t = (const U *)g.ptr;
        for (uint64_t i0 = 0; i0 < g.n; i0 += blockDim.x) {
            const uint64_t i = i0 + threadIdx.x;
            U k = 0, rid = 0;
            bool keep = false;
            if (i < g.n) {
                k = t[2 * i];
                rid = t[2 * i + 1];
                keep = pf.keep(key_hash<W>(k));
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            unsigned long long base = 0;
            if (lane == 0 && m) base = atomicAdd(count, (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (keep) {
                const unsigned long long at = base + __popc(m & lt);
                if (at < cap) {
                    o[2 * at] = k;
                    o[2 * at + 1] = rid;
                } else {  // cannot happen (cap is the ranges' total): reported, never written
                    atomicOr(fault, (unsigned long long)kStatusBadInput);
                }
            }
        }
    }
}

// Gather the rows of `ranges` into a new array; *rows gets the number kept.
hj_status gather_rows(hj_ctx *c, int W, const std::vector<GatherRange> &ranges, DevBuf &out, uint64_t *rows) {
    uint64_t cap = 0;
    for (const GatherRange &g : ranges) cap += g.n;
    *rows = 0;
    if (!cap) return HJ_OK;
    // pieces of at most 2^16 rows, so that a large partition spreads over the SMs
    constexpr uint64_t kPiece = 1ull << 16;
    std::vector<GatherRange> pieces;
    for (const GatherRange &g : ranges)
        for (uint64_t at = 0; at < g.n; at += kPiece)
            pieces.push_back(GatherRange{(const char *)g.ptr + at * tuple_bytes(W), std::min(kPiece, g.n - at), g.p,
                                         g.b1, g.b2});
    const uint64_t tb = tuple_bytes(W);
    DevBuf rg(c), cnt(c);
    HJ_TRY(out.alloc(cap * tb + 64));
    HJ_TRY(rg.alloc(pieces.size() * sizeof(GatherRange)));
    HJ_TRY(cnt.alloc(8));
    HJ_CUDA(c, cudaMemcpyAsync(rg.p, pieces.data(), pieces.size() * sizeof(GatherRange), cudaMemcpyHostToDevice,
                               c->stream));
    HJ_CUDA(c, cudaMemsetAsync(cnt.p, 0, 8, c->stream));
    const unsigned grid = (unsigned)std::min<uint64_t>(pieces.size(), (uint64_t)num_sms(c) * 8);
    if (W == 4)
        HJ_LAUNCH(c, "fallback_gather", gather_rows_kernel<4>, grid, 256, 0, rg.as<GatherRange>(),
                  (uint64_t)pieces.size(), out.p, cap, cnt.as<unsigned long long>(), &c->d_ctr->fault);
    else
        HJ_LAUNCH(c, "fallback_gather", gather_rows_kernel<8>, grid, 256, 0, rg.as<GatherRange>(),
                  (uint64_t)pieces.size(), out.p, cap, cnt.as<unsigned long long>(), &c->d_ctr->fault);
    HJ_CUDA(c, cudaMemcpyAsync(rows, cnt.p, 8, cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    return HJ_OK;
}

}  // namespace fallback

FallbackGroup::~FallbackGroup() { table_destroy(c, t); }

hj_status fallback_reprobe(hj_ctx *c, bool chk, const FallbackRedo &redo, const JoinSlot &slot) {
    for (const auto &g : redo.groups)
        HJ_TRY(keylist_probe(c, g->t, g->S, g->ns, g->pf, slot.pairs, slot.pcap, slot.ctr, chk));
    return HJ_OK;
}

hj_status oversize_fallback(hj_ctx *c, int W, bool agg, bool chk, const PartTask *tasks, const uint32_t *list_dev,
                            uint64_t nov, const std::vector<JoinSlot> &slots_host, FallbackRedo *redo) {
    hj_counters prev{};
    if (redo) prev = *c->h_ctr;  // the caller read the counters last
    std::vector<PartTask> tk(nov);
    {
        DevBuf picked(c);
        HJ_TRY(picked.alloc(nov * sizeof(PartTask)));
        const unsigned grid = (unsigned)std::min<uint64_t>((nov + 255) / 256, (uint64_t)num_sms(c) * 8);
        HJ_LAUNCH(c, "fallback_tasks", fallback::pick_tasks_kernel, grid ? grid : 1, 256, 0, tasks, list_dev, nov,
                  picked.as<PartTask>());
        HJ_CUDA(c, cudaMemcpyAsync(tk.data(), picked.p, nov * sizeof(PartTask), cudaMemcpyDeviceToHost, c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    // the tasks of each join; the R side of a partition once (its S slices share it)
    std::sort(tk.begin(), tk.end(), [](const PartTask &a, const PartTask &b) {
        return a.join != b.join ? a.join < b.join : a.R < b.R;
    });
    for (size_t i = 0; i < tk.size();) {
        const uint32_t join = tk[i].join;
        std::vector<fallback::GatherRange> rr, ss;
        size_t j = i;
        for (; j < tk.size() && tk[j].join == join; ++j) {
            const PartTask &t = tk[j];
            if (j == i || t.R != tk[j - 1].R) rr.push_back(fallback::GatherRange{t.R, t.nr, t.p, t.b1, t.b2});
            ss.push_back(fallback::GatherRange{t.S, t.ns, t.p, t.b1, t.b2});
        }
        i = j;
        if (join >= slots_host.size()) return set_err(c, HJ_E_CUDA, "fallback task of unknown join %u", join);
        const JoinSlot &js = slots_host[join];
        DevBuf Rg(c), Sg(c);
        const void *Rt, *St;
        uint64_t nr = 0, ns = 0;
        PartFilter pf{0, 0, 0, 0};
        if (rr.size() == 1) {
            // one partition: its rows in place, padding dropped by the partition
            // filter; its S slices too when they are one gapless run (a slice whose
            // own build fitted has been probed already and must not be again)
            const uint64_t tb = tuple_bytes(W);
            std::sort(ss.begin(), ss.end(), [](const fallback::GatherRange &a, const fallback::GatherRange &b) {
                return (const char *)a.ptr < (const char *)b.ptr;
            });
            bool run = true;
            for (size_t q = 1; q < ss.size(); ++q)
                run &= (const char *)ss[q].ptr == (const char *)ss[q - 1].ptr + ss[q - 1].n * tb;
            Rt = rr[0].ptr;
            nr = rr[0].n;
            pf = PartFilter{rr[0].p, (int)rr[0].b1, (int)rr[0].b2, 1};
            if (run) {
                St = ss[0].ptr;
                for (const auto &g : ss) ns += g.n;
            } else {
                HJ_TRY(fallback::gather_rows(c, W, ss, Sg, &ns));
                St = Sg.p;
            }
        } else {
            HJ_TRY(fallback::gather_rows(c, W, rr, Rg, &nr));
            HJ_TRY(fallback::gather_rows(c, W, ss, Sg, &ns));
            Rt = Rg.p;
            St = Sg.p;
        }
        if (!nr || !ns) continue;
        TableHold tg{c};
        if (!agg) {
            HJ_TRY(keylist_build(c, W, Rt, nr, pf, &tg.t));
            HJ_TRY(keylist_probe(c, tg.t, St, ns, pf, js.pairs, js.pcap, js.ctr, chk));
            if (redo) {
                HJ_TRY(read_counters(c));
                if (!redo->crossed && c->h_ctr->count > js.pcap) {
                    redo->crossed = true;
                    redo->from = prev;
                }
                prev = *c->h_ctr;
                if (redo->crossed) {  // this group's pairs are written again after the buffer grows
                    auto g = std::make_unique<FallbackGroup>(c);
                    g->t = tg.t;
                    tg.t = nullptr;
                    g->Sg.p = Sg.release();
                    g->S = St;
                    g->ns = ns;
                    g->pf = pf;
                    redo->groups.push_back(std::move(g));
                }
            }
            continue;
        }
        HJ_TRY(table_create(c, W, agg, nr, &tg.t));
        HJ_TRY(table_build(c, tg.t, Rt, 0, nr, nr, pf));
        const RecArea none{nullptr, nullptr, 0};
        HJ_TRY(table_probe(c, tg.t, St, 0, ns, ns, js.pairs, js.pcap, chk, none, pf, js.ctr, 1));
    }
    return HJ_OK;
}

}  // namespace hj

namespace {

hj_status check_rel(hj_ctx *c, const hj_rel *r, const char *name) {
    if (!r) return set_err(c, HJ_E_INVALID, "%s is NULL", name);
    if (r->width != HJ_U32 && r->width != HJ_U64)
        return set_err(c, HJ_E_INVALID, "%s width %d is not 4 or 8", name, r->width);
    if (r->n && !r->tuples) return set_err(c, HJ_E_INVALID, "%s has %llu tuples but a NULL pointer", name,
                                           (unsigned long long)r->n);
    if (r->n && ((uintptr_t)r->tuples & 15))
        return set_err(c, HJ_E_INVALID, "%s tuples are not 16-byte aligned", name);
    if (r->n >= 0xFFFFFFFFull)  // partition passes keep 32-bit row offsets
        return set_err(c, HJ_E_INVALID, "%s: a relation holds fewer than 2^32 - 1 tuples", name);
    return HJ_OK;
}

hj_status check_ctx(hj_ctx *c) {
    if (!c) return HJ_E_INVALID;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    return HJ_OK;
}

hj_opts default_opts() {
    hj_opts o;
    o.algo = HJ_ALGO_AUTO;
    o.mode = HJ_MATERIALIZE;
    o.radix_bits = 0;
    o.passes = 0;
    o.out_capacity = 0;
    o.flags = 0;
    return o;
}

bool is_agg(int mode) { return mode == HJ_COUNT || mode == HJ_COUNT_CHECKSUM; }
bool wants_checksum(const hj_opts &o) {
    return o.mode == HJ_COUNT_CHECKSUM || (o.mode == HJ_MATERIALIZE && (o.flags & HJ_FLAG_CHECKSUM));
}

__global__ void set_pair_kernel(uint64_t *p, uint64_t a, uint64_t b) {
    p[0] = a;
    p[1] = b;
}

// Device array {a, b}, written by a one-thread kernel so that the host need not wait.
hj_status device_pair(hj_ctx *c, uint64_t a, uint64_t b, DevBuf &out) {
    HJ_TRY(out.alloc(16));
    HJ_LAUNCH(c, "set_pair", set_pair_kernel, 1, 1, 0, out.as<uint64_t>(), a, b);
    return HJ_OK;
}

// Partition a whole relation in one or two passes (Alg. 2); on success `tuples`
// and `offsets` (2^(b1+b2) + 1 entries) hold the result and *rows the number of
// rows allocated for the tuples (more than in->n when padded).
hj_status partition_rel(hj_ctx *c, const hj_rel *in, int b1, int b2, int pad, DevBuf &tuples, DevBuf &offsets,
                        uint64_t *rows) {
    const uint64_t n = in->n, tb = tuple_bytes(in->width);
    DevBuf seg(c), A(c), off1(c);
    const uint64_t rows1 = partition_out_rows(c, in->width, n, 1, b1, pad);
    // run offsets inside a pass are 32-bit: the padded output must stay below 2^32 rows
    if (rows1 >= 0xFFFFFFFFull || (b2 && partition_out_rows(c, in->width, rows1, 1ull << b1, b2, pad) >= 0xFFFFFFFFull))
        return set_err(c, HJ_E_UNSUPPORTED, "%llu tuples padded to whole sectors pass 2^32 rows",
                       (unsigned long long)n);
    HJ_TRY(A.alloc(rows1 * tb + 64));
    HJ_TRY(off1.alloc(((1ull << b1) + 1) * 8));
    if (pad && b1 <= 11) {  // the first pass is one segment: the fused form
        HJ_TRY(partition_pass1(c, in->width, in->tuples, n, b1, A.p, off1.as<uint64_t>()));
    } else {
        HJ_TRY(device_pair(c, 0ull, n, seg));
        HJ_TRY(partition_pass(c, in->width, in->tuples, n, seg.as<uint64_t>(), 1, 0, b1, A.p, off1.as<uint64_t>(),
                              pad));
    }
    if (b2 == 0) {
        tuples.reset();
        offsets.reset();
        tuples.p = A.release();
        offsets.p = off1.release();
        *rows = rows1;
        return HJ_OK;
    }
    DevBuf B(c), off2(c);
    const uint64_t rows2 = partition_out_rows(c, in->width, rows1, 1ull << b1, b2, pad);
    HJ_TRY(B.alloc(rows2 * tb + 64));
    HJ_TRY(off2.alloc(((1ull << (b1 + b2)) + 1) * 8));
    HJ_TRY(partition_pass(c, in->width, A.p, rows1, off1.as<uint64_t>(), 1ull << b1, b1, b2, B.p,
                          off2.as<uint64_t>(), pad));
    tuples.reset();
    offsets.reset();
    tuples.p = B.release();
    offsets.p = off2.release();
    *rows = rows2;
    return HJ_OK;
}

void fill_result(hj_ctx *c, hj_result *res, int width, int algo, int bits, int passes) {
    res->count = c->h_ctr->count;
    res->checksum[0] = c->h_ctr->c0;
    res->checksum[1] = c->h_ctr->c1;
    res->width = width;
    res->algo = algo;
    res->radix_bits = algo == HJ_ALGO_PHJ ? bits : 0;
    res->passes = algo == HJ_ALGO_PHJ ? passes : 0;
}

struct TableGuard {
    hj_ctx *c;
    hj_table *t = nullptr;
    ~TableGuard() { table_destroy(c, t); }
};

hj_status check_output_status(hj_ctx *c) {
    if (c->h_ctr->status & kStatusRecords) return set_err(c, HJ_E_CUDA, "output record area overflow");
    if (c->h_ctr->status & kStatusCompact) return set_err(c, HJ_E_CUDA, "output compaction mismatch");
    return HJ_OK;
}

// Initial pair capacity: the caller's hint, else |S| (every probe tuple matching
// once), plus one chunk per emitting warp for the holes of partly filled chunks.
uint64_t first_capacity(const hj_opts &o, uint64_t nS, uint64_t warps) {
    uint64_t want = o.out_capacity ? o.out_capacity : nS;
    return want + warps * kChunkPairs;
}

// ----------------------------------------------------------------------- SHJ
// With `after_build` the counters hold the status of a build queued just before
// (no host synchronisation in between): the first attempt keeps them, and a full
// table is reported after the probe.  A build that met a run of repeated keys
// (kStatusLongRun) sets *long_run and leaves the result alone: the caller builds
// a key-list table and probes again.
hj_status probe_into(hj_ctx *c, const hj_table *t, const hj_rel *S, const hj_opts &o, hj_result *res,
                     bool after_build = false, bool *long_run = nullptr) {
    const bool mat = o.mode == HJ_MATERIALIZE, chk = wants_checksum(o);
    PairSink sink(c, t->width);
    // exact output leaves no holes: the caller's hint, else one pair per probe tuple
    uint64_t cap = mat ? std::max<uint64_t>(o.out_capacity ? o.out_capacity : S->n, 1) : 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        // warps stage their pairs in shared memory and claim exact rows: the
        // output is dense as written, no compaction pass
        RecArea ra{nullptr, nullptr, 0};
        if (mat) HJ_TRY(sink.reset(cap));
        if (!(after_build && attempt == 0)) HJ_TRY(zero_counters(c));
        if (t->keylist)
            HJ_TRY(keylist_probe(c, t, S->tuples, S->n, PartFilter{0, 0, 0, 0}, sink.pairs.p, sink.pcap, c->d_ctr,
                                 chk));
        else
            HJ_TRY(table_probe(c, t, S->tuples, 0, S->n, S->n, sink.pairs.p, sink.pcap, chk, ra,
                               PartFilter{0, 0, 0, 0}, nullptr, 2));
        HJ_TRY(read_counters(c));
        if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
        if (c->h_ctr->status & kStatusLongRun) {
            if (!long_run) return set_err(c, HJ_E_CUDA, "pair table with a run of repeated keys");
            *long_run = true;
            return HJ_OK;
        }
        HJ_TRY(check_output_status(c));
        if (!mat || c->h_ctr->count <= sink.pcap) break;
        // more pairs than the capacity: run the probe again at the exact size
        cap = c->h_ctr->count;
        if (attempt == 1) return set_err(c, HJ_E_CUDA, "pair capacity still too small after resizing");
    }
    fill_result(c, res, t->width, HJ_ALGO_SHJ, 0, 0);
    res->pairs = mat ? sink.pairs.release() : nullptr;
    res->pairs_cap = mat ? sink.pcap : 0;
    return HJ_OK;
}

hj_status join_shj(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts &o, hj_result *res) {
    TableGuard tg{c};
    HJ_TRY(zero_counters(c));
    HJ_TRY(table_create(c, R->width, is_agg(o.mode), R->n, &tg.t));
    HJ_TRY(table_build(c, tg.t, R->tuples, 0, R->n, R->n, PartFilter{0, 0, 0, 0}));
    bool long_run = false;
    HJ_TRY(probe_into(c, tg.t, S, o, res, true, &long_run));
    if (!long_run) return HJ_OK;
    // heavily repeated build keys: one entry per distinct key with its rid list
    table_destroy(c, tg.t);
    tg.t = nullptr;
    HJ_TRY(zero_counters(c));
    HJ_TRY(keylist_build(c, R->width, R->tuples, R->n, PartFilter{0, 0, 0, 0}, &tg.t));
    return probe_into(c, tg.t, S, o, res, true);
}

// ----------------------------------------------------------------------- PHJ
__global__ void set_slot_kernel(JoinSlot *s, void *pairs, unsigned long long pcap, hj_counters *ctr) {
    s->pairs = pairs;
    s->pcap = pcap;
    s->ctr = ctr;
    s->pad = 0;
}

hj_status run_partition_join(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts &o, const void *Rp,
                             const uint64_t *roff, const void *Sp, const uint64_t *soff, uint64_t NP, uint64_t ntasks,
                             int b1, int b2, PairSink *sink, uint32_t *oversize, PartTask *tasks, JoinSlot *slot_dev) {
    const bool agg = is_agg(o.mode), chk = wants_checksum(o), mat = o.mode == HJ_MATERIALIZE;
    const int W = R->width;
    RecArea ra{nullptr, nullptr, 0};
    if (mat) HJ_TRY(sink->new_area(partition_join_warps(c), &ra));
    HJ_TRY(zero_counters(c));
    void *pairs = mat ? sink->pairs.p : nullptr;
    const uint64_t pcap = mat ? sink->pcap : 0;
    HJ_LAUNCH(c, "set_slot", set_slot_kernel, 1, 1, 0, slot_dev, pairs, (unsigned long long)pcap, c->d_ctr);
    const uint64_t expect = NP ? (R->n + NP - 1) / NP : 0;
    HJ_TRY(partition_join(c, W, agg, tasks, ntasks, slot_dev, expect, chk, oversize, ra, nullptr, 0));
    if (mat) HJ_TRY(sink->finalize_device(c->d_ctr));
    HJ_TRY(read_counters(c));
    HJ_TRY(check_output_status(c));
    const uint64_t nov = c->h_ctr->n_oversize;
    if (nov == 0) return HJ_OK;
    // partitions whose table did not fit shared memory: global tables, pairs claimed
    // exactly after the compacted ones (counted even past the capacity)
    const hj_counters before = *c->h_ctr;
    std::vector<JoinSlot> slots_host{JoinSlot{pairs, pcap, c->d_ctr, 0}};
    // (pairs whose partition join fitted its buffer: the fallback keeps what it
    // needs to write the pairs that pass the buffer again)
    const bool keep = mat && before.cursor <= pcap && before.count <= pcap;
    FallbackRedo redo;
    HJ_TRY(oversize_fallback(c, W, agg, chk, tasks, oversize, nov, slots_host, keep ? &redo : nullptr));
    HJ_TRY(read_counters(c));
    if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
    if (keep && redo.crossed && c->h_ctr->count > pcap) {
        // only fallback pairs passed the buffer (heavy keys in oversize partitions):
        // the buffer grows to the exact count, keeping every pair written before the
        // first group that passed it, and that group and the later ones probe again
        // from the counters they started from (no partition join, no table rebuilt)
        HJ_TRY(sink->grow(c->h_ctr->count, redo.from.count));
        HJ_CUDA(c, cudaMemcpyAsync(c->d_ctr, &redo.from, offsetof(hj_counters, work), cudaMemcpyHostToDevice,
                                   c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));  // (`redo` lives on this stack)
        HJ_TRY(fallback_reprobe(c, chk, redo, JoinSlot{sink->pairs.p, sink->pcap, c->d_ctr, 0}));
        HJ_TRY(read_counters(c));
        if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
    }
    return HJ_OK;
}

hj_status join_phj(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts &o, int bits, int passes,
                   hj_result *res) {
    const bool mat = o.mode == HJ_MATERIALIZE;
    const int b1 = passes == 2 ? bits - bits / 2 : bits, b2 = passes == 2 ? bits / 2 : 0;
    if (b1 < 1 || b1 > 12 || b2 < 0 || b2 > 12)
        return set_err(c, HJ_E_INVALID, "radix bits %d in %d passes: each pass takes 1..12 bits", bits, passes);
    const uint64_t NP = 1ull << bits;
    DevBuf Rp(c), Sp(c), roff(c), soff(c), oversize(c), tasks(c), slot(c);
    PairSink sink(c, R->width);
    uint64_t r_rows = 0, s_rows = 0;
    HJ_TRY(partition_rel(c, R, b1, b2, 1, Rp, roff, &r_rows));
    HJ_TRY(partition_rel(c, S, b1, b2, 1, Sp, soff, &s_rows));
    const uint64_t tail = tail_split_from(c, R->width, is_agg(o.mode), NP, NP ? (R->n + NP - 1) / NP : 0);
    const uint64_t slice = task_slice_rows(R->width, S->n, NP),
                   ntasks = max_tasks(NP, s_rows, slice) + (NP - tail);
    HJ_TRY(oversize.alloc(ntasks * 4));
    HJ_TRY(tasks.alloc(ntasks * sizeof(PartTask) + 8));
    HJ_TRY(slot.alloc(sizeof(JoinSlot)));
    HJ_TRY(make_tasks(c, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, 0, b1, b2, R->width, slice, ntasks,
                      tasks.as<PartTask>(), tail));
    const uint64_t warps = partition_join_warps(c);
    uint64_t cap = mat ? first_capacity(o, S->n, warps) : 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (mat) HJ_TRY(sink.reset(cap));
        HJ_TRY(run_partition_join(c, R, S, o, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, ntasks, b1, b2,
                                  &sink, oversize.as<uint32_t>(), tasks.as<PartTask>(), slot.as<JoinSlot>()));
        if (!mat || (c->h_ctr->cursor <= sink.pcap && c->h_ctr->count <= sink.pcap)) break;
        // more pairs than the buffer holds: the count is exact, run again at that size
        cap = c->h_ctr->count + warps * kChunkPairs;
        if (attempt == 1) return set_err(c, HJ_E_CUDA, "pair capacity still too small after resizing");
    }
    fill_result(c, res, R->width, HJ_ALGO_PHJ, bits, passes);
    res->pairs = mat ? sink.pairs.release() : nullptr;
    res->pairs_cap = mat ? sink.pcap : 0;
    return HJ_OK;
}


// ------------------------------------------------------- pipelined host join
// hj_join_host for a large S: R is copied and partitioned once; S travels in
// chunks through two device buffers, and each chunk is partitioned and joined
// against the partitioned R while the next chunk is copied in (copy stream) and
// the previous chunk's pairs are copied out (output stream):
//
//   copy stream   H2D(0)  H2D(1)        H2D(2)        ...
//   ctx stream            join(0)       join(1)       join(2)
//   out stream                          D2H(0)        D2H(1)
//
// A chunk whose pairs overflow its buffer, or that needed the global-table
// fallback, is joined again on its own afterwards.
constexpr uint64_t kHostChunk = 1ull << 24;  // S rows per chunk

struct PipeSet {
    explicit PipeSet(hj_ctx *c, int w) : sink(c, w), dS(c) {}
    PairSink sink;
    DevBuf dS;
    hj_counters *h = nullptr;  // page-locked copy of the chunk's counters
    cudaEvent_t arrived = nullptr, computed = nullptr, drained = nullptr;
    uint64_t chunk = ~0ull, n = 0;
    bool taken = false;  // the chunk's counters were read (and its pairs sent home or queued for a rerun)
};

hj_status join_host_pipelined(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts &o, int bits,
                              uint64_t chunk_rows, void *pairs_host, uint64_t pairs_host_cap, hj_result *res) {
    const int W = Rh->width;
    const uint64_t tb = tuple_bytes(W), NP = 1ull << bits;
    const bool mat = o.mode == HJ_MATERIALIZE;
    cudaStream_t &cs = c->pipe_in, &os = c->pipe_out;
    std::vector<std::unique_ptr<PipeSet>> sets;
    std::vector<uint64_t> redo;
    uint64_t count = 0, c0 = 0, c1 = 0, written = 0;
    hj_status st = HJ_OK;
    DevBuf dR(c), Rp(c), roff(c);
    uint64_t r_rows = 0;
    // streams, events and counter copies are the context's, kept across calls
    auto cleanup = [&]() {
        if (cs) cudaStreamSynchronize(cs);
        if (os) cudaStreamSynchronize(os);
        cudaStreamSynchronize(c->stream);
        sets.clear();
    };
    // take a finished chunk: counters, then its pairs to the host (output stream)
    auto drain = [&](PipeSet &ps) -> hj_status {
        HJ_CUDA(c, cudaEventSynchronize(ps.computed));
        ps.taken = true;
        const hj_counters &h = *ps.h;
        if (h.fault) {  // a partition pass reported a fault: clear the sticky word, report it once
            HJ_CUDA(c, cudaMemsetAsync(&c->d_ctr->fault, 0, sizeof(unsigned long long), c->stream));
            if (h.fault & kStatusTimeout)
                return set_err(c, HJ_E_TIMEOUT, "chunk %llu: a bounded device wait expired",
                               (unsigned long long)ps.chunk);
            return set_err(c, HJ_E_INVALID, "chunk %llu: a partition pass rejected its input",
                           (unsigned long long)ps.chunk);
        }
        if (h.status & (kStatusTimeout | kStatusBadInput | kStatusRecords | kStatusCompact | kStatusTableFull))
            return set_err(c, HJ_E_CUDA, "chunk %llu: kernel status %llu", (unsigned long long)ps.chunk,
                           (unsigned long long)h.status);
        if (h.n_oversize || (mat && (h.cursor > ps.sink.pcap || h.count > ps.sink.pcap))) {
            redo.push_back(ps.chunk);  // joined again on its own below
            return HJ_OK;
        }
        count += h.count;
        c0 += h.c0;
        c1 += h.c1;
        if (mat && h.count) {
            const uint64_t n = written < pairs_host_cap ? std::min<uint64_t>(h.count, pairs_host_cap - written) : 0;
            HJ_CUDA(c, cudaStreamWaitEvent(os, ps.computed, 0));
            if (n && pairs_host)
                HJ_CUDA(c, cudaMemcpyAsync((char *)pairs_host + written * tb, ps.sink.pairs.p, n * tb,
                                           cudaMemcpyDeviceToHost, os));
            written += n;
        }
        HJ_CUDA(c, cudaEventRecord(ps.drained, os));
        return HJ_OK;
    };
    auto body = [&]() -> hj_status {
        if (!cs) HJ_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        if (!os) HJ_CUDA(c, cudaStreamCreateWithFlags(&os, cudaStreamNonBlocking));
        if (!c->pipe_h) HJ_CUDA(c, cudaMallocHost(&c->pipe_h, 2 * sizeof(hj_counters)));
        for (int i = 0; i < 2; ++i) {
            for (cudaEvent_t &e : c->pipe_ev[i])
                if (!e) HJ_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            // a fresh call must not wait on the last call's events: record them here
            for (cudaEvent_t e : c->pipe_ev[i]) HJ_CUDA(c, cudaEventRecord(e, c->stream));
            sets.push_back(std::make_unique<PipeSet>(c, W));
            PipeSet &ps = *sets.back();
            ps.arrived = c->pipe_ev[i][0];
            ps.computed = c->pipe_ev[i][1];
            ps.drained = c->pipe_ev[i][2];
            ps.h = (hj_counters *)c->pipe_h + i;
            HJ_TRY(ps.dS.alloc(chunk_rows * tb + 64));
        }
        // R: copied and partitioned once
        HJ_TRY(dR.alloc(Rh->n * tb + 64));
        HJ_TRY(copy_wide(c, dR.p, Rh->tuples, Rh->n * tb, cudaMemcpyHostToDevice));
        hj_rel R = *Rh;
        R.tuples = dR.p;
        HJ_TRY(partition_rel(c, &R, bits, 0, 1, Rp, roff, &r_rows));
        const uint64_t nchunks = (Sh->n + chunk_rows - 1) / chunk_rows;
        const uint64_t warps = partition_join_warps(c);
        for (uint64_t k = 0; k < nchunks; ++k) {
            PipeSet &ps = *sets[k & 1];
            if (ps.chunk != ~0ull && !ps.taken) HJ_TRY(drain(ps));
            const uint64_t r0 = k * chunk_rows, n = std::min(chunk_rows, Sh->n - r0);
            // the set's S buffer is free once chunk k - 2's join is done
            HJ_CUDA(c, cudaStreamWaitEvent(cs, ps.computed, 0));
            HJ_CUDA(c, cudaMemcpyAsync(ps.dS.p, (const char *)Sh->tuples + r0 * tb, n * tb, cudaMemcpyHostToDevice,
                                       cs));
            HJ_CUDA(c, cudaEventRecord(ps.arrived, cs));
            ps.chunk = k;
            ps.n = n;
            ps.taken = false;
            // join of chunk k on the context's stream, after its copy and after the
            // set's pairs of chunk k - 2 have left for the host
            HJ_CUDA(c, cudaStreamWaitEvent(c->stream, ps.arrived, 0));
            HJ_CUDA(c, cudaStreamWaitEvent(c->stream, ps.drained, 0));
            hj_rel S{ps.dS.p, n, W, 0};
            DevBuf Sp(c), soff(c), tasks(c), oversize(c), slot(c);
            uint64_t s_rows = 0;
            HJ_TRY(partition_rel(c, &S, bits, 0, 1, Sp, soff, &s_rows));
            const uint64_t slice = task_slice_rows(W, n, NP), ntasks = max_tasks(NP, s_rows, slice);
            HJ_TRY(oversize.alloc(ntasks * 4));
            HJ_TRY(tasks.alloc(ntasks * sizeof(PartTask) + 8));
            HJ_TRY(slot.alloc(sizeof(JoinSlot)));
            HJ_TRY(make_tasks(c, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, 0, bits, 0, W, slice,
                              ntasks, tasks.as<PartTask>()));
            if (mat) HJ_TRY(ps.sink.reset(n + warps * kChunkPairs));
            RecArea ra{nullptr, nullptr, 0};
            if (mat) HJ_TRY(ps.sink.new_area(warps, &ra));
            HJ_TRY(zero_counters(c));
            HJ_LAUNCH(c, "set_slot", set_slot_kernel, 1, 1, 0, slot.as<JoinSlot>(), mat ? ps.sink.pairs.p : nullptr,
                      (unsigned long long)(mat ? ps.sink.pcap : 0), c->d_ctr);
            HJ_TRY(partition_join(c, W, is_agg(o.mode), tasks.as<PartTask>(), ntasks, slot.as<JoinSlot>(),
                                  (Rh->n + NP - 1) / NP, wants_checksum(o), oversize.as<uint32_t>(), ra, nullptr, 0));
            if (mat) HJ_TRY(ps.sink.finalize_device(c->d_ctr));
            HJ_CUDA(c, cudaMemcpyAsync(ps.h, c->d_ctr, sizeof(hj_counters), cudaMemcpyDeviceToHost, c->stream));
            HJ_CUDA(c, cudaEventRecord(ps.computed, c->stream));
            // the previous chunk is done or nearly: send its pairs home
            if (k >= 1) HJ_TRY(drain(*sets[(k - 1) & 1]));
        }
        if (nchunks) HJ_TRY(drain(*sets[(nchunks - 1) & 1]));
        HJ_CUDA(c, cudaStreamSynchronize(os));
        // chunks that did not fit their pair buffer: on their own, exact capacity
        for (uint64_t k : redo) {
            const uint64_t r0 = k * chunk_rows, n = std::min(chunk_rows, Sh->n - r0);
            DevBuf dS(c);
            HJ_TRY(dS.alloc(n * tb + 64));
            HJ_CUDA(c, cudaMemcpyAsync(dS.p, (const char *)Sh->tuples + r0 * tb, n * tb, cudaMemcpyHostToDevice,
                                       c->stream));
            hj_rel S{dS.p, n, W, 0};
            hj_result r{};
            HJ_TRY(join_phj(c, &R, &S, o, bits, 1, &r));
            count += r.count;
            c0 += r.checksum[0];
            c1 += r.checksum[1];
            if (mat && r.count) {
                const uint64_t m = written < pairs_host_cap ? std::min<uint64_t>(r.count, pairs_host_cap - written) : 0;
                if (m && pairs_host)
                    HJ_CUDA(c, cudaMemcpyAsync((char *)pairs_host + written * tb, r.pairs, m * tb,
                                               cudaMemcpyDeviceToHost, c->stream));
                HJ_CUDA(c, cudaStreamSynchronize(c->stream));
                written += m;
            }
            dfree(c, r.pairs);
        }
        return HJ_OK;
    };
    st = body();
    cleanup();
    if (st != HJ_OK) return st;
    res->count = count;
    res->checksum[0] = c0;
    res->checksum[1] = c1;
    res->width = W;
    res->algo = HJ_ALGO_PHJ;
    res->radix_bits = bits;
    res->passes = 1;
    res->pairs = nullptr;
    res->pairs_cap = 0;
    if (mat && count > pairs_host_cap)
        return set_err(c, HJ_E_OVERFLOW, "%llu pairs do not fit in %llu", (unsigned long long)count,
                       (unsigned long long)pairs_host_cap);
    if (mat && count && !pairs_host) return set_err(c, HJ_E_INVALID, "pairs_host is NULL but the join produced pairs");
    return HJ_OK;
}

// ------------------------------------------------------- CPU/GPU co-processing
// The PHJ with its join step divided between the GPU and the host CPU (the
// paper's data dividing, Sec. 3.2, on the join step; coexec.cu has the CPU side).
// The GPU partitions both relations; the partition pairs [0, p_cpu) -- the first
// cpu_share of S's rows -- are copied to page-locked host memory by a host thread
// (its own stream, after the partition passes) and joined there by cpu_threads
// threads, while the GPU joins the pairs [p_cpu, NP) (the CPU's tasks are emptied
// first).  The CPU's pairs are then appended to the GPU's in the result buffer.

__global__ void drop_tasks_kernel(PartTask *tasks, uint64_t ntasks, uint32_t p_cpu) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ntasks; i += (uint64_t)gridDim.x * blockDim.x)
        if (tasks[i].p < p_cpu) {
            tasks[i].nr = 0;
            tasks[i].ns = 0;
        }
}

hj_status join_coproc(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts &o, int bits, int passes,
                      double cpu_share, int threads, hj_result *res, double *times) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    const bool mat = o.mode == HJ_MATERIALIZE, chk = wants_checksum(o);
    const int W = R->width;
    const uint64_t tb = tuple_bytes(W);
    const int b1 = passes == 2 ? bits - bits / 2 : bits, b2 = passes == 2 ? bits / 2 : 0;
    if (b1 < 1 || b1 > 12 || b2 < 0 || b2 > 12)
        return set_err(c, HJ_E_INVALID, "radix bits %d in %d passes: each pass takes 1..12 bits", bits, passes);
    const uint64_t NP = 1ull << bits;
    cudaEvent_t ev[4] = {};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 4; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } eg{ev};
    for (auto &e : ev) HJ_CUDA(c, cudaEventCreate(&e));
    DevBuf Rp(c), Sp(c), roff(c), soff(c), oversize(c), tasks(c), slot(c);
    PairSink sink(c, W);
    uint64_t r_rows = 0, s_rows = 0;
    HJ_CUDA(c, cudaEventRecord(ev[0], c->stream));
    HJ_TRY(partition_rel(c, R, b1, b2, 1, Rp, roff, &r_rows));
    HJ_TRY(partition_rel(c, S, b1, b2, 1, Sp, soff, &s_rows));
    HJ_CUDA(c, cudaEventRecord(ev[1], c->stream));
    // partition offsets on the host (this waits for the partition passes)
    std::vector<uint64_t> ro(NP + 1), so(NP + 1);
    HJ_CUDA(c, cudaMemcpyAsync(ro.data(), roff.p, (NP + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaMemcpyAsync(so.data(), soff.p, (NP + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    HJ_TRY(read_counters(c));  // synchronises; a partition pass's fault is reported here
    // the CPU's partitions: the first ones holding cpu_share of S's rows
    uint32_t p_cpu = 0;
    if (cpu_share >= 1.0) {
        p_cpu = (uint32_t)NP;
    } else if (cpu_share > 0.0) {
        const double want = cpu_share * (double)(so[NP] - so[0]);
        while (p_cpu < NP && (double)(so[p_cpu] - so[0]) < want) ++p_cpu;
    }
    // host buffers for the CPU's rows, kept on the context
    const uint64_t rb = (ro[p_cpu] - ro[0]) * tb, sb = (so[p_cpu] - so[0]) * tb;
    for (int side = 0; side < 2; ++side) {
        const uint64_t need = side ? sb : rb;
        if (need && c->host_cap[side] < need) {
            if (c->host_buf[side]) cudaFreeHost(c->host_buf[side]);
            c->host_buf[side] = nullptr;
            c->host_cap[side] = 0;
            HJ_CUDA(c, cudaMallocHost(&c->host_buf[side], need));
            c->host_cap[side] = need;
        }
    }
    if (!c->pipe_in) HJ_CUDA(c, cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking));
    if (!c->cpu_pool) c->cpu_pool = cpu_pool_new();
    // CPU side: copy the CPU's rows home and join them, beside the GPU's join
    CpuJoinResult cres;
    cudaError_t cerr = cudaSuccess;
    double t_copy = 0.0, t_cpu = 0.0;
    std::thread cpu_side;
    if (p_cpu) {
        cpu_side = std::thread([&, rb, sb, p_cpu]() {
            const auto t0 = clk::now();
            cerr = cudaSetDevice(c->device);
            if (cerr == cudaSuccess && rb)
                cerr = cudaMemcpyAsync(c->host_buf[0], (const char *)Rp.p + ro[0] * tb, rb, cudaMemcpyDeviceToHost,
                                       c->pipe_in);
            if (cerr == cudaSuccess && sb)
                cerr = cudaMemcpyAsync(c->host_buf[1], (const char *)Sp.p + so[0] * tb, sb, cudaMemcpyDeviceToHost,
                                       c->pipe_in);
            if (cerr == cudaSuccess) cerr = cudaStreamSynchronize(c->pipe_in);
            const auto t1 = clk::now();
            t_copy = std::chrono::duration<double>(t1 - t0).count();
            if (cerr != cudaSuccess) return;
            cpu_join_partitions(c->cpu_pool, W, c->host_buf[0], ro.data(), c->host_buf[1], so.data(), p_cpu, b1, b2,
                                mat, chk, threads, &cres);
            t_cpu = std::chrono::duration<double>(clk::now() - t1).count();
        });
    }
    struct Joiner {
        std::thread &t;
        ~Joiner() {
            if (t.joinable()) t.join();
        }
    } joiner{cpu_side};
    // GPU side: the remaining partition pairs, as join_phj does
    const uint64_t slice = task_slice_rows(W, S->n, NP), ntasks = max_tasks(NP, s_rows, slice);
    HJ_TRY(oversize.alloc(ntasks * 4));
    HJ_TRY(tasks.alloc(ntasks * sizeof(PartTask) + 8));
    HJ_TRY(slot.alloc(sizeof(JoinSlot)));
    HJ_TRY(make_tasks(c, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, 0, b1, b2, W, slice, ntasks,
                      tasks.as<PartTask>()));
    if (p_cpu) {
        const unsigned grid = (unsigned)std::min<uint64_t>((ntasks + 255) / 256, (uint64_t)num_sms(c) * 8);
        HJ_LAUNCH(c, "drop_tasks", drop_tasks_kernel, grid ? grid : 1, 256, 0, tasks.as<PartTask>(), ntasks, p_cpu);
    }
    const uint64_t warps = partition_join_warps(c);
    // the GPU's pairs: at most one per S row of its partitions (unique R keys), else resized
    uint64_t cap = mat ? first_capacity(o, S->n, warps) : 0;
    HJ_CUDA(c, cudaEventRecord(ev[2], c->stream));
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (mat) HJ_TRY(sink.reset(cap));
        HJ_TRY(run_partition_join(c, R, S, o, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, ntasks, b1, b2,
                                  &sink, oversize.as<uint32_t>(), tasks.as<PartTask>(), slot.as<JoinSlot>()));
        if (!mat || (c->h_ctr->cursor <= sink.pcap && c->h_ctr->count <= sink.pcap)) break;
        cap = c->h_ctr->count + warps * kChunkPairs;
        if (attempt == 1) return set_err(c, HJ_E_CUDA, "pair capacity still too small after resizing");
    }
    HJ_CUDA(c, cudaEventRecord(ev[3], c->stream));
    const uint64_t g_count = c->h_ctr->count, g_c0 = c->h_ctr->c0, g_c1 = c->h_ctr->c1;
    if (cpu_side.joinable()) cpu_side.join();
    if (cerr != cudaSuccess) return cuda_err(c, cerr, "copy of the CPU's partitions");
    // merge: counts and checksums add; the CPU's pairs follow the GPU's
    res->count = g_count + cres.count;
    res->checksum[0] = g_c0 + cres.c0;
    res->checksum[1] = g_c1 + cres.c1;
    res->width = W;
    res->algo = HJ_ALGO_PHJ;
    res->radix_bits = bits;
    res->passes = passes;
    res->pairs = nullptr;
    res->pairs_cap = 0;
    if (mat) {
        if (sink.pcap < res->count) {  // room for both parts
            DevBuf all(c);
            HJ_TRY(all.alloc(res->count * tb));
            if (g_count)
                HJ_CUDA(c, cudaMemcpyAsync(all.p, sink.pairs.p, g_count * tb, cudaMemcpyDeviceToDevice, c->stream));
            sink.pairs.reset();
            sink.pairs.p = all.release();
            sink.pcap = res->count;
        }
        uint64_t at = g_count;
        for (const auto &v : cres.pairs) {
            if (v.empty()) continue;
            HJ_CUDA(c, cudaMemcpyAsync((char *)sink.pairs.p + at * tb, v.data(), v.size(), cudaMemcpyHostToDevice,
                                       c->stream));
            at += v.size() / tb;
        }
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        res->pairs = sink.pairs.release();
        res->pairs_cap = sink.pcap;
    }
    if (times) {
        HJ_CUDA(c, cudaEventSynchronize(ev[3]));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        times[0] = ms / 1e3;
        cudaEventElapsedTime(&ms, ev[2], ev[3]);
        times[1] = ms / 1e3;
        times[2] = t_copy;
        times[3] = t_cpu;
        times[4] = std::chrono::duration<double>(clk::now() - t_start).count();
    }
    return HJ_OK;
}

}  // namespace

namespace hj {

// Device bytes of join_host_pipelined with chunks of `chunk_rows` S rows at `bits`
// radix bits: R and its padded partitioned copy, two S chunk buffers and (pairs)
// two pair buffers with one chunk of slack per emitting warp, one chunk's padded
// partitioned copy, and 64 MiB for counters, histograms, task lists and records.
uint64_t host_streamed_bytes(hj_ctx *c, int width, bool mat, uint64_t nR, uint64_t chunk_rows, int bits) {
    const uint64_t tb = tuple_bytes(width);
    uint64_t b = nR * tb + partition_out_rows(c, width, nR, 1, bits, 1) * tb + ((1ull << bits) + 1) * 8;
    b += 2 * (chunk_rows * tb + 64);
    if (mat) b += 2 * (chunk_rows + partition_join_warps(c) * kChunkPairs) * tb;
    b += partition_out_rows(c, width, chunk_rows, 1, bits, 1) * tb;
    return b + (64ull << 20);
}

bool host_streamed_plan(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts &o, uint64_t device_bytes,
                        uint64_t *chunk_rows, int *bits) {
    if (Rh->n == 0 || Rh->n >= 0xFFFFFFFFull) return false;
    if (!c->model_ready) {
        c->model = cost_model_for(c->device);
        c->model_ready = true;
    }
    const bool mat = o.mode == HJ_MATERIALIZE;
    for (uint64_t ch = kHostChunk; ch >= (1ull << 20); ch >>= 1) {
        const std::vector<PlanCand> pcs =
            plan_candidates(c->model, Rh->width, !mat, mat, Rh->n, std::min<uint64_t>(Sh->n, ch), HJ_ALGO_PHJ, 0, 1);
        if (pcs.empty() || pcs[0].passes != 1) return false;  // R needs two passes: no streamed plan
        if (host_streamed_bytes(c, Rh->width, mat, Rh->n, ch, pcs[0].bits) <= device_bytes) {
            *chunk_rows = ch;
            *bits = pcs[0].bits;
            return true;
        }
    }
    return false;
}

hj_status host_streamed_join(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts &o, int bits,
                             uint64_t chunk_rows, void *pairs_host, uint64_t pairs_host_cap, hj_result *res) {
    *res = hj_result{};
    return join_host_pipelined(c, Rh, Sh, o, bits, chunk_rows, pairs_host, pairs_host_cap, res);
}

}  // namespace hj

extern "C" {

hj_status hj_join_coproc(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts *opts, double cpu_share,
                         int cpu_threads, hj_result *res, double *times) {
    HJ_TRY(check_ctx(c));
    if (!res) return set_err(c, HJ_E_INVALID, "result is NULL");
    HJ_TRY(check_rel(c, R, "R"));
    HJ_TRY(check_rel(c, S, "S"));
    if (R->width != S->width) return set_err(c, HJ_E_INVALID, "R and S widths differ (%d, %d)", R->width, S->width);
    if (!(cpu_share >= 0.0 && cpu_share <= 1.0)) return set_err(c, HJ_E_INVALID, "cpu_share outside [0, 1]");
    if (cpu_threads < 0) return set_err(c, HJ_E_INVALID, "cpu_threads %d < 0", cpu_threads);
    hj_opts o = opts ? *opts : default_opts();
    if (o.mode < HJ_COUNT || o.mode > HJ_MATERIALIZE) return set_err(c, HJ_E_INVALID, "bad mode %d", o.mode);
    if (o.algo == HJ_ALGO_SHJ) return set_err(c, HJ_E_INVALID, "co-processing divides the PHJ's join step");
    if (o.passes < 0 || o.passes > 2) return set_err(c, HJ_E_INVALID, "passes %d not in {1, 2}", o.passes);
    if (o.radix_bits < 0 || o.radix_bits > 24) return set_err(c, HJ_E_INVALID, "radix bits %d > 24", o.radix_bits);
    *res = hj_result{};
    int algo, bits, passes;
    choose_plan(c, R->width, o.mode, R->n, S->n, HJ_ALGO_PHJ, o.radix_bits, o.passes, &algo, &bits, &passes);
    int threads = cpu_threads;
    if (!threads) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    return join_coproc(c, R, S, o, bits, passes, cpu_share, threads, res, times);
}

hj_status hj_build(hj_ctx *c, const hj_rel *R, const hj_opts *opts, hj_table **out) {
    HJ_TRY(check_ctx(c));
    if (!out) return set_err(c, HJ_E_INVALID, "out is NULL");
    *out = nullptr;
    HJ_TRY(check_rel(c, R, "R"));
    hj_opts o = opts ? *opts : default_opts();
    if (o.mode < HJ_COUNT || o.mode > HJ_MATERIALIZE) return set_err(c, HJ_E_INVALID, "bad mode %d", o.mode);
    TableGuard tg{c};
    HJ_TRY(zero_counters(c));
    HJ_TRY(table_create(c, R->width, is_agg(o.mode), R->n, &tg.t));
    HJ_TRY(table_build(c, tg.t, R->tuples, 0, R->n, R->n, PartFilter{0, 0, 0, 0}));
    HJ_TRY(read_counters(c));
    if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
    if (c->h_ctr->status & kStatusLongRun) {  // heavily repeated keys: a key-list table
        table_destroy(c, tg.t);
        tg.t = nullptr;
        HJ_TRY(zero_counters(c));
        HJ_TRY(keylist_build(c, R->width, R->tuples, R->n, PartFilter{0, 0, 0, 0}, &tg.t));
        HJ_TRY(read_counters(c));
        if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
    }
    *out = tg.t;
    tg.t = nullptr;
    return HJ_OK;
}

hj_status hj_probe(hj_ctx *c, const hj_table *t, const hj_rel *S, const hj_opts *opts, hj_result *res) {
    HJ_TRY(check_ctx(c));
    if (!t || !res) return set_err(c, HJ_E_INVALID, "table or result is NULL");
    HJ_TRY(check_rel(c, S, "S"));
    hj_opts o = opts ? *opts : default_opts();
    if (S->width != t->width) return set_err(c, HJ_E_INVALID, "S width %d differs from the table's %d", S->width, t->width);
    if (is_agg(o.mode) != (t->agg != 0))
        return set_err(c, HJ_E_INVALID, "probe mode %d does not match the table's build mode", o.mode);
    *res = hj_result{};
    return probe_into(c, t, S, o, res);
}

hj_status hj_table_free(hj_ctx *c, hj_table *t) {
    if (!c || !t) return HJ_E_INVALID;
    cudaSetDevice(c->device);
    table_destroy(c, t);
    return HJ_OK;
}

hj_status hj_partition(hj_ctx *c, const hj_rel *in, int b1, int b2, hj_rel *out_tuples, uint64_t **out_offsets) {
    HJ_TRY(check_ctx(c));
    HJ_TRY(check_rel(c, in, "in"));
    if (!out_tuples || !out_offsets) return set_err(c, HJ_E_INVALID, "output pointers are NULL");
    if (b1 < 1 || b1 > 12 || b2 < 0 || b2 > 12)
        return set_err(c, HJ_E_INVALID, "bits (%d, %d): pass one takes 1..12 bits, pass two 0..12", b1, b2);
    DevBuf tup(c), off(c);
    uint64_t rows = 0;
    HJ_TRY(partition_rel(c, in, b1, b2, 0, tup, off, &rows));
    HJ_TRY(read_counters(c));  // synchronises; reports a pass's expired wait or rejected input
    out_tuples->tuples = tup.release();
    out_tuples->n = in->n;
    out_tuples->width = in->width;
    out_tuples->reserved = 0;
    *out_offsets = off.as<uint64_t>();
    off.release();
    return HJ_OK;
}

hj_status hj_partition_free(hj_ctx *c, hj_rel *tuples, uint64_t *offsets) {
    if (!c) return HJ_E_INVALID;
    cudaSetDevice(c->device);
    if (tuples) {
        dfree(c, (void *)tuples->tuples);
        tuples->tuples = nullptr;
        tuples->n = 0;
    }
    dfree(c, offsets);
    return HJ_OK;
}

hj_status hj_join(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts *opts, hj_result *res) {
    HJ_TRY(check_ctx(c));
    if (!res) return set_err(c, HJ_E_INVALID, "result is NULL");
    HJ_TRY(check_rel(c, R, "R"));
    HJ_TRY(check_rel(c, S, "S"));
    if (R->width != S->width) return set_err(c, HJ_E_INVALID, "R and S widths differ (%d, %d)", R->width, S->width);
    hj_opts o = opts ? *opts : default_opts();
    if (o.mode < HJ_COUNT || o.mode > HJ_MATERIALIZE) return set_err(c, HJ_E_INVALID, "bad mode %d", o.mode);
    if (o.algo < HJ_ALGO_AUTO || o.algo > HJ_ALGO_PHJ) return set_err(c, HJ_E_INVALID, "bad algo %d", o.algo);
    if (o.passes < 0 || o.passes > 2) return set_err(c, HJ_E_INVALID, "passes %d not in {1, 2}", o.passes);
    if (o.radix_bits < 0 || o.radix_bits > 24) return set_err(c, HJ_E_INVALID, "radix bits %d > 24", o.radix_bits);
    *res = hj_result{};
    int algo, bits, passes;
    choose_plan(c, R->width, o.mode, R->n, S->n, o.algo, o.radix_bits, o.passes, &algo, &bits, &passes);
    hj_status st = algo == HJ_ALGO_SHJ ? join_shj(c, R, S, o, res) : join_phj(c, R, S, o, bits, passes, res);
    return st;
}

hj_status hj_copy(hj_ctx *c, void *dst, const void *src, uint64_t bytes) {
    HJ_TRY(check_ctx(c));
    if (!bytes) return HJ_OK;
    if (!dst || !src) return set_err(c, HJ_E_INVALID, "copy with a NULL pointer");
    HJ_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    return HJ_OK;
}

hj_status hj_join_host(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts *opts, void *pairs_host,
                       uint64_t pairs_host_cap, hj_result *res) {
    HJ_TRY(check_ctx(c));
    if (!res) return set_err(c, HJ_E_INVALID, "result is NULL");
    if (!Rh || !Sh) return set_err(c, HJ_E_INVALID, "relation is NULL");
    if (Rh->width != HJ_U32 && Rh->width != HJ_U64) return set_err(c, HJ_E_INVALID, "bad width %d", Rh->width);
    if (Rh->width != Sh->width) return set_err(c, HJ_E_INVALID, "R and S widths differ");
    if ((Rh->n && !Rh->tuples) || (Sh->n && !Sh->tuples)) return set_err(c, HJ_E_INVALID, "NULL host tuples");
    const uint64_t tb = tuple_bytes(Rh->width);
    {
        // a large S: chunked, copies overlapping a one-pass PHJ
        hj_opts o = opts ? *opts : default_opts();
        int algo, bits, passes;
        choose_plan(c, Rh->width, o.mode, Rh->n, Sh->n, o.algo, o.radix_bits, o.passes, &algo, &bits, &passes);
        bool pipe = algo == HJ_ALGO_PHJ && passes == 1;
        if (!pipe && o.algo == HJ_ALGO_AUTO && o.passes <= 0) {
            // the in-memory plan is SHJ or two passes; the chunked join is bound by
            // the host link, so a one-pass PHJ serves as well when R's partitions
            // fit shared memory at some fan-out
            if (!c->model_ready) {
                c->model = cost_model_for(c->device);
                c->model_ready = true;
            }
            const bool mat = o.mode == HJ_MATERIALIZE;
            std::vector<PlanCand> pcs = plan_candidates(c->model, Rh->width, !mat, mat, Rh->n,
                                                        std::min<uint64_t>(Sh->n, kHostChunk), HJ_ALGO_PHJ,
                                                        o.radix_bits, 1);
            if (!pcs.empty() && pcs[0].passes == 1) {
                pipe = true;
                bits = pcs[0].bits;
            }
        }
        if (pipe && Sh->n >= 2 * kHostChunk && Rh->n < 0xFFFFFFFFull && o.mode >= HJ_COUNT &&
            o.mode <= HJ_MATERIALIZE) {
            *res = hj_result{};
            return join_host_pipelined(c, Rh, Sh, o, bits, kHostChunk, pairs_host, pairs_host_cap, res);
        }
    }
    DevBuf dR(c), dS(c);
    HJ_TRY(dR.alloc(Rh->n * tb + 64));
    HJ_TRY(dS.alloc(Sh->n * tb + 64));
    if (Rh->n) HJ_TRY(copy_wide(c, dR.p, Rh->tuples, Rh->n * tb, cudaMemcpyHostToDevice));
    if (Sh->n) HJ_TRY(copy_wide(c, dS.p, Sh->tuples, Sh->n * tb, cudaMemcpyHostToDevice));
    hj_rel R = *Rh, S = *Sh;
    R.tuples = dR.p;
    S.tuples = dS.p;
    HJ_TRY(hj_join(c, &R, &S, opts, res));
    DevBuf pairs(c);
    pairs.p = res->pairs;  // released below whatever happens
    res->pairs = nullptr;
    res->pairs_cap = 0;
    if (pairs.p && res->count) {
        if (!pairs_host) return set_err(c, HJ_E_INVALID, "pairs_host is NULL but the join produced pairs");
        uint64_t n = std::min(res->count, pairs_host_cap);
        if (n) HJ_TRY(copy_wide(c, pairs_host, pairs.p, n * tb, cudaMemcpyDeviceToHost));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        if (n < res->count)
            return set_err(c, HJ_E_OVERFLOW, "%llu pairs do not fit in %llu", (unsigned long long)res->count,
                           (unsigned long long)pairs_host_cap);
    }
    return HJ_OK;
}

hj_status hj_result_free(hj_ctx *c, hj_result *res) {
    if (!c || !res) return HJ_E_INVALID;
    cudaSetDevice(c->device);
    dfree(c, res->pairs);
    *res = hj_result{};
    return HJ_OK;
}

}  // extern "C"
