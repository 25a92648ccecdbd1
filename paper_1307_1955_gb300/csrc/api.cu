// api.cu -- the C ABI of include/hj.h: argument checks, plan choice, and the
// SHJ / PHJ drivers that sequence the kernels of join.cu and partition.cu.
#include <algorithm>
#include <cmath>
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

// Partitions whose table did not fit in shared memory: SHJ with a global table,
// task by task (host loop over the listed tasks).
hj_status oversize_fallback(hj_ctx *c, int W, bool agg, bool chk, const PartTask *tasks, const uint32_t *list_dev,
                            uint64_t nov, const std::vector<JoinSlot> &slots_host) {
    std::vector<uint32_t> list(nov);
    HJ_CUDA(c, cudaMemcpyAsync(list.data(), list_dev, nov * 4, cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    for (uint32_t ti : list) {
        PartTask tk;
        HJ_CUDA(c, cudaMemcpyAsync(&tk, tasks + ti, sizeof tk, cudaMemcpyDeviceToHost, c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        const PartFilter pf{tk.p, (int)tk.b1, (int)tk.b2, 1};
        const JoinSlot &js = slots_host[tk.join];
        TableHold tg{c};
        HJ_TRY(table_create(c, W, agg, tk.nr, &tg.t));
        HJ_TRY(table_build(c, tg.t, tk.R, 0, tk.nr, tk.nr, pf));
        const RecArea none{nullptr, nullptr, 0};
        HJ_TRY(table_probe(c, tg.t, tk.S, 0, tk.ns, tk.ns, js.pairs, js.pcap, chk, none, pf, js.ctr, 1));
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
    if (r->width == HJ_U32 && r->n >= 0xFFFFFFFFull)
        return set_err(c, HJ_E_INVALID, "%s: 4-byte relations hold fewer than 2^32 - 1 tuples", name);
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
    HJ_TRY(device_pair(c, 0ull, n, seg));
    const uint64_t rows1 = partition_out_rows(c, in->width, n, 1, b1, pad);
    HJ_TRY(A.alloc(rows1 * tb + 64));
    HJ_TRY(off1.alloc(((1ull << b1) + 1) * 8));
    HJ_TRY(partition_pass(c, in->width, in->tuples, n, seg.as<uint64_t>(), 1, 0, b1, A.p, off1.as<uint64_t>(), pad));
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
// table is reported after the probe.
hj_status probe_into(hj_ctx *c, const hj_table *t, const hj_rel *S, const hj_opts &o, hj_result *res,
                     bool after_build = false) {
    const bool mat = o.mode == HJ_MATERIALIZE, chk = wants_checksum(o);
    const uint64_t warps = table_probe_warps(c, S->n);
    PairSink sink(c, t->width);
    uint64_t cap = mat ? first_capacity(o, S->n, warps) : 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        RecArea ra{nullptr, nullptr, 0};
        if (mat) {
            HJ_TRY(sink.reset(cap));
            HJ_TRY(sink.new_area(warps, &ra));
        }
        if (!(after_build && attempt == 0)) HJ_TRY(zero_counters(c));
        HJ_TRY(table_probe(c, t, S->tuples, 0, S->n, S->n, sink.pairs.p, sink.pcap, chk, ra, PartFilter{0, 0, 0, 0}));
        if (mat) HJ_TRY(sink.finalize_device(c->d_ctr));
        HJ_TRY(read_counters(c));
        if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
        HJ_TRY(check_output_status(c));
        if (!mat || c->h_ctr->cursor <= sink.pcap) break;
        // more pairs than the capacity: run the probe again at the exact size
        cap = c->h_ctr->count + warps * kChunkPairs;
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
    std::vector<JoinSlot> slots_host{JoinSlot{pairs, pcap, c->d_ctr, 0}};
    HJ_TRY(oversize_fallback(c, W, agg, chk, tasks, oversize, nov, slots_host));
    HJ_TRY(read_counters(c));
    if (c->h_ctr->status & kStatusTableFull) return set_err(c, HJ_E_CUDA, "hash table unexpectedly full");
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
    const uint64_t slice = task_slice_rows(R->width, S->n, NP), ntasks = max_tasks(NP, s_rows, slice);
    HJ_TRY(oversize.alloc(ntasks * 4));
    HJ_TRY(tasks.alloc(ntasks * sizeof(PartTask) + 8));
    HJ_TRY(slot.alloc(sizeof(JoinSlot)));
    HJ_TRY(make_tasks(c, Rp.p, roff.as<uint64_t>(), Sp.p, soff.as<uint64_t>(), NP, 0, b1, b2, R->width, slice, ntasks,
                      tasks.as<PartTask>()));
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

}  // namespace

extern "C" {

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
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
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
    DevBuf dR(c), dS(c);
    HJ_TRY(dR.alloc(Rh->n * tb + 64));
    HJ_TRY(dS.alloc(Sh->n * tb + 64));
    if (Rh->n) HJ_CUDA(c, cudaMemcpyAsync(dR.p, Rh->tuples, Rh->n * tb, cudaMemcpyHostToDevice, c->stream));
    if (Sh->n) HJ_CUDA(c, cudaMemcpyAsync(dS.p, Sh->tuples, Sh->n * tb, cudaMemcpyHostToDevice, c->stream));
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
        if (n) HJ_CUDA(c, cudaMemcpyAsync(pairs_host, pairs.p, n * tb, cudaMemcpyDeviceToHost, c->stream));
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
