// outcore.cu -- joins of relations held in host memory that need not fit the
// device (hj_join_host_large), after the paper's larger-than-buffer scheme
// (App. A: partition each relation chunk by chunk through a bounded buffer, keep
// the partitions, then join every partition pair).
//
// When R alone fits the budget with room for two S chunks in flight, the split is
// skipped: R is partitioned once on the device and S streamed past it in chunks
// (host_streamed_join, api.cu), so that each tuple crosses the host link once
// instead of three times.  Otherwise:
//
//   1. partition: each relation is streamed to the device in chunks that fit the
//      budget; every chunk is split on hash bits [kTopShift, kTopShift + bt) by the
//      partition pass and copied back whole, with its partition offsets, into a
//      page-locked host buffer: partition p of the relation is the concatenation
//      of its slice of every chunk.
//   2. join: partition pair p is gathered onto the device (one copy per chunk
//      slice) and joined by the PHJ, whose own partitioning uses hash bits from 0
//      up -- disjoint from the top-level bits, so partition p's keys still spread
//      over all of its digits.  Pairs go to the caller's host buffer; counts and
//      checksums (order-free sums) add up.  A pair whose S side alone is too large
//      for the budget (skew) is joined in S groups against the whole R partition.
#include <algorithm>
#include <vector>

#include "ctx.cuh"
#include "engine.cuh"

namespace {

using namespace hj;

constexpr int kTopShift = 20;  // first hash bit of the top-level split
constexpr int kTopMaxBits = 8;

constexpr uint64_t kMinGroup = 1ull << 16;  // smallest S group joined against an R partition

// Device bytes hj_join needs whatever the sizes: counters, histograms, task lists
// and (materialising) the pair buffer's slack of one chunk per emitting warp.
uint64_t fixed_bytes(uint64_t tb, bool mat) { return (64ull << 20) + (mat ? (1ull << 20) * tb : 0); }

// Device bytes a join of nr x ns tuples takes in hj_join (inputs, partitioned
// copies with padding, pair buffer, fixed workspace).
uint64_t join_bytes(uint64_t nr, uint64_t ns, uint64_t tb, bool mat) {
    uint64_t b = (nr + ns) * tb * 2 + (nr + ns) * tb / 10 + fixed_bytes(tb, mat);
    if (mat) b += ns * tb;
    return b;
}

// The same with a second input set (the next join's inputs, copied in meanwhile)
// and the pairs of the two joins before it, still being copied home.
uint64_t pipe_bytes(uint64_t nr, uint64_t ns, uint64_t tb, bool mat) {
    return join_bytes(nr, ns, tb, mat) + (nr + ns) * tb + (mat ? 2 * ns * tb : 0);
}

struct HostPart {
    // one relation split into 2^bt partitions, chunk by chunk
    std::vector<uint64_t> chunk_row;               // first row of chunk c in `rows`
    std::vector<std::vector<uint64_t>> off;        // off[c][p]: offsets inside chunk c (2^bt + 1)
    void *rows = nullptr;                          // page-locked (the context's), partitioned chunks back to back
    uint64_t n = 0;
    uint64_t part_rows(uint32_t p) const {
        uint64_t t = 0;
        for (size_t c = 0; c < off.size(); ++c) t += off[c][p + 1] - off[c][p];
        return t;
    }
};

// Streams and events of the overlapped copies: copies in on pipe_in, kernels on the
// context's stream, copies out on pipe_out.
struct Lanes {
    hj_ctx *c;
    std::vector<cudaEvent_t> ev;
    explicit Lanes(hj_ctx *ctx) : c(ctx) {}
    hj_status open() {
        if (!c->pipe_in) HJ_CUDA(c, cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking));
        if (!c->pipe_out) HJ_CUDA(c, cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking));
        return HJ_OK;
    }
    hj_status event(cudaEvent_t *e) {
        HJ_CUDA(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        ev.push_back(*e);
        return HJ_OK;
    }
    // `to` waits for everything queued so far on `from`
    hj_status order(cudaStream_t from, cudaStream_t to) {
        cudaEvent_t e;
        HJ_TRY(event(&e));
        HJ_CUDA(c, cudaEventRecord(e, from));
        HJ_CUDA(c, cudaStreamWaitEvent(to, e, 0));
        return HJ_OK;
    }
    // the context's stream waits for both copy streams (before buffers are freed on it)
    hj_status join() {
        HJ_TRY(order(c->pipe_in, c->stream));
        return order(c->pipe_out, c->stream);
    }
    ~Lanes() {
        if (c->pipe_in) cudaStreamSynchronize(c->pipe_in);
        if (c->pipe_out) cudaStreamSynchronize(c->pipe_out);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Stream `in` (host) through the device in chunks of at most `chunk` tuples and
// split it on bits [kTopShift, kTopShift + bt).  Two buffer sets: chunk i + 1's
// copy in, chunk i's partition pass and chunk i - 1's copy out run at once.
hj_status split_host(hj_ctx *c, const hj_rel *in, int bt, uint64_t chunk, int side, HostPart &hp) {
    const uint64_t tb = tuple_bytes(in->width), P = 1ull << bt;
    hp.n = in->n;
    if (in->n == 0) return HJ_OK;
    // the context keeps one page-locked buffer per side, grown when too small
    if (c->host_cap[side] < in->n * tb) {
        if (c->host_buf[side]) cudaFreeHost(c->host_buf[side]);
        c->host_buf[side] = nullptr;
        c->host_cap[side] = 0;
        HJ_CUDA(c, cudaMallocHost(&c->host_buf[side], in->n * tb));
        c->host_cap[side] = in->n * tb;
    }
    hp.rows = c->host_buf[side];
    const uint64_t nchunks = (in->n + chunk - 1) / chunk;
    const uint64_t out_rows = partition_out_rows(c, in->width, chunk, 1, bt, 0);
    DevBuf d_in0(c), d_in1(c), d_out0(c), d_out1(c), d_seg(c), h_off_dev(c);
    DevBuf *d_in[2] = {&d_in0, &d_in1}, *d_out[2] = {&d_out0, &d_out1};
    for (int k = 0; k < 2; ++k) {
        HJ_TRY(d_in[k]->alloc(chunk * tb + 64));
        HJ_TRY(d_out[k]->alloc(out_rows * tb + 64));
    }
    HJ_TRY(h_off_dev.alloc(nchunks * (P + 1) * 8));  // every chunk's partition offsets
    HJ_TRY(d_seg.alloc(nchunks * 16));               // every chunk's segment {0, n}
    std::vector<uint64_t> seg(2 * nchunks);
    for (uint64_t i = 0; i < nchunks; ++i) {
        seg[2 * i] = 0;
        seg[2 * i + 1] = std::min(chunk, in->n - i * chunk);
    }
    HJ_CUDA(c, cudaMemcpyAsync(d_seg.p, seg.data(), nchunks * 16, cudaMemcpyHostToDevice, c->stream));
    // (declared after the buffers: on an early return the copy streams are drained
    // before the buffers are freed)
    Lanes ln(c);
    HJ_TRY(ln.open());
    cudaStream_t cin = c->pipe_in, cout = c->pipe_out;
    // the copy streams see the buffers only after their allocation on the context's stream
    HJ_TRY(ln.order(c->stream, cin));
    HJ_TRY(ln.order(c->stream, cout));
    cudaEvent_t copied[2], parted[2], sent[2];
    for (int k = 0; k < 2; ++k) {
        HJ_TRY(ln.event(&copied[k]));
        HJ_TRY(ln.event(&parted[k]));
        HJ_TRY(ln.event(&sent[k]));
    }
    for (uint64_t i = 0; i < nchunks; ++i) {
        const int k = (int)(i & 1);
        const uint64_t r0 = i * chunk, n = seg[2 * i + 1];
        // d_in[k] is free once chunk i - 2 was partitioned, d_out[k] once it was sent
        if (i >= 2) HJ_CUDA(c, cudaStreamWaitEvent(cin, parted[k], 0));
        HJ_CUDA(c, cudaMemcpyAsync(d_in[k]->p, (const char *)in->tuples + r0 * tb, n * tb, cudaMemcpyHostToDevice,
                                   cin));
        HJ_CUDA(c, cudaEventRecord(copied[k], cin));
        HJ_CUDA(c, cudaStreamWaitEvent(c->stream, copied[k], 0));
        if (i >= 2) HJ_CUDA(c, cudaStreamWaitEvent(c->stream, sent[k], 0));
        HJ_TRY(partition_pass(c, in->width, d_in[k]->p, n, d_seg.as<uint64_t>() + 2 * i, 1, kTopShift, bt,
                              d_out[k]->p, h_off_dev.as<uint64_t>() + i * (P + 1), 0));
        HJ_CUDA(c, cudaEventRecord(parted[k], c->stream));
        HJ_CUDA(c, cudaStreamWaitEvent(cout, parted[k], 0));
        HJ_CUDA(c, cudaMemcpyAsync((char *)hp.rows + r0 * tb, d_out[k]->p, n * tb, cudaMemcpyDeviceToHost, cout));
        HJ_CUDA(c, cudaEventRecord(sent[k], cout));
        hp.chunk_row.push_back(r0);
    }
    std::vector<uint64_t> offs(nchunks * (P + 1));
    HJ_TRY(ln.join());
    HJ_CUDA(c, cudaMemcpyAsync(offs.data(), h_off_dev.p, offs.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    for (uint64_t i = 0; i < nchunks; ++i)
        hp.off.emplace_back(offs.begin() + i * (P + 1), offs.begin() + (i + 1) * (P + 1));
    return HJ_OK;
}

// Rows [lo, hi) of partition p (in chunk order) onto the device at `dst`.
hj_status gather(hj_ctx *c, const HostPart &hp, uint32_t p, uint64_t lo, uint64_t hi, uint64_t tb, void *dst,
                 cudaStream_t st) {
    uint64_t at = 0, put = 0;
    for (size_t ci = 0; ci < hp.off.size() && at < hi; ++ci) {
        const uint64_t b = hp.off[ci][p], e = hp.off[ci][p + 1], len = e - b;
        const uint64_t s0 = std::max(lo, at), s1 = std::min(hi, at + len);
        if (s1 > s0) {
            const char *src = (const char *)hp.rows + (hp.chunk_row[ci] + b + (s0 - at)) * tb;
            HJ_CUDA(c, cudaMemcpyAsync((char *)dst + put * tb, src, (s1 - s0) * tb, cudaMemcpyHostToDevice, st));
            put += s1 - s0;
        }
        at += len;
    }
    return HJ_OK;
}

}  // namespace

extern "C" hj_status hj_join_host_large(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts *opts,
                                        uint64_t device_bytes, void *pairs_host, uint64_t pairs_host_cap,
                                        hj_result *out) {
    if (!c) return HJ_E_INVALID;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(c, cudaGetLastError(), "cudaSetDevice");
    if (!out || !Rh || !Sh) return set_err(c, HJ_E_INVALID, "NULL argument");
    if ((Rh->width != HJ_U32 && Rh->width != HJ_U64) || Rh->width != Sh->width)
        return set_err(c, HJ_E_INVALID, "bad or differing widths");
    if ((Rh->n && !Rh->tuples) || (Sh->n && !Sh->tuples)) return set_err(c, HJ_E_INVALID, "NULL host tuples");
    hj_opts o{};
    o.mode = HJ_MATERIALIZE;
    if (opts) o = *opts;
    if (o.mode < HJ_COUNT || o.mode > HJ_MATERIALIZE) return set_err(c, HJ_E_INVALID, "bad mode %d", o.mode);
    const bool mat = o.mode == HJ_MATERIALIZE;
    const uint64_t tb = tuple_bytes(Rh->width);
    if (device_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        device_bytes = (uint64_t)(fr * 0.4);
    }
    *out = hj_result{};
    if (device_bytes < 2 * fixed_bytes(tb, mat))
        return set_err(c, HJ_E_INVALID, "device budget %llu below the minimum %llu", (unsigned long long)device_bytes,
                       (unsigned long long)(2 * fixed_bytes(tb, mat)));
    // everything fits: one join
    if (join_bytes(Rh->n, Sh->n, tb, mat) <= device_bytes)
        return hj_join_host(c, Rh, Sh, &o, pairs_host, pairs_host_cap, out);
    // R fits with room to stream S past it: R is partitioned once and kept, S goes
    // through in chunks (every tuple crosses the link once, where the split below
    // takes three crossings)
    {
        uint64_t sc = 0;
        int sb = 0;
        if (c->outcore_mode != HJ_OUTCORE_SPLIT && host_streamed_plan(c, Rh, Sh, o, device_bytes, &sc, &sb))
            return host_streamed_join(c, Rh, Sh, o, sb, sc, pairs_host, pairs_host_cap, out);
    }
    // top-level fan-out: partition pairs of a uniform split fit with room for skew
    int bt = 1;
    while (bt < kTopMaxBits && 3 * pipe_bytes(Rh->n >> bt, Sh->n >> bt, tb, mat) / 2 > device_bytes) ++bt;
    // two chunk sets (input and partitioned copy each) in flight
    const uint64_t chunk = std::max<uint64_t>(1ull << 16, device_bytes / (6 * tb) / 1024 * 1024);
    HostPart hr, hs;
    HJ_TRY(split_host(c, Rh, bt, chunk, 0, hr));
    HJ_TRY(split_host(c, Sh, bt, chunk, 1, hs));
    // join every partition pair (PHJ: its digits use hash bits below kTopShift)
    hj_opts oj = o;
    oj.algo = HJ_ALGO_PHJ;
    oj.radix_bits = 0;
    oj.passes = 0;
    oj.out_capacity = 0;
    uint64_t count = 0, c0 = 0, c1 = 0, written = 0;
    // the joins to run: (partition, S group) in order, each S group fitting beside
    // the whole R partition and a second input set (the next unit's, copied in
    // while this one joins)
    struct Unit {
        uint32_t p;
        uint64_t nr, s0, s1;
    };
    std::vector<Unit> units;
    uint64_t max_r = 0, max_s = 0;
    for (uint32_t p = 0; p < (1u << bt); ++p) {
        const uint64_t nr = hr.part_rows(p), ns = hs.part_rows(p);
        if (nr == 0 || ns == 0) continue;
        uint64_t sg = ns;
        while (sg > kMinGroup && pipe_bytes(nr, sg, tb, mat) > device_bytes) sg = (sg + 1) / 2;
        if (pipe_bytes(nr, std::min(sg, ns), tb, mat) > device_bytes)
            return set_err(c, HJ_E_NOMEM, "partition %u (%llu R tuples) does not fit the device budget", p,
                           (unsigned long long)nr);
        for (uint64_t s0 = 0; s0 < ns; s0 += sg) units.push_back(Unit{p, nr, s0, std::min(ns, s0 + sg)});
        max_r = std::max(max_r, nr);
        max_s = std::max(max_s, std::min(sg, ns));
    }
    if (units.empty()) {
        out->count = 0;
        out->width = Rh->width;
        out->algo = HJ_ALGO_PHJ;
        out->radix_bits = bt;
        return HJ_OK;
    }
    DevBuf dR0(c), dR1(c), dS0(c), dS1(c);
    DevBuf *dR[2] = {&dR0, &dR1}, *dS[2] = {&dS0, &dS1};
    for (int k = 0; k < 2; ++k) {
        HJ_TRY(dR[k]->alloc(max_r * tb + 64));
        HJ_TRY(dS[k]->alloc(max_s * tb + 64));
    }
    // joined units whose pairs are still on their way home (freed however the loop ends)
    struct Inflight {
        hj_ctx *c;
        std::vector<hj_result> r;
        ~Inflight() {
            for (hj_result &x : r) hj_result_free(c, &x);
        }
    } inflight{c, {}};
    // (declared after the buffers: on an early return the copy streams are drained
    // before the buffers and results are freed)
    Lanes ln(c);
    HJ_TRY(ln.open());
    cudaStream_t cin = c->pipe_in, cout = c->pipe_out;
    HJ_TRY(ln.order(c->stream, cin));
    HJ_TRY(ln.order(c->stream, cout));
    cudaEvent_t arrived[2];
    for (int k = 0; k < 2; ++k) HJ_TRY(ln.event(&arrived[k]));
    // unit u's inputs into set k (R only when the partition changes)
    auto fetch = [&](size_t u, int k) -> hj_status {
        const Unit &x = units[u];
        // set k still holds R of partition p when unit u - 2 (the last one in set k) had it
        if (u < 2 || units[u - 2].p != x.p) HJ_TRY(gather(c, hr, x.p, 0, x.nr, tb, dR[k]->p, cin));
        HJ_TRY(gather(c, hs, x.p, x.s0, x.s1, tb, dS[k]->p, cin));
        HJ_CUDA(c, cudaEventRecord(arrived[k], cin));
        return HJ_OK;
    };
    HJ_TRY(fetch(0, 0));
    for (size_t u = 0; u < units.size(); ++u) {
        const int k = (int)(u & 1);
        const Unit &x = units[u];
        // the next unit's inputs go into the other set, whose last join has returned
        if (u + 1 < units.size()) HJ_TRY(fetch(u + 1, k ^ 1));
        HJ_CUDA(c, cudaStreamWaitEvent(c->stream, arrived[k], 0));
        hj_rel R{dR[k]->p, x.nr, Rh->width, 0}, S{dS[k]->p, x.s1 - x.s0, Rh->width, 0};
        hj_result r{};
        HJ_TRY(hj_join(c, &R, &S, &oj, &r));  // returns once its counters are read
        count += r.count;
        c0 += r.checksum[0];
        c1 += r.checksum[1];
        if (mat && r.count && r.pairs) {
            const uint64_t n = written < pairs_host_cap ? std::min(r.count, pairs_host_cap - written) : 0;
            if (n && pairs_host) {
                HJ_TRY(ln.order(c->stream, cout));
                HJ_CUDA(c, cudaMemcpyAsync((char *)pairs_host + written * tb, r.pairs, n * tb, cudaMemcpyDeviceToHost,
                                           cout));
            }
            written += n;
        }
        inflight.r.push_back(r);
        // a result's pairs are freed (on the context's stream) after the copies queued so far
        if (inflight.r.size() > 2) {
            HJ_TRY(ln.order(cout, c->stream));
            hj_result_free(c, &inflight.r.front());
            inflight.r.erase(inflight.r.begin());
        }
    }
    HJ_TRY(ln.join());
    for (hj_result &r : inflight.r) hj_result_free(c, &r);
    inflight.r.clear();
    HJ_CUDA(c, cudaStreamSynchronize(c->stream));
    out->count = count;
    out->checksum[0] = c0;
    out->checksum[1] = c1;
    out->width = Rh->width;
    out->algo = HJ_ALGO_PHJ;
    out->radix_bits = bt;
    out->passes = 0;
    if (mat && count > pairs_host_cap)
        return set_err(c, HJ_E_OVERFLOW, "%llu pairs do not fit in %llu", (unsigned long long)count,
                       (unsigned long long)pairs_host_cap);
    if (mat && count && !pairs_host) return set_err(c, HJ_E_INVALID, "pairs_host is NULL but the join has pairs");
    return HJ_OK;
}
