// outcore.cu -- joins of relations held in host memory that need not fit the
// device (hj_join_host_large), after the paper's larger-than-buffer scheme
// (App. A: partition each relation chunk by chunk through a bounded buffer, keep
// the partitions, then join every partition pair).
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

// Stream `in` (host) through the device in chunks of at most `chunk` tuples and
// split it on bits [kTopShift, kTopShift + bt).
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
    DevBuf d_in(c), d_out(c), d_off(c), d_seg(c);
    const uint64_t out_rows = partition_out_rows(c, in->width, chunk, 1, bt, 0);
    HJ_TRY(d_in.alloc(chunk * tb + 64));
    HJ_TRY(d_out.alloc(out_rows * tb + 64));
    HJ_TRY(d_off.alloc((P + 1) * 8));
    HJ_TRY(d_seg.alloc(16));
    std::vector<uint64_t> off(P + 1);
    for (uint64_t r0 = 0; r0 < in->n; r0 += chunk) {
        const uint64_t n = std::min(chunk, in->n - r0);
        const uint64_t seg[2] = {0, n};
        HJ_CUDA(c, cudaMemcpyAsync(d_seg.p, seg, 16, cudaMemcpyHostToDevice, c->stream));
        HJ_TRY(copy_wide(c, d_in.p, (const char *)in->tuples + r0 * tb, n * tb, cudaMemcpyHostToDevice));
        HJ_TRY(partition_pass(c, in->width, d_in.p, n, d_seg.as<uint64_t>(), 1, kTopShift, bt, d_out.p,
                              d_off.as<uint64_t>(), 0));
        HJ_TRY(copy_wide(c, (char *)hp.rows + r0 * tb, d_out.p, n * tb, cudaMemcpyDeviceToHost));
        HJ_CUDA(c, cudaMemcpyAsync(off.data(), d_off.p, (P + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
        HJ_CUDA(c, cudaStreamSynchronize(c->stream));
        hp.chunk_row.push_back(r0);
        hp.off.push_back(off);
    }
    return HJ_OK;
}

// Rows [lo, hi) of partition p (in chunk order) onto the device at `dst`.
hj_status gather(hj_ctx *c, const HostPart &hp, uint32_t p, uint64_t lo, uint64_t hi, uint64_t tb, void *dst) {
    uint64_t at = 0, put = 0;
    for (size_t ci = 0; ci < hp.off.size() && at < hi; ++ci) {
        const uint64_t b = hp.off[ci][p], e = hp.off[ci][p + 1], len = e - b;
        const uint64_t s0 = std::max(lo, at), s1 = std::min(hi, at + len);
        if (s1 > s0) {
            const char *src = (const char *)hp.rows + (hp.chunk_row[ci] + b + (s0 - at)) * tb;
            HJ_CUDA(c, cudaMemcpyAsync((char *)dst + put * tb, src, (s1 - s0) * tb, cudaMemcpyHostToDevice, c->stream));
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
    // top-level fan-out: partition pairs of a uniform split fit with room for skew
    int bt = 1;
    while (bt < kTopMaxBits && 3 * join_bytes(Rh->n >> bt, Sh->n >> bt, tb, mat) / 2 > device_bytes) ++bt;
    const uint64_t chunk = std::max<uint64_t>(1ull << 16, device_bytes / (3 * tb) / 1024 * 1024);
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
    for (uint32_t p = 0; p < (1u << bt); ++p) {
        const uint64_t nr = hr.part_rows(p), ns = hs.part_rows(p);
        if (nr == 0 || ns == 0) continue;
        // S groups that fit next to the whole R partition
        uint64_t sg = ns;
        while (sg > kMinGroup && join_bytes(nr, sg, tb, mat) > device_bytes) sg = (sg + 1) / 2;
        if (join_bytes(nr, std::min(sg, ns), tb, mat) > device_bytes)
            return set_err(c, HJ_E_NOMEM, "partition %u (%llu R tuples) does not fit the device budget", p,
                           (unsigned long long)nr);
        DevBuf dR(c), dS(c);
        HJ_TRY(dR.alloc(nr * tb + 64));
        HJ_TRY(dS.alloc(std::min(sg, ns) * tb + 64));
        HJ_TRY(gather(c, hr, p, 0, nr, tb, dR.p));
        for (uint64_t s0 = 0; s0 < ns; s0 += sg) {
            const uint64_t s1 = std::min(ns, s0 + sg);
            HJ_TRY(gather(c, hs, p, s0, s1, tb, dS.p));
            hj_rel R{dR.p, nr, Rh->width, 0}, S{dS.p, s1 - s0, Rh->width, 0};
            hj_result r{};
            HJ_TRY(hj_join(c, &R, &S, &oj, &r));
            count += r.count;
            c0 += r.checksum[0];
            c1 += r.checksum[1];
            if (mat && r.count && r.pairs) {
                const uint64_t n = written < pairs_host_cap ? std::min(r.count, pairs_host_cap - written) : 0;
                if (n && pairs_host)
                    HJ_TRY(copy_wide(c, (char *)pairs_host + written * tb, r.pairs, n * tb, cudaMemcpyDeviceToHost));
                HJ_CUDA(c, cudaStreamSynchronize(c->stream));
                written += n;
            }
            hj_result_free(c, &r);
        }
    }
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
