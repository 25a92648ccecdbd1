// engine.cuh -- internal launchers shared by the C ABI implementation.
#pragma once

#include <memory>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"

namespace hj {

struct RecArea;  // emit.cuh

// ----------------------------------------------------------------- join.cu
// Global-memory table (SHJ, Alg. 1): allocate + initialise, build, probe.
hj_status table_create(hj_ctx *c, int width, int agg, uint64_t n_build, hj_table **out);
void table_destroy(hj_ctx *c, hj_table *t);
// Insert tuples [lo, hi) of the array `R` (n_total tuples long) into the table.
// With pf.on only tuples of partition pf.p are inserted (padding is skipped).
hj_status table_build(hj_ctx *c, hj_table *t, const void *R, uint64_t lo, uint64_t hi, uint64_t n_total,
                      PartFilter pf);
// Probe with tuples [lo, hi) of S; counts and checksums accumulate into the
// context counters, pairs into `pairs` (capacity pcap; unused in count modes).
// Warps that leave a partly filled output chunk record it in `ra`.
hj_status table_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                      void *pairs, uint64_t pcap, int checksum, RecArea ra, PartFilter pf);
// Number of warps table_probe launches for n probe tuples (record-area size).
uint64_t table_probe_warps(hj_ctx *c, uint64_t n);

// Per-partition join (Alg. 2's "apply SHJ on each partition pair") with the
// table in shared memory, persistent CTAs over nparts pairs.  roff/soff hold
// nparts+1 row offsets into Rp/Sp.  Partitions whose table does not fit are
// appended to `oversize` (device, nparts entries) and counted in
// counters.n_oversize.  counters.work must be zero at launch.  With `filter`,
// tuples whose hash belongs to another partition (padding) are skipped.
hj_status partition_join(hj_ctx *c, int width, int agg, const void *Rp, const uint64_t *roff, uint64_t nR_total,
                         const void *Sp, const uint64_t *soff, uint64_t nS_total, uint64_t nparts,
                         uint64_t expect_r, void *pairs, uint64_t pcap, int checksum, uint32_t *oversize,
                         RecArea ra, int b1, int b2, int filter);
uint64_t partition_join_warps(hj_ctx *c);

// ------------------------------------------------------------ partition.cu
// One radix-partition pass over nseg independent segments of `in` (segment s is
// rows [seg_off[s], seg_off[s+1]), device offsets): each segment is split on
// hash bits [shift, shift + bits) into 2^bits partitions written to the same row
// range of `out`.  part_off (device, nseg * 2^bits + 1 entries) receives the row
// offset of every (segment, digit) partition.  With `pad`, every (chunk, digit)
// run is rounded up to whole 32-byte sectors with padding tuples whose key
// hashes to another digit, so the output holds up to partition_out_rows() rows
// and segment s of the output starts where the padded segments before it end.
hj_status partition_pass(hj_ctx *c, int width, const void *in, uint64_t n_total, const uint64_t *seg_off,
                         uint64_t nseg, int shift, int bits, void *out, uint64_t *part_off, int pad);
uint64_t partition_out_rows(hj_ctx *c, int width, uint64_t n_total, uint64_t nseg, int bits, int pad);

// --------------------------------------------------------------- output.cu
// The pair buffer of a materialising join: warps append whole chunks, then
// finalize() moves tail pairs into the holes so that pairs[0, count) is dense.
struct PairSink {
    hj_ctx *c;
    int width;
    DevBuf pairs;
    uint64_t pcap = 0;
    std::vector<std::unique_ptr<DevBuf>> areas;
    std::vector<uint64_t> caps;
    PairSink(hj_ctx *ctx, int w) : c(ctx), width(w), pairs(ctx) {}
    hj_status reset(uint64_t cap_pairs);                 // (re)allocate the buffer, drop records
    hj_status new_area(uint64_t warps, RecArea *ra);     // record area for one launch
    hj_status finalize(uint64_t count, uint64_t cursor);
};

// Tuple bytes of a relation of `width`-byte fields.
inline uint64_t tuple_bytes(int width) { return 2ull * (uint64_t)width; }

}  // namespace hj
