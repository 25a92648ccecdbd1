// engine.cuh -- internal launchers shared by the C ABI implementation.
#pragma once

#include "ctx.cuh"

namespace hj {

// ----------------------------------------------------------------- join.cu
// Global-memory table (SHJ, Alg. 1): allocate + initialise, build, probe.
hj_status table_create(hj_ctx *c, int width, int agg, uint64_t n_build, hj_table **out);
void table_destroy(hj_ctx *c, hj_table *t);
// Insert tuples [lo, hi) of the array `R` (n_total tuples long) into the table.
hj_status table_build(hj_ctx *c, hj_table *t, const void *R, uint64_t lo, uint64_t hi, uint64_t n_total);
// Probe with tuples [lo, hi) of S; results accumulate into the context counters
// (count = output cursor) and `pairs` (capacity pcap, may be null in count modes).
hj_status table_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                      void *pairs, uint64_t pcap, int checksum);

// Per-partition join (Alg. 2's "apply SHJ on each partition pair") with the
// table in shared memory: one CTA per partition pair.  roff/soff hold nparts+1
// row offsets into Rp/Sp.  Partitions whose table does not fit are appended to
// `oversize` (device, nparts entries) and counted in counters.n_oversize.
hj_status partition_join(hj_ctx *c, int width, int agg, const void *Rp, const uint64_t *roff, uint64_t nR_total,
                         const void *Sp, const uint64_t *soff, uint64_t nS_total, uint64_t nparts,
                         uint64_t expect_r, void *pairs, uint64_t pcap, int checksum, uint32_t *oversize);

// ------------------------------------------------------------ partition.cu
// One radix-partition pass over nseg independent segments of `in` (segment s is
// rows [seg_off[s], seg_off[s+1]), device offsets): each segment is split on
// hash bits [shift, shift + bits) into 2^bits partitions written to the same row
// range of `out`.  part_off (device, nseg * 2^bits + 1 entries) receives the row
// offset of every (segment, digit) partition.
hj_status partition_pass(hj_ctx *c, int width, const void *in, uint64_t n_total, const uint64_t *seg_off,
                         uint64_t nseg, int shift, int bits, void *out, uint64_t *part_off);

// Tuple bytes of a relation of `width`-byte fields.
inline uint64_t tuple_bytes(int width) { return 2ull * (uint64_t)width; }

}  // namespace hj
