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
// Key-list table (keylist.cu): aggregate-table slots over the kept tuples of
// R[0, n) plus the rid lists (t->rids, every key's rids contiguous at the offset
// its slot holds).  For build relations with heavily repeated keys.
hj_status keylist_build(hj_ctx *c, int width, const void *R, uint64_t n, PartFilter pf, hj_table **out);
// Pairs of the kept tuples of S[0, ns) against a key-list table, claimed exactly
// from ctr->count (dense output); checksums with `chk`.
hj_status keylist_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t ns, PartFilter pf, void *pairs,
                        uint64_t pcap, hj_counters *ctr, int chk);
// Insert tuples [lo, hi) of the array `R` (n_total tuples long) into the table.
// With pf.on only tuples of partition pf.p are inserted (padding is skipped).
hj_status table_build(hj_ctx *c, hj_table *t, const void *R, uint64_t lo, uint64_t hi, uint64_t n_total,
                      PartFilter pf);
// Probe with tuples [lo, hi) of S; counts and checksums accumulate into the
// context counters, pairs into `pairs` (capacity pcap; unused in count modes).
// Warps that leave a partly filled output chunk record it in `ra`.
// ctr: the counters to accumulate into (NULL: the context's).  dense: 0 = warps
// take whole chunks of the cursor (holes recorded in `ra`); 1 = every append
// claims exactly its rows from ctr->count; 2 = each warp stages its pairs in
// shared memory and claims exactly that many rows per full buffer (no holes,
// one atomic per 256 pairs).
hj_status table_probe(hj_ctx *c, const hj_table *t, const void *S, uint64_t lo, uint64_t hi, uint64_t n_total,
                      void *pairs, uint64_t pcap, int checksum, RecArea ra, PartFilter pf,
                      hj_counters *ctr = nullptr, int dense = 0);
// Number of warps table_probe launches for n probe tuples (record-area size).
uint64_t table_probe_warps(hj_ctx *c, uint64_t n);

// A partition pair for the shared-memory join: padded partitions (every row
// range starts on a 32-byte sector, its row count is a multiple of the sector's
// tuples), their partition index p under pass bits (b1, b2) -- rows hashing
// elsewhere are padding -- and the join (output target) they belong to.
struct PartTask {
    const void *R;
    const void *S;
    uint32_t nr, ns;
    uint32_t join, p;
    uint16_t b1, b2;
    uint32_t pad;
    uint64_t ek1;  // second empty-slot marker candidate for (b1, b2)
    // Keys a padding row of this partition can carry: 0 and each padded pass's
    // second sentinel (pass_pad_key); a build row with another key is a real tuple
    // of the partition and needs no hash to be kept.
    uint64_t pk1, pk2;
};
// Output of one join: its pair buffer and its counters.
struct JoinSlot {
    void *pairs;
    unsigned long long pcap;
    hj_counters *ctr;
    unsigned long long pad;
};
uint64_t empty_key2(int width, int b1, int b2);
// The second padding key of a padded pass over `bits` digits from bit `shift`
// (the first is 0): the smallest key whose digit differs from 0's.
uint64_t pass_pad_key(int width, int shift, int bits);
// Tasks for one join's NP partitions (device array `tasks` of `ntasks` entries
// plus 8 bytes, ntasks = max_tasks(NP, S rows, slice)): one per slice of at most
// `slice` S rows of every partition; unused entries are empty.
uint64_t task_slice_rows(int width, uint64_t n_s, uint64_t NP);
uint64_t max_tasks(uint64_t NP, uint64_t s_rows, uint64_t slice);
// Partitions p >= tail_from have their S rows probed in two halves (at most: the
// slice bound still holds); each such partition may add one task, so ntasks must
// then hold NP - tail_from more.
hj_status make_tasks(hj_ctx *c, const void *Rp, const uint64_t *roff, const void *Sp, const uint64_t *soff,
                     uint64_t NP, uint32_t join, int b1, int b2, int width, uint64_t slice, uint64_t ntasks,
                     PartTask *tasks, uint64_t tail_from = ~0ull);
// First partition of the persistent join's last, partly filled round of NP equal
// tasks (NP when the tasks fill whole rounds).
uint64_t tail_split_from(hj_ctx *c, int width, int agg, uint64_t NP, uint64_t expect_r);


// Per-partition join (Alg. 2's "apply SHJ on each partition pair") with the
// table in shared memory; persistent CTAs take tasks from c->d_ctr->work (which
// must be zero at launch).  Tasks whose table does not fit are appended to
// `oversize` (task indices) and counted in c->d_ctr->n_oversize.  Pairs go to
// each task's join slot: with `stage` (a staging area of scap pairs per warp, for
// partition_join_warps(c) warps) by
// exact claims, otherwise by per-warp chunks recorded in `ra`.
hj_status partition_join(hj_ctx *c, int width, int agg, const PartTask *tasks, uint64_t ntasks, const JoinSlot *slots,
                         uint64_t expect_r, int checksum, uint32_t *oversize, RecArea ra, void *stage,
                         uint32_t scap);
uint64_t partition_join_warps(hj_ctx *c);
uint64_t partition_join_ctas(hj_ctx *c, int width, int agg, uint64_t expect_r);

// ------------------------------------------------------------ api.cu (host joins)
// hj_join_host_large with R kept on the device: the device bytes of the streamed
// join (R partitioned once, S in chunks of chunk_rows through two buffer sets),
// the largest chunk (2^24 .. 2^20 rows) and one-pass radix bits that fit
// device_bytes (false if none does, or R needs two passes), and the join itself.
uint64_t host_streamed_bytes(hj_ctx *c, int width, bool mat, uint64_t nR, uint64_t chunk_rows, int bits);
bool host_streamed_plan(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts &o, uint64_t device_bytes,
                        uint64_t *chunk_rows, int *bits);
hj_status host_streamed_join(hj_ctx *c, const hj_rel *Rh, const hj_rel *Sh, const hj_opts &o, int bits,
                             uint64_t chunk_rows, void *pairs_host, uint64_t pairs_host_cap, hj_result *res);

struct PairSink;
// Tasks listed in `list_dev` (nov task indices) whose table did not fit in shared
// memory: SHJ with a global table per task, into the task's join slot (slots_host
// mirrors the device slots).  Pairs are claimed exactly at the slot's count, after
// the pairs already there.
// With `redo` (one join writing pairs into the context's counters), the counters
// are read after each task group's probe; from the first group whose pairs passed
// the slot's capacity on, each group's key-list table and S rows are kept in
// `redo`, with the counters from before that group, so that fallback_reprobe can
// write those groups' pairs again into a larger buffer without rebuilding.
struct FallbackGroup {
    hj_ctx *c;
    hj_table *t = nullptr;
    DevBuf Sg;                  // gathered S rows (empty when S is probed in place)
    const void *S = nullptr;
    uint64_t ns = 0;
    PartFilter pf{0, 0, 0, 0};
    explicit FallbackGroup(hj_ctx *ctx) : c(ctx), Sg(ctx) {}
    ~FallbackGroup();
};
struct FallbackRedo {
    bool crossed = false;
    hj_counters from{};  // counters before the first group that passed the capacity
    std::vector<std::unique_ptr<FallbackGroup>> groups;
};
hj_status oversize_fallback(hj_ctx *c, int W, bool agg, bool chk, const PartTask *tasks, const uint32_t *list_dev,
                            uint64_t nov, const std::vector<JoinSlot> &slots_host, FallbackRedo *redo = nullptr);
hj_status fallback_reprobe(hj_ctx *c, bool chk, const FallbackRedo &redo, const JoinSlot &slot);

// ------------------------------------------------------------ partition.cu
// One radix-partition pass over nseg independent segments of `in` (segment s is
// rows [seg_off[s], seg_off[s+1]), device offsets): each segment is split on
// hash bits [shift, shift + bits) into 2^bits partitions written to the same row
// range of `out`.  part_off (device, nseg * 2^bits + 1 entries) receives the row
// offset of every (segment, digit) partition.  With `pad`, every (chunk, digit)
// run is rounded up to whole 32-byte sectors with padding tuples whose key
// hashes to another digit, so the output holds up to partition_out_rows() rows
// and segment s of the output starts where the padded segments before it end.
// With seg_ptrs (device array of nseg pointers, 16-byte aligned), segment s is read
// from its own array seg_ptrs[s] instead of from `in` (fan-out at most 2^11).
hj_status partition_pass(hj_ctx *c, int width, const void *in, uint64_t n_total, const uint64_t *seg_off,
                         uint64_t nseg, int shift, int bits, void *out, uint64_t *part_off, int pad,
                         const void *const *seg_ptrs = nullptr);
// One padded pass over a single segment of n rows at 2^bits <= 2^11 digits:
// partition_pass's output with two launches (histogram, scatter).
hj_status partition_pass1(hj_ctx *c, int width, const void *in, uint64_t n, int bits, void *out, uint64_t *part_off);
uint64_t partition_out_rows(hj_ctx *c, int width, uint64_t n_total, uint64_t nseg, int bits, int pad);
// Exclusive scan of n uint32 counts into n + 1 uint64 offsets (out[n] = total).
hj_status scan_counts(hj_ctx *c, const uint32_t *in, uint64_t n, unsigned long long *out);

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
    hj_status grow(uint64_t cap_pairs, uint64_t keep);  // larger buffer holding the first `keep` pairs
    hj_status new_area(uint64_t warps, RecArea *ra);     // record area for one launch
    // Device-planned compaction of the single record area, stream-ordered after the
    // join: no host round trip.  Does nothing when the cursor ran past the capacity.
    hj_status finalize_device(hj_counters *ctr);
};

// ----------------------------------------------------------------- tune.cu
// Plan choice: the cost model (Sec. 4, Eq. 1-2 with every step on the GPU) and the
// plans hj_tune measured.  A candidate is (algo, total radix bits, passes) with
// its predicted seconds.
struct PlanCand {
    int algo, bits, passes;
    double sec;
};
CostModel cost_model_for(int device);
double predict_seconds(const CostModel &m, int width, bool agg, bool mat, uint64_t nR, uint64_t nS, int algo,
                       int bits, int passes, double *steps);
// Candidates allowed by the forced fields (0 = free), cheapest first.
std::vector<PlanCand> plan_candidates(const CostModel &m, int width, bool agg, bool mat, uint64_t nR, uint64_t nS,
                                      int algo, int bits, int passes);
uint64_t plan_key(int width, bool agg, uint64_t nR, uint64_t nS);
// The plan hj_join runs: a tuned plan for the size class if any, else the model's.
void choose_plan(hj_ctx *c, int width, int mode, uint64_t nR, uint64_t nS, int algo, int bits, int passes,
                 int *a_out, int *b_out, int *g_out);

// --------------------------------------------------------------- coexec.cu
// Host threads join partition pairs 0 .. np - 1 of padded partitioned copies in
// HOST memory (pass bits b1, b2): R rows roff[p] - roff[0] .. roff[p + 1] - roff[0]
// of `R`, likewise for S.  Counts and checksums add up in `out`; with `mat` each
// thread's (rid_R, rid_S) pairs (fields of `width` bytes) are in out->pairs[t].
struct CpuJoinPart {
    uint64_t count = 0, c0 = 0, c1 = 0;
};
struct CpuJoinResult {
    uint64_t count = 0, c0 = 0, c1 = 0;
    std::vector<CpuJoinPart> parts;
    std::vector<std::vector<uint8_t>> pairs;
};
struct CpuPool;  // host worker threads, kept on a context
CpuPool *cpu_pool_new();
void cpu_pool_delete(CpuPool *p);
void cpu_join_partitions(CpuPool *pool, int width, const void *R, const uint64_t *roff, const void *S,
                         const uint64_t *soff, uint32_t np, int b1, int b2, bool mat, bool chk, int threads,
                         CpuJoinResult *out);

// Tuple bytes of a relation of `width`-byte fields.
inline uint64_t tuple_bytes(int width) { return 2ull * (uint64_t)width; }

}  // namespace hj
