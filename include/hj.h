/*
 * hj.h -- C ABI of the GB300 hash-join engine (libhj.so).
 *
 * The engine computes the equi-join of two relations R and S of <key, rid> tuples:
 * the multiset of pairs (r.rid, s.rid) with r.key == s.key.  Its two algorithms are
 * the simple hash join (SHJ: build a table on R, probe it with S -- Sec. 3.1,
 * Alg. 1) and the radix-partitioned hash join (PHJ: partition R and S on low bits
 * of the key hash in one or two passes, then run SHJ on every partition pair --
 * Sec. 3.1, Alg. 2).  Tuples are two integer attributes (Sec. 5.1); here both are
 * 4 bytes (HJ_U32) or both 8 bytes (HJ_U64).
 *
 * Conventions shared by every call:
 *   - Tuple and offset pointers are DEVICE pointers on the context's device unless
 *     a call says otherwise.  The caller owns its inputs; the library never frees
 *     or writes them.  Buffers the library returns (tables, pairs, partitions) are
 *     library-owned and released with the matching *_free call.
 *   - Work is ordered on the context's CUDA stream.  Calls that return a count
 *     (hj_probe, hj_join, hj_join_batch, hj_partition) synchronise that stream
 *     before returning.
 *   - Relations are arrays of n tuples, AoS, key first then rid, each field
 *     `width` bytes, little-endian; `tuples` must be 16-byte aligned (n = 0 allows
 *     NULL).  No key or rid value is reserved: 0 and 2^(8*width)-1 are ordinary.
 *   - Every call returns an hj_status; nothing aborts, traps or prints.
 *     hj_last_error() describes the last failure on a context.
 *   - The radix digit and the table bucket come from MurmurHash2 (Sec. 5.1) of the
 *     key's little-endian bytes with seed 0: the 32-bit variant for 4-byte keys,
 *     MurmurHash64A for 8-byte keys.  The digit of pass one is bits [0, b1) of the
 *     hash, of pass two bits [b1, b1 + b2) (Alg. 2: "lower bits of the integer hash
 *     values"); table buckets use the high bits.
 */
#ifndef HJ_H
#define HJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hj_status;
#define HJ_OK 0
#define HJ_E_INVALID 1     /* bad argument: NULL, width, alignment, sizes          */
#define HJ_E_NOMEM 2       /* device allocation failed or HBM budget exceeded      */
#define HJ_E_OVERFLOW 3    /* caller capacity too small; the required size is set */
#define HJ_E_CUDA 4        /* a CUDA runtime call failed                           */
#define HJ_E_TIMEOUT 5     /* a bounded device-side wait expired                   */
#define HJ_E_UNSUPPORTED 6 /* valid request this build does not implement         */
#define HJ_E_PENDING 7     /* serving: request not finished yet                    */

#define HJ_U32 4
#define HJ_U64 8

/* A relation: n tuples of <key, rid>, both fields `width` bytes (HJ_U32 or HJ_U64).
 * The device entry points take relations of fewer than 2^32 - 1 tuples (row offsets
 * inside a partition pass are 32-bit); hj_join_host_large splits larger host
 * relations into partition pairs below that size. */
typedef struct hj_rel {
    const void *tuples;
    uint64_t n;
    int32_t width;
    int32_t reserved;
} hj_rel;

/* Output modes.  COUNT returns |J|; COUNT_CHECKSUM adds two order-independent sums
 * over J, c0 = sum A(rid_R) * B(rid_S) and c1 = sum A(rid_R) + B(rid_S) (mod 2^64),
 * with A(x) the SplitMix64 finaliser of x and B(x) = A(x ^ 0x9E3779B97F4A7C15);
 * both are computed per key without forming pairs.  MATERIALIZE also returns the
 * pairs in a device buffer. */
#define HJ_COUNT 0
#define HJ_COUNT_CHECKSUM 1
#define HJ_MATERIALIZE 2

#define HJ_ALGO_AUTO 0
#define HJ_ALGO_SHJ 1
#define HJ_ALGO_PHJ 2

/* opts.flags */
#define HJ_FLAG_CHECKSUM 1u /* MATERIALIZE: also compute c0, c1 over the pairs           */
#define HJ_FLAG_GRAPH 2u    /* hj_join_batch: capture each wave's launches in a CUDA graph */

typedef struct hj_opts {
    int32_t algo;          /* HJ_ALGO_*                                              */
    int32_t mode;          /* HJ_COUNT, HJ_COUNT_CHECKSUM, HJ_MATERIALIZE            */
    int32_t radix_bits;    /* PHJ: total radix bits b1 + b2 (0: the tuner chooses)  */
    int32_t passes;        /* PHJ: 1 or 2 partition passes (0: the tuner chooses)   */
    uint64_t out_capacity; /* MATERIALIZE: initial pair capacity (0: |S|); a join
                              with more pairs is re-run once at the exact size     */
    uint64_t flags;        /* HJ_FLAG_*                                              */
} hj_opts;

/* Result of a join.  `pairs` holds `count` pairs (rid_R, rid_S), each field `width`
 * bytes (the relations' width), in no particular order; NULL in the count modes.
 * It is library-owned: release it with hj_result_free. */
typedef struct hj_result {
    uint64_t count;
    uint64_t checksum[2];
    void *pairs;
    uint64_t pairs_cap;
    int32_t width;
    int32_t algo;       /* algorithm that ran: HJ_ALGO_SHJ or HJ_ALGO_PHJ */
    int32_t radix_bits; /* PHJ: total radix bits used                     */
    int32_t passes;     /* PHJ: partition passes used                     */
} hj_result;

typedef struct hj_ctx hj_ctx;
typedef struct hj_table hj_table;

/* Create a context on `device`.  `cuda_stream` is a cudaStream_t to order work on
 * (NULL: the library creates its own non-blocking stream, which is NOT ordered
 * after work on the legacy default stream -- pass cudaStreamLegacy to order the
 * context's work with that stream, e.g. after kernels that produced the inputs
 * there).  Any stream may be given, the legacy one included: the library captures
 * CUDA graphs on private streams.  `hbm_budget_bytes`
 * caps the device memory the library holds at once (0: no cap).  Every later call
 * on the context must run with that device current or will make it current. */
hj_status hj_create(hj_ctx **ctx, int device, void *cuda_stream, uint64_t hbm_budget_bytes);

/* Release the context and every buffer it still owns. */
hj_status hj_destroy(hj_ctx *ctx);

/* Text of the last error on the context ("" if none).  Valid until the next call. */
const char *hj_last_error(const hj_ctx *ctx);

/* SHJ build phase (Alg. 1, steps b1-b4): a device hash table on R.  For the
 * MATERIALIZE mode the table holds every R tuple (duplicates kept as separate
 * entries; if a key repeats so often that an insert walks past 1024 slots, the
 * table is rebuilt in the paper's key-list form -- one entry per distinct key
 * with the list of its rids -- within the same call); for the count modes it
 * holds one entry per distinct key with the tuple count and the sum of A(rid).  `opts->mode` fixes which; the table is only
 * valid for probes in a mode of the same family.  R is read during the call's
 * stream work only; the table does not point into R. */
hj_status hj_build(hj_ctx *ctx, const hj_rel *R, const hj_opts *opts, hj_table **out);

/* SHJ probe phase (Alg. 1, steps p1-p4): look every S tuple up in `table` and
 * produce the join result in `out` (count, checksums, pairs as `opts->mode` says).
 * HJ_E_INVALID if S's width differs from the table's or the modes differ. */
hj_status hj_probe(hj_ctx *ctx, const hj_table *table, const hj_rel *S, const hj_opts *opts,
                   hj_result *out);

hj_status hj_table_free(hj_ctx *ctx, hj_table *table);

/* Radix partitioning (Alg. 2, steps n1-n3): split `in` into 2^(b1+b2) partitions,
 * pass one on hash bits [0, b1), pass two (if b2 > 0) on bits [b1, b1 + b2) within
 * each pass-one partition.  Partition p = d1 * 2^b2 + d2 is rows
 * [offsets[p], offsets[p+1]) of `out_tuples`; the order of tuples inside a
 * partition is unspecified.  b1 in [1, 12], b2 in [0, 12].
 * `out_tuples->tuples` and `*out_offsets` (2^(b1+b2) + 1 uint64 entries) are
 * library-owned device buffers; release them with hj_partition_free. */
hj_status hj_partition(hj_ctx *ctx, const hj_rel *in, int b1, int b2, hj_rel *out_tuples,
                       uint64_t **out_offsets);
hj_status hj_partition_free(hj_ctx *ctx, hj_rel *tuples, uint64_t *offsets);

/* The whole join: SHJ or PHJ (opts->algo, HJ_ALGO_AUTO lets the tuner pick), with
 * partitioning, per-partition build and probe, and output.  `out` as for hj_probe. */
hj_status hj_join(hj_ctx *ctx, const hj_rel *R, const hj_rel *S, const hj_opts *opts,
                  hj_result *out);

/* Many independent joins: outs[j] receives the join of Rs[j] and Ss[j] exactly as
 * hj_join would return it (count, checksums, library-owned pairs).  All relations
 * share one width; each must have fewer than 2^32 - 1 tuples.  Joins are grouped
 * by the radix bits their build side needs; every group is partitioned in one
 * pass per relation side and all (join, partition) pairs of all groups are joined
 * by ONE persistent launch that takes them from a work counter, so small and large
 * joins share the GPU.  If the joins' workspace exceeds the HBM budget (the
 * context's, else 70% of free device memory) they run in several such waves.
 * opts->flags & HJ_FLAG_GRAPH captures each wave's device work in a CUDA graph and
 * launches it as one.  opts->algo, radix_bits and passes are ignored. */
hj_status hj_join_batch(hj_ctx *ctx, int n, const hj_rel *Rs, const hj_rel *Ss, const hj_opts *opts,
                        hj_result *outs);

/* ------------------------------------------------------------ plan choice
 * hj_join with HJ_ALGO_AUTO (and radix_bits, passes left 0) picks SHJ or PHJ, the
 * radix bits and the pass count from a cost model of the GPU-only join: the
 * paper's T = sum over steps of computation + memory time (Sec. 4, Eq. 1-2, with
 * every step on the GPU so that the pipeline delay is zero), where a step's memory
 * time is the bytes it must move over the HBM bandwidth and its computation time
 * its per-item instruction count over the SMs' issue rate; a step costs the larger
 * of the two.  hj_tune refines the choice on the device. */
typedef struct hj_plan_info {
    int32_t algo;        /* HJ_ALGO_SHJ or HJ_ALGO_PHJ                               */
    int32_t radix_bits;  /* PHJ: total radix bits                                    */
    int32_t passes;      /* PHJ: partition passes                                    */
    int32_t reserved;
    double predicted_ms; /* the model's time for the whole join                      */
    double step_ms[4];   /* PHJ: histogram, scatter, join, 0; SHJ: 0, 0, build, probe */
    double measured_ms;  /* hj_tune: best measured time (-1 from hj_plan)            */
} hj_plan_info;

/* The plan hj_join would run for R and S under `opts` (forced fields honoured).
 * With ctx NULL the model uses GB300's figures and no tuned plan; no GPU work is
 * done either way.  R and S are only read for their sizes and width. */
hj_status hj_plan(hj_ctx *ctx, const hj_rel *R, const hj_rel *S, const hj_opts *opts, hj_plan_info *out);

/* Time the model's `top_k` cheapest plans (0: 4) on R and S (each run once to warm
 * up and twice timed, in opts->mode) and remember the fastest for their size class
 * (width, count or pair mode, floor(log2) of |R| + 1 and of |S| + 1) on this
 * context: later hj_join calls with HJ_ALGO_AUTO in that class run it.  `out`
 * (NULL allowed) receives the chosen plan with its predicted and measured time. */
hj_status hj_tune(hj_ctx *ctx, const hj_rel *R, const hj_rel *S, const hj_opts *opts, int top_k, hj_plan_info *out);

/* Forget every tuned plan of the context. */
hj_status hj_tune_clear(hj_ctx *ctx);

/* End-to-end join on HOST buffers: copies R and S from host memory (page-locked
 * memory gives full link speed; pageable works) to device buffers the library
 * allocates, runs hj_join, and copies the pairs into `pairs_host` (room for
 * `pairs_host_cap` pairs of 2 * width bytes; may be NULL in the count modes).
 * `out->pairs` is NULL on return: nothing stays on the device.  If the join has
 * more pairs than `pairs_host_cap`, the first pairs_host_cap are copied and
 * HJ_E_OVERFLOW is returned with out->count set to the full count. */
hj_status hj_join_host(hj_ctx *ctx, const hj_rel *R_host, const hj_rel *S_host, const hj_opts *opts,
                       void *pairs_host, uint64_t pairs_host_cap, hj_result *out);

/* Join of relations in HOST memory that need not fit the device.  When R,
 * partitioned, fits `device_bytes` beside two S chunks of at least 2^20 tuples in
 * flight (and R's partitions fit shared memory after one pass), R is copied and
 * partitioned once and S streamed past it in chunks, as hj_join_host does
 * (out->passes = 1, out->radix_bits = the PHJ's bits).  Otherwise the paper's
 * larger-than-buffer join (App. A; out->passes = 0): each relation is streamed
 * to the device in chunks, split there on hash bits [20, 20 + bt) (bt <= 8,
 * chosen so that every partition pair of a uniform split fits) and copied back
 * into page-locked host partitions; then every partition pair is gathered onto
 * the device and joined by the PHJ (whose digits use hash bits below 20), its
 * pairs copied into `pairs_host`.  A pair whose S side is too large next to its R
 * partition (skew) is joined in S groups.  The device memory used is sized to
 * `device_bytes` (0: 40% of free memory); when everything fits at once this is
 * hj_join_host.  `out` receives count and checksums (out->radix_bits = bt for the
 * split, out->pairs = NULL); the
 * pairs land in `pairs_host` (room for pairs_host_cap pairs; HJ_E_OVERFLOW with
 * the full count if too small).  HJ_E_INVALID if device_bytes is below twice
 * the fixed workspace of one join (64 MiB, plus 2^20 pairs when materialising);
 * HJ_E_NOMEM if a partition of R with an S group of 2^16 tuples exceeds it.  Host
 * memory: one page-locked copy of R and of S, kept by the context for later calls
 * (released by hj_destroy). */
hj_status hj_join_host_large(hj_ctx *ctx, const hj_rel *R_host, const hj_rel *S_host, const hj_opts *opts,
                             uint64_t device_bytes, void *pairs_host, uint64_t pairs_host_cap, hj_result *out);

/* Release a result's pairs (no-op for the count modes) and zero the struct. */
hj_status hj_result_free(hj_ctx *ctx, hj_result *res);

/* Simple hash join that allocates nothing.  (The paper has no counterpart: this
 * entry exists for callers that may not allocate device memory -- for example a
 * host process whose device memory is owned by another allocator that reserves
 * it all, or a latency-critical or certified loop that forbids allocation after
 * start-up.)  It needs no context: it runs on the current device and on
 * `cuda_stream` (NULL: the default stream), and returns when the join is done.
 * The caller provides R, S (device, 16-byte aligned, same width) and the pair
 * buffer `pairs` (device, room for `pairs_cap` pairs of 2 * width bytes; may be
 * NULL when pairs_cap is 0).  *count receives the number of pairs; checksum
 * (NULL allowed) receives c0, c1 as in HJ_COUNT_CHECKSUM; the pairs are written
 * densely in no particular order.  Returns HJ_E_OVERFLOW, with *count set, if
 * the join has more than pairs_cap pairs (the first pairs_cap are written).  Its
 * table keeps one slot per build tuple, so a build key repeated so often that an
 * insert walks past 65536 slots makes the call return HJ_E_UNSUPPORTED (nothing
 * useful in *count or the pairs): hj_join handles such relations.
 *
 * Its scratch -- counters and the hash table -- is one file-scope device array of
 * HJ_STATIC_SCRATCH_BYTES bytes in the library, which every GPU that loads the
 * library holds until the process exits.  The table needs 2 * width bytes for
 * each of the next power of two at least 2|R| + 1 slots, so |R| may be at most
 * 2097151 tuples for HJ_U32 and 1048575 for HJ_U64; a larger R is rejected with
 * HJ_E_NOMEM before any work is queued.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call reuses the same
 * array, so calls whose work overlaps on the GPU (other streams, other threads)
 * race and corrupt each other's results: serialise them. */
#define HJ_STATIC_SCRATCH_BYTES (64ull << 20)
hj_status hj_join_static(const hj_rel *R, const hj_rel *S, void *cuda_stream, void *pairs, uint64_t pairs_cap,
                         uint64_t *count, uint64_t *checksum);

/* ------------------------------------------------------------------ serving
 * A request loop over the join (the paper has no serving layer: it joins one R
 * and one S at a time, Sec. 3.1).  Clients submit joins of any size from any
 * thread; the server admits them in FIFO order against an HBM budget, groups the
 * admitted ones into waves (one hj_join_batch launch sequence per wave, or hj_join
 * for a wave of one) and runs up to `workers` waves at once, each on its own CUDA
 * stream.  Requests that arrive while waves run are admitted as soon as a worker
 * and budget are free (continuous batching); their work overlaps the running
 * waves on the device.  Every result is exactly what hj_join returns for the same
 * R, S and mode (count, checksums, the pair multiset), whatever it was batched
 * with.
 *
 * Budget: a request reserves an estimate of its join workspace (partitioned R
 * and S, pair buffer) from admission to completion; afterwards its pairs stay
 * charged until hj_server_result_free.  A request whose estimate exceeds the whole
 * budget is refused at submission (HJ_E_NOMEM).  All worker streams allocate from
 * one memory pool owned by the server. */
typedef struct hj_server hj_server;

typedef struct hj_server_opts {
    uint64_t budget_bytes; /* HBM admission budget (0: min(120 GiB, 60% of free memory)) */
    int32_t workers;       /* waves in flight at once, one stream each (0: 4; at most 16) */
    int32_t max_wave;      /* most requests in one wave (0: 512)                       */
    uint64_t wave_tuples;  /* a wave stops growing past this many tuples of R and S;
                              a request above it runs alone (0: 2^26)                 */
    uint64_t flags;        /* HJ_FLAG_GRAPH: waves of several joins run as a CUDA graph */
} hj_server_opts;

/* Host clock (seconds since hj_server_create, steady clock) of a request's steps. */
typedef struct hj_req_times {
    double submit; /* hj_server_submit accepted it                          */
    double admit;  /* its workspace was reserved and it joined a wave       */
    double start;  /* its wave's work began                                 */
    double done;   /* its result was complete on the device and read back   */
} hj_req_times;

typedef struct hj_server_stats {
    uint64_t submitted, completed, waves, wave_max, queued;
    uint64_t in_use, peak_in_use, budget; /* bytes charged now / at most / allowed */
    uint64_t launches;                    /* kernels the workers have launched       */
} hj_server_stats;

/* Start a server on ctx's device with its own worker threads, streams and memory
 * pool (ctx is only consulted for the device and error text). */
hj_status hj_server_create(hj_server **srv, hj_ctx *ctx, const hj_server_opts *opts);

/* Queue the join of R and S (device pointers, same width, 16-byte aligned, fewer
 * than 2^32 - 1 tuples each) in `mode` (HJ_COUNT, HJ_COUNT_CHECKSUM,
 * HJ_MATERIALIZE).  The workers run on streams of their own: R and S must be
 * completely written when this is called (synchronise the stream that produced
 * them), and must stay valid and unchanged until the request is collected.
 * *req_id identifies it for hj_server_poll / hj_server_wait. */
hj_status hj_server_submit(hj_server *srv, const hj_rel *R, const hj_rel *S, int32_t mode, uint64_t *req_id);

/* HJ_E_PENDING while the request runs.  Once done, returns the request's own
 * status, moves its result into *out (NULL: the pairs are released at once) and
 * its times into *t (NULL allowed), and forgets the request. */
hj_status hj_server_poll(hj_server *srv, uint64_t req_id, hj_result *out, hj_req_times *t);

/* As hj_server_poll, but blocks until the request is done or `timeout_s` seconds
 * pass (HJ_E_PENDING; a negative timeout waits for ever). */
hj_status hj_server_wait(hj_server *srv, uint64_t req_id, double timeout_s, hj_result *out, hj_req_times *t);

/* Release the pairs of a result collected from this server (and their budget). */
hj_status hj_server_result_free(hj_server *srv, hj_result *res);

hj_status hj_server_stats_get(hj_server *srv, hj_server_stats *st);
const char *hj_server_last_error(const hj_server *srv);

/* Run every queued request to completion, stop the workers and free everything,
 * including pairs of results not yet released (their pointers become invalid). */
hj_status hj_server_destroy(hj_server *srv);

/* Wait for all work queued on the context's stream. */
hj_status hj_sync(hj_ctx *ctx);

/* Copy `bytes` between any two host or device buffers (cudaMemcpyDefault
 * semantics), ordered on the context's stream; returns after the copy is done.
 * Used to read library-owned results (pairs, offsets) into caller memory. */
hj_status hj_copy(hj_ctx *ctx, void *dst, const void *src, uint64_t bytes);

/* Pipelined CPU/GPU co-processing cost model (PL, Sec. 3.2 and Sec. 4, Eq. 1-5) as
 * host arithmetic; no device is touched.  A series of n (1..16) steps: step i has
 * x[i] items, of which the share r_i runs on the CPU at cpu_s[i] seconds per item
 * and the rest on the GPU at gpu_s[i] seconds per item (computation and memory
 * stalls, Eq. 2-3); intermediate items between steps of different ratios,
 * |r_i - r_(i-1)| x_i, cost xfer_s seconds each on the receiving processor; the
 * pipeline delays are Eq. 4 (r_i > r_(i-1)) and Eq. 5 (r_i < r_(i-1)), clamped at
 * 0, with the running sums taken without the delay being computed.  The elapsed
 * time is T = max(T_CPU, T_GPU) (Eq. 1).
 * hj_coproc_time: T for the given ratios (each in [0, 1]); t_cpu and t_gpu (NULL
 * allowed) receive T_CPU and T_GPU.
 * hj_coproc_ratios: the ratios minimising T over r_i in {0, delta, 2 delta, ...,
 * 1} for every step (the paper's exhaustive search; it uses delta = 0.02), and
 * that T; ties go to smaller CPU shares.  HJ_E_INVALID for bad arguments (negative
 * sizes or costs, delta outside (0, 1]); HJ_E_UNSUPPORTED when the grid^n search
 * would exceed 10^9 ratio vectors. */
hj_status hj_coproc_time(int n, const double *x, const double *cpu_s, const double *gpu_s, double xfer_s,
                         const double *ratios, double *t_out, double *t_cpu, double *t_gpu);
hj_status hj_coproc_ratios(int n, const double *x, const double *cpu_s, const double *gpu_s, double xfer_s,
                           double delta, double *ratios_out, double *t_out);

/* Per-kernel timing on the context's stream.  While enabled, every kernel launch
 * is bracketed by CUDA events; hj_prof_read synchronises, then reports, for up to
 * `cap` distinct kernel names, the name (NUL-terminated, at most 47 chars), the
 * number of launches and the summed device milliseconds, and returns how many
 * names exist in *n_out.  hj_prof_reset clears the record.  hj_launch_count returns
 * the number of kernels this context has launched since creation. */
typedef struct hj_prof_entry {
    char name[48];
    uint64_t launches;
    double ms;
} hj_prof_entry;
hj_status hj_prof_enable(hj_ctx *ctx, int on);
/* Restrict the event brackets to launches of the kernel named `name` (as reported
 * by hj_prof_read); NULL or "" brackets every launch again.  Timing one kernel
 * costs two event records per launch of it and nothing for the others.  Copies
 * the name; HJ_E_INVALID for a NULL context or a name of 48 chars or more. */
hj_status hj_prof_only(hj_ctx *ctx, const char *name);
hj_status hj_prof_reset(hj_ctx *ctx);
hj_status hj_prof_read(hj_ctx *ctx, hj_prof_entry *entries, int cap, int *n_out);
uint64_t hj_launch_count(const hj_ctx *ctx);

/* ------------------------------------------------------ CPU/GPU co-processing
 * The PHJ with its join step divided between the GPU and the host CPU: the
 * paper's data dividing (DD, Sec. 3.2) applied to the join step, whose share the
 * cost model (Sec. 4, Eq. 1-5; hj_coproc_time / hj_coproc_ratios) prices.  The GPU
 * partitions R and S (Alg. 2); the partition pairs holding the first `cpu_share`
 * of S's rows are copied to page-locked host memory (kept on the context) and
 * joined by `cpu_threads` host threads (0: one per host core) while the GPU joins
 * the other pairs.  The result is what hj_join returns -- count, checksums, and in
 * HJ_MATERIALIZE the pairs in one library-owned device buffer (the CPU's after the
 * GPU's) -- for the PHJ plan hj_join would pick (or opts' radix bits and passes).
 * cpu_share in [0, 1]: 0 is the GPU join alone, 1 every partition on the CPU.
 * times (optional, 5 doubles, seconds measured in this call): GPU partitioning,
 * GPU join, copy of the CPU's share to the host, CPU join, the whole call.
 * Synchronises the context's stream.  HJ_E_INVALID for an SHJ algo, a share
 * outside [0, 1] or cpu_threads < 0. */
hj_status hj_join_coproc(hj_ctx *ctx, const hj_rel *R, const hj_rel *S, const hj_opts *opts, double cpu_share,
                         int cpu_threads, hj_result *out, double *times);

/* ---------------------------------------------------------------- sharding
 * The local step of one join sharded over several GPUs (the partitioning of
 * Alg. 2 applied across GPUs, Sec. 3.1): every GPU splits its slices of R and S
 * into `nparts` groups, group g of every GPU goes to GPU g (one all-to-all by the
 * caller's collective library), and each GPU joins what it received -- equal keys
 * meet on one GPU, so the local joins together are the whole join.
 * hj_split writes the n tuples of `in` to `out` (device, caller-owned, room for
 * in->n tuples of in's width, 16-byte aligned, not overlapping `in`) grouped by
 * group = (high 32 bits of the SplitMix64 finaliser of the key) * nparts >> 32, a
 * hash that no local join uses (their digits and buckets come from MurmurHash2
 * and from a Fibonacci multiply), so a GPU's keys still spread over all of its
 * digits and buckets.  Group g is rows [offsets[g], offsets[g+1]) of `out`;
 * `offsets` is a HOST array of nparts + 1 entries, filled before the call returns
 * (it synchronises the context's stream).  Order inside a group is unspecified.
 * nparts in [1, 4096]; HJ_E_INVALID otherwise or for bad pointers. */
hj_status hj_split(hj_ctx *ctx, const hj_rel *in, int nparts, void *out, uint64_t *offsets);

/* Host-side fault injection for tests (no GPU fault is involved):
 * hj_debug_fail_alloc makes the n-th device allocation from now fail with
 * HJ_E_NOMEM (n < 0 disarms); hj_debug_bytes_in_use reports the device bytes the
 * context currently holds (0 after every buffer has been released). */
hj_status hj_debug_fail_alloc(hj_ctx *ctx, int64_t n);
uint64_t hj_debug_bytes_in_use(const hj_ctx *ctx);
/* Test hook for the bounded device waits (the paper has no counterpart): the
 * ring partition scatter (2^9 .. 2^11 digits) runs flush warps that wait
 * on the CTA's insert warps; after n passes (default 2^22; n = 0 restores both
 * defaults) they give up, set a sticky fault bit and return.  The TMA-staged
 * scatter of unpadded passes (hj_partition and the host-memory split, fan-out
 * <= 2^11) polls the mbarrier of each staged tile at most n - 1 times (default
 * 2^26; so n = 1 gives up at the first wait): a CTA that gives up sets the same
 * bit, waits for its copy in flight to land and returns.  The call that reads the
 * counters next returns HJ_E_TIMEOUT (its results are then undefined).  The fault
 * is reported once; later calls on the context run normally.  Only the limits
 * change: no GPU fault is involved.  HJ_E_INVALID for a NULL context. */
hj_status hj_debug_wait_limit(hj_ctx *ctx, uint64_t n);
/* Test and measurement hook: which kernel scatters a padded partition pass at
 * 2^9 .. 2^11 digits.  HJ_SCATTER_AUTO (the default) takes the ring scatter where
 * it measured faster than the region scatter (4-byte tuples at 2^10 and 2^11
 * digits, 8-byte tuples at 2^9 .. 2^11) and the region scatter elsewhere; HJ_SCATTER_REGION and HJ_SCATTER_RING force one
 * (other fan-outs always take the region scatter).  Results are identical either
 * way; only the kernel changes.  HJ_E_INVALID for a NULL context or another
 * value. */
#define HJ_SCATTER_AUTO 0
#define HJ_SCATTER_REGION 1
#define HJ_SCATTER_RING 2
hj_status hj_debug_scatter(hj_ctx *ctx, int kind);
/* Test and measurement hook: hj_join_host_large's plan.  HJ_OUTCORE_AUTO (the
 * default) keeps R on the device and streams S past it when that fits
 * device_bytes, else splits both relations (App. A); HJ_OUTCORE_SPLIT always
 * splits.  Results are identical either way.  HJ_E_INVALID for a NULL context or
 * another value. */
#define HJ_OUTCORE_AUTO 0
#define HJ_OUTCORE_SPLIT 1
hj_status hj_debug_outcore(hj_ctx *ctx, int mode);
/* Test hook: the most device bytes the context held at once (its own buffers, as
 * hj_debug_bytes_in_use counts them) since it was created or since the last call
 * with reset != 0, which then restarts the count from the bytes held now.  0 for
 * a NULL context. */
uint64_t hj_debug_peak_bytes(hj_ctx *ctx, int reset);

#ifdef __cplusplus
}
#endif

#endif /* HJ_H */
