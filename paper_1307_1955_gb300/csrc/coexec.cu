// coexec.cu -- the CPU side of co-processing: host threads join partition pairs.
//
// In the paper's data dividing (DD, Sec. 3.2) a step's items are shared between
// the CPU and the GPU by a ratio.  hj_join_coproc (api.cu) applies it to the join
// step of the PHJ: the GPU partitions R and S, then the partition pairs that hold
// the first share of S's rows are copied to page-locked host memory and joined
// here by host threads while the GPU joins the rest.  A thread takes one partition
// pair at a time from a shared counter and runs Alg. 1 on it with the table of
// Sec. 3.1: a key list (open addressing, one slot per distinct key, linear
// probing) whose slots head rid lists (the R rows of that key, linked), built over
// the pair's R rows; then one lookup per S row, every rid of the key's list
// appended as a pair (rid_R, rid_S).  Repeated build keys cost one list step each.
// Padding rows of the partitioned copies carry keys of another partition: they
// are skipped when the table is built (their digit is checked with the same
// MurmurHash2 the GPU partitioned by) and can match nothing when it is probed.
// Count and the two checksums (SplitMix64 finaliser A of rid_R times / plus
// A(rid_S ^ golden), summed modulo 2^64) are those of the library's GPU joins.
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "engine.cuh"

namespace hj {
namespace {

inline uint64_t host_fin(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Partition index of a key under pass bits (b1, b2): the GPU's PartFilter formula.
inline uint32_t host_part(uint64_t h, int b1, int b2) {
    const uint32_t h32 = (uint32_t)h, m1 = (1u << b1) - 1u, m2 = b2 ? (1u << b2) - 1u : 0u;
    return ((h32 & m1) << b2) | ((h32 >> b1) & m2);
}

template <int W> struct HostTup { using U = uint32_t; };
template <> struct HostTup<8> { using U = uint64_t; };

// Per-thread scratch of the table: Sec. 3.1's key list and rid lists, as arrays.
template <int W> struct HostTable {
    using U = typename HostTup<W>::U;
    std::vector<U> keys;        // distinct key of a slot
    std::vector<int64_t> head;  // first R row of the slot's key (-1: empty slot)
    std::vector<int64_t> next;  // next R row with the same key (-1: the list ends)
};

template <int W>
void join_one(const typename HostTup<W>::U *R, uint64_t nr, const typename HostTup<W>::U *S, uint64_t ns, uint32_t p,
              int b1, int b2, bool mat, bool chk, HostTable<W> &t, CpuJoinPart *acc,
              std::vector<typename HostTup<W>::U> &pairs) {
    using U = typename HostTup<W>::U;
    if (!nr || !ns) return;
    int lg = 4;
    while ((1ull << lg) < 2 * nr) ++lg;
    const uint64_t cap = 1ull << lg, mask = cap - 1;
    t.keys.resize(cap);
    t.head.assign(cap, -1);
    t.next.resize(nr);
    auto home = [&](U k) { return (uint64_t)(((uint64_t)k * 0x9E3779B97F4A7C15ull) >> (64 - lg)); };
    // build: one slot per distinct key, its rows linked in a list
    for (uint64_t i = 0; i < nr; ++i) {
        const U k = R[2 * i];
        const uint64_t h = W == 4 ? (uint64_t)murmur2_u32((uint32_t)k) : murmur2_u64((uint64_t)k);
        if (host_part(h, b1, b2) != p) continue;  // padding row
        uint64_t s = home(k);
        while (t.head[s] >= 0 && t.keys[s] != k) s = (s + 1) & mask;
        if (t.head[s] < 0) t.keys[s] = k;
        t.next[i] = t.head[s];
        t.head[s] = (int64_t)i;
    }
    // probe: the slot of the key, then its list
    for (uint64_t i = 0; i < ns; ++i) {
        const U k = S[2 * i], rs = S[2 * i + 1];
        uint64_t s = home(k);
        while (t.head[s] >= 0 && t.keys[s] != k) s = (s + 1) & mask;
        if (t.head[s] < 0) continue;
        const uint64_t bs = chk ? host_fin((uint64_t)rs ^ 0x9E3779B97F4A7C15ull) : 0;
        for (int64_t j = t.head[s]; j >= 0; j = t.next[j]) {
            const U rr = R[2 * j + 1];
            acc->count++;
            if (chk) {
                const uint64_t a = host_fin((uint64_t)rr);
                acc->c0 += a * bs;
                acc->c1 += a + bs;
            }
            if (mat) {
                pairs.push_back(rr);
                pairs.push_back(rs);
            }
        }
    }
}

}  // namespace

// Host worker threads kept on a context: run(n, f) calls f(0) .. f(n - 1) on the
// calling thread and n - 1 workers and returns when all are done.  Workers sleep
// on a condition variable between jobs, so a co-processing call pays no thread
// creation.
struct CpuPool {
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable wake, done;
    std::function<void(int)> job;
    uint64_t gen = 0;       // job generation; a worker runs each generation once
    int want = 0, left = 0;  // workers the job uses, workers still running it
    bool stop = false;

    void loop(int id) {
        uint64_t seen = 0;
        for (;;) {
            std::function<void(int)> f;
            {
                std::unique_lock<std::mutex> lk(mu);
                wake.wait(lk, [&] { return stop || gen != seen; });
                if (stop) return;
                seen = gen;
                if (id >= want) continue;  // not needed this time
                f = job;
            }
            f(id + 1);
            std::lock_guard<std::mutex> lk(mu);
            if (--left == 0) done.notify_all();
        }
    }
    void run(int n, const std::function<void(int)> &f) {
        while ((int)workers.size() < n - 1) {
            const int id = (int)workers.size();
            workers.emplace_back([this, id] { loop(id); });
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            job = f;
            want = n - 1;
            left = n - 1;
            ++gen;
        }
        wake.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(mu);
        done.wait(lk, [&] { return left == 0; });
    }
    ~CpuPool() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        wake.notify_all();
        for (auto &t : workers) t.join();
    }
};

CpuPool *cpu_pool_new() { return new CpuPool(); }
void cpu_pool_delete(CpuPool *p) { delete p; }

namespace {

template <int W>
void run_threads(CpuPool *pool, const void *R, const uint64_t *roff, const void *S, const uint64_t *soff, uint32_t np,
                 int b1, int b2, bool mat, bool chk, int threads, CpuJoinResult *out) {
    using U = typename HostTup<W>::U;
    std::atomic<uint32_t> next{0};
    out->parts.assign(threads, CpuJoinPart{});
    out->pairs.assign(threads, std::vector<uint8_t>());
    auto work = [&](int t) {
        HostTable<W> tab;
        std::vector<U> pairs;
        CpuJoinPart acc{};
        for (uint32_t p = next++; p < np; p = next++) {
            const U *r = (const U *)R + 2 * (roff[p] - roff[0]);
            const U *s = (const U *)S + 2 * (soff[p] - soff[0]);
            join_one<W>(r, roff[p + 1] - roff[p], s, soff[p + 1] - soff[p], p, b1, b2, mat, chk, tab, &acc, pairs);
        }
        out->parts[t] = acc;
        out->pairs[t].resize(pairs.size() * sizeof(U));
        if (!pairs.empty()) memcpy(out->pairs[t].data(), pairs.data(), pairs.size() * sizeof(U));
    };
    pool->run(threads, work);
}

}  // namespace

void cpu_join_partitions(CpuPool *pool, int width, const void *R, const uint64_t *roff, const void *S,
                         const uint64_t *soff, uint32_t np, int b1, int b2, bool mat, bool chk, int threads,
                         CpuJoinResult *out) {
    if (threads < 1) threads = 1;
    if ((uint32_t)threads > np) threads = np ? (int)np : 1;  // no more threads than partition pairs
    if (width == 4) run_threads<4>(pool, R, roff, S, soff, np, b1, b2, mat, chk, threads, out);
    else run_threads<8>(pool, R, roff, S, soff, np, b1, b2, mat, chk, threads, out);
    out->count = out->c0 = out->c1 = 0;
    for (const auto &q : out->parts) {
        out->count += q.count;
        out->c0 += q.c0;
        out->c1 += q.c1;
    }
}

}  // namespace hj
