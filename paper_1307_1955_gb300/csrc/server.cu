// server.cu -- the serving loop (hj_server_*): join requests of any size arrive
// one by one, are admitted against an HBM budget, grouped into waves and run on
// several CUDA streams at once.  The paper has no serving layer; this is the
// request-level form of its data-parallel join: continuous batching of whole joins.
//
//   client threads --submit--> FIFO queue --admit (budget)--> wave --> worker w
//                                                                      (own stream,
//   client threads <--poll/wait-- results (+ times) <--done-- hj_join / hj_join_batch)
//
// Each of the `workers` host threads owns a context (stream) of its own; all of
// them allocate from one memory pool that the server owns, so the device memory
// the server holds is bounded by what its admitted requests use, not by the sum of
// per-worker high-water marks.  A worker that is free takes every queued request
// that fits the remaining budget (FIFO, same width and mode as the queue head, up
// to `max_wave` requests and `wave_tuples` tuples) and runs them as one batched
// join (or alone, with hj_join, if it is a single request).  Requests that arrive
// while other waves are on the GPU are therefore admitted as soon as a worker and
// budget are free, and their work overlaps the running waves on the device.
//
// Budget: a request reserves its join workspace (partitioned copies of R and S,
// the pair buffer) when admitted; after it finishes it keeps only its pairs, which
// stay charged until the client releases them with hj_server_result_free.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.cuh"
#include "engine.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued = 0, kAdmitted, kRunning, kDone };

struct Req {
    hj_rel R{}, S{};
    int32_t mode = HJ_MATERIALIZE;
    uint64_t need = 0;     // bytes reserved while admitted or running
    uint64_t held = 0;     // bytes of its pairs, charged from completion until released
    ReqState state = kQueued;
    hj_status status = HJ_OK;
    hj_result res{};
    int worker = -1;
    hj_req_times t{};
};

// Workspace of one join while it runs: partitioned copies of R and S (padding
// included) and, when materialising, a pair buffer of |S| pairs (a larger result
// is re-run at its exact size inside the join).
uint64_t join_need(const hj_rel &R, const hj_rel &S, int mode) {
    const uint64_t tb = 2ull * (uint64_t)R.width;
    uint64_t b = (R.n + S.n) * tb * 11 / 10 + (16ull << 20);
    if (mode == HJ_MATERIALIZE) b += (S.n + 65536) * tb;
    return b;
}

}  // namespace

struct hj_server {
    int device = 0;
    hj_server_opts opts{};
    cudaMemPool_t pool = nullptr;
    std::vector<hj_ctx *> ctxs;
    std::vector<std::thread> threads;
    std::vector<std::vector<void *>> to_free;  // per worker: pairs released by clients
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    std::unordered_map<void *, int> pair_owner;
    uint64_t next_id = 1;
    uint64_t in_use = 0, peak = 0;
    uint64_t submitted = 0, completed = 0, waves = 0, wave_max = 0;
    int running = 0;  // waves on the GPU
    bool stop = false;
    Clock::time_point epoch;
    std::string err;

    double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }
    void charge(uint64_t b) {
        in_use += b;
        if (in_use > peak) peak = in_use;
    }
    void worker_loop(int w);
    // Take the wave worker w runs next; mu held.  Empty when nothing fits.
    std::vector<uint64_t> take_wave();
};

std::vector<uint64_t> hj_server::take_wave() {
    std::vector<uint64_t> wave;
    if (queue.empty()) return wave;
    const Req &head = reqs[queue.front()];
    const int width = head.R.width, mode = head.mode;
    uint64_t tuples = 0;
    for (auto it = queue.begin(); it != queue.end() && (int)wave.size() < opts.max_wave;) {
        Req &r = reqs[*it];
        if (r.R.width != width || r.mode != mode) break;  // keep FIFO order across kinds
        const uint64_t t = r.R.n + r.S.n;
        if (!wave.empty() && tuples + t > opts.wave_tuples) break;
        if (in_use + r.need > opts.budget_bytes) break;
        charge(r.need);
        r.state = kAdmitted;
        r.t.admit = now();
        tuples += t;
        wave.push_back(*it);
        it = queue.erase(it);
    }
    return wave;
}

void hj_server::worker_loop(int w) {
    hj_ctx *c = ctxs[w];
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_work.wait(lk, [&] {
            if (!to_free[w].empty() || stop) return true;
            if (queue.empty()) return false;
            const Req &h = reqs[queue.front()];
            return in_use + h.need <= opts.budget_bytes;
        });
        // pairs released by clients: freed on this worker's context, which owns them
        std::vector<void *> frees;
        frees.swap(to_free[w]);
        std::vector<uint64_t> wave = take_wave();
        if (wave.empty() && frees.empty() && stop) {
            if (queue.empty()) break;
            if (running == 0) {
                // shutting down with queued requests that can never be admitted (the
                // budget is held by results nobody releases now): fail them
                for (uint64_t id : queue) {
                    Req &r = reqs[id];
                    r.status = HJ_E_NOMEM;
                    r.state = kDone;
                    completed++;
                }
                queue.clear();
                cv_done.notify_all();
                break;
            }
            cv_work.wait(lk);  // a running wave will return budget
            continue;
        }
        // requests' relations are copied out under the lock
        std::vector<hj_rel> Rs, Ss;
        int32_t mode = HJ_MATERIALIZE;
        for (uint64_t id : wave) {
            Req &r = reqs[id];
            r.state = kRunning;
            r.worker = w;
            Rs.push_back(r.R);
            Ss.push_back(r.S);
            mode = r.mode;
        }
        if (!wave.empty()) {
            waves++;
            running++;
            if (wave.size() > wave_max) wave_max = wave.size();
        }
        lk.unlock();
        for (void *p : frees) hj::dfree(c, p);
        std::vector<hj_result> outs(wave.size());
        hj_status st = HJ_OK;
        std::string why;
        const double t_start = now();
        if (!wave.empty()) {
            hj_opts o{};
            o.algo = HJ_ALGO_AUTO;
            o.mode = mode;
            o.flags = opts.flags & HJ_FLAG_GRAPH;
            if (wave.size() == 1) {
                o.flags = 0;
                st = hj_join(c, &Rs[0], &Ss[0], &o, &outs[0]);
            } else {
                st = hj_join_batch(c, (int)wave.size(), Rs.data(), Ss.data(), &o, outs.data());
            }
            if (st != HJ_OK) why = c->err;
        }
        const double t_done = now();
        lk.lock();
        for (size_t i = 0; i < wave.size(); ++i) {
            Req &r = reqs[wave[i]];
            r.t.start = t_start;
            r.t.done = t_done;
            r.status = st;
            in_use -= r.need;
            r.need = 0;
            if (st == HJ_OK) {
                r.res = outs[i];
                if (r.res.pairs) {
                    r.held = r.res.pairs_cap * 2ull * (uint64_t)r.res.width;
                    charge(r.held);
                    pair_owner[r.res.pairs] = w;
                }
            }
            r.state = kDone;
            completed++;
        }
        if (st != HJ_OK) err = why;
        if (!wave.empty()) running--;
        cv_done.notify_all();
        cv_work.notify_all();  // budget came back: other idle workers may now admit
    }
}

namespace {

hj_status srv_err(hj_server *s, hj_status code, const char *msg) {
    if (s) s->err = msg;
    return code;
}

// Move a finished request's result to the caller; mu held.
hj_status hand_over(hj_server *s, uint64_t id, Req &r, hj_result *out, hj_req_times *t) {
    if (t) *t = r.t;
    const hj_status st = r.status;
    if (out) {
        *out = st == HJ_OK ? r.res : hj_result{};
    } else if (r.res.pairs) {  // nobody takes the pairs: release them
        auto it = s->pair_owner.find(r.res.pairs);
        if (it != s->pair_owner.end()) {
            s->to_free[it->second].push_back(r.res.pairs);
            s->pair_owner.erase(it);
        }
        s->in_use -= r.held;
        s->cv_work.notify_all();
    }
    // pairs handed over stay charged until hj_server_result_free
    s->reqs.erase(id);
    return st;
}

}  // namespace

extern "C" {

hj_status hj_server_create(hj_server **out, hj_ctx *ctx, const hj_server_opts *opts) {
    if (!out || !ctx) return HJ_E_INVALID;
    *out = nullptr;
    hj_server_opts o{};
    if (opts) o = *opts;
    if (o.workers < 0 || o.workers > 16 || o.max_wave < 0) return hj::set_err(ctx, HJ_E_INVALID, "bad server options");
    if (o.workers == 0) o.workers = 4;  // measured: 3 -> 4 raised saturated throughput 4 %, 6 only 1 % more
    if (o.max_wave == 0) o.max_wave = 512;
    if (o.wave_tuples == 0) o.wave_tuples = 1ull << 26;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return hj::cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
    if (o.budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        o.budget_bytes = std::min<uint64_t>(120ull << 30, (uint64_t)(fr * 0.6));
    }
    hj_server *s = new hj_server();
    s->device = ctx->device;
    s->opts = o;
    s->epoch = Clock::now();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = o.budget_bytes;  // reuse freed blocks up to the budget
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) {
        int no = 0;  // no hidden cross-stream waits between workers
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    if (e != cudaSuccess) {
        hj_status st = hj::cuda_err(ctx, e, "server memory pool");
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return st;
    }
    for (int w = 0; w < o.workers; ++w) {
        hj_ctx *c = nullptr;
        hj_status st = hj::ctx_create(&c, ctx->device, nullptr, 0, s->pool);
        if (st != HJ_OK) {
            for (hj_ctx *x : s->ctxs) hj_destroy(x);
            cudaMemPoolDestroy(s->pool);
            delete s;
            return hj::set_err(ctx, st, "server worker context creation failed");
        }
        s->ctxs.push_back(c);
    }
    s->to_free.resize(o.workers);
    for (int w = 0; w < o.workers; ++w) s->threads.emplace_back([s, w] { s->worker_loop(w); });
    *out = s;
    return HJ_OK;
}

hj_status hj_server_submit(hj_server *s, const hj_rel *R, const hj_rel *S, int32_t mode, uint64_t *req_id) {
    if (!s || !R || !S || !req_id) return HJ_E_INVALID;
    if (R->width != HJ_U32 && R->width != HJ_U64) return srv_err(s, HJ_E_INVALID, "width is not 4 or 8");
    if (R->width != S->width) return srv_err(s, HJ_E_INVALID, "R and S widths differ");
    if (mode < HJ_COUNT || mode > HJ_MATERIALIZE) return srv_err(s, HJ_E_INVALID, "bad mode");
    for (const hj_rel *r : {R, S}) {
        if (r->n && (!r->tuples || ((uintptr_t)r->tuples & 15)))
            return srv_err(s, HJ_E_INVALID, "tuples NULL or not 16-byte aligned");
        if (r->n >= 0xFFFFFFFFull) return srv_err(s, HJ_E_INVALID, "a relation has 2^32 - 1 tuples or more");
    }
    Req r;
    r.R = *R;
    r.S = *S;
    r.mode = mode;
    r.need = join_need(*R, *S, mode);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return srv_err(s, HJ_E_INVALID, "server is shutting down");
    if (r.need > s->opts.budget_bytes) return srv_err(s, HJ_E_NOMEM, "request needs more than the whole budget");
    r.t.submit = s->now();
    const uint64_t id = s->next_id++;
    s->reqs.emplace(id, r);
    s->queue.push_back(id);
    s->submitted++;
    *req_id = id;
    s->cv_work.notify_one();
    return HJ_OK;
}

hj_status hj_server_poll(hj_server *s, uint64_t id, hj_result *out, hj_req_times *t) {
    if (!s) return HJ_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return srv_err(s, HJ_E_INVALID, "unknown or already collected request");
    if (it->second.state != kDone) return HJ_E_PENDING;
    return hand_over(s, id, it->second, out, t);
}

hj_status hj_server_wait(hj_server *s, uint64_t id, double timeout_s, hj_result *out, hj_req_times *t) {
    if (!s) return HJ_E_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->reqs.find(id);
        return it == s->reqs.end() || it->second.state == kDone;
    };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return HJ_E_PENDING;
    }
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return srv_err(s, HJ_E_INVALID, "unknown or already collected request");
    return hand_over(s, id, it->second, out, t);
}

hj_status hj_server_result_free(hj_server *s, hj_result *res) {
    if (!s || !res) return HJ_E_INVALID;
    if (res->pairs) {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->pair_owner.find(res->pairs);
        if (it == s->pair_owner.end()) return srv_err(s, HJ_E_INVALID, "pairs not owned by this server");
        s->to_free[it->second].push_back(res->pairs);
        s->pair_owner.erase(it);
        const uint64_t held = res->pairs_cap * 2ull * (uint64_t)res->width;
        s->in_use -= std::min(held, s->in_use);
        s->cv_work.notify_all();
    }
    *res = hj_result{};
    return HJ_OK;
}

hj_status hj_server_stats_get(hj_server *s, hj_server_stats *st) {
    if (!s || !st) return HJ_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->waves = s->waves;
    st->wave_max = s->wave_max;
    st->queued = s->queue.size();
    st->in_use = s->in_use;
    st->peak_in_use = s->peak;
    st->budget = s->opts.budget_bytes;
    st->launches = 0;
    for (hj_ctx *c : s->ctxs) st->launches += c->launches;  // read racily while waves run
    return HJ_OK;
}

const char *hj_server_last_error(const hj_server *s) { return s ? s->err.c_str() : "null server"; }

hj_status hj_server_destroy(hj_server *s) {
    if (!s) return HJ_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    // results nobody collected, and pairs released after the workers stopped
    for (auto &kv : s->reqs)
        if (kv.second.res.pairs) {
            auto it = s->pair_owner.find(kv.second.res.pairs);
            if (it != s->pair_owner.end()) s->to_free[it->second].push_back(kv.second.res.pairs);
        }
    for (size_t w = 0; w < s->ctxs.size(); ++w) {
        for (void *p : s->to_free[w]) hj::dfree(s->ctxs[w], p);
        hj_destroy(s->ctxs[w]);  // also frees pairs still handed out to clients
    }
    cudaMemPoolDestroy(s->pool);
    delete s;
    return HJ_OK;
}

}  // extern "C"
