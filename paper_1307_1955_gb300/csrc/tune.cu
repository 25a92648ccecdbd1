// tune.cu -- plan choice for hj_join (SHJ or PHJ, radix bits, passes): a cost model
// of the GPU-only join, and an on-device tuner that refines it.
//
// The paper's model (Sec. 4) prices a join as T = max(T_CPU, T_GPU) (Eq. 1) with
// T_XPU = sum over steps i of C_i + M_i + D_i (Eq. 2): computation C_i = #I_i x
// items / IPC (Eq. 3), memory stalls M_i, and the CPU/GPU pipeline delay D_i.  With
// every step on the GPU the ratio r is 0, T = T_GPU and D_i = 0.  Re-derived for
// GB300:
//   * M_i = bytes the step must move / HBM bandwidth (nominal from the device's
//     memory clock and bus width, times the fraction a plain copy reaches);
//   * C_i = items_i x thread instructions per item / issue rate (SMs x 4
//     schedulers x clock x 32 lanes x a sustained issue fraction).  As in the
//     paper's instantiation (Sec. 4.2, instruction counts from a profiler), the
//     per-item instruction counts are measured (ncu, smsp__inst_executed);
//   * a GPU overlaps the two within a kernel, so a step costs max(C_i, M_i), plus
//     a launch latency per kernel;
//   * the SHJ table's random accesses cost nothing extra while the table stays in
//     L2 and one sector per access from HBM once it does not (the "leap" of the
//     paper's end-to-end results once the table outgrows the cache, Sec. 5.5).
// hj_tune then times the model's best few plans on the caller's relations and
// caches the fastest for the relations' size class on the context; hj_join with
// HJ_ALGO_AUTO uses a cached plan when one exists, else the model's choice.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "engine.cuh"

namespace hj {

namespace {

// Effective thread instructions per item of each kernel at the sustained issue
// rate below: ncu's smsp__inst_executed x 32 / items, scaled so that the model's
// time equals the kernel's measured time on GB300 (4-byte tuples: the 2^24 x 2^28
// join at 11 radix bits -- scatter 1.302 ms, join 1.019 ms -- and the build-heavy
// 2^24 x 2^24 join -- join 0.229 ms, which with the first fixes the probe and build
// costs --, 12 bits in one and two passes, and SHJ at 2^20 and 2^24 build tuples).
// hj_tune measures the real thing on the caller's relations.
constexpr double kIptHist = 22.0;            // per input tuple (bandwidth-bound)
constexpr double kIptScatterRing = 101.0;    // per input tuple, ring scatter (2^10 and 2^11 digits)
constexpr double kIptScatterRegion = 131.0;  // per input tuple, region scatter at 2^8 and 2^9 digits
constexpr double kIptScatterRegionLow = 115.0;  // per input tuple, region scatter at <= 2^7 digits (measured per pass of 6 + 6 bits)
constexpr double kIptScatterWide = 293.0;    // per input tuple, fan-out 2^12
constexpr double kIptJoinProbe = 70.0;       // per S tuple, shared-memory table
constexpr double kIptJoinBuild = 232.0;      // per R tuple, shared-memory table (latency-bound build)
constexpr double kIptShjBuild = 40.0;     // per R tuple, global table
constexpr double kIptShjProbe = 60.0;     // per S tuple, global table
constexpr double kIssueFraction = 0.55;   // sustained share of the issue slots
constexpr double kCopyFraction = 0.83;    // share of nominal HBM bandwidth a copy reaches
constexpr double kRandomFraction = 0.2;   // share for 32-byte random sectors (table probes)
constexpr double kLaunchS = 4e-6;         // per kernel launch
constexpr double kShjFixedS = 55e-6;      // per SHJ call: table fill, allocations, one host synchronisation
constexpr double kPhjFixedS = 50e-6;      // per PHJ call: allocations, launch gaps, one host synchronisation

}  // namespace

CostModel cost_model_for(int device) {
    CostModel m;  // defaults: GB300
    int v = 0;
    if (device >= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && v > 0) m.sms = v;
        int clk = 0, mclk = 0, bus = 0, l2 = 0;
        if (cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device) == cudaSuccess && clk > 0)
            m.sm_hz = clk * 1e3;
        if (cudaDeviceGetAttribute(&mclk, cudaDevAttrMemoryClockRate, device) == cudaSuccess &&
            cudaDeviceGetAttribute(&bus, cudaDevAttrGlobalMemoryBusWidth, device) == cudaSuccess && mclk > 0 && bus > 0)
            m.hbm_bps = 2.0 * mclk * 1e3 * bus / 8.0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) == cudaSuccess && l2 > 0) m.l2_bytes = l2;
        cudaGetLastError();
    }
    return m;
}

static double issue_rate(const CostModel &m) { return m.sms * 4.0 * m.sm_hz * 32.0 * kIssueFraction; }
static double bw(const CostModel &m) { return m.hbm_bps * kCopyFraction; }

// Largest mean build partition whose shared-memory table stays at most half full
// (the join kernel's biggest shape: 200 KiB of slots).
static double fit_tuples(int width, bool agg) {
    // aggregate slots: key, count and (with checksums, assumed) a 64-bit sum
    const double slot = agg ? width + 12.0 : 2.0 * width;
    return (200.0 * 1024 - 4096) / slot / 2.0;
}

double predict_seconds(const CostModel &m, int width, bool agg, bool mat, uint64_t nR, uint64_t nS, int algo,
                       int bits, int passes, double *steps) {
    const double t = 2.0 * width, o = 2.0 * width, ir = issue_rate(m), b = bw(m);
    const double n = (double)nR + (double)nS, M = mat ? (double)nS : 0.0;  // one match per probe tuple
    double s[4] = {0, 0, 0, 0};  // hist, scatter, join / build, probe
    if (algo == HJ_ALGO_SHJ) {
        const double cap = std::exp2(std::ceil(std::log2(2.0 * nR + 1.0)));
        const double slot = agg ? (width == 4 ? 16.0 : 32.0) : t;
        const bool in_l2 = cap * slot <= 0.5 * m.l2_bytes;
        const double rnd = b * kRandomFraction;
        s[2] = std::max(t * nR / b + cap * slot / b + (in_l2 ? 0.0 : 64.0 * nR / rnd), nR * kIptShjBuild / ir);
        s[3] = std::max((t * nS + o * M) / b + (in_l2 ? 0.0 : 32.0 * nS / rnd), nS * kIptShjProbe / ir);
        s[3] += 5 * kLaunchS + kShjFixedS;
    } else {
        const int b1 = passes == 2 ? bits - bits / 2 : bits, b2 = passes == 2 ? bits / 2 : 0;
        for (int p = 0; p < passes; ++p) {
            const int bp = p == 0 ? b1 : b2;
            const double ipt = bp >= 10 && bp <= 11 ? kIptScatterRing
                               : bp <= 7               ? kIptScatterRegionLow
                               : bp <= 9               ? kIptScatterRegion
                                                       : kIptScatterWide;
            // a first pass at <= 2^11 digits is two launches per relation (histogram
            // and scatter place the runs themselves), any other pass eight
            s[0] += std::max(t * n / b, n * kIptHist / ir) + (p == 0 && bp <= 11 ? 2 * 2 : 2 * 8) * kLaunchS;
            s[1] += std::max(2.0 * t * n / b, n * ipt / ir);
        }
        // fewer partition pairs than join CTAs leave SMs idle
        const double busy = std::min(1.0, std::exp2(bits) / (2.0 * m.sms));
        s[2] = std::max((t * n + o * M) / b, (nS * kIptJoinProbe + nR * kIptJoinBuild) / ir) / busy + 6 * kLaunchS +
               kPhjFixedS;
        // the (chunk, digit) count matrix: written, scanned and read once per pass
        s[0] += passes * 24.0 * m.sms * std::exp2(std::max(b1, b2)) / b;
    }
    if (steps)
        for (int i = 0; i < 4; ++i) steps[i] = s[i];
    return s[0] + s[1] + s[2] + s[3];
}

std::vector<PlanCand> plan_candidates(const CostModel &m, int width, bool agg, bool mat, uint64_t nR, uint64_t nS,
                                      int algo, int bits, int passes) {
    std::vector<PlanCand> out;
    auto add = [&](int a, int bb, int g) {
        PlanCand pc{a, bb, g, predict_seconds(m, width, agg, mat, nR, nS, a, bb, g, nullptr)};
        out.push_back(pc);
    };
    // the SHJ table must stay well inside the device (it is 2^ceil(log2(2|R|+1)) slots)
    if (algo == HJ_ALGO_AUTO || algo == HJ_ALGO_SHJ) add(HJ_ALGO_SHJ, 0, 0);
    if (algo == HJ_ALGO_AUTO || algo == HJ_ALGO_PHJ) {
        const double fit = fit_tuples(width, agg);
        for (int b = 1; b <= 24; ++b) {
            if (bits > 0 && b != bits) continue;
            // every partition table must fit: skip fan-outs whose mean partition plus
            // six standard deviations exceeds the half-full table (unless forced)
            const double mean = (double)nR / std::exp2(b);
            if (bits <= 0 && mean + 6.0 * std::sqrt(mean + 1.0) + 64.0 > fit && b < 24) continue;
            for (int g = 1; g <= 2; ++g) {
                if (passes > 0 && g != passes) continue;
                if (g == 1 && b > 12) continue;
                if (g == 2 && (b < 2 || b - b / 2 > 12)) continue;
                add(HJ_ALGO_PHJ, b, g);
            }
            // the smallest fitting fan-outs are the cheapest; a few more are kept
            // as candidates for the tuner
            if (bits <= 0 && out.size() >= 8) break;
        }
    }
    std::sort(out.begin(), out.end(), [](const PlanCand &x, const PlanCand &y) { return x.sec < y.sec; });
    return out;
}

uint64_t plan_key(int width, bool agg, uint64_t nR, uint64_t nS) {
    auto lg = [](uint64_t x) {
        int l = 0;
        while (x > 1) {
            x >>= 1;
            ++l;
        }
        return (uint64_t)l;
    };
    return ((uint64_t)width << 40) | ((uint64_t)agg << 32) | (lg(nR + 1) << 8) | lg(nS + 1);
}

void choose_plan(hj_ctx *c, int width, int mode, uint64_t nR, uint64_t nS, int algo, int bits, int passes,
                 int *a_out, int *b_out, int *g_out) {
    const bool agg = mode != HJ_MATERIALIZE, mat = mode == HJ_MATERIALIZE;
    if (algo == HJ_ALGO_AUTO && bits <= 0 && passes <= 0 && c) {
        auto it = c->tuned.find(plan_key(width, agg, nR, nS));
        if (it != c->tuned.end()) {
            *a_out = it->second.algo;
            *b_out = it->second.bits;
            *g_out = it->second.passes;
            return;
        }
    }
    if (algo == HJ_ALGO_SHJ) {
        *a_out = HJ_ALGO_SHJ;
        *b_out = 0;
        *g_out = 0;
        return;
    }
    if (!c->model_ready) {
        c->model = cost_model_for(c->device);
        c->model_ready = true;
    }
    std::vector<PlanCand> pcs = plan_candidates(c->model, width, agg, mat, nR, nS, algo, bits, passes);
    if (pcs.empty()) {  // forced shape the filters rejected: honour it
        *a_out = HJ_ALGO_PHJ;
        *b_out = bits > 0 ? bits : 12;
        *g_out = passes > 0 ? passes : (*b_out <= 12 ? 1 : 2);
        return;
    }
    *a_out = pcs[0].algo;
    *b_out = pcs[0].bits;
    *g_out = pcs[0].passes;
}

}  // namespace hj

using namespace hj;

extern "C" {

hj_status hj_plan(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts *opts, hj_plan_info *out) {
    if (!R || !S || !out) return c ? set_err(c, HJ_E_INVALID, "NULL argument") : HJ_E_INVALID;
    if ((R->width != HJ_U32 && R->width != HJ_U64) || R->width != S->width)
        return c ? set_err(c, HJ_E_INVALID, "bad or differing widths") : HJ_E_INVALID;
    hj_opts o{};
    o.mode = HJ_MATERIALIZE;
    if (opts) o = *opts;
    const bool agg = o.mode != HJ_MATERIALIZE, mat = o.mode == HJ_MATERIALIZE;
    CostModel m = c ? cost_model_for(c->device) : CostModel{};
    int a = o.algo, b = o.radix_bits, g = o.passes;
    if (c) {
        choose_plan(c, R->width, o.mode, R->n, S->n, o.algo, o.radix_bits, o.passes, &a, &b, &g);
    } else {
        std::vector<PlanCand> pcs = plan_candidates(m, R->width, agg, mat, R->n, S->n, o.algo, o.radix_bits, o.passes);
        if (pcs.empty()) return HJ_E_INVALID;
        a = pcs[0].algo;
        b = pcs[0].bits;
        g = pcs[0].passes;
    }
    *out = hj_plan_info{};
    out->algo = a;
    out->radix_bits = a == HJ_ALGO_PHJ ? b : 0;
    out->passes = a == HJ_ALGO_PHJ ? g : 0;
    double st[4];
    out->predicted_ms = 1e3 * predict_seconds(m, R->width, agg, mat, R->n, S->n, a, b, g, st);
    for (int i = 0; i < 4; ++i) out->step_ms[i] = 1e3 * st[i];
    out->measured_ms = -1.0;
    return HJ_OK;
}

hj_status hj_tune(hj_ctx *c, const hj_rel *R, const hj_rel *S, const hj_opts *opts, int top_k, hj_plan_info *out) {
    if (!c || !R || !S) return c ? set_err(c, HJ_E_INVALID, "NULL argument") : HJ_E_INVALID;
    if ((R->width != HJ_U32 && R->width != HJ_U64) || R->width != S->width)
        return set_err(c, HJ_E_INVALID, "bad or differing widths");
    hj_opts o{};
    o.mode = HJ_MATERIALIZE;
    if (opts) o = *opts;
    if (top_k <= 0) top_k = 4;
    const bool agg = o.mode != HJ_MATERIALIZE, mat = o.mode == HJ_MATERIALIZE;
    if (!c->model_ready) {
        c->model = cost_model_for(c->device);
        c->model_ready = true;
    }
    std::vector<PlanCand> pcs = plan_candidates(c->model, R->width, agg, mat, R->n, S->n, HJ_ALGO_AUTO, 0, 0);
    if ((int)pcs.size() > top_k) pcs.resize(top_k);
    if (pcs.empty()) return set_err(c, HJ_E_UNSUPPORTED, "no plan candidate");
    cudaEvent_t e0, e1;
    HJ_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_err(c, HJ_E_CUDA, "cudaEventCreate");
    }
    double best = 1e30;
    PlanCand pick = pcs[0];
    hj_status st = HJ_OK;
    for (const PlanCand &pc : pcs) {
        hj_opts oj = o;
        oj.algo = pc.algo;
        oj.radix_bits = pc.bits;
        oj.passes = pc.passes;
        double t_min = 1e30;
        for (int rep = 0; rep < 3 && st == HJ_OK; ++rep) {  // one warm-up, two timed
            hj_result res{};
            cudaEventRecord(e0, c->stream);
            st = hj_join(c, R, S, &oj, &res);
            cudaEventRecord(e1, c->stream);
            if (st != HJ_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            hj_result_free(c, &res);
            if (rep > 0) t_min = std::min(t_min, (double)ms);
        }
        if (st != HJ_OK) break;
        if (t_min < best) {
            best = t_min;
            pick = pc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HJ_OK) return st;
    c->tuned[plan_key(R->width, agg, R->n, S->n)] = TunedPlan{pick.algo, pick.bits, pick.passes};
    if (out) {
        *out = hj_plan_info{};
        out->algo = pick.algo;
        out->radix_bits = pick.algo == HJ_ALGO_PHJ ? pick.bits : 0;
        out->passes = pick.algo == HJ_ALGO_PHJ ? pick.passes : 0;
        double s4[4];
        out->predicted_ms = 1e3 * predict_seconds(c->model, R->width, agg, mat, R->n, S->n, pick.algo, pick.bits,
                                                  pick.passes, s4);
        for (int i = 0; i < 4; ++i) out->step_ms[i] = 1e3 * s4[i];
        out->measured_ms = best;
    }
    return HJ_OK;
}

hj_status hj_tune_clear(hj_ctx *c) {
    if (!c) return HJ_E_INVALID;
    c->tuned.clear();
    return HJ_OK;
}

}  // extern "C"
