// coproc.cu -- the paper's cost model of pipelined CPU/GPU co-processing (PL,
// Sec. 3.2 and Sec. 4) and its search for the workload ratios, as host logic.
//
// A step series has n steps; step i has x_i input items, of which the share r_i
// runs on the CPU and 1 - r_i on the GPU.  Per item a step costs c_i seconds on
// the CPU and g_i on the GPU (computation plus memory stalls: C_i + M_i of Eq. 2-3
// divided by the items).  Then
//   T = max(T_CPU, T_GPU)                                   (Eq. 1)
//   T_XPU = sum_i (C^i + M^i + D^i)                         (Eq. 2)
// with the pipeline delays of Eq. 4 (r_i > r_{i-1}: the CPU waits for the GPU's
// step i-1 output) and Eq. 5 (r_i < r_{i-1}: the GPU waits), clamped at 0.  The
// intermediate results between two steps of different ratios, |r_i - r_{i-1}| x_i
// items (Sec. 4), cost `xfer` seconds per item on the processor that receives them.
// Readings where the paper is silent: the running sums inside Eq. 4 and 5 are the
// steps' times up to step i without the delay being computed; the search takes
// r_i from {0, delta, 2 delta, ..., floor(1 / delta) delta, 1}, 0 and 1 included so
// that the GPU-only and CPU-only plans (OL's extremes) are candidates.
//
// GB300 runs every step on the GPU (r = 0): with the oracle's single-core rate
// against the GPU's, the search returns that too.  The model is exposed so that a
// caller can evaluate the trade-off on other processors or costs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/hj.h"

namespace {

struct Series {
    int n;
    const double *x, *c, *g;
    double xfer;
};

// Running sums over the steps before i, each step's time with its delay.
struct Acc {
    double cpu = 0.0, gpu = 0.0;  // sum over steps < i of T^j (delays included)
    double last_gpu = 0.0;        // T^{i-1}_GPU
};

// Times of step i on the CPU and the GPU for its ratio r, the previous step's rp.
void step_times(const Series &s, int i, double r, double rp, const Acc &a, double *tc, double *tg) {
    double cpu = s.c[i] * r * s.x[i], gpu = s.g[i] * (1.0 - r) * s.x[i];
    if (i > 0 && r != rp) {  // intermediate results, charged to the receiver
        const double items = std::fabs(r - rp) * s.x[i] * s.xfer;
        if (r > rp) cpu += items;
        else gpu += items;
    }
    double dc = 0.0, dg = 0.0;
    if (i > 0 && r > rp && rp < 1.0) {  // Eq. 4
        dc = (a.gpu - a.last_gpu * (1.0 - r) / (1.0 - rp)) - (a.cpu + cpu);
    } else if (i > 0 && r < rp && r < 1.0) {  // Eq. 5
        dg = a.cpu - ((a.gpu + gpu) - gpu * (1.0 - rp) / (1.0 - r));
    }
    *tc = cpu + std::max(dc, 0.0);
    *tg = gpu + std::max(dg, 0.0);
}

Acc series_times(const Series &s, const double *r) {
    Acc a;
    for (int i = 0; i < s.n; ++i) {
        double tc, tg;
        step_times(s, i, r[i], i ? r[i - 1] : r[i], a, &tc, &tg);
        a.cpu += tc;
        a.gpu += tg;
        a.last_gpu = tg;
    }
    return a;
}

struct Search {
    const Series &s;
    const std::vector<double> &grid;
    std::vector<double> r, best_r;
    double best = INFINITY;
    void go(int i, const Acc &a) {
        if (i == s.n) {
            const double t = std::max(a.cpu, a.gpu);
            if (t < best) {
                best = t;
                best_r = r;
            }
            return;
        }
        for (double ri : grid) {
            double tc, tg;
            step_times(s, i, ri, i ? r[i - 1] : ri, a, &tc, &tg);
            Acc b{a.cpu + tc, a.gpu + tg, tg};
            if (std::max(b.cpu, b.gpu) >= best) continue;  // step times only add up: cannot win
            r[i] = ri;
            go(i + 1, b);
        }
    }
};

bool bad_series(int n, const double *x, const double *c, const double *g, double xfer) {
    if (n < 1 || n > 16 || !x || !c || !g || !(xfer >= 0.0)) return true;
    for (int i = 0; i < n; ++i)
        if (!(x[i] >= 0.0) || !(c[i] >= 0.0) || !(g[i] >= 0.0)) return true;
    return false;
}

}  // namespace

extern "C" hj_status hj_coproc_time(int n, const double *x, const double *cpu_s, const double *gpu_s, double xfer_s,
                                    const double *ratios, double *t_out, double *t_cpu, double *t_gpu) {
    if (bad_series(n, x, cpu_s, gpu_s, xfer_s) || !ratios || !t_out) return HJ_E_INVALID;
    for (int i = 0; i < n; ++i)
        if (!(ratios[i] >= 0.0 && ratios[i] <= 1.0)) return HJ_E_INVALID;
    const Acc a = series_times(Series{n, x, cpu_s, gpu_s, xfer_s}, ratios);
    *t_out = std::max(a.cpu, a.gpu);
    if (t_cpu) *t_cpu = a.cpu;
    if (t_gpu) *t_gpu = a.gpu;
    return HJ_OK;
}

extern "C" hj_status hj_coproc_ratios(int n, const double *x, const double *cpu_s, const double *gpu_s,
                                      double xfer_s, double delta, double *ratios_out, double *t_out) {
    if (bad_series(n, x, cpu_s, gpu_s, xfer_s) || !ratios_out || !t_out) return HJ_E_INVALID;
    if (!(delta > 0.0 && delta <= 1.0)) return HJ_E_INVALID;
    // the search visits up to (points per ratio)^n ratio vectors: refuse sizes it
    // cannot finish before building the grid (a tiny delta would otherwise ask for
    // a grid larger than memory, or overflow the int count)
    const double steps = std::floor(1.0 / delta + 1e-9);
    if (std::pow(steps + 2.0, n) > 1e9) return HJ_E_UNSUPPORTED;
    const int m = (int)steps;
    std::vector<double> grid{0.0};
    for (int k = 1; k <= m; ++k) grid.push_back(std::min(1.0, k * delta));
    if (grid.back() < 1.0) grid.push_back(1.0);
    const Series s{n, x, cpu_s, gpu_s, xfer_s};
    Search sr{s, grid, std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};
    sr.go(0, Acc{});
    for (int i = 0; i < n; ++i) ratios_out[i] = sr.best_r[i];
    *t_out = sr.best;
    return HJ_OK;
}
