// Tile / block-shape autotuner of the step kernel.
//
// Candidates: every variant of the one-pass direct kernel and of the TMA-staged one compiled
// for the solver's precision, and the one-warp-per-cell kernel on small grids.  Each runs `trial` steps after two warm-up
// steps, timed with CUDA events on the solver's stream; the fastest wins.
// Results are cached per (lattice, precision, order, Nx class, Ny class) for
// the life of the process and, when LBM_AUTOTUNE_CACHE names a file, across
// processes (one "key kernel variant ms" line per class).
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "launchers.h"
#include "lbm_internal.h"

namespace lbm {

namespace {

struct Choice {
    int kernel, variant;
    double ms;
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;
bool g_loaded = false;

int size_class(int n) {
    int c = 1;
    while (c < n) c <<= 1;
    return c;
}

std::string class_key(const SolverImpl &s) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "Q%d_p%d_o%d_x%d_y%d", s.L.kind, s.p.precision, s.p.eq_order,
                  size_class(s.p.Nx), size_class(s.p.Ny));
    return buf;
}

void load_file_cache() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("LBM_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *fh = std::fopen(path, "r");
    if (!fh) return;
    char key[100];
    Choice c;
    while (std::fscanf(fh, "%99s %d %d %lf", key, &c.kernel, &c.variant, &c.ms) == 4)
        g_cache[key] = c;
    std::fclose(fh);
}

void append_file_cache(const std::string &key, const Choice &c) {
    const char *path = std::getenv("LBM_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *fh = std::fopen(path, "a");
    if (!fh) return;
    std::fprintf(fh, "%s %d %d %.6f\n", key.c_str(), c.kernel, c.variant, c.ms);
    std::fclose(fh);
}

int time_candidate(SolverImpl &s, int kernel, int variant, int trial, double *ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LBM_ECUDA; }
    int rc = LBM_OK;
    for (int i = 0; i < 2 && !rc; ++i) {
        if (launch_step_variant(s, s.cur, s.cur ^ 1, kernel, variant)) rc = LBM_ECUDA;
        s.cur ^= 1;
    }
    cudaEventRecord(e0, s.stream);
    for (int i = 0; i < trial && !rc; ++i) {
        if (launch_step_variant(s, s.cur, s.cur ^ 1, kernel, variant)) rc = LBM_ECUDA;
        s.cur ^= 1;
    }
    cudaEventRecord(e1, s.stream);
    float t = 0;
    if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
        *ms = t / trial;
    else
        rc = LBM_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

int autotune_solver(SolverImpl &s, int trial) {
    const std::string key = class_key(s);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_file_cache();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            s.p.kernel = it->second.kernel;
            s.variant = it->second.variant;
            s.tuned_ms = it->second.ms;
            return LBM_OK;
        }
    }
    // a valid state to step on; the caller re-initialises afterwards
    int rc = dispatch_init_rest(s);
    if (rc) return rc;
    Choice best{LBM_KERNEL_DIRECT, 0, 1e30};
    double ms = 0;
    const int nd = direct_variant_count(s.p.precision);
    for (int v = 0; v < nd; ++v) {
        if ((rc = time_candidate(s, LBM_KERNEL_DIRECT, v, trial, &ms))) return rc;
        if (ms < best.ms) best = Choice{LBM_KERNEL_DIRECT, v, ms};
    }
    // the staged kernel: grids stored as one x-tile only
    const int nv = s.nt == 1 ? staged_variant_count(s.p.precision) : 0;
    for (int v = 0; v < nv; ++v) {
        if ((rc = time_candidate(s, LBM_KERNEL_STAGED, v, trial, &ms))) return rc;
        if (ms < best.ms) best = Choice{LBM_KERNEL_STAGED, v, ms};
    }
    // one warp per cell: only a candidate for small grids (32 threads a cell)
    if ((long long)s.p.Nx * s.p.Ny <= 16 * kCellwarpAutoCells) {
        if ((rc = time_candidate(s, LBM_KERNEL_CELLWARP, 0, trial, &ms))) return rc;
        if (ms < best.ms) best = Choice{LBM_KERNEL_CELLWARP, 0, ms};
    }
    s.p.kernel = best.kernel;
    s.variant = best.variant;
    s.tuned_ms = best.ms;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = best;
        append_file_cache(key, best);
    }
    return dispatch_init_rest(s);
}

}  // namespace lbm
