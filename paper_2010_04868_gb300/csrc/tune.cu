// Plan selection: which kernel family a run uses, with its tile and T_b.
//
// The paper picks blocking sizes by trying every power-of-two, symmetric
// size and keeping the fastest (Section 4.1), and leaves an auto-tuner to
// future work (Section 6). Here the tuner measures instead of guessing:
//   * Jacobi: the plain per-step kernel, the temporally blocked kernels (the
//     overlapped tiles, and in 2D/3D the streaming tiles) over a small set of
//     tiles and depths T_b, and the split (diamond) tiles over a few periods
//     and band heights are each timed for a few steps on private
//     buffers of the run's extents; the fastest per step wins, a plan other
//     than plain only if it is more than 3% faster. On GB300 the FP64 pipe, not HBM, bounds large grids, so the plain
//     kernel usually wins there and blocking wins where launches dominate.
//   * Gauss-Seidel: the wavefront kernel whenever it is legal (constant
//     boundary); it was faster than per-sweep execution in every measured
//     case by one to two orders of magnitude, so the plain sweep is not
//     timed. In 2D and 3D its parameters are: CTAs per SM of the persistent
//     kernel (tile[0]), skewed rows per tile (tile[1], 2D) and points per
//     lane and step or the decoupled tile (tile[2], 2D radius 1); a few
//     combinations around the default are timed like the Jacobi plans.
// Results are cached per (stencil, extent class, T class) in memory and, when
// the environment variable STENCIL_TUNE_CACHE names a file, in that file (one
// JSON object per line). A run inside CUDA stream capture never tunes; it
// uses a cached plan or the static default.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tune.h"

namespace gbst {

namespace {

std::mutex g_mu;
std::map<std::string, Plan> g_cache;
bool g_loaded = false;

int log2_bucket(int64_t n)
{
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

std::string plan_key(const stencil_handle_s* h, const Geo& g, int64_t T)
{
    char buf[160];
    const int tcls = T < 8 ? 0 : (T < 64 ? 1 : (T < 512 ? 2 : 3));
    snprintf(buf, sizeof buf, "d%d_s%d_r%d_m%d_b%d_a%d_f%d_e%d.%d.%d_t%d", h->dim, h->shape, h->r, h->method, h->bc,
             h->arith, h->field ? 1 : 0, log2_bucket(g.n0), log2_bucket(g.n1), log2_bucket(g.n2), tcls);
    return buf;
}

void load_file()
{
    if (g_loaded) return;
    g_loaded = true;
    const char* path = getenv("STENCIL_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char key[200];
        Plan p{};
        long long t0 = 0, t1 = 0, t2 = 0;
        if (sscanf(line, "{\"key\": \"%199[^\"]\", \"kernel\": %d, \"tb\": %d, \"tile\": [%lld, %lld, %lld]", key,
                   &p.kernel, &p.tb, &t0, &t1, &t2) == 6) {
            p.tile[0] = t0;
            p.tile[1] = t1;
            p.tile[2] = t2;
            g_cache[key] = p;
        }
    }
    fclose(f);
}

void save_entry(const std::string& key, const Plan& p, double ms_per_step)
{
    const char* path = getenv("STENCIL_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"kernel\": %d, \"tb\": %d, \"tile\": [%lld, %lld, %lld], \"ms_per_step\": %.6f}\n",
            key.c_str(), p.kernel, p.tb, (long long)p.tile[0], (long long)p.tile[1], (long long)p.tile[2],
            ms_per_step);
    fclose(f);
}

Plan default_plan(const stencil_handle_s* h, const Geo& g)
{
    Plan p{STENCIL_KERNEL_PLAIN, 1, {0, 0, 0}};
    if (h->method == GAUSS_SEIDEL) {
        if (gs_wavefront_supported(h, g)) p.kernel = STENCIL_KERNEL_WAVEFRONT;
    } else if (h->dim == 1 && jacobi_blocked_supported(h, g)) {
        p.kernel = STENCIL_KERNEL_BLOCKED;
        p.tb = 64 / h->r;
        p.tile[2] = 256;
    }
    return p;
}

std::vector<Plan> jacobi_candidates(const stencil_handle_s* h, const Geo& g, int64_t T)
{
    std::vector<Plan> c;
    c.push_back(Plan{STENCIL_KERNEL_PLAIN, 1, {0, 0, 0}});
    if (T < 2) return c;
    // split (diamond) tiles: no redundant work, so they compete where the FP64 pipe binds
    if (jacobi_diamond_supported(h, g)) {
        auto dia = [&](int H, int64_t t0, int64_t t1, int64_t t2) {
            if (H <= T) c.push_back(Plan{STENCIL_KERNEL_DIAMOND, H, {t0, t1, t2}});
        };
        if (h->dim == 1) {
            for (int H : {54, 100}) dia(H / h->r > 0 ? H / h->r : 1, 0, 0, 0);
            dia(100 / h->r > 0 ? 100 / h->r : 1, 0, 0, (g.n2 + 303) / 304 < 64 ? 64 : (g.n2 + 303) / 304);
        } else if (h->dim == 2) {
            dia(16, 0, 80, 80);
            dia(16, 0, 88, 88);
        }
    }
    // streaming blocked tiles (2D/3D): the slowest axis streamed, redundancy on the cross-section only
    if (jacobi_stream_supported(h, g)) {
        auto st = [&](int tb, int64_t w1, int64_t w2) {
            if (tb <= T) c.push_back(Plan{STENCIL_KERNEL_STREAM, tb, {0, w1, w2}});
        };
        if (h->dim == 2) {
            for (int tb : {1, 2, 4}) st(tb, 0, 256);
            st(2, 0, 192);
            if (h->r == 1) st(3, 0, 256);
        } else {
            st(1, 16, 64);
            st(1, 24, 128);
            st(2, 12, 64);
        }
    }
    if (!jacobi_blocked_supported(h, g)) return c;
    auto add = [&](int tb, int64_t t0, int64_t t1, int64_t t2) {
        if (tb <= T) c.push_back(Plan{STENCIL_KERNEL_BLOCKED, tb, {t0, t1, t2}});
    };
    if (h->dim == 1) {
        // tiles that spread the grid evenly over 1-4 CTAs per SM (one even wave), and two fixed sizes
        int nsm = 152, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        std::vector<int64_t> tiles = {256, 1024};
        for (int m = 1; m <= 4; ++m) {
            int64_t t = (g.n2 + (int64_t)nsm * m - 1) / ((int64_t)nsm * m);
            t = (t + 1) & ~int64_t(1);
            if (t >= 64 && t <= 4096) tiles.push_back(t);
        }
        for (int64_t tile : tiles)
            for (int tb : {16, 32, 64}) add(tb / h->r > 0 ? tb / h->r : 1, 0, 0, tile);
    } else if (h->dim == 2) {
        for (int tb : {2, 3, 4}) {
            add(tb, 0, 32, 64);
            add(tb, 0, 16, 128);
        }
    } else {
        add(2, 8, 16, 32);
    }
    return c;
}

// Wavefront Gauss-Seidel parameter sets (the first is the default, the reference).
std::vector<Plan> gs_candidates(const stencil_handle_s* h)
{
    std::vector<Plan> c;
    auto add = [&](int64_t ctas, int64_t rows, int64_t pts) {
        c.push_back(Plan{STENCIL_KERNEL_WAVEFRONT, 0, {ctas, rows, pts}});
    };
    add(0, 0, 0);
    if (h->dim == 2) {
        add(3, 16, 16);
        add(4, 16, 16);
        add(3, 8, 16);
        if (h->r == 1) add(2, 32, 8);
        if (h->r == 1 && h->shape == STAR && !h->field) add(3, 32, 1);   // the decoupled tile
    } else {
        add(3, 0, 0);
        add(4, 0, 0);
    }
    return c;
}

// Time one candidate: ms per time step over probe steps (after one warm-up).
double time_candidate(stencil_handle_s* h, const Plan& p, double* a, double* b, const int64_t ext[3], int64_t probe,
                      cudaStream_t st)
{
    const int saved_k = h->plan_kernel, saved_tb = h->plan_tb;
    int64_t saved_tile[3] = {h->plan_tile[0], h->plan_tile[1], h->plan_tile[2]};
    h->plan_kernel = p.kernel;
    h->plan_tb = p.tb;
    for (int d = 0; d < 3; ++d) h->plan_tile[d] = p.tile[d];
    stencil_grid g;
    g.data = a;
    g.scratch = b;
    for (int d = 0; d < 3; ++d) g.ext[d] = ext[d];
    double ms = INFINITY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (stencil_run(h, &g, probe, st) == STENCIL_OK) {
        cudaEventRecord(e0, st);
        int rc = stencil_run(h, &g, probe, st);
        cudaEventRecord(e1, st);
        if (rc == STENCIL_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float f = 0;
            cudaEventElapsedTime(&f, e0, e1);
            ms = f / (double)probe;
        }
    }
    cudaStreamSynchronize(st);
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->plan_kernel = saved_k;
    h->plan_tb = saved_tb;
    for (int d = 0; d < 3; ++d) h->plan_tile[d] = saved_tile[d];
    return ms;
}

}  // namespace

Plan plan_for(const stencil_handle_s* hc, const Geo& g, int64_t T, cudaStream_t caller)
{
    stencil_handle_s* h = const_cast<stencil_handle_s*>(hc);
    if (h->plan_kernel != STENCIL_KERNEL_AUTO) {
        Plan p{h->plan_kernel, h->plan_tb, {h->plan_tile[0], h->plan_tile[1], h->plan_tile[2]}};
        return p;
    }
    const bool gs_tuned = h->method == GAUSS_SEIDEL && h->dim >= 2 && h->bc == BC_CONSTANT &&
                          gs_wavefront_supported(h, g);
    if (h->method == GAUSS_SEIDEL && !gs_tuned) return default_plan(h, g);
    const std::string key = plan_key(h, g, T);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return it->second;
    }
    // never tune while the caller's stream is being captured into a graph
    cudaStream_t st;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(caller, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return default_plan(h, g);
    }
    if (getenv("STENCIL_NO_TUNE")) return default_plan(h, g);
    if (!gs_tuned && !jacobi_blocked_supported(h, g) && !jacobi_diamond_supported(h, g) &&
        !jacobi_stream_supported(h, g))
        return default_plan(h, g);  // the plain kernel is the only candidate
    const size_t n = (size_t)(g.n0 * g.n1 * g.n2);
    double *a = nullptr, *b = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return default_plan(h, g);
    }
    if (cudaMalloc(&a, n * sizeof(double)) != cudaSuccess || cudaMalloc(&b, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a);
        cudaStreamDestroy(st);
        return default_plan(h, g);
    }
    cudaMemsetAsync(a, 0x3f, n * sizeof(double), st);  // every double 0x3f3f... ~ 4.8e-4: no subnormals
    int64_t ext[3] = {1, 1, 1};
    if (h->dim == 1) ext[0] = g.n2;
    if (h->dim == 2) { ext[0] = g.n1; ext[1] = g.n2; }
    if (h->dim == 3) { ext[0] = g.n0; ext[1] = g.n1; ext[2] = g.n2; }
    // probe length: enough steps to amortise a pass of the deepest candidate, bounded by T
    int64_t probe = h->dim == 1 ? 128 : (h->dim == 2 ? 48 : 8);
    // two sweep blocks of the one-warp tiles; in 2D enough sweeps that the rows-as-lanes pipeline's
    // fill (a fixed number of steps) does not decide the choice
    if (gs_tuned) probe = h->dim == 2 ? 128 : 32;
    if (probe > T) probe = T;
    std::vector<Plan> cands = gs_tuned ? gs_candidates(h) : jacobi_candidates(h, g, T);
    // the plain kernel is the reference: another plan must beat it by a clear
    // margin, so that run-to-run noise of a few percent never flips the choice
    constexpr double MARGIN = 0.97;
    Plan best = cands[0];
    double best_ms = time_candidate(h, cands[0], a, b, ext, probe, st) * MARGIN;
    for (size_t q = 1; q < cands.size(); ++q) {
        double ms = time_candidate(h, cands[q], a, b, ext, probe, st);
        if (ms < best_ms) {
            best_ms = ms;
            best = cands[q];
        }
    }
    cudaFree(a);
    cudaFree(b);
    cudaStreamDestroy(st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best;
    save_entry(key, best, best_ms);
    return best;
}

}  // namespace gbst
