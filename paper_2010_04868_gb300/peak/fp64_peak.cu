// FP64 pipe micro-benchmark: the ALU roofline the stencil kernels are measured against.
// Also the 32-bit integer logic (LOP3) and funnel-shift (SHF) rates, the roofline of the
// bit-packed Game of Life kernels.
//
// Streams of independent __fma_rn / __dadd_rn / __dmul_rn on every resident warp. Each CTA
// records its SM (%smid) and the SM clock (clock64) at its start and end; an SM's rate is
// the lane operations of all its CTAs over the span from its first start to its last end,
// so the result is a per-clock rate independent of the clock the GPU happened to run at.
// The rate is swept over the shapes that could limit it:
//   * chains per thread (independent accumulators: latency hiding inside a warp),
//   * warps per SM (CTAs per SM x warps per CTA: latency hiding across warps),
//   * the instruction (DFMA, DADD, DMUL, and the three interleaved),
//   * the operands (two shared scalars, or a distinct register triple per chain),
//   * stencil-shaped streams: 5-term weighted sums, weights from the constant bank or registers,
// and the best rate is the FP64 peak reported. Also: the dependent-chain latency of one
// DFMA and the cost of a warp instruction with one active lane.
//
//   fp64_peak            one JSON object: the best rate of a short sweep (about a second)
//   fp64_peak --sweep    one JSON object per swept shape, then the summary
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess) {                                                                  \
            printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__);         \
            exit(1);                                                                              \
        }                                                                                         \
    } while (0)

__device__ __forceinline__ unsigned smid()
{
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// OP: 0 DFMA x = fma(x, a, b); 1 DADD; 2 DMUL; 3 DFMA, DADD, DMUL in turn;
//     4 DFMA with a distinct register triple per chain: x = fma(y, x, z)
template <int CH, int OP>
__global__ void stream_ops(double* out, long long* rec, int iters, double a, double b, int active)
{
    const long long t0 = clock64();
    double x[CH], y[CH], z[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        x[c] = threadIdx.x * 1e-9 + c * 0.1;
        y[c] = a + c * 1e-12;
        z[c] = b * (1 + c);
    }
    if ((int)(threadIdx.x & 31) < active) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (OP == 0) x[c] = __fma_rn(x[c], a, b);
                else if (OP == 1) x[c] = __dadd_rn(x[c], b);
                else if (OP == 2) x[c] = __dmul_rn(x[c], a);
                else if (OP == 3) {
                    if (c % 3 == 0) x[c] = __fma_rn(x[c], a, b);
                    else if (c % 3 == 1) x[c] = __dadd_rn(x[c], b);
                    else x[c] = __dmul_rn(x[c], a);
                } else x[c] = __fma_rn(y[c], x[c], z[c]);
            }
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

// A stencil-shaped stream: per chain a 5-term weighted sum (one DMUL, four dependent DFMAs) whose
// result feeds the chain's next sum, weights read from the constant bank (REGW = 0) or forced into
// registers with an empty asm (REGW = 1), the values in registers.
__constant__ double c_w5[5] = {0.2, 0.21, 0.18, 0.22, 0.19};

template <int CH, int REGW>
__global__ void stream_stencil(double* out, long long* rec, int iters, double a, double b, int active)
{
    const long long t0 = clock64();
    double wq[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        wq[q] = c_w5[q];
        if (REGW) asm volatile("" : "+d"(wq[q]));
    }
    double v[CH][5];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            v[c][q] = threadIdx.x * 1e-9 + c * 0.1 + q * a + b;
            asm volatile("" : "+d"(v[c][q]));
        }
    if ((int)(threadIdx.x & 31) < active) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                double acc = __dmul_rn(wq[0], v[c][0]);
#pragma unroll
                for (int q = 1; q < 5; ++q) acc = __fma_rn(wq[q], v[c][q], acc);
                v[c][0] = acc;
            }
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += v[c][0];
    if (s == 12345.678) out[0] = s;
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

// Independent chains of one 3-input logic op (LOP3) or one funnel shift (SHF) per step, written
// in PTX so that the compiler cannot fold the repeated bitwise operations.
template <int CH, int OP>
__global__ void stream_int(double* out, long long* rec, int iters, double fa, double fb, int active)
{
    const long long t0 = clock64();
    const unsigned a = (unsigned)(fa * 1e7) | 1u, b = (unsigned)(fb * 1e9) + 3u;
    unsigned x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 7u + c;
    if ((int)(threadIdx.x & 31) < active) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (OP == 0)
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(a), "r"(b));
                else
                    asm volatile("shf.l.wrap.b32 %0, %0, %1, 1;" : "+r"(x[c]) : "r"(b));
            }
        }
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s ^= x[c];
    if (s == 0x12345678u) out[0] = s;
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

typedef void (*Kern)(double*, long long*, int, double, double, int);

struct Shape {
    const char* op;
    Kern k;
    int chains, threads, ctas_per_sm, active;
};

static int g_nsm = 0;
static double* g_out = nullptr;
static long long* g_rec = nullptr;
static cudaEvent_t g_e0, g_e1;

// Lane operations per SM clock (median over SMs), or 0 if the CTAs cannot all be resident.
static double measure(const Shape& s, int iters, double* ops_per_s, double* ms_out)
{
    int fit = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, s.k, s.threads, 0));
    if (fit < s.ctas_per_sm) return 0.0;
    const int nblk = g_nsm * s.ctas_per_sm;
    s.k<<<nblk, s.threads>>>(g_out, g_rec, iters / 8 + 1, 1.0000001, 1e-7, s.active);  // warm-up
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(g_e0));
    s.k<<<nblk, s.threads>>>(g_out, g_rec, iters, 1.0000001, 1e-7, s.active);
    CK(cudaEventRecord(g_e1));
    CK(cudaEventSynchronize(g_e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, g_e0, g_e1));
    std::vector<long long> rec(3 * (size_t)nblk);
    CK(cudaMemcpy(rec.data(), g_rec, rec.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    const int maxsm = 1024;
    std::vector<long long> lo(maxsm, -1), hi(maxsm, -1);
    std::vector<int> cnt(maxsm, 0);
    for (int b = 0; b < nblk; ++b) {
        const int sm = (int)rec[3 * b];
        if (sm < 0 || sm >= maxsm) continue;
        if (lo[sm] < 0 || rec[3 * b + 1] < lo[sm]) lo[sm] = rec[3 * b + 1];
        if (hi[sm] < 0 || rec[3 * b + 2] > hi[sm]) hi[sm] = rec[3 * b + 2];
        cnt[sm]++;
    }
    const double lanes = (double)(s.active < 32 ? s.active : 32);
    const double ops_per_cta = (s.threads / 32.0) * lanes * (double)iters * s.chains;
    std::vector<double> rates;
    for (int sm = 0; sm < maxsm; ++sm)
        if (cnt[sm] > 0 && hi[sm] > lo[sm]) rates.push_back(ops_per_cta * cnt[sm] / (double)(hi[sm] - lo[sm]));
    if (rates.empty()) return 0.0;
    std::sort(rates.begin(), rates.end());
    if (ops_per_s) *ops_per_s = ops_per_cta * nblk / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return rates[rates.size() / 2];
}

template <int CH>
static void add_shapes(std::vector<Shape>& v, bool full)
{
    const int warps[] = {4, 8, 16, 32, 64};
    for (int wps : warps) {
        if (!full && wps != 8 && wps != 32) continue;
        // CTAs of 8 warps (one of 4 for the smallest count)
        const int threads = wps < 8 ? wps * 32 : 256;
        const int ctas = wps < 8 ? 1 : wps / 8;
        v.push_back(Shape{"dfma", stream_ops<CH, 0>, CH, threads, ctas, 32});
        if (full) {
            v.push_back(Shape{"dadd", stream_ops<CH, 1>, CH, threads, ctas, 32});
            v.push_back(Shape{"dmul", stream_ops<CH, 2>, CH, threads, ctas, 32});
            v.push_back(Shape{"mix", stream_ops<CH, 3>, CH, threads, ctas, 32});
        }
        v.push_back(Shape{"dfma_reg3", stream_ops<CH, 4>, CH, threads, ctas, 32});
        if (full && CH <= 4) {
            // 5 FP64 instructions per chain and iteration: counted as 5 "chains" of one
            v.push_back(Shape{"stencil5_const", stream_stencil<CH, 0>, 5 * CH, threads, ctas, 32});
            v.push_back(Shape{"stencil5_reg", stream_stencil<CH, 1>, 5 * CH, threads, ctas, 32});
        }
    }
}

int main(int argc, char** argv)
{
    const bool full = argc > 1 && strcmp(argv[1], "--sweep") == 0;
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    g_nsm = p.multiProcessorCount;
    CK(cudaMalloc(&g_out, 64));
    CK(cudaMalloc(&g_rec, sizeof(long long) * 3 * 1024 * 16));
    CK(cudaEventCreate(&g_e0));
    CK(cudaEventCreate(&g_e1));

    std::vector<Shape> shapes;
    if (full) {
        add_shapes<1>(shapes, true);
        add_shapes<2>(shapes, true);
        add_shapes<4>(shapes, true);
        add_shapes<8>(shapes, true);
        add_shapes<16>(shapes, true);
    } else {
        add_shapes<2>(shapes, false);
        add_shapes<4>(shapes, false);
        add_shapes<8>(shapes, false);
    }
    // a fixed number of FP64 instructions per SM for every shape (about 40 ms at the peak)
    const double target_lane_ops = 1.2e8;
    double best = 0, best_ops_s = 0;
    const Shape* best_s = nullptr;
    for (const Shape& s : shapes) {
        const double per_iter = (s.threads / 32.0) * 32.0 * s.chains * s.ctas_per_sm;
        const int iters = (int)std::max(64.0, target_lane_ops / per_iter);
        double ops_s = 0, ms = 0;
        const double r = measure(s, iters, &ops_s, &ms);
        if (full)
            printf("{\"op\": \"%s\", \"chains\": %d, \"warps_per_sm\": %d, \"lane_ops_per_sm_clk\": %.4f, "
                   "\"gops\": %.1f, \"ms\": %.3f}\n",
                   s.op, s.chains, s.threads / 32 * s.ctas_per_sm, r, ops_s / 1e9, ms);
        if (r > best) {
            best = r;
            best_ops_s = ops_s;
            best_s = &s;
        }
    }
    // one active lane, and the dependent-chain latency (one warp of one lane per SM)
    const double one_lane = measure(Shape{"dfma", stream_ops<8, 0>, 8, 128, 1, 1}, 4096, nullptr, nullptr);
    const double chain = measure(Shape{"dfma", stream_ops<1, 0>, 1, 32, 1, 1}, 4096, nullptr, nullptr);
    const double lop = measure(Shape{"lop3", stream_int<8, 0>, 8, 512, 1, 32}, 4096, nullptr, nullptr);
    const double shf = measure(Shape{"shf", stream_int<8, 1>, 8, 512, 1, 32}, 4096, nullptr, nullptr);
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    printf("{\"device\": \"%s\", \"sms\": %d, \"max_sm_mhz\": %.0f, \"shapes_swept\": %zu, "
           "\"fp64_lane_ops_per_sm_clk\": %.4f, \"best_shape\": {\"op\": \"%s\", \"chains\": %d, "
           "\"warps_per_sm\": %d}, \"fp64_gops_measured\": %.1f, \"fp64_gops_at_max_clock\": %.1f, "
           "\"one_active_lane_lane_ops_per_sm_clk\": %.4f, \"dependent_dfma_latency_clk\": %.1f, "
           "\"int_lop3_lane_ops_per_sm_clk\": %.2f, \"int_shf_lane_ops_per_sm_clk\": %.2f}\n",
           p.name, g_nsm, clk_khz / 1e3, shapes.size(), best, best_s ? best_s->op : "", best_s ? best_s->chains : 0,
           best_s ? best_s->threads / 32 * best_s->ctas_per_sm : 0, best_ops_s / 1e9, best * g_nsm * clk_khz / 1e6,
           one_lane, chain > 0 ? 1.0 / chain : 0.0, lop, shf);
    return 0;
}
