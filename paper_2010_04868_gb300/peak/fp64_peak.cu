// FP64 pipe micro-benchmark: the ALU roofline the stencil kernels are measured against.
// Also the 32-bit integer logic (LOP3) and funnel-shift (SHF) rates, the roofline of the
// bit-packed Game of Life kernels.
//
// Streams of independent __fma_rn / __dadd_rn / __dmul_rn on every resident
// warp, timed with clock64() per CTA (SM clocks, so the result is a per-clock
// rate independent of the clock the GPU happened to run at) and with CUDA
// events. Also: the dependent-chain latency of one DFMA, and the cost of a
// warp instruction with only some lanes active. Prints one JSON object.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__); exit(1); } } while (0)

template <int CH, int OP>
__global__ void stream_ops(double* out, long long* cyc, int iters, double a, double b, int active)
{
    if ((int)(threadIdx.x & 31) >= active) return;
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-9 + c * 0.1;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (OP == 0) x[c] = __fma_rn(x[c], a, b);
            else if (OP == 1) x[c] = __dadd_rn(x[c], b);
            else x[c] = __dmul_rn(x[c], a);
        }
    }
    const long long t1 = clock64();
    double s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// Independent chains of one 3-input logic op (LOP3) or one funnel shift (SHF) per step, written
// in PTX so that the compiler cannot fold the repeated bitwise operations.
template <int CH, int OP>
__global__ void stream_int(double* out, long long* cyc, int iters, double fa, double fb, int active)
{
    if ((int)(threadIdx.x & 31) >= active) return;
    const unsigned a = (unsigned)(fa * 1e7) | 1u, b = (unsigned)(fb * 1e9) + 3u;
    unsigned x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 7u + c;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (OP == 0)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(a), "r"(b));
            else
                asm volatile("shf.l.wrap.b32 %0, %0, %1, 1;" : "+r"(x[c]) : "r"(b));
        }
    }
    const long long t1 = clock64();
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s ^= x[c];
    if (s == 0x12345678u) out[0] = s;
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

static double median(std::vector<long long> v)
{
    std::sort(v.begin(), v.end());
    return (double)v[v.size() / 2];
}

int main()
{
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    const int nsm = p.multiProcessorCount;
    double* dout;
    long long* dcyc;
    CK(cudaMalloc(&dout, 64));
    CK(cudaMalloc(&dcyc, 8 * 4096));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // per-SM rate: 4 warps (one per SM sub-partition) x 8 chains, one CTA per SM
    auto rate = [&](auto kern, int threads, int iters, int chains, int active, double& ops_per_s) {
        kern<<<nsm, threads>>>(dout, dcyc, iters / 8, 1.0000001, 1e-7, active);
        CK(cudaDeviceSynchronize());
        CK(cudaEventRecord(e0));
        kern<<<nsm, threads>>>(dout, dcyc, iters, 1.0000001, 1e-7, active);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        std::vector<long long> c(nsm);
        CK(cudaMemcpy(c.data(), dcyc, 8 * nsm, cudaMemcpyDeviceToHost));
        const double warps = threads / 32.0;
        const double lane_ops_per_sm = warps * (active < 32 ? active : 32) * (double)iters * chains;
        ops_per_s = lane_ops_per_sm * nsm / (ms * 1e-3);
        return lane_ops_per_sm / median(c);  // lane operations per SM clock
    };
    double s_fma, s_add, s_mul, s_lat, s_one;
    const double fma_clk = rate(stream_ops<8, 0>, 128, 4096, 8, 32, s_fma);
    const double add_clk = rate(stream_ops<8, 1>, 128, 4096, 8, 32, s_add);
    const double mul_clk = rate(stream_ops<8, 2>, 128, 4096, 8, 32, s_mul);
    const double one_lane_clk = rate(stream_ops<8, 0>, 128, 4096, 8, 1, s_one);
    const double chain_clk = rate(stream_ops<1, 0>, 32, 4096, 1, 1, s_lat);  // 1 lane, dependent chain
    double s_lop, s_shf;
    const double lop_clk = rate(stream_int<8, 0>, 512, 4096, 8, 32, s_lop);  // 16 warps: the integer pipes are wider
    const double shf_clk = rate(stream_int<8, 1>, 512, 4096, 8, 32, s_shf);
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    printf("{\"device\": \"%s\", \"sms\": %d, \"max_sm_mhz\": %.0f, "
           "\"fp64_fma_lane_ops_per_sm_clk\": %.4f, \"fp64_add_lane_ops_per_sm_clk\": %.4f, "
           "\"fp64_mul_lane_ops_per_sm_clk\": %.4f, \"fp64_fma_gops_measured\": %.1f, "
           "\"fp64_fma_gops_at_max_clock\": %.1f, \"one_active_lane_lane_ops_per_sm_clk\": %.4f, "
           "\"dependent_dfma_latency_clk\": %.1f, \"int_lop3_lane_ops_per_sm_clk\": %.2f, "
           "\"int_shf_lane_ops_per_sm_clk\": %.2f, \"int_lop3_gops_measured\": %.1f}\n",
           p.name, nsm, clk_khz / 1e3, fma_clk, add_clk, mul_clk, s_fma / 1e9, fma_clk * nsm * clk_khz / 1e6,
           one_lane_clk, 1.0 / chain_clk, lop_clk, shf_clk, s_lop / 1e9);
    return 0;
}
