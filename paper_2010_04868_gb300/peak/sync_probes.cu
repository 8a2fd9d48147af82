// Latency probes behind the design of the split-tiled and wavefront kernels: what one
// shared-memory level loop with a CTA barrier per level costs, and how the FP64 pipe is shared
// between the warps of an SM. Timed with clock64() (SM clocks). Prints one JSON object.
//
//   level_loop: a 1D 3-point stencil level (three shared loads, DMUL + two dependent DFMA, one
//               store per point) followed by __syncthreads(), repeated; clocks per level for a
//               given number of points per CTA, threads per CTA and CTAs (one grid wave)
//   chain:      one warp doing 16 dependent DFMAs per batch between barriers, alone and with
//               other warps of the CTA issuing 16 independent DMUL + DFMA pairs per batch
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__); exit(1); } } while (0)

__global__ void level_loop(double* out, long long* cyc, int pts, int levels, double a, double b, double c)
{
    __shared__ double s[2][1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        s[0][i] = i * 1e-3;
        s[1][i] = 0;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int k = 1; k <= levels; ++k) {
        const double* src = s[(k - 1) & 1];
        double* dst = s[k & 1];
        for (int i = 1 + threadIdx.x; i <= pts; i += blockDim.x) {
            double acc = __dmul_rn(a, src[i + 1]);
            acc = __fma_rn(b, src[i], acc);
            acc = __fma_rn(c, src[i - 1], acc);
            dst[i] = acc;
        }
        __syncthreads();
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        cyc[blockIdx.x] = t1 - t0;
        out[blockIdx.x] = s[levels & 1][5];
    }
}

__global__ void chain(double* out, long long* cyc, int batches, int loaders, double w0, double w1, double w2)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double nw = lane * 1e-3, acc[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) acc[d] = (lane + d) * 1e-4;
    __syncthreads();
    const long long t0 = clock64();
    for (int m = 0; m < batches; ++m) {
        if (warp == 0) {
#pragma unroll
            for (int d = 0; d < 16; ++d) nw = __fma_rn(w2, nw, acc[d]);
        } else if (warp <= loaders) {
#pragma unroll
            for (int d = 0; d < 16; ++d) acc[d] = __fma_rn(w1, acc[d], __dmul_rn(w0, acc[d]));
        }
        __syncthreads();
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
    double s = nw;
#pragma unroll
    for (int d = 0; d < 16; ++d) s += acc[d];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
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
    CK(cudaMalloc(&dout, sizeof(double) * 8 * nsm * 256));
    CK(cudaMalloc(&dcyc, sizeof(long long) * 8 * nsm));
    printf("{\"device\": \"%s\", \"level_loop\": [", p.name);
    // points per CTA x threads x CTAs per SM: one CTA of 431 points per SM is the 1D heat grid (65536 / 152)
    const int cfg[][3] = {{100, 128, 1}, {100, 128, 4}, {200, 256, 2}, {431, 512, 1}, {54, 128, 8}};
    for (int q = 0; q < 5; ++q) {
        const int pts = cfg[q][0], thr = cfg[q][1], blocks = cfg[q][2] * nsm, levels = 200;
        level_loop<<<blocks, thr>>>(dout, dcyc, pts, levels, 0.25, 0.5, 0.25);
        CK(cudaDeviceSynchronize());
        std::vector<long long> c(blocks);
        CK(cudaMemcpy(c.data(), dcyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
        const double clk = median(c) / levels;
        const double lane_ops_per_sm_clk = 3.0 * pts * cfg[q][2] / clk;
        printf("%s{\"points_per_cta\": %d, \"threads\": %d, \"ctas_per_sm\": %d, \"clk_per_level\": %.0f, "
               "\"fp64_lane_ops_per_sm_clk\": %.3f}",
               q ? ", " : "", pts, thr, cfg[q][2], clk, lane_ops_per_sm_clk);
    }
    printf("], \"chain\": [");
    const int loaders[] = {0, 1, 3, 6};
    for (int q = 0; q < 4; ++q) {
        const int batches = 20000;
        chain<<<nsm, 256>>>(dout, dcyc, batches, loaders[q], 0.25, 0.5, 0.25);
        CK(cudaDeviceSynchronize());
        std::vector<long long> c(nsm);
        CK(cudaMemcpy(c.data(), dcyc, sizeof(long long) * nsm, cudaMemcpyDeviceToHost));
        printf("%s{\"loader_warps\": %d, \"clk_per_batch_of_16_dependent_dfma\": %.0f}", q ? ", " : "", loaders[q],
               median(c) / batches);
    }
    printf("]}\n");
    return 0;
}
