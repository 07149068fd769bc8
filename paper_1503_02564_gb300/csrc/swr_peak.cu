// FP64 throughput probes: the denominators of the marches' roofline.
//
// The subdomain marches are bound by FP64 arithmetic, whose rate on this part is
// not a published constant one can trust to a few percent; these kernels measure
// it.  Two paths:
//   kind 0, DFMA: the vector FP64 pipe.  Every thread runs NCH independent
//           fused multiply-add chains x <- x * b + c (b slightly below 1, so the
//           values stay bounded), enough chains per warp to cover the pipe's
//           latency;
//   kind 1, DMMA: the FP64 tensor path, mma.sync.aligned.m8n8k4 (f64 operands,
//           f64 accumulators; 2 * 8 * 8 * 4 = 512 flops per warp instruction), with
//           NACC independent accumulator tiles per warp.
//   kind 2, both at once: every warp issues the DFMA chains and the DMMA tiles of
//           kinds 0 and 1 in each round (do the two paths share one unit?).
// Results are written to a sink so that nothing is optimised away.
#include "swr_internal.cuh"

namespace {

constexpr int NCH = 8;    // independent DFMA chains per thread
constexpr int NACC = 4;   // independent DMMA accumulator tiles per warp

__global__ void __launch_bounds__(256) k_peak_dfma(long long iters, double b, double c,
                                                   double* __restrict__ sink) {
    double x[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void dmma_m8n8k4(double& d0, double& d1, double a, double b,
                                            double c0, double c1) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%4, %5};"
                 : "=d"(d0), "=d"(d1)
                 : "d"(a), "d"(b), "d"(c0), "d"(c1));
}

__global__ void __launch_bounds__(256) k_peak_dmma(long long iters, double b, double c,
                                                   double* __restrict__ sink) {
    const int lane = threadIdx.x & 31;
    // A: 8 x 4 and B: 4 x 8, one element per lane; scaled so that the accumulators,
    // d <- A B + d with |A B| small, stay bounded over many iterations
    const double a = b * (1.0 + 1e-3 * lane);
    const double bb = c * (1.0 - 1e-3 * lane);
    double d0[NACC], d1[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        d0[k] = 1e-3 * (k + 1);
        d1[k] = -1e-3 * (k + 1);
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NACC; ++k) dmma_m8n8k4(d0[k], d1[k], a, bb, d0[k], d1[k]);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NACC; ++k) s += d0[k] + d1[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// kind 2: both at once in every warp, equal flops per round (NCH DFMA chains per
// thread: 64 NCH = 512 flops per warp; one DMMA tile: 512 flops): about twice the
// single-path rate if the two paths are separate units, about the same if shared.
__global__ void __launch_bounds__(256) k_peak_mixed(long long iters, double b, double c,
                                                    double* __restrict__ sink) {
    const int lane = threadIdx.x & 31;
    const double a = 1e-4 * (1.0 + 1e-3 * lane), bb = 1e-4 * (1.0 - 1e-3 * lane);
    double x[NCH], d0 = 1e-3, d1 = -1e-3;
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (long long i = 0; i < iters; ++i) {
        dmma_m8n8k4(d0, d1, a, bb, d0, d1);
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], b, c);
    }
    double s = d0 + d1;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" swr_status swr_fp64_peak(int32_t kind, int64_t iters, int32_t blocks,
                                    int32_t threads, double* sink, double* flops,
                                    float* ms, void* stream) {
    if (kind < 0 || kind > 2 || iters < 1 || blocks < 1 || threads < 32 ||
        threads > 256 || (threads & 31) || !sink || !flops || !ms)
        return SWR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SWR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SWR_ERR_CUDA;
    }
    cudaEventRecord(e0, s);
    if (kind == 0) {
        k_peak_dfma<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7, sink);
        *flops = 2.0 * NCH * (double)iters * (double)blocks * (double)threads;
    } else if (kind == 1) {
        k_peak_dmma<<<blocks, threads, 0, s>>>(iters, 1e-4, 1e-4, sink);
        *flops = 512.0 * NACC * (double)iters * (double)blocks * (double)(threads / 32);
    } else {
        k_peak_mixed<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7, sink);
        *flops = (2.0 * NCH * (double)threads + 512.0 * (double)(threads / 32)) *
                 (double)iters * (double)blocks;
    }
    swr_count_launch(1);
    cudaEventRecord(e1, s);
    swr_status st = SWR_OK;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        st = SWR_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
