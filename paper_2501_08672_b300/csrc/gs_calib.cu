// Throughput microbenchmarks of the FP32 FMA pipe and of the MUFU ex2 unit
// on the current device: the measured denominators of the compositing
// kernels' ALU roofline (the nominal one is SMs x 128 lanes x 2 FLOP x the
// maximum SM clock).  Each thread runs kChains independent dependency
// chains so that latency is hidden at full occupancy; the results are kept
// live by a store that never happens.
#include "gs_internal.cuh"

namespace gsb {

namespace {

constexpr int kCalThreads = 256;
constexpr int kCalBlocksPerSM = 8;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kCalThreads) k_ffma_rate(int iters, float a, float b, float* sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.f) *sink = s;  // a, b > 0 keep every chain positive
}

__global__ void __launch_bounds__(kCalThreads) k_ex2_rate(int iters, float* sink) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0.25f + (float)((threadIdx.x + k) & 63) * (1.f / 128.f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = ex2_approx(-x[k]);  // stays in [0.5, 1]
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.f) *sink = s;
}

}  // namespace

cudaError_t measure_alu(int sm_count, float* sink, cudaStream_t s, double* ffma_tflops, double* ex2_gops) {
    const int blocks = sm_count * kCalBlocksPerSM;
    const double threads = (double)blocks * kCalThreads;
    const int ffma_iters = 4096, ex2_iters = 512;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    double best_f = 0.0, best_x = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        float ms = 0.f;
        cudaEventRecord(e0, s);
        k_ffma_rate<<<blocks, kCalThreads, 0, s>>>(ffma_iters, 0.9999f, 1e-4f, sink);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
        const double f = 2.0 * threads * ffma_iters * kUnroll * kChains / (ms * 1e-3) / 1e12;
        if (f > best_f) best_f = f;
        cudaEventRecord(e0, s);
        k_ex2_rate<<<blocks, kCalThreads, 0, s>>>(ex2_iters, sink);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
        const double x = threads * ex2_iters * kUnroll * kChains / (ms * 1e-3) / 1e9;
        if (x > best_x) best_x = x;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ffma_tflops = best_f;
    *ex2_gops = best_x;
    return e;
}

}  // namespace gsb
