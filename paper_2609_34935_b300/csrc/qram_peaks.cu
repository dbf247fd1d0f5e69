// Roofline denominators measured on the device: the throughput of FP64
// fused multiply-adds and of 32-bit integer add/logic instructions.  The
// trajectory kernel is neither a dense contraction nor bandwidth bound; its
// instruction mix is integer bit arithmetic with some FP64, so these two
// rates, taken on the same GPU, are the peaks its work is compared with.
// A measurement utility; the simulation method has no counterpart.
#include <cuda_runtime.h>

#include "../../include/qram_sim.h"

namespace {

constexpr int kChains = 8;     // independent dependency chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

// x <- x * b + c on kChains independent chains: 2 FLOP per FMA
__global__ void __launch_bounds__(kThreads) dfma_peak_kernel(double *out, int iters, double b, double c) {
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 1e-3 * (double)(threadIdx.x + 37 * q);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;     // keeps every chain live
}

// x <- x ^ (x + k) on kChains independent chains: one add and one logic
// instruction, 2 integer ops per step
__global__ void __launch_bounds__(kThreads) int_peak_kernel(uint32_t *out, int iters, uint32_t k) {
    uint32_t x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = threadIdx.x * 2654435761u + (uint32_t)q;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] ^= x[q] + (k + (uint32_t)q);
    }
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s ^= x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (after one untimed), in seconds
template <typename F>
cudaError_t time_best(F launch, int reps, float *best_ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    launch();
    *best_ms = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < *best_ms) *best_ms = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" int qram_measure_peaks(int device, double *fp64_flops, double *int32_ops) {
    if (!fp64_flops || !int32_ops) return QRAM_E_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return QRAM_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return QRAM_E_CUDA;
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_peak_kernel, kThreads, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    void *buf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)grid * kThreads * sizeof(double));
    const int iters_fp = 1 << 14, iters_int = 1 << 16;
    float ms_fp = 0.f, ms_int = 0.f;
    if (e == cudaSuccess)
        e = time_best([&] { dfma_peak_kernel<<<grid, kThreads>>>((double *)buf, iters_fp, 0.9999999, 1e-7); }, 5,
                      &ms_fp);
    if (e == cudaSuccess)
        e = time_best([&] { int_peak_kernel<<<grid, kThreads>>>((uint32_t *)buf, iters_int, 0x9E3779B9u); }, 5,
                      &ms_int);
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return QRAM_E_CUDA;
    const double lanes = (double)grid * kThreads * kChains;
    *fp64_flops = 2.0 * lanes * iters_fp / (ms_fp * 1e-3);
    *int32_ops = 2.0 * lanes * iters_int / (ms_int * 1e-3);
    return QRAM_OK;
}
