// d3gb_peaks.cu -- measured arithmetic rates of the GPU, the denominators of the
// rooflines that bench.py reports for the pair passes (FP32 FMA lanes, FP64 FMA
// lanes, MUFU reciprocals per second).
//
// Each rate is taken from a kernel of independent dependency chains (8 per
// thread, enough to keep the pipe full) over 8 resident blocks of 256 threads
// per SM, timed with events on the given stream, best of 3 runs.  Every loop
// has a fixed trip count; the results are written to a small device buffer so
// that the chains are not removed by the compiler.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/d3gb.h"

namespace {

constexpr int kIters = 1024;

__global__ void __launch_bounds__(256) k_ffma(float* out, float a) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j);
    for (int k = 0; k < kIters; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, 1.0f);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_dfma(double* out, double a) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (double)(threadIdx.x + j);
    for (int k = 0; k < kIters / 16; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, 1.0);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_mufu(float* out, float a) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j + 1);
    for (int k = 0; k < kIters / 4; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float r;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[j]));
            x[j] = r + a;
        }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" d3_status d3_peak_rates(double* rates, void* stream) {
    if (!rates) return D3_ERR_ARG;
    for (int k = 0; k < 3; ++k) rates[k] = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return D3_ERR_CUDA;
    const int blocks = 8 * sms, threads = 256;
    const size_t n = (size_t)blocks * threads;
    double* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, n * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // lane operations per launch: FP32 and MUFU 8 chains x iterations, FP64 the same / 16
    const double ops[3] = {(double)n * 8 * kIters, (double)n * 8 * (kIters / 16), (double)n * 8 * (kIters / 4)};
    for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
            e = cudaEventRecord(e0, st);
            if (kind == 0) k_ffma<<<blocks, threads, 0, st>>>((float*)buf, 0.999f);
            else if (kind == 1) k_dfma<<<blocks, threads, 0, st>>>(buf, 0.999);
            else k_mufu<<<blocks, threads, 0, st>>>((float*)buf, 0.5f);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
        }
        if (e == cudaSuccess) rates[kind] = ops[kind] / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    return e == cudaSuccess ? D3_OK : D3_ERR_CUDA;
}
