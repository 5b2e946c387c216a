// Measured FP32 pipe throughput of the current device (include/mmpc_peaks.h).
//
// Each kernel runs 8 independent dependent chains per thread for ITERS steps
// (with 64 warps per SM, 16 per scheduler, this covers the pipe latency) and
// writes one value per thread, so nothing is dead code; grids are 8 CTAs of
// 256 threads per SM, and every write index is below grid x block, the
// buffer's length.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/mmpc.h"
#include "../../include/mmpc_peaks.h"

namespace {

constexpr int ITERS = 4096;
constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 8;

__global__ void __launch_bounds__(THREADS) peak_ffma_kernel(float* out, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = (float)(threadIdx.x + j);
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) peak_ffma2_kernel(float* out, float a, float b)
{
    float2 x[CHAINS];
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = make_float2((float)(threadIdx.x + j), (float)(threadIdx.x + j) + 0.5f);
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) x[j] = __ffma2_rn(x[j], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j].x + x[j].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) peak_rsqrt_kernel(float* out, float a)
{
    float x[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = (float)(threadIdx.x + j + 1);
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) x[j] = rsqrtf(x[j]) + a;
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mmpc_measure_peaks(mmpc_peaks* out, int reps, void* stream)
{
    if (!out || reps < 1) return MMPC_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, clk = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess || sms < 1) return MMPC_ERR_CUDA;
    const int blocks = sms * CTAS_PER_SM;
    float* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&buf, sizeof(float) * (size_t)blocks * THREADS);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best[3] = {1e30f, 1e30f, 1e30f};
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {  // the first round warms up
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            cudaEventRecord(e0, st);
            if (k == 0) peak_ffma_kernel<<<blocks, THREADS, 0, st>>>(buf, 0.999f, 0.001f);
            else if (k == 1) peak_ffma2_kernel<<<blocks, THREADS, 0, st>>>(buf, 0.999f, 0.001f);
            else peak_rsqrt_kernel<<<blocks, THREADS, 0, st>>>(buf, 0.5f);
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && r > 0) best[k] = std::min(best[k], ms);
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return MMPC_ERR_CUDA;
    const double lanes = (double)blocks * THREADS * ITERS * CHAINS;  // lane operations per kernel (FFMA2: x 2)
    out->ffma = lanes / (best[0] * 1e-3);
    out->ffma2 = 2.0 * lanes / (best[1] * 1e-3);
    out->rsqrt = lanes / (best[2] * 1e-3);
    out->ms_ffma = best[0];
    out->ms_ffma2 = best[1];
    out->ms_rsqrt = best[2];
    out->sms = sms;
    out->clock_khz = clk;
    return MMPC_OK;
}
