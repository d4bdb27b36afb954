// Throughput probes for the ALU roofline: how many ex2.approx.ftz.f32 (the
// MUFU exponential every interpolation term needs) and how many packed FP32x2
// FMA instructions this GPU retires per second, measured with many independent
// dependency chains at full occupancy. Diagnostics, not a step of the method.
#include "internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ex2(float *sink, int iters) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 0.001f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) {
            // x <- 2^-x stays in (0.5, 1]: one MUFU per step, no other work
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(-x[k]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 12345.f) sink[threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma2(float *sink, int iters) {
    float2 x[PROBE_CHAINS];
    const float2 a = make_float2(0.999f, 0.998f), c = make_float2(1e-3f, 2e-3f);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = make_float2(0.001f * threadIdx.x, 0.002f * k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    if (s == 12345.f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" es_status es_probe_rates(int device, double *ex2_per_s, double *ffma2_per_s) {
    if (!ex2_per_s || !ffma2_per_s) return ES_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return ES_ECUDA;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_ex2, PROBE_THREADS, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 4096;
    float *sink = nullptr;
    if (cudaMalloc(&sink, PROBE_THREADS * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return ES_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_ms = [&](auto kern) {
        kern<<<grid, PROBE_THREADS>>>(sink, 64);   // warm-up
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0);
            kern<<<grid, PROBE_THREADS>>>(sink, iters);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = ms < best ? ms : best;
        }
        return best;
    };
    const double ops = (double)grid * PROBE_THREADS * iters * PROBE_CHAINS;
    const float ms_ex2 = time_ms(k_probe_ex2);
    const float ms_fma = time_ms(k_probe_ffma2);
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return ES_ECUDA;
    *ex2_per_s = ops / (ms_ex2 * 1e-3);
    *ffma2_per_s = ops / (ms_fma * 1e-3);   // packed instructions (two FMAs each)
    return ES_OK;
}
