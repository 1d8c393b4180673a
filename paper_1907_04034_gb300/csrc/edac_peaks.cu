// edac_fma_peak: the FMA-pipe peak of the current GPU, measured with FMA chains.
//
// The roofline of the pair passes is the FP32 pipe (mixed path) or the FP64 pipe (fp64 path),
// so the peak used as denominator is measured on the device, at the clocks it runs under load,
// instead of being taken from a data sheet.  Each thread runs 8 independent FMA chains
// (a <- a b + c, with 0 < b < 1 and c > 0 so the values stay bounded and positive); enough
// blocks are resident on every SM to hide the FMA latency.  FP32 is measured with scalar FFMA
// and with the paired FFMA2 form (two FMAs per instruction), and the larger rate is the peak.
// A flop is counted as 2 per FMA.
#include <algorithm>

#include "edac.h"

namespace {

static __device__ float g_sink_f;
static __device__ double g_sink_d;

constexpr int CHAINS = 8;
constexpr int PK_TPB = 256;

__global__ void __launch_bounds__(PK_TPB) k_fma32(int iters, float b, float c)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s < 0.0f) g_sink_f = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(PK_TPB) k_fma32x2(int iters, float b, float c)
{
    float2 a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        a[k] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + k), 1.5f + 1e-3f * (float)k);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k].x + a[k].y;
    if (s < 0.0f) g_sink_f = s;
}

__global__ void __launch_bounds__(PK_TPB) k_fma64(int iters, double b, double c)
{
    double a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s < 0.0) g_sink_d = s;
}

// launch form f (0 fp32, 1 fp32 paired, 2 fp64) with `iters` iterations; returns ms, < 0 on error
float run_once(int f, int blocks, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0f;
    if (f == 0) k_fma32<<<blocks, PK_TPB, 0, st>>>(iters, 0.999999f, 1e-6f);
    else if (f == 1) k_fma32x2<<<blocks, PK_TPB, 0, st>>>(iters, 0.999999f, 1e-6f);
    else k_fma64<<<blocks, PK_TPB, 0, st>>>(iters, 0.999999999, 1e-9);
    if (cudaGetLastError() != cudaSuccess) return -1.0f;
    if (cudaEventRecord(e1, st) != cudaSuccess) return -1.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
    return ms;
}

// best rate (TFLOP/s) of form f over 3 launches of about target_ms each
double measure(int f, cudaStream_t st, double target_ms, cudaEvent_t e0, cudaEvent_t e1)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
    const void *fn = f == 0 ? (const void *)k_fma32 : (f == 1 ? (const void *)k_fma32x2 : (const void *)k_fma64);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PK_TPB, 0) != cudaSuccess) return -1.0;
    const int blocks = sms * std::max(per_sm, 1);
    const double fma_per_iter = (double)blocks * PK_TPB * CHAINS * (f == 1 ? 2.0 : 1.0);
    // calibrate: grow the iteration count until one launch takes >= 2 ms
    int iters = 256;
    float ms = 0.0f;
    for (;;) {
        ms = run_once(f, blocks, iters, st, e0, e1);
        if (ms < 0.0f) return -1.0;
        if (ms >= 2.0f || iters >= (1 << 28)) break;
        iters *= 4;
    }
    const double scale = target_ms / std::max((double)ms, 1e-3);
    iters = (int)std::min(std::max((double)iters * scale, 256.0), (double)(1 << 28));
    double best = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        ms = run_once(f, blocks, iters, st, e0, e1);
        if (ms <= 0.0f) return -1.0;
        best = std::max(best, 2.0 * fma_per_iter * (double)iters / ((double)ms * 1e-3) * 1e-12);
    }
    return best;
}

}  // namespace

extern "C" edac_status edac_fma_peak(int kind, void *cuda_stream, double *tflops)
{
    if (!tflops || (kind != EDAC_PEAK_FP32 && kind != EDAC_PEAK_FP64)) return EDAC_E_INVALID;
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EDAC_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EDAC_E_CUDA;
    }
    double r;
    if (kind == EDAC_PEAK_FP32) {
        const double r1 = measure(0, st, 30.0, e0, e1);
        const double r2 = r1 < 0 ? -1.0 : measure(1, st, 30.0, e0, e1);
        r = (r1 < 0 || r2 < 0) ? -1.0 : std::max(r1, r2);
    } else {
        r = measure(2, st, 30.0, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r < 0) return EDAC_E_CUDA;
    *tflops = r;
    return EDAC_OK;
}
