// probe.cu -- measured arithmetic peaks of the device: throughput of long
// chains of independent fused multiply-adds (FP32 scalar FFMA, FP32 packed
// FFMA2, FP64 DFMA) over the whole GPU, timed with CUDA events. They are the
// denominators of the kick's (FP32 pipe) and the Kepler drift's (FP64 pipe)
// roofline fractions; nothing of the integrator runs here.
#include "qym_internal.cuh"

namespace qym {

// results are kept alive by a store that never happens (a value the chains
// cannot reach), so the chains cost no memory traffic
static __device__ int g_probe_sink;

constexpr int kProbeChains = 8;   // independent accumulators per thread

__global__ void __launch_bounds__(256) k_probe_ffma(int64_t iters, float b, float c) {
    float acc[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc[k] = (float)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) acc[k] = fmaf(acc[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += acc[k];
    if (s == -1.25e-37f) g_probe_sink = 1;
}

__global__ void __launch_bounds__(256) k_probe_ffma2(int64_t iters, float b, float c) {
    float2 acc[kProbeChains];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc[k] = make_float2((float)(threadIdx.x + k), (float)k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) acc[k] = __ffma2_rn(acc[k], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += acc[k].x + acc[k].y;
    if (s == -1.25e-37f) g_probe_sink = 1;
}

__global__ void __launch_bounds__(256) k_probe_dfma(int64_t iters, double b, double c) {
    double acc[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc[k] = (double)(threadIdx.x + k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) acc[k] = fma(acc[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += acc[k];
    if (s == -1.25e-300) g_probe_sink = 1;
}

}  // namespace qym

using namespace qym;

extern "C" qym_status qym_probe_fma(int32_t kind, int64_t iters, int32_t blocks_per_sm,
                                    double *tflops, double *ms, void *stream) {
    if (kind < 0 || kind > 2 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !tflops) {
        set_thread_error("qym_probe_fma: kind 0..2, iters >= 1, 1..8 blocks per SM, tflops != NULL");
        return QYM_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_thread_error(std::string("qym_probe_fma: ") + cudaGetErrorString(e));
        return QYM_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256;
    const int grid = sms * blocks_per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        // b, c keep the chains bounded: a -> a b + c converges to c / (1 - b)
        if (kind == 0) k_probe_ffma<<<grid, threads, 0, st>>>(iters, 0.999f, 0.001f);
        else if (kind == 1) k_probe_ffma2<<<grid, threads, 0, st>>>(iters, 0.999f, 0.001f);
        else k_probe_dfma<<<grid, threads, 0, st>>>(iters, 0.999, 0.001);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float f = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_thread_error(std::string("qym_probe_fma: ") + cudaGetErrorString(e));
        return QYM_ECUDA;
    }
    // two flops per lane and FMA; FFMA2 does two lanes' worth per instruction
    const double lanes = kind == 1 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes * kProbeChains * (double)iters * (double)grid * threads;
    *tflops = flops / ((double)f * 1e-3) / 1e12;
    if (ms) *ms = f;
    return QYM_OK;
}
