// FP32 throughput of this GPU's CUDA cores, measured: the denominator of the
// FP32-pipe fractions that are reported beside the HBM roofline (the FFT
// passes and the ring epilogue are bound by arithmetic and latency, not by
// DRAM).  Each thread runs CHAINS independent dependency chains of fused
// multiply-adds (scalar, or on packed FP32 pairs), x <- x a + b with
// |a| < 1, so that the values stay normal; one FMA is two flops, one packed
// FMA four.
#include <cuda_runtime.h>

#include "../../include/lenia.h"
#include "lenia_internal.cuh"

namespace lenia {

constexpr int PEAK_CHAINS = 8;

template <bool PAIR>
__global__ void __launch_bounds__(256) k_fma_peak(float* out, int iters, float a, float b)
{
    const float seed = 1e-3f * (float)(threadIdx.x + 1);
    if constexpr (PAIR) {
        float2 x[PEAK_CHAINS];
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) x[c] = make_float2(seed + c, seed - c);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; c++) x[c] = __ffma2_rn(x[c], a2, b2);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) s += x[c].x + x[c].y;
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else {
        float x[PEAK_CHAINS];
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) x[c] = seed + c;
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; c++) x[c] = fmaf(x[c], a, b);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) s += x[c];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

// Best of `reps` timed launches of each form, in TFLOP/s.
cudaError_t measure_fp32_peak(cudaStream_t s, double* scalar_tflops, double* pair_tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256, iters = 4096, reps = 5;
    float* out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    double best[2] = {0.0, 0.0};
    for (int form = 0; form < 2 && e == cudaSuccess; form++) {
        for (int r = 0; r <= reps && e == cudaSuccess; r++) {          // the first launch warms up
            e = cudaEventRecord(t0, s);
            if (form == 0) k_fma_peak<false><<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);
            else k_fma_peak<true><<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && r > 0 && ms > 0.f) {
                const double flops = (double)blocks * threads * iters * PEAK_CHAINS * (form == 0 ? 2.0 : 4.0);
                const double tf = flops / (ms * 1e-3) / 1e12;
                if (tf > best[form]) best[form] = tf;
            }
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (out) cudaFree(out);
    *scalar_tflops = best[0];
    *pair_tflops = best[1];
    return e;
}

}  // namespace lenia

extern "C" lenia_status lenia_measure_fp32_peak(double* scalar_tflops, double* pair_tflops, void* stream)
{
    if (!scalar_tflops || !pair_tflops) return LENIA_EINVAL;
    return lenia::measure_fp32_peak((cudaStream_t)stream, scalar_tflops, pair_tflops) == cudaSuccess ? LENIA_OK
                                                                                                     : LENIA_ECUDA;
}
