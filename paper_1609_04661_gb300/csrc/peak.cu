// FP32 fused multiply-add throughput of this GPU, measured: the denominator
// of the ALU rooflines the benchmark reports for the kernels that are bound
// by instruction issue rather than by memory (the projector, the
// back-projector, blocked TV).  One FFMA is one warp instruction per 32
// lanes, so the same figure is the FP32 issue peak.
//
// Every thread runs kChains independent FMA chains (enough to cover the FMA
// pipe's latency) for `iters` unrolled rounds on operands the compiler
// cannot fold, and writes a sum so that nothing is eliminated.  The grid is
// blocks_per_sm blocks of 256 threads on every SM.  A second kernel runs the
// chains as packed FP32 pairs, which on this GPU reach the same FMA rate:
// the pairs save issue slots, they do not raise the peak.  Nothing here
// changes a clock or any other setting of the GPU.
#include "internal.cuh"

namespace dgct {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads)
k_fma_peak(float a, float b, int iters, float* __restrict__ out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // every chain stays in (0, 0.3) for the operands used, so this never
    // stores; it keeps the chains live
    if (s > 1234.5f) out[blockIdx.x] = s;
}

// The same chains as packed FP32 pairs (__ffma2_rn, two FMAs per
// instruction): whether the pairs raise the FMA rate or only save issue slots.
__global__ void __launch_bounds__(kPeakThreads)
k_fma2_peak(float a, float b, int iters, float* __restrict__ out) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)(threadIdx.x + c) * 2e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s > 1234.5f) out[blockIdx.x] = s;
}

template <bool PACKED>
static int measure(int32_t reps, double* h_tflops, int32_t* h_sms, cudaStream_t st) {
    if (!h_tflops || reps < 1) return DGAMP_CT_ERR_INVALID_ARG;
    const void* kfn = PACKED ? (const void*)k_fma2_peak : (const void*)k_fma_peak;
    int dev = 0, sms = 0, per_sm = 0;
    DGCT_CUDA(cudaGetDevice(&dev));
    DGCT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DGCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kPeakThreads, 0));
    if (sms < 1 || per_sm < 1) return DGAMP_CT_ERR_CUDA;
    if (h_sms) *h_sms = sms;
    const int grid = sms * per_sm;
    const int iters = 4096;
    // a < 1 and b > 0: x <- a x + b stays between 0 and its start (< 0.3)
    const float a = 0.99999905f, b = 1e-7f;
    float* sink = nullptr;
    DGCT_CUDA(cudaMalloc((void**)&sink, (size_t)grid * sizeof(float)));
    auto launch = [&](int it) {
        if (PACKED)
            k_fma2_peak<<<grid, kPeakThreads, 0, st>>>(a, b, it, sink);
        else
            k_fma_peak<<<grid, kPeakThreads, 0, st>>>(a, b, it, sink);
    };
    launch(64);   // warm-up
    cudaError_t e = cudaGetLastError();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        launch(iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e);
    const double flop = (PACKED ? 4.0 : 2.0) * kChains * 16.0 * iters * (double)grid * kPeakThreads * reps;
    *h_tflops = flop / ((double)ms * 1e-3) / 1e12;
    return DGAMP_CT_OK;
}

}  // namespace dgct

using namespace dgct;

extern "C" int dgamp_ct_measure_fp32_peak(int32_t reps, double* h_tflops, int32_t* h_sms, void* stream) {
    return measure<false>(reps, h_tflops, h_sms, (cudaStream_t)stream);
}

extern "C" int dgamp_ct_measure_fp32x2_peak(int32_t reps, double* h_tflops, int32_t* h_sms, void* stream) {
    return measure<true>(reps, h_tflops, h_sms, (cudaStream_t)stream);
}
