// Arithmetic-peak probe of the GPU the library runs on: the FP32, packed
// FP32x2 and FP64 fused multiply-add rates that the operator's roofline is
// judged against (the HBM copy rate is measured outside the library).
//
// Every thread runs NCHAIN independent multiply-add chains; the grid holds
// 8 blocks of 256 threads per SM.  The kernel is timed with CUDA events on
// the default stream (best of 3 after one warm-up) and the rate counts 2
// flops per FMA lane.
#include "bk_common.cuh"

namespace {

constexpr int NCHAIN = 8;

__global__ void k_fma32(float* out, float a, float b, int n) {
    float acc[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) acc[c] = fmaf(acc[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += acc[c];
    if (s == 12345.678f) out[threadIdx.x] = s;  // keeps the chains live
}

__global__ void k_fma32x2(float* out, float a, float b, int n) {
    unsigned long long acc[NCHAIN], va, vb;
    asm("mov.b64 %0, {%1, %1};" : "=l"(va) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(vb) : "f"(b));
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) {
        const float lo = threadIdx.x * 1e-3f + c, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(acc[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(va), "l"(vb));
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[c]));
        s += lo + hi;
    }
    if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void k_fma64(double* out, double a, double b, int n) {
    double acc[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) acc[c] = fma(acc[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += acc[c];
    if (s == 12345.678) out[threadIdx.x] = s;
}

}  // namespace

extern "C" bk_status bk_probe_peak(int kind, int device, double* tflops) {
    if (!tflops || kind < 0 || kind > 2) {
        bk_set_error("bk_probe_peak: kind must be 0 (FP32), 1 (FP32x2) or 2 (FP64)");
        return BK_ERR_INVALID_ARG;
    }
    BK_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    BK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int threads = 256, blocks = 8 * sms;
    const int n = kind == 2 ? 1 << 12 : 1 << 16;
    void* buf = nullptr;
    BK_CUDA_TRY(cudaMalloc(&buf, threads * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        if (kind == 0) k_fma32<<<blocks, threads>>>((float*)buf, 0.999f, 1e-4f, n);
        else if (kind == 1) k_fma32x2<<<blocks, threads>>>((float*)buf, 0.999f, 1e-4f, n);
        else k_fma64<<<blocks, threads>>>((double*)buf, 0.999, 1e-4, n);
        cudaEventRecord(e1, 0);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    BK_CUDA_TRY(err);
    const double lanes = (double)blocks * threads * NCHAIN * n * (kind == 1 ? 2.0 : 1.0);
    *tflops = 2.0 * lanes / (best * 1e-3) / 1e12;
    return BK_OK;
}
