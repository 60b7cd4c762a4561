// osc_probe.cu -- the FP32 FMA throughput of the device, the peak the FP32
// path's roofline is measured against (the vendor's figure assumes the
// maximum clock; under an FMA load the clock settles lower).
#include <algorithm>

#include "osc_internal.h"

namespace osc {

// Eight independent FMA chains per thread (enough instruction-level
// parallelism to hide the FMA latency at any occupancy), unrolled 16 times per
// iteration; the result is stored so the chains cannot be removed.
__global__ void __launch_bounds__(256) k_fma_peak(float *out, float a, float b, int iters) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-7f + k * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace osc

using namespace osc;

extern "C" osc_status osc_measure_fp32_peak(int device, double *tflops) {
    if (!tflops) return OSC_E_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return OSC_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return OSC_E_ARG;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = std::max(sms, 1) * 8, threads = 256, iters = 4096;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
    if (!e) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    double best = 0.0;
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    for (int rep = 0; rep < 7 && !e; ++rep) {
        e = cudaEventRecord(e0, st);
        k_fma_peak<<<blocks, threads, 0, st>>>(out, 0.9999999f, 1e-7f, iters);
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e1, st);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e && rep >= 2 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // two warm-up launches
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    if (e) return OSC_E_CUDA;
    *tflops = best;
    return OSC_OK;
}
