// Histogram and reweight kernel instantiations for one precision (fp32).
#include "osc_kernels.cuh"
#include "osc_launch.h"

namespace osc {

const void *hist_kernel_fn_fp32(int pt) {
    switch (pt) {
        case 1: return (const void *)k_hist<kFP32, 1>;
        case 4: return (const void *)k_hist<kFP32, 4>;
        case 16: return (const void *)k_hist<kFP32, 16>;
        case 64: return (const void *)k_hist<kFP32, 64>;
        case 256: return (const void *)k_hist<kFP32, 256>;
        default: return nullptr;
    }
}

cudaError_t launch_hist_fp32(int pt, const HistParams &p, int grid, cudaStream_t st) {
    switch (pt) {
        case 1: k_hist<kFP32, 1><<<grid, hist_block_threads<kFP32, 1>(), 0, st>>>(p); break;
        case 4: k_hist<kFP32, 4><<<grid, kNT, 0, st>>>(p); break;
        case 16: k_hist<kFP32, 16><<<grid, kNT, 0, st>>>(p); break;
        case 64: k_hist<kFP32, 64><<<grid, kNT, 0, st>>>(p); break;
        case 256: k_hist<kFP32, 256><<<grid, kNT, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reweight_fp32(const ReweightParams &p, cudaStream_t st) {
    int64_t blocks = (p.s.n + 255) / 256;
    if (blocks > device_sms() * 16) blocks = device_sms() * 16;
    k_reweight<kFP32><<<(int)blocks, 256, 0, st>>>(p);
    return cudaGetLastError();
}

const void *redo_kernel_fn_fp32() { return (const void *)k_redo<kFP32>; }

}  // namespace osc
