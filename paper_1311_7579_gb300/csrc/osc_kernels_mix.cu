// Histogram and reweight kernel instantiations for one precision (FP64 eigen-solve, FP32 amplitude).
#include "osc_kernels.cuh"
#include "osc_launch.h"

namespace osc {

const void *hist_kernel_fn_mix(int pt) {
    switch (pt) {
        case 1: return (const void *)k_hist<kMix, 1>;
        case 4: return (const void *)k_hist<kMix, 4>;
        case 16: return (const void *)k_hist<kMix, 16>;
        case 64: return (const void *)k_hist<kMix, 64>;
        case 256: return (const void *)k_hist<kMix, 256>;
        default: return nullptr;
    }
}

cudaError_t launch_hist_mix(int pt, const HistParams &p, int grid, cudaStream_t st) {
    switch (pt) {
        case 1: k_hist<kMix, 1><<<grid, kNT, 0, st>>>(p); break;
        case 4: k_hist<kMix, 4><<<grid, kNT, 0, st>>>(p); break;
        case 16: k_hist<kMix, 16><<<grid, kNT, 0, st>>>(p); break;
        case 64: k_hist<kMix, 64><<<grid, kNT, 0, st>>>(p); break;
        case 256: k_hist<kMix, 256><<<grid, kNT, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reweight_mix(const ReweightParams &p, cudaStream_t st) {
    int64_t blocks = (p.s.n + 255) / 256;
    if (blocks > device_sms() * 16) blocks = device_sms() * 16;
    k_reweight<kMix><<<(int)blocks, 256, 0, st>>>(p);
    return cudaGetLastError();
}

const void *redo_kernel_fn_mix() { return (const void *)k_redo<kMix>; }

}  // namespace osc
