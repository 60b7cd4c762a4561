// Histogram and reweight kernel instantiations for one precision (fp32).
#include "osc_kernels.cuh"
#include "osc_launch.h"

namespace osc {

// With its constants read in place rather than held in registers it fits five
// 128-thread blocks per SM (20 warps) without spilling, where k_hist<FP32, 1> fits four.
constexpr int kInlineMinBlocks = 5;
__global__ void __launch_bounds__((hist_block_threads<kFP32, 1>()), kInlineMinBlocks)
    k_hist_inline(const HistParams prm, const __grid_constant__ PointInline pin) {
    grid_dependents_launch();
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < C32_STRIDE; i += blockDim.x) const_cast<float *>(prm.pc32)[i] = pin.c32[i];
        for (int i = threadIdx.x; i < C64_STRIDE; i += blockDim.x) const_cast<double *>(prm.pc64)[i] = pin.c64[i];
    }
    hist_items_per_warp<kFP32>(prm, pin.c32);
    if (prm.fuse_final && !prm.redo) fused_final_warp(prm);
}

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

const void *hist_inline_kernel_fn() { return (const void *)k_hist_inline; }
size_t point_inline_bytes() { return sizeof(PointInline); }
int hist_inline_blocks_per_sm() {
    static int per_sm = 0;  // the same on every device of a process (one GPU model)
    if (!per_sm) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hist_inline, hist_block_threads<kFP32, 1>(), 0);
        per_sm = n > 0 ? n : 1;
    }
    return per_sm;
}

}  // namespace osc
