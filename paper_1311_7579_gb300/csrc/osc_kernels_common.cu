// Constants and finalize kernels, and the precision dispatch of the launch helpers.
#include <algorithm>

#include "osc_kernels.cuh"
#include "osc_launch.h"

namespace osc {

__global__ void __launch_bounds__(kConstThreads) k_point_consts(const osc_point *pts, int n, float *pc32, double *pc64) {
    grid_dependents_launch();
    const int i = blockIdx.x;
    if (i >= n) return;
    point_consts_block(pts[i], pc32 + (int64_t)i * C32_STRIDE, pc64 + (int64_t)i * C64_STRIDE);
}

// The table is read in place from the parameter space (a grid constant): the
// block's point is selected by a run-time index, which would otherwise make the
// compiler copy it to the thread's stack first.
template <int N>
__global__ void __launch_bounds__(kConstThreads)
    k_point_consts_v(const __grid_constant__ PointsByValueT<N> pv, float *pc32, double *pc64) {
    grid_dependents_launch();
    const int i = blockIdx.x;
    if (i >= pv.n) return;
    point_consts_block(pv.p[i], pc32 + (int64_t)i * C32_STRIDE, pc64 + (int64_t)i * C64_STRIDE);
}

// Converts the exact bins to doubles and clears them for the next launch.  It
// is launched programmatically after the histogram kernel: its blocks may be
// resident before that grid ends, and griddepcontrol.wait returns once the grid
// has completed and its reductions are visible.  Each thread loads the digit
// columns of up to kFinPerThread bins before converting any (one memory round
// trip rather than one per bin).
constexpr int kFinPerThread = 4;
__global__ void __launch_bounds__(256) k_final(const FinalParams f) {
    grid_dependency_wait();
    const int64_t n = f.n_hist * (int64_t)f.nbins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += stride * kFinPerThread) {
        Digits d[kFinPerThread];
#pragma unroll
        for (int k = 0; k < kFinPerThread; ++k) {
            const int64_t i = i0 + k * stride;
            if (i < n) d[k] = load_digits(f.acc, i);
        }
#pragma unroll
        for (int k = 0; k < kFinPerThread; ++k) {
            const int64_t i = i0 + k * stride;
            if (i < n) {
                clear_digits(f.acc, i);
                f.out[i] = final_bin(d[k], f.hmeta + 4 * (i / f.nbins), f.pc64);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *f.counter = 0;
}

const void *redo_kernel_fn_fp32();
const void *redo_kernel_fn_mix();

int device_sms() {
    constexpr int kMaxDev = 64;
    static int cached[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

const void *hist_kernel_fn_fp32(int pt);
const void *hist_kernel_fn_fp64(int pt);
const void *hist_kernel_fn_mix(int pt);
cudaError_t launch_hist_mix(int pt, const HistParams &p, int grid, cudaStream_t st);
cudaError_t launch_reweight_mix(const ReweightParams &p, cudaStream_t st);
cudaError_t launch_hist_fp32(int pt, const HistParams &p, int grid, cudaStream_t st);
cudaError_t launch_hist_fp64(int pt, const HistParams &p, int grid, cudaStream_t st);
cudaError_t launch_reweight_fp32(const ReweightParams &p, cudaStream_t st);
cudaError_t launch_reweight_fp64(const ReweightParams &p, cudaStream_t st);

int hist_threads() { return kNT; }
int hist_threads_for(int prec, int pt) { return (prec == kFP32 && pt == 1) ? hist_block_threads<kFP32, 1>() : kNT; }

const void *hist_kernel_fn(int prec, int pt) {
    return prec == kFP32 ? hist_kernel_fn_fp32(pt) : prec == kMix ? hist_kernel_fn_mix(pt) : hist_kernel_fn_fp64(pt);
}

const void *final_kernel_fn() { return (const void *)k_final; }

cudaError_t launch_point_consts(const osc_point *d_pts, int n, float *pc32, double *pc64, cudaStream_t st) {
    k_point_consts<<<n, kConstThreads, 0, st>>>(d_pts, n, pc32, pc64);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_by_value(const osc_point *h_pts, int n, float *pc32, double *pc64, cudaStream_t st) {
    PointsByValueT<N> pv;
    pv.n = n;
    for (int i = 0; i < n; ++i) pv.p[i] = h_pts[i];
    k_point_consts_v<N><<<n, kConstThreads, 0, st>>>(pv, pc32, pc64);
    return cudaGetLastError();
}

const void *point_consts_one_fn() { return (const void *)k_point_consts_v<1>; }
int point_consts_threads() { return kConstThreads; }

cudaError_t launch_point_consts_host(const osc_point *h_pts, int n, float *pc32, double *pc64, cudaStream_t st) {
    if (n < 1 || n > kPointsByValue) return cudaErrorInvalidValue;
    // a small parameter block launches faster than the full one (one point: a fit step)
    return n == 1   ? launch_by_value<1>(h_pts, n, pc32, pc64, st)
           : n <= 8 ? launch_by_value<8>(h_pts, n, pc32, pc64, st)
                    : launch_by_value<kPointsByValue>(h_pts, n, pc32, pc64, st);
}

cudaError_t launch_hist(int prec, int pt, const HistParams &p, int grid, cudaStream_t st) {
    return prec == kFP32 ? launch_hist_fp32(pt, p, grid, st)
           : prec == kMix ? launch_hist_mix(pt, p, grid, st)
                          : launch_hist_fp64(pt, p, grid, st);
}

// The same launch with programmatic stream serialization: the kernel may start
// while the preceding kernel of the stream still runs (its work that reads no
// kernel output overlaps it; everything else waits in griddepcontrol.wait).
cudaError_t launch_hist_programmatic(int prec, int pt, const HistParams &p, int grid, cudaStream_t st) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(hist_threads_for(prec, pt));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HistParams q = p;
    void *args[] = {&q};
    return cudaLaunchKernelExC(&cfg, hist_kernel_fn(prec, pt), args);
}

// Serving finalize: k_final's conversion, then a completion flag in host-mapped
// memory.  Every thread's bin stores go to host-mapped memory and are fenced at
// system scope before its block takes a ticket; the block that takes the last
// ticket stores the batch's sequence number with release semantics at system
// scope, so a host thread that reads the new value and then acquires sees every
// bin.  The host polls the flag instead of waiting for a stream callback.
__global__ void __launch_bounds__(256) k_final_flag(const FinalFlag p) {
    grid_dependency_wait();
    const FinalParams &f = p.f;
    const int64_t n = f.n_hist * (int64_t)f.nbins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const Digits g = load_digits(f.acc, i);
        clear_digits(f.acc, i);
        f.out[i] = final_bin(g, f.hmeta + 4 * (i / f.nbins), f.pc64);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *f.counter = 0;
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(p.ticket, 1) == (int)gridDim.x - 1) {
        *p.ticket = 0;
        __threadfence_system();
        asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p.flag), "l"(p.seq) : "memory");
    }
}

cudaError_t launch_final_flag(const FinalFlag &p, cudaStream_t st) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(final_blocks(p.f.n_hist * (int64_t)p.f.nbins));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FinalFlag q = p;
    void *args[] = {&q};
    return cudaLaunchKernelExC(&cfg, (const void *)k_final_flag, args);
}

int final_blocks(int64_t n_bins) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n_bins + 255) / 256, (int64_t)device_sms() * 8));
}

cudaError_t launch_final(const FinalParams &p, cudaStream_t st) {
    k_final<<<final_blocks(p.n_hist * (int64_t)p.nbins), 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_final_programmatic(const FinalParams &p, cudaStream_t st) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(final_blocks(p.n_hist * (int64_t)p.nbins));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FinalParams q = p;
    void *args[] = {&q};
    return cudaLaunchKernelExC(&cfg, (const void *)k_final, args);
}

// Exact sharded histograms: the accumulators' digit columns copied out (and
// cleared) instead of converted, launched programmatically after the histogram
// kernel (or its FP64 recomputation pass); the caller sums such columns over
// ranks exactly and converts them with k_from_digits.
__global__ void __launch_bounds__(256) k_digits_out(const FinalParams f, unsigned long long *out) {
    grid_dependency_wait();
    const int64_t n = f.n_hist * (int64_t)f.nbins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const Digits g = load_digits(f.acc, i);
        clear_digits(f.acc, i);
#pragma unroll
        for (int q = 0; q < kDigits; ++q) out[kDigits * i + q] = g.d[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *f.counter = 0;
}

// Bins from digit columns (summed over ranks): the same conversion as every
// finalize (final_bin), so the bins equal those of one launch over all events.
__global__ void __launch_bounds__(256) k_from_digits(const unsigned long long *digits, const double *hmeta,
                                                    const double *pc64, double *out, int64_t n, int32_t nbins) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        Digits g;
#pragma unroll
        for (int q = 0; q < kDigits; ++q) g.d[q] = digits[kDigits * i + q];
        out[i] = final_bin(g, hmeta + 4 * (i / nbins), pc64);
    }
}

cudaError_t launch_digits_out_programmatic(const FinalParams &p, unsigned long long *out, cudaStream_t st) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(final_blocks(p.n_hist * (int64_t)p.nbins));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FinalParams q = p;
    void *args[] = {&q, &out};
    return cudaLaunchKernelExC(&cfg, (const void *)k_digits_out, args);
}

cudaError_t launch_from_digits(const unsigned long long *digits, const double *hmeta, const double *pc64, double *out,
                               int64_t n, int32_t nbins, cudaStream_t st) {
    k_from_digits<<<final_blocks(n), 256, 0, st>>>(digits, hmeta, pc64, out, n, nbins);
    return cudaGetLastError();
}

const void *redo_kernel_fn(int prec) {
    return prec == kFP32 ? redo_kernel_fn_fp32() : prec == kMix ? redo_kernel_fn_mix() : nullptr;
}

// Two blocks of eight warps per SM: the pass has work only where events were
// left out, and one warp takes one marked item.
int redo_grid() { return 2 * device_sms(); }

cudaError_t launch_redo_programmatic(int prec, const HistParams &p, cudaStream_t st) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(redo_grid());
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HistParams q = p;
    void *args[] = {&q};
    return cudaLaunchKernelExC(&cfg, redo_kernel_fn(prec), args);
}

cudaError_t launch_reweight(int prec, const ReweightParams &p, cudaStream_t st) {
    return prec == kFP32 ? launch_reweight_fp32(p, st) : prec == kMix ? launch_reweight_mix(p, st) : launch_reweight_fp64(p, st);
}

}  // namespace osc
