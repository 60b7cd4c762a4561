// Constants and finalize kernels, and the precision dispatch of the launch helpers.
#include "osc_kernels.cuh"
#include "osc_launch.h"

namespace osc {

__global__ void __launch_bounds__(kConstThreads) k_point_consts(const osc_point *pts, int n, float *pc32, double *pc64) {
    grid_dependents_launch();
    const int i = blockIdx.x;
    if (i >= n) return;
    point_consts_block(pts[i], pc32 + (int64_t)i * C32_STRIDE, pc64 + (int64_t)i * C64_STRIDE);
}

template <int N>
__global__ void __launch_bounds__(kConstThreads) k_point_consts_v(const PointsByValueT<N> pv, float *pc32, double *pc64) {
    grid_dependents_launch();
    const int i = blockIdx.x;
    if (i >= pv.n) return;
    point_consts_block(pv.p[i], pc32 + (int64_t)i * C32_STRIDE, pc64 + (int64_t)i * C64_STRIDE);
}

__global__ void k_final(const FinalParams f) {
    const int64_t n = f.n_hist * (int64_t)f.nbins;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long d0 = f.acc[3 * i], d1 = f.acc[3 * i + 1], d2 = f.acc[3 * i + 2];
        f.acc[3 * i] = 0ull;
        f.acc[3 * i + 1] = 0ull;
        f.acc[3 * i + 2] = 0ull;
        f.out[i] = final_bin(d0, d1, d2, f.hmeta + 4 * (i / f.nbins), f.pc64);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *f.counter = 0;
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

cudaError_t launch_point_consts_host(const osc_point *h_pts, int n, float *pc32, double *pc64, cudaStream_t st) {
    if (n < 1 || n > kPointsByValue) return cudaErrorInvalidValue;
    // a small parameter block launches faster than the full one
    return n <= 8 ? launch_by_value<8>(h_pts, n, pc32, pc64, st) : launch_by_value<kPointsByValue>(h_pts, n, pc32, pc64, st);
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
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HistParams q = p;
    void *args[] = {&q};
    return cudaLaunchKernelExC(&cfg, hist_kernel_fn(prec, pt), args);
}

cudaError_t launch_final(const FinalParams &p, cudaStream_t st) {
    int64_t n = p.n_hist * (int64_t)p.nbins;
    int64_t blocks = (n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_final<<<(int)blocks, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_reweight(int prec, const ReweightParams &p, cudaStream_t st) {
    return prec == kFP32 ? launch_reweight_fp32(p, st) : prec == kMix ? launch_reweight_mix(p, st) : launch_reweight_fp64(p, st);
}

}  // namespace osc
