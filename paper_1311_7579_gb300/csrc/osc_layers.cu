// Kernels for samples whose path is a sequence of constant-density layers:
// the event-by-event histogram (per-warp work items, the same exact fixed-point
// accumulation as the single-layer kernels) and the per-event reweight.  Each
// event's probability is the layered mass-basis propagation of osc_layers.cuh.
#include <algorithm>

#include "osc_layers.cuh"
#include "osc_launch.h"

namespace osc {

// Per-point constants of the layered path for one precision.
template <int PREC>
struct LayPoint {
    Pt32 c;
    Pt64 c64;
    const double *d64;    // sorted vacuum eigenvalues, FP64
    const float *lu32;    // sorted-order PMNS, FP32
    const double *lu64;   // sorted-order PMNS, FP64
    float sf;             // energy scale of E_reco
};

template <int PREC>
__device__ __forceinline__ void load_lay_point(LayPoint<PREC> &lp, const float *pc32, const double *pc64) {
    if (PREC != kFP64) {
        load_pt32(pc32, lp.c);
        lp.lu32 = pc32 + C32_LU;
        lp.sf = pc32[C32_ESCALE];
    }
    if (PREC != kFP32) {
        load_pt64(pc64, lp.c64);
        lp.d64 = pc64 + C64_LD;
        lp.lu64 = pc64 + C64_LU;
    }
    if (PREC == kFP64) lp.sf = (float)pc64[C64_ESCALE];
}

template <int PREC>
__global__ void __launch_bounds__(kNT) k_hist_layers(const HistParams prm) {
    grid_dependents_launch();  // lets a finalize kernel after it (programmatic launch) become resident early
    const int lane = threadIdx.x & 31;
    int it = 0;
    if (lane == 0) it = atomicAdd(prm.counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    LayPoint<PREC> lp;
    LayU<float> u32;
    LayU<double> u64;
    int cur_point = -1, cur_nb = -1;
    while (it < prm.n_items) {
        const WorkItem wi = prm.items[it];
        const SampleDev &sd = prm.samples[wi.sample];
        if (wi.point_base != cur_point) {
            cur_point = wi.point_base;
            cur_nb = -1;
            load_lay_point<PREC>(lp, prm.pc32 + (int64_t)cur_point * C32_STRIDE,
                                 prm.pc64 + (int64_t)cur_point * C64_STRIDE);
        }
        unsigned long long *accp = prm.acc + kDigits * wi.acc_base * (int64_t)prm.nbins;
        const int sh = sd.frac_bits - 150;
        const double hs = sd.hscale_d;
        typename AccOf<PREC>::T r;
        const float4 *ev = sd.ev + wi.ev_begin;
        const bool valid = debug_ok(wi.ev_begin >= 0 && wi.ev_count >= 0 && wi.ev_begin + wi.ev_count <= sd.n,
                                    prm.counter, kDbgItem) &&
                           debug_ok(sd.n_layers >= 1 && sd.n_layers <= kMaxLayers, prm.counter, kDbgLayers);
        for (int e = lane; valid && e < wi.ev_count; e += 32) {
            const float4 q = ev[e];
            const int ch = __float_as_int(q.w);
            const int nb = ch >= 9;
            if (nb != cur_nb) {
                cur_nb = nb;
                if (PREC == kFP64)
                    load_layu(lp.lu64, nb, u64);
                else
                    load_layu(lp.lu32, nb, u32);
            }
            if constexpr (PREC == kFP64) {
                const double P = prob_layers64(lp.c64, lp.d64, u64, sd, ch, q.x);
                acc_event_f64(r, accp, prm, lp.sf, q.y, P * (double)q.z, hs, true);
            } else {
                const float P = prob_layers32<PREC>(lp.c, lp.c64, lp.d64, u32, sd, ch, q.x);
                acc_event_f32(r, accp, prm, lp.sf, q.y, P * q.z, sh, true);
            }
        }
        acc_finish_warp(r, accp);
        if (lane == 0) it = atomicAdd(prm.counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
    }
    if (prm.fuse_final) fused_final_warp(prm);
}

template <int PREC>
__global__ void __launch_bounds__(256) k_reweight_layers(const ReweightParams r) {
    const SampleDev &sd = r.s;
    LayPoint<PREC> lp;
    load_lay_point<PREC>(lp, r.pc32 + (int64_t)r.point * C32_STRIDE, r.pc64 + (int64_t)r.point * C64_STRIDE);
    LayU<float> u32;
    LayU<double> u64;
    int cur_nb = -1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.n; i += stride) {
        const float4 q = sd.ev[i];
        const int ch = __float_as_int(q.w);
        const int nb = ch >= 9;
        if (nb != cur_nb) {
            cur_nb = nb;
            if (PREC == kFP64)
                load_layu(lp.lu64, nb, u64);
            else
                load_layu(lp.lu32, nb, u32);
        }
        double P, w;
        if (PREC == kFP64) {
            P = prob_layers64(lp.c64, lp.d64, u64, sd, ch, q.x);
            w = P * (double)q.z;
        } else {
            const float p = prob_layers32<PREC>(lp.c, lp.c64, lp.d64, u32, sd, ch, q.x);
            P = (double)p;
            w = (double)(p * q.z);
        }
        const int32_t o = sd.perm[i];
        if (r.out_prob) r.out_prob[o] = P;
        if (r.out_weight) r.out_weight[o] = w * r.norm;
    }
}

const void *layers_hist_kernel_fn(int prec) {
    return prec == kFP32 ? (const void *)k_hist_layers<kFP32>
           : prec == kMix ? (const void *)k_hist_layers<kMix>
                          : (const void *)k_hist_layers<kFP64>;
}

cudaError_t launch_hist_layers(int prec, const HistParams &p, int grid, cudaStream_t st) {
    if (prec == kFP32)
        k_hist_layers<kFP32><<<grid, kNT, 0, st>>>(p);
    else if (prec == kMix)
        k_hist_layers<kMix><<<grid, kNT, 0, st>>>(p);
    else
        k_hist_layers<kFP64><<<grid, kNT, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_reweight_layers(int prec, const ReweightParams &p, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((p.s.n + 255) / 256, (int64_t)device_sms() * 8);
    if (prec == kFP32)
        k_reweight_layers<kFP32><<<blocks, 256, 0, st>>>(p);
    else if (prec == kMix)
        k_reweight_layers<kMix><<<blocks, 256, 0, st>>>(p);
    else
        k_reweight_layers<kFP64><<<blocks, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace osc
