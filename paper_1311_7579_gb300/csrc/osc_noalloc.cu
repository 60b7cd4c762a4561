// osc_noalloc.cu -- osc_histogram_noalloc: the one-point histogram for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has reserved all
// device memory for its own allocator, or a fit loop where an allocation (which
// may synchronise the device or fail under fragmentation) is not allowed in
// the middle of a step.  This entry point takes every input and the output as
// caller-owned device pointers, creates no context and allocates nothing.  Its
// working memory -- the point's constants, the histogram accumulators, a work
// counter and an error flag -- lives in one file-scope device array of fixed
// size, g_noalloc_scratch below, which every GPU that loads this library holds
// until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "osc_kernels.cuh"

namespace osc {

constexpr int kNoAllocMaxBins = 4096;    // largest histogram the scratch can hold
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    double pc64[C64_STRIDE];
    float pc32[C32_STRIDE];
    unsigned long long acc[kDigits * kNoAllocMaxBins];  // bin digit columns, as in the main path
    int counter;                                        // work-item counter
    int error;  // bit 0: an invalid event; bit 1: an event outside the pass's precision domain
};

// The scratch array (about 130 KB).  Host code must not use this name as an
// address: it is resolved per device with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

struct NoAllocParams {
    const float *e_true, *e_reco, *w_mc;
    const uint8_t *flav_in, *flav_out, *is_nubar;
    int64_t n;
    int32_t chunk, n_items;
    SampleDev sd;        // only the scalar fields are used
    float lo_f, inv_f, nb_f, w_abs_max;
    float a_lim;         // this pass's precision domain: |A| <= a_lim (FP32 bulk: 10 |dm31|, F64EIG: 1000 |dm31|)
    int32_t nbins;
    NoAllocScratch *s;
};

__global__ void __launch_bounds__(kConstThreads) k_noalloc_consts(osc_point P, NoAllocScratch *s) {
    point_consts_block(P, s->pc32, s->pc64);
}

// Same per-warp scheme as the one-point histogram path, over events in the
// caller's order (any order gives the same exact bin sums; events sorted by
// channel and E_reco flush least often).  Invalid events set the error flag; so
// do events outside the pass's precision domain, and the host then runs the call
// again in the next precision (FP32 bulk -> FP32_F64EIG -> FP64).  Unsorted
// events may flush once per event: the 32-bit digit columns absorb 2^32 flushes
// a bin, more than the 2^31 - 1 events a call may hold.
template <int PREC>
__global__ void __launch_bounds__(kNT, 1) k_noalloc_hist(const NoAllocParams p) {
    const int lane = threadIdx.x & 31;
    HistParams hp;
    hp.lo_f = p.lo_f;
    hp.inv_f = p.inv_f;
    hp.nb_f = p.nb_f;
    NoAllocScratch *s = p.s;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&s->counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= p.n_items) return;
        const int64_t beg = (int64_t)it * p.chunk;
        const int64_t end = min(p.n, beg + p.chunk);
        typename AccOf<PREC>::T r;
        int cur_ch = -1;
        Pt32 c32;
        Ch32 h32;
        Pt64 c64;
        Ch64 h64;
        if (PREC != kFP64) load_pt32(s->pc32, c32);
        if (PREC != kFP32) load_pt64(s->pc64, c64);
        for (int64_t e = beg + lane; e < end; e += 32) {
            const float E = p.e_true[e], er = p.e_reco[e], w = p.w_mc[e];
            const int a = p.flav_in[e], b = p.flav_out[e], nb = p.is_nubar[e];
            if (!(E > 0.0f && E <= 3.0e38f) || !(fabsf(er) <= 3.0e38f) || !(fabsf(w) <= p.w_abs_max) || a > 2 ||
                b > 2 || nb > 1) {
                atomicOr(&s->error, 1);
                continue;
            }
            const int ch = chan_id(a, b, nb);
            if constexpr (PREC != kFP64) {
                if (ch != cur_ch) {
                    cur_ch = ch;
                    load_ch32(s->pc32, ch, h32);
                }
                float A, th, tl;
                event_terms32(p.sd, E, ch, A, th, tl);
                if (fabsf(A) > p.a_lim) atomicOr(&s->error, 2);  // the host re-runs the call in the next precision
                bool x;
                float P;
                if (PREC == kFP32) {
                    P = prob_fp32(c32, h32, A, th, tl, x);
                } else {
                    const double Ad = p.sd.kA_rhoye * (double)E;
                    P = prob_mix(c32, h32, c64, (ch >= 9) ? -Ad : Ad, (double)th + (double)tl, x);
                }
                if (x) P = (float)prob_redo64(s->pc64, ch, E, p.sd.kA_rhoye, p.sd.cLL);
                acc_event_f32(r, s->acc, hp, s->pc32[C32_ESCALE], er, P * w, p.sd.frac_bits - 150, true);
            } else {
                if (ch != cur_ch) {
                    cur_ch = ch;
                    load_ch64(s->pc64, ch, h64);
                }
                const double Ad = p.sd.kA_rhoye * (double)E;
                const double P = prob_fp64(c64, h64, (ch >= 9) ? -Ad : Ad, tau64(p.sd.cLL, E));
                acc_event_f64(r, s->acc, hp, (float)s->pc64[C64_ESCALE], er, P * (double)w, p.sd.hscale_d, true);
            }
        }
        acc_finish_warp(r, s->acc);
    }
}

__global__ void k_noalloc_final(double *out, int nbins, double s_hi, double s_lo, NoAllocScratch *s) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins || s->error) return;
    out[b] = bin_value(load_digits(s->acc, b), s_hi, s_lo, s->pc64[C64_NORM]);
}

static void put_err(char *err, size_t len, const char *msg) {
    if (err && len) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = 0;
    }
}

static bool fin(double x) { return std::isfinite(x); }

}  // namespace osc

using namespace osc;

extern "C" osc_status osc_histogram_noalloc(const float *d_e_true, const float *d_e_reco, const float *d_w_mc,
                                            const uint8_t *d_flav_in, const uint8_t *d_flav_out,
                                            const uint8_t *d_is_nubar, int64_t n, double baseline_km,
                                            double density_gcc, double ye, double w_abs_max, const osc_point *pt,
                                            osc_precision prec, double lo, double hi, int32_t nbins, double *d_out,
                                            void *cuda_stream, char *err, size_t err_len) {
    if (!d_e_true || !d_e_reco || !d_w_mc || !d_flav_in || !d_flav_out || !d_is_nubar || !pt || !d_out) {
        put_err(err, err_len, "null pointer argument");
        return OSC_E_ARG;
    }
    if (prec != OSC_FP64 && prec != OSC_FP32_BULK && prec != OSC_FP32_F64EIG) {
        put_err(err, err_len, "bad precision");
        return OSC_E_ARG;
    }
    if (n < 1 || n > (int64_t)INT32_MAX) {
        put_err(err, err_len, "n must be in [1, 2^31 - 1]");
        return OSC_E_ARG;
    }
    if (nbins < 1 || nbins > kNoAllocMaxBins) {
        put_err(err, err_len, "nbins must be in [1, 4096]: the fixed scratch array holds at most 4096 bins");
        return OSC_E_ARG;
    }
    if (!(fin(lo) && fin(hi) && hi > lo) || !(fin(baseline_km) && baseline_km > 0) ||
        !(fin(density_gcc) && density_gcc >= 0) || !(ye >= 0 && ye <= 1) || !(fin(w_abs_max) && w_abs_max > 0) ||
        w_abs_max > 3.0e38) {
        put_err(err, err_len, "need finite lo < hi, baseline > 0, density >= 0, Y_e in [0, 1], 0 < w_abs_max < 3e38");
        return OSC_E_RANGE;
    }
    const osc_point P = *pt;
    if (!(fin(P.s2_12) && fin(P.s2_13) && fin(P.s2_23) && fin(P.dm21) && fin(P.dm32) && fin(P.dcp) &&
          fin(P.escale) && fin(P.norm)) ||
        !(P.s2_12 > 0 && P.s2_12 < 1) || !(P.s2_13 > 0 && P.s2_13 < 1) || !(P.s2_23 >= 0 && P.s2_23 <= 1) ||
        !(P.dm21 > 0) || !(std::fabs(P.dm32) > P.dm21) || !(P.escale > 0) || !(std::fabs(P.dcp) <= 1e6)) {
        put_err(err, err_len, "invalid parameter point (same rules as osc_set_params)");
        return OSC_E_RANGE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        put_err(err, err_len, "no usable current CUDA device");
        return OSC_E_CUDA;
    }
    // One-time set-up per device (with that device current): resolve the device
    // address of the scratch array.  The first call on each device does this.
    static std::mutex mu;
    static void *scratch_ptr[kNoAllocMaxDevices] = {};
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!scratch_ptr[dev]) {
            void *q = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
            if (e != cudaSuccess || !q) {
                put_err(err, err_len, "cudaGetSymbolAddress(g_noalloc_scratch) failed");
                return OSC_E_CUDA;
            }
            scratch_ptr[dev] = q;
        }
        ptr = scratch_ptr[dev];
    }
    NoAllocScratch *s = (NoAllocScratch *)ptr;
    // sample scalars and the fixed-point scale (as osc_load_sample derives them)
    NoAllocParams p;
    std::memset(&p, 0, sizeof(p));
    p.e_true = d_e_true;
    p.e_reco = d_e_reco;
    p.w_mc = d_w_mc;
    p.flav_in = d_flav_in;
    p.flav_out = d_flav_out;
    p.is_nubar = d_is_nubar;
    p.n = n;
    int F = 62 - (int)std::ceil(std::log2(w_abs_max));
    F = std::max(8, std::min(F, 190));
    p.sd.kA_rhoye = matter_k_A() * density_gcc * ye;
    p.sd.cLL = kCL * baseline_km;
    p.sd.kA_rhoye_f = (float)p.sd.kA_rhoye;
    const double rev = kCL * baseline_km / kTwoPi;
    p.sd.rev_hi = (float)rev;
    p.sd.rev_lo = (float)(rev - (double)p.sd.rev_hi);
    p.sd.hscale_d = std::ldexp(1.0, F - 64);
    p.sd.hscale_f = (float)p.sd.hscale_d;
    p.sd.frac_bits = F;
    p.lo_f = (float)lo;
    p.inv_f = (float)((double)nbins / (hi - lo));
    p.nb_f = (float)nbins;
    p.w_abs_max = (float)w_abs_max;
    p.nbins = nbins;
    p.s = s;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // The precision of the first pass: FP32 bulk needs the sample's matter phase
    // c_L L k_A rho Y_e within kFp32BulkMatterPhase (else its shifts and phases
    // go to FP64: F64EIG).  A pass whose kernel flags an event outside its
    // domain (FP32 bulk: |A| > kFp32BulkMatterRatio |dm31|; F64EIG: |A| >
    // kFp32MatterRatio |dm31|) is followed by a pass in the next precision.
    const double adm31 = std::fabs(P.dm32 + P.dm21);
    int kind = prec == OSC_FP64 ? kFP64 : prec == OSC_FP32_F64EIG ? kMix : kFP32;
    if (kind == kFP32 && !(kCL * baseline_km * p.sd.kA_rhoye <= kFp32BulkMatterPhase)) kind = kMix;
    int flag = 0;
    for (;;) {
        p.a_lim = (float)((kind == kFP32 ? kFp32BulkMatterRatio : kFp32MatterRatio) * adm31);
        int per_sm = 1;
        const void *fn = kind == kFP32 ? (const void *)k_noalloc_hist<kFP32>
                         : kind == kMix ? (const void *)k_noalloc_hist<kMix>
                                        : (const void *)k_noalloc_hist<kFP64>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kNT, 0);
        per_sm = std::max(per_sm, 1);
        const int64_t warps = (int64_t)std::max(n_sm, 1) * per_sm * (kNT / 32);
        int64_t chunk = (n + 4 * warps - 1) / (4 * warps);
        chunk = std::max<int64_t>(64, (chunk + 63) / 64 * 64);
        p.chunk = (int32_t)chunk;
        p.n_items = (int32_t)((n + chunk - 1) / chunk);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)n_sm * per_sm, (p.n_items + 7) / 8));
        // Calls share the scratch and it keeps the previous call's contents: clear
        // the accumulators, the counter and the error flag first.
        cudaError_t e = cudaMemsetAsync(s->acc, 0, sizeof(unsigned long long) * kDigits * (size_t)nbins, st);
        if (!e) e = cudaMemsetAsync(&s->counter, 0, 2 * sizeof(int), st);
        if (e) {
            put_err(err, err_len, "cudaMemsetAsync on the scratch array failed");
            return OSC_E_CUDA;
        }
        k_noalloc_consts<<<1, kConstThreads, 0, st>>>(P, s);
        if (kind == kFP32)
            k_noalloc_hist<kFP32><<<grid, kNT, 0, st>>>(p);
        else if (kind == kMix)
            k_noalloc_hist<kMix><<<grid, kNT, 0, st>>>(p);
        else
            k_noalloc_hist<kFP64><<<grid, kNT, 0, st>>>(p);
        k_noalloc_final<<<(nbins + 255) / 256, 256, 0, st>>>(d_out, nbins, std::ldexp(1.0, 64 - F),
                                                              std::ldexp(1.0, -F), s);
        e = cudaGetLastError();
        flag = 0;
        if (!e) e = cudaMemcpyAsync(&flag, &s->error, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) {
            char buf[256];
            std::snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
            put_err(err, err_len, buf);
            return OSC_E_CUDA;
        }
        if (kind != kFP64 && flag == 2) {
            kind = kind == kFP32 ? kMix : kFP64;
            continue;
        }
        break;
    }
    if (flag & 1) {
        put_err(err, err_len, "invalid event (E_true <= 0 or non-finite, non-finite E_reco, |w_mc| > w_abs_max, "
                              "or bad flavour); output left unwritten");
        return OSC_E_RANGE;
    }
    put_err(err, err_len, "");
    return OSC_OK;
}
