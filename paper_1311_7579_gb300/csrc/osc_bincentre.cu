// Binned ("bin-centre") reweighting, the quicker alternative that Sec. 1.1.1
// contrasts with event-by-event reweighting: every event's probability is taken
// at the centre of its true-energy bin.  Two kernels:
//   k_bc_table  one thread per (table row, true bin): P at the bin centre, where
//               a row is a (sample, point, channel present in the sample);
//   k_bc_hist   per-warp work items (sample, point, event range): true bin of
//               each event by the FP32 binning rule, gather of P from the table,
//               weight P * w_mc binned by E_reco into the same exact fixed-point
//               accumulators as the event-by-event kernel.
// The table is tiny next to the event stream, so the histogram kernel is bound
// by reading the 16-byte event records: each lane works on four records while
// the next four are loaded, and the kernel is launched programmatically after
// the table kernel so that its first loads overlap the table computation (and
// the finalize kernel programmatically after it).
#include "osc_layers.cuh"
#include "osc_launch.h"

namespace osc {

// FP64 probabilities enter the table as the integer P * 2^63, rounded (P <= 1 up
// to rounding, so the value stays below 2^64).
__device__ __forceinline__ unsigned long long prob_fixed(double P) {
    return __double2ull_rn(fmin(fmax(P, 0.0), 1.5) * 9223372036854775808.0);
}

// Adds P * w * 2^F to the lane's 128-bit run accumulator with integer
// instructions only: Pq = P * 2^63 (integer), w = m * 2^(e - 150) (FP32
// mantissa m with its implicit bit), so the addend is Pq * m * 2^(e + F - 213),
// truncated.  |w| * 2^F < 2^63 makes e + F - 213 <= -24, so it is a right
// shift of the 88-bit product and the addend fits in 63 bits.
__device__ __forceinline__ void fx_add_pw(unsigned long long &lo, unsigned long long &hi, unsigned long long pq,
                                          float w, int frac_bits) {
    const uint32_t u = __float_as_uint(w);
    const int ef = (int)((u >> 23) & 0xFFu);
    const unsigned long long m = (unsigned long long)((u & 0x7FFFFFu) | (ef ? 0x800000u : 0u));
    const int rs = 213 - frac_bits - (ef ? ef : 1);
    const unsigned long long plo = pq * m, phi = __umul64hi(pq, m);
    unsigned long long v;
    if (rs >= 128)
        v = 0ull;
    else if (rs >= 64)
        v = phi >> (rs - 64);
    else
        v = (plo >> rs) | (phi << (64 - rs));  // rs >= 24 here
    if (u >> 31) {
        asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(v));
    } else {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(v));
    }
}

// Small blocks spread the table over many SMs: its FP64 evaluations are few
// but long, and the FP64 pipe of one SM would serialise them.
constexpr int kBcTableThreads = 64;

template <int PREC>
__global__ void __launch_bounds__(kBcTableThreads) k_bc_table(const BcParams b) {
    grid_dependents_launch();
    const int64_t n = (int64_t)b.n_rows * b.t_nbins;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(idx / b.t_nbins);
        const int32_t t = (int32_t)(idx - (int64_t)r * b.t_nbins);
        const BcRow rw = b.rows[r];
        const SampleDev &sd = b.h.samples[rw.sample];
        // centre t_lo + (t + 1/2) w in double (no contraction), stored in FP32 like an event energy
        const float E = __double2float_rn(__dadd_rn(b.t_lo, __dmul_rn((double)t + 0.5, b.t_w)));
        const int ch = rw.chan;
        if (sd.n_layers > 1) {
            // layered path: the sample's layer sequence, same precision split
            const double *pc64 = b.h.pc64 + (int64_t)rw.point * C64_STRIDE;
            Pt64 c64;
            load_pt64(pc64, c64);
            if (PREC == kFP64) {
                LayU<double> u;
                load_layu(pc64 + C64_LU, ch >= 9, u);
                b.tabq[idx] = prob_fixed(prob_layers64(c64, pc64 + C64_LD, u, sd, ch, E));
            } else {
                const float *pc = b.h.pc32 + (int64_t)rw.point * C32_STRIDE;
                Pt32 c;
                load_pt32(pc, c);
                LayU<float> u;
                load_layu(pc + C32_LU, ch >= 9, u);
                b.tab32[idx] = prob_layers32<PREC>(c, c64, pc64 + C64_LD, u, sd, ch, E);
            }
            continue;
        }
        if (PREC == kFP32) {
            const float *pc = b.h.pc32 + (int64_t)rw.point * C32_STRIDE;
            Pt32 c;
            load_pt32(pc, c);
            Ch32 h;
            load_ch32(pc, ch, h);
            float A, th, tl;
            event_terms32(sd, E, ch, A, th, tl);
            bool x;
            float P = prob_fp32(c, h, A, th, tl, x);
            if (x) P = (float)prob_redo64(b.h.pc64 + (int64_t)rw.point * C64_STRIDE, ch, E, sd.kA_rhoye, sd.cLL);
            b.tab32[idx] = P;
        } else if (PREC == kMix) {
            const float *pc = b.h.pc32 + (int64_t)rw.point * C32_STRIDE;
            Pt32 c;
            load_pt32(pc, c);
            Ch32 h;
            load_ch32(pc, ch, h);
            Pt64 c64;
            load_pt64(b.h.pc64 + (int64_t)rw.point * C64_STRIDE, c64);
            float A, th, tl;
            event_terms32(sd, E, ch, A, th, tl);
            const double Ad = sd.kA_rhoye * (double)E;
            bool x;
            float P = prob_mix(c, h, c64, (ch >= 9) ? -Ad : Ad, (double)th + (double)tl, x);
            if (x) P = (float)prob_redo64(b.h.pc64 + (int64_t)rw.point * C64_STRIDE, ch, E, sd.kA_rhoye, sd.cLL);
            b.tab32[idx] = P;
        } else {
            const double *pc = b.h.pc64 + (int64_t)rw.point * C64_STRIDE;
            Pt64 c;
            load_pt64(pc, c);
            Ch64 h;
            load_ch64(pc, ch, h);
            const double Ad = sd.kA_rhoye * (double)E;
            b.tabq[idx] = prob_fixed(prob_fp64(c, h, (ch >= 9) ? -Ad : Ad, tau64(sd.cLL, E)));
        }
    }
}

constexpr int kBcUnroll = 4;  // event records per lane per step; the next step's are loaded meanwhile

template <bool F64>
__global__ void __launch_bounds__(kNT) k_bc_hist(const BcParams b) {
    grid_dependents_launch();  // the finalize kernel after this one may become resident early
    const HistParams &prm = b.h;
    const int lane = threadIdx.x & 31;
    // first item of every warp assigned statically, later ones from the counter
    const int n_warps = (int)(gridDim.x * (blockDim.x >> 5));
    int it = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    WorkItem wi{};
    const float4 *ev = nullptr;
    int end = 0;
    float4 q[kBcUnroll];
    auto load_step = [&](float4 *dst, int e0) {
#pragma unroll
        for (int k = 0; k < kBcUnroll; ++k) {
            const int e = e0 + lane + 32 * k;
            dst[k] = (e < end) ? ev[e] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    };
    auto fetch = [&](int idx) {
        wi = prm.items[idx];
        const SampleDev &s = prm.samples[wi.sample];
        ev = s.ev + wi.ev_begin;
        end = debug_ok(wi.ev_begin >= 0 && wi.ev_count >= 0 && wi.ev_begin + wi.ev_count <= s.n, prm.counter,
                       kDbgItem) ? wi.ev_count : 0;
        load_step(q, 0);
    };
    // items and events are never written by a kernel: the first item's events are
    // in flight before the wait for the table kernel (programmatic launch)
    if (it < prm.n_items) fetch(it);
    grid_dependency_wait();
    while (it < prm.n_items) {
        const SampleDev &sd = prm.samples[wi.sample];
        const float sf = F64 ? (float)prm.pc64[(int64_t)wi.point_base * C64_STRIDE + C64_ESCALE]
                             : prm.pc32[(int64_t)wi.point_base * C32_STRIDE + C32_ESCALE];
        const int sh = sd.frac_bits - 150;
        const int32_t *rmap = b.row_map + wi.acc_base * kChannels;
        unsigned long long *accp = prm.acc + kDigits * wi.acc_base * (int64_t)prm.nbins;
        // FP64: the 128-bit run of fx_add_pw; FP32: the 96-bit run of acc_event_f32
        typename AccOf<F64 ? kFP64 : kFP32>::T r;
        int cur_ch = -1;
        int64_t row_off = 0;
        for (int e0 = 0; e0 < end; e0 += 32 * kBcUnroll) {
            float4 qn[kBcUnroll];
            load_step(qn, e0 + 32 * kBcUnroll);
#pragma unroll
            for (int k = 0; k < kBcUnroll; ++k) {
                const int e = e0 + lane + 32 * k;
                const int ch = __float_as_int(q[k].w);
                const float tb = __fsub_rn(q[k].x, b.t_lo_f);
                const float u = __fmul_rn(tb, b.t_inv_f);
                const bool keep = e < end && tb >= 0.0f && u < b.t_nb_f;
                if (keep && ch != cur_ch) {
                    cur_ch = ch;
                    row_off = (int64_t)rmap[ch] * b.t_nbins;
                }
                const int64_t ti = row_off + (keep ? __float2int_rz(u) : 0);
                if (keep && !debug_ok(row_off >= 0 && ti < (int64_t)b.n_rows * b.t_nbins, prm.counter, kDbgRow))
                    continue;
                if constexpr (F64) {
                    // binning as in acc_event_f64, integer addend
                    const float x = __fmul_rn(sf, q[k].y);
                    const float tr = __fsub_rn(x, prm.lo_f);
                    const float ur = __fmul_rn(tr, prm.inv_f);
                    if (keep && tr >= 0.0f && ur < prm.nb_f) {
                        const int bn = __float2int_rz(ur);
                        if (bn != r.cur_b) {
                            if (r.cur_b >= 0 && (r.lo | r.hi)) fx_flush(accp + kDigits * r.cur_b, r.lo, r.hi);
                            r.lo = r.hi = 0;
                            r.cur_b = bn;
                        }
                        fx_add_pw(r.lo, r.hi, b.tabq[ti], q[k].z, sd.frac_bits);
                    }
                } else {
                    const float P = keep ? b.tab32[ti] : 0.0f;
                    acc_event_f32(r, accp, prm, sf, q[k].y, P * q[k].z, sh, keep);
                }
            }
#pragma unroll
            for (int k = 0; k < kBcUnroll; ++k) q[k] = qn[k];
        }
        if (lane == 0) it = atomicAdd(prm.counter, 1) + n_warps;
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it < prm.n_items) fetch(it);
        acc_finish_warp(r, accp);
    }
}

const void *bc_hist_kernel_fn(int prec) {
    return prec == kFP64 ? (const void *)k_bc_hist<true> : (const void *)k_bc_hist<false>;
}

int bc_table_threads() { return kBcTableThreads; }

const void *bc_table_kernel_fn(int prec) {
    return prec == kFP32 ? (const void *)k_bc_table<kFP32>
           : prec == kMix ? (const void *)k_bc_table<kMix>
                          : (const void *)k_bc_table<kFP64>;
}

}  // namespace osc
