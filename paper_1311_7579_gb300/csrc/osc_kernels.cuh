// osc_kernels.cuh -- CUDA kernels of the reweighting hot path (sm_103a).
//
//   k_point_consts  per parameter point, FP64: PMNS matrix, vacuum Hamiltonian
//                   invariants, cubic coefficients, sorted vacuum spectrum and the
//                   per-channel (M)_ba, (M^2)_ba pieces (Sec. 2.1: the components
//                   that depend only on the oscillation parameters).
//   k_hist<P, PT>   persistent fused kernel: streams the (channel, E_reco)-sorted
//                   event SoA through shared memory with 128-bit loads, computes
//                   P, weight and bin for PT points x the tile's events, and
//                   accumulates each lane's bins run-length in exact 128-bit fixed
//                   point in registers, flushing with integer atomics (Sec. 1.1.1).
//   k_final         128-bit bins -> double * norm, and clears the accumulators.
//   k_reweight<P>   per-event probability and weight in the caller's event order.
#pragma once

#include "osc_internal.h"
#include "osc_math.cuh"

namespace osc {

constexpr int kNT = 256;          // threads per block of the histogram kernel
constexpr int kET = 4 * kNT;      // events per shared-memory tile

// ------------------------------------------------------------- debug checks
// Built with OSC_DEBUG_CHECKS, the kernels verify work-item and index ranges
// against their buffers; a violation skips the access and sets a bit of the
// error word (int kDebugWord of the launch's counter block), which the host
// reads after it synchronises.  Release builds compile the checks away.
__device__ __forceinline__ bool debug_ok(bool ok, int32_t *counter, unsigned code) {
#ifdef OSC_DEBUG_CHECKS
    if (!ok) atomicOr(reinterpret_cast<unsigned *>(counter + kDebugWord), code);
    return ok;
#else
    (void)ok;
    (void)counter;
    (void)code;
    return true;
#endif
}

// ------------------------------------------------ programmatic dependent launch
// A kernel launched with programmatic stream serialization may start before the
// preceding kernel of its stream has finished; it must wait here before it reads
// anything that kernel writes.  Without that launch attribute the wait returns
// at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the dependent kernel of a programmatic launch start (its wait still
// covers all of this kernel's writes).
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- constants
struct cplx64 {
    double re, im;
};
// The constants are written with explicit fma wherever a product is added (and
// explicit adds where no product may be fused), so that every kernel inlining
// them (the constants kernels, the allocation-free call) and the host's copy of
// the computation (host_point_consts) round identically and give bitwise the
// same constants.
__device__ __forceinline__ cplx64 cmul_conj(cplx64 a, double m, cplx64 b) {
    // a * m * conj(b)
    return {m * fma(a.re, b.re, a.im * b.im), m * fma(a.im, b.re, -(a.re * b.im))};
}

__device__ __forceinline__ void split_ff(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// sin and cos of delta in FP64, evaluated by two lanes in the same instruction
// stream (lane 0 the sine, lane 1 the cosine), so that the chain is one
// polynomial long.  Cody and Waite's reduction by pi/2 with a two-part constant
// (the high part has 33 significant bits, so k * hi is exact for |k| < 2^20)
// leaves r in [-pi/4, pi/4]; the Taylor series of sin r / r and cos r in u = r^2
// through u^8 truncate below 3e-18.  Returns (sin, cos) of delta on lane 0.
__device__ __forceinline__ void sincos_lanes(double x, int lane, double *sn, double *cs) {
    constexpr double kTwoOverPi = 0.63661977236758134308;
    constexpr double kPio2Hi = 1.5707963267341256;        // pi/2 to 33 bits
    constexpr double kPio2Lo = 6.077100506506192e-11;     // pi/2 - kPio2Hi
    const double k = rint(x * kTwoOverPi);
    const double r = fma(-k, kPio2Lo, fma(-k, kPio2Hi, x));
    const double u = r * r;
    const bool c = lane == 1;
    // coefficients (-1)^j / (2j + 1)! (sine) and (-1)^j / (2j)! (cosine), j = 8 .. 1
    double p = c ? 1.0 / 20922789888000.0 : 1.0 / 355687428096000.0;
    p = fma(p, u, c ? -1.0 / 87178291200.0 : -1.0 / 1307674368000.0);
    p = fma(p, u, c ? 1.0 / 479001600.0 : 1.0 / 6227020800.0);
    p = fma(p, u, c ? -1.0 / 3628800.0 : -1.0 / 39916800.0);
    p = fma(p, u, c ? 1.0 / 40320.0 : 1.0 / 362880.0);
    p = fma(p, u, c ? -1.0 / 720.0 : -1.0 / 5040.0);
    p = fma(p, u, c ? 1.0 / 24.0 : 1.0 / 120.0);
    p = fma(p, u, c ? -1.0 / 2.0 : -1.0 / 6.0);
    p = fma(p, u, 1.0);
    const double v = c ? p : p * r;
    const double w = __shfl_xor_sync(0x3u, v, 1);
    const int q = (int)k & 3;  // quadrant, two's complement for negative k
    *sn = q == 0 ? v : q == 1 ? w : q == 2 ? -v : -w;
    *cs = q == 0 ? w : q == 1 ? -v : q == 2 ? -w : v;
}

// PMNS entry U[f][m] (PDG: U_e3 = s13 e^{-i delta}, e^{+i delta} in the mu and
// tau rows of the first two mass columns), written for every (f, m) as
// a + b s13 (cos delta + i g sin delta), with a and b products of two of the
// sines and cosines; each lane of one instruction stream picks its operands.
// t = (s12, c12, s13, c13, s23, c23, sin delta, cos delta).
__device__ __forceinline__ cplx64 pmns_entry(const double *t, int f, int m) {
    const double s12 = t[0], c12 = t[1], s13 = t[2], c13 = t[3], s23 = t[4], c23 = t[5], sd = t[6], cd = t[7];
    double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0, g = 1.0;
    if (f == 0) {
        if (m == 0) { ax = c12; ay = c13; }
        else if (m == 1) { ax = s12; ay = c13; }
        else { bx = 1.0; by = 1.0; g = -1.0; }
    } else if (m == 2) {
        ax = (f == 1) ? s23 : c23; ay = c13;
    } else if (f == 1) {
        ax = (m == 0) ? -s12 : c12; ay = c23;
        bx = (m == 0) ? -c12 : -s12; by = s23;
    } else {
        ax = (m == 0) ? s12 : -c12; ay = s23;
        bx = (m == 0) ? -c12 : -s12; by = c23;
    }
    const double bs = bx * by * s13;
    return {fma(bs, cd, ax * ay), bs * (g * sd)};
}

// Barrier of warps 0 and 1 only (named barrier id 1..15; warps 2, 3 never wait).
__device__ __forceinline__ void pair_barrier(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// One block of four warps (one per scheduler) per point.  FP64 runs at a small
// fraction of the FP32 rate on this GPU: a warp instruction occupies its
// scheduler's FP64 unit for many cycles whatever the number of active lanes, and
// a dependent one waits about a hundred cycles, so the kernel's latency is the
// number of FP64 instructions on its longest path.  Independent work therefore
// runs on different warps, and parallel work as one instruction stream over
// lanes with per-lane operands (never as divergent branches, which would issue
// each path in turn).  Only the chain s^2, delta -> U -> H0, H0^2 -> channel
// fields needs barriers; it runs on warps 0 and 1, which wait for each other
// alone, while warps 2 and 3 write everything that depends on the inputs
// directly and never wait:
//   warp 0 lanes 0-5: the six square roots | warp 1 lanes 0-1: sin, cos delta
//   -- barrier --
//   warp 0 lanes 0-8: one PMNS entry each
//   -- barrier --
//   warp 0 lanes 0-8: one entry each of H0 = U diag(m) U^dagger and H0^2
//   | warp 1 lanes 0-8: U with its columns in the sorted vacuum order
//   -- barrier --
//   warps 0, 1 lanes 0-26: one field of one channel each
// | warp 2 lanes 0-1: shifted-cubic constants of sorted root lane (from the
//   sorted vacuum spectrum and |U_e|^2 = products of the s^2 inputs), then
//   lanes 0-4: one depressed-cubic coefficient each
// | warp 3 lanes 0-13: one each of the sorted spectrum, gaps (float-float
//   differences), T0, c1(0), T0 / 3 - d0,1 and the systematics.
// The cubic's coefficients need two invariants of H0 besides T0 and c1(0), and
// both follow from the s^2 inputs alone (the eigenvalues in matter depend on U
// only through |U_e|^2):
//   smt = H0_mumu + H0_tautau = T0 - H0_ee,  H0_ee = dm21 |U_e2|^2 + dm31 |U_e3|^2,
//   mee = H0_mumu H0_tautau - |H0_mutau|^2 = (adj H0)_ee = dm21 dm31 |U_e1|^2,
// since adj(U D U^dagger) = U adj(D) U^dagger and adj(diag(0, dm21, dm31)) =
// diag(dm21 dm31, 0, 0); written this way neither carries a cancellation.
constexpr int kConstThreads = 128;
__device__ inline void point_consts_block(const osc_point &P, float *c32, double *c64) {
    __shared__ double t[8];
    __shared__ cplx64 Us[9];     // U[f][m] at 3 f + m
    __shared__ double Hs[4][9];  // H re, H im, H2 re, H2 im, entry (b, a) at 3 b + a
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double dm21 = P.dm21, dm31 = P.dm32 + P.dm21;
    const double T0 = dm21 + dm31;
    const double c10 = dm21 * dm31;
    // sorted vacuum spectrum d0 <= d1 <= d2 (normal ordering 0, dm21, dm31;
    // inverted dm31, 0, dm21) and the matching |U_e|^2
    const bool no = dm31 > 0;
    const double d0 = no ? 0.0 : dm31, d1 = no ? dm21 : 0.0, d2 = no ? dm31 : dm21;
    if (warp <= 1) {
        if (warp == 0 && lane < 6) {
            const double x = (lane == 0) ? P.s2_12 : (lane == 1) ? 1.0 - P.s2_12 : (lane == 2) ? P.s2_13
                           : (lane == 3) ? 1.0 - P.s2_13 : (lane == 4) ? P.s2_23 : 1.0 - P.s2_23;
            t[lane] = sqrt(x);
        }
        if (warp == 1 && lane < 2) {
            double sn, cs;
            sincos_lanes(P.dcp, lane, &sn, &cs);
            if (lane == 0) {
                t[6] = sn;
                t[7] = cs;
            }
        }
        pair_barrier(1);
        if (warp == 0 && lane < 9) Us[lane] = pmns_entry(t, lane / 3, lane % 3);
        pair_barrier(2);
        if (warp == 0 && lane < 9) {
            // entry (b, a) of H0 and H0^2: sum over the mass columns 1, 2 (column 0 carries m = 0)
            const int b = lane / 3, a = lane % 3;
            const double m[3] = {0.0, dm21, dm31};
            cplx64 h = {0, 0}, h2 = {0, 0};
            for (int k = 1; k < 3; ++k) {
                const cplx64 q = cmul_conj(Us[3 * b + k], m[k], Us[3 * a + k]);
                h.re = __dadd_rn(h.re, q.re);  // an explicit add: no product is fused into it
                h.im = __dadd_rn(h.im, q.im);
                h2.re = fma(q.re, m[k], h2.re); h2.im = fma(q.im, m[k], h2.im);
            }
            Hs[0][lane] = h.re; Hs[1][lane] = h.im; Hs[2][lane] = h2.re; Hs[3][lane] = h2.im;
        }
        if (warp == 1 && lane < 9) {
            // PMNS entry U[f][m] with its mass column m in the sorted vacuum order,
            // for the mass-basis propagation through layered matter
            const int f = lane / 3, l = lane % 3;
            const int m = no ? l : (l + 2) % 3;
            const cplx64 u = Us[3 * f + m];
            c32[C32_LU + 2 * lane] = (float)u.re;
            c32[C32_LU + 2 * lane + 1] = (float)u.im;
            c64[C64_LU + 2 * lane] = u.re;
            c64[C64_LU + 2 * lane + 1] = u.im;
        }
        pair_barrier(3);
        if (lane < 27) {
            // FP64 block: channel (alpha -> beta) = ch (alpha * 3 + beta), field j of
            // (Xr, Xi, Yr, Yi, Zr, Zi) with X = M0_ba, Y = (M0^2)_ba,
            // Z = M0_be [alpha = e] + [beta = e] M0_ea: one field per lane of warps 0, 1
            const int ch = lane / 3, j = 3 * warp + lane % 3;
            const int a = ch / 3, b = ch % 3;
            const int cmp = j < 4 ? j : j - 4;
            const double z = (a == 0 ? Hs[cmp][3 * b] : 0.0) + (b == 0 ? Hs[cmp][a] : 0.0);
            c64[C64_CH + 6 * ch + j] = j < 4 ? Hs[cmp][3 * b + a] : z;
        }
        // FP32 block: the channels in the vacuum mass basis, field j of
        // (X0r, X0i, X1r, X1i, X2r, X2i, Zr, Zi) with X_l = U_bm conj(U_am) (m the mass
        // state of sorted vacuum root l) and Z as above; 72 fields over the 64 lanes
        for (int f = 32 * warp + lane; f < 72; f += 64) {
            const int ch = f >> 3, j = f & 7, a = ch / 3, b = ch % 3;
            double v;
            if (j < 6) {
                const int l = j >> 1, m = no ? l : (l + 2) % 3;
                const cplx64 ub = Us[3 * b + m], ua = Us[3 * a + m];
                v = (j & 1) ? fma(ub.im, ua.re, -(ub.re * ua.im)) : fma(ub.re, ua.re, ub.im * ua.im);
            } else {
                const int cmp = j - 6;
                v = (a == 0 ? Hs[cmp][3 * b] : 0.0) + (b == 0 ? Hs[cmp][a] : 0.0);
            }
            c32[C32_CH + 8 * ch + j] = (float)v;
        }
    } else if (warp == 2) {
        // |U_e1|^2, |U_e2|^2, |U_e3|^2 and their sorted-order counterparts
        const double ze0 = (1.0 - P.s2_12) * (1.0 - P.s2_13), ze1 = P.s2_12 * (1.0 - P.s2_13), ze2 = P.s2_13;
        if (lane < 2) {
            // sorted root l = lane and the other two j, k: a_j = d_l - d_j, a_k = d_l - d_k
            const double z0 = no ? ze0 : ze2, z1 = no ? ze1 : ze0, z2 = no ? ze2 : ze1;
            const double dl = lane ? d1 : d0, dj = lane ? d2 : d1, dk = lane ? d0 : d2;
            const double zl = lane ? z1 : z0, zj = lane ? z2 : z1, zk = lane ? z0 : z2;
            const double aj = dl - dj, ak = dl - dk;
            const int o = lane ? (C32_S1 - C32_S0) : 0;
            const double S = aj + ak, PI = aj * ak, W = fma(zl, aj + ak, fma(zj, ak, zk * aj)), E = zl * aj * ak;
            c32[C32_S0 + o] = (float)S;
            c32[C32_PI0 + o] = (float)PI;
            c32[C32_W0 + o] = (float)W;
            c32[C32_E0 + o] = (float)E;
            c64[C64_SH + 4 * lane] = S;
            c64[C64_SH + 4 * lane + 1] = PI;
            c64[C64_SH + 4 * lane + 2] = W;
            c64[C64_SH + 4 * lane + 3] = E;
        }
        if (lane < 5) {
            // depressed cubic mu^3 + p mu + q, lambda = mu + (T0 + A) / 3:
            //   p = c1 - c2^2/3, q = -2 c2^3/27 + c1 c2 / 3 - c0, c2 = T0 + A, c1 = c10 + A smt, c0 = A mee;
            // lane j forms coefficient j of (p0, p1, q0, q1, q2) as one weighted sum
            //   w3 T0^3 + w2 T0^2 + w1 T0 + wc c10 + wct c10 T0 + ws smt + wst smt T0 - [j = 3] mee
            constexpr double k3 = 1.0 / 3.0, k9 = 1.0 / 9.0, k27 = 1.0 / 27.0;
            const double smt = T0 - fma(dm21, ze1, dm31 * ze2);
            const double mee = c10 * ze0;
            const double w3 = lane == 2 ? -2.0 * k27 : 0.0;
            const double w2 = lane == 0 ? -k3 : lane == 3 ? -2.0 * k9 : 0.0;
            const double w1 = lane == 1 ? -2.0 * k3 : lane == 4 ? -2.0 * k9 : 0.0;
            const double wc = lane == 0 ? 1.0 : lane == 3 ? k3 : 0.0;
            const double wct = lane == 2 ? k3 : 0.0;
            const double ws = lane == 1 ? 1.0 : lane == 4 ? k3 : 0.0;
            const double wst = lane == 3 ? k3 : 0.0;
            const double wm = lane == 3 ? -1.0 : 0.0;
            const double T2 = T0 * T0;
            double v = wm * mee;
            v = fma(wst, smt * T0, v);
            v = fma(ws, smt, v);
            v = fma(wct, c10 * T0, v);
            v = fma(wc, c10, v);
            v = fma(w1, T0, v);
            v = fma(w2, T2, v);
            v = fma(w3, T2 * T0, v);
            const int o32 = lane == 0 ? C32_P0 : lane == 1 ? C32_P1 : lane == 2 ? C32_Q0 : lane == 3 ? C32_Q1 : C32_Q2;
            const int o64 = lane == 0 ? C64_P0 : lane == 1 ? C64_P1 : lane == 2 ? C64_Q0 : lane == 3 ? C64_Q1 : C64_Q2;
            // FP32 seed coefficients of -p/3 and -q/2 (the forms the seed uses)
            c32[o32] = (float)(v * (lane < 2 ? -1.0 / 3.0 : -0.5));
            c64[o64] = v;
            if (lane == 0) {
                c32[C32_SMT] = (float)smt;
                c64[C64_SMT] = smt;
            }
        }
    } else if (lane >= 14) {
        // warp 3, lanes 14, 15: T0 less one sorted vacuum eigenvalue (the e -> e term of the FP32 amplitude)
        if (lane == 14) c32[C32_SD02] = (float)(d0 + d2);
        if (lane == 15) c32[C32_SD01] = (float)(d0 + d1);
    } else {
        // warp 3: one value per lane, x = a s - b: the sorted spectrum, its gaps
        // (two as float-float), T0, c1(0), T0 / 3 - d0, T0 / 3 - d1 and the
        // systematics; o64 / o32 are its FP64 / FP32 slots (-1: none)
        const double a = lane == 0 || lane == 6 || lane == 7 ? d0
                       : lane == 1 || lane == 3 || lane == 5 ? d1
                       : lane == 2 || lane == 4            ? d2
                       : lane == 9                         ? c10
                       : lane == 12                        ? P.escale
                       : lane == 13                        ? P.norm
                                                           : T0;
        const double b = lane == 3 || lane == 4 || lane == 10 ? d0
                       : lane == 6 || lane == 11            ? d1
                       : lane == 5 || lane == 7             ? d2
                                                            : 0.0;
        const double x = fma(a, (lane == 10 || lane == 11) ? 1.0 / 3.0 : 1.0, -b);
        const int o64 = lane <= 2 ? C64_LD + lane : (lane >= 3 && lane <= 5) ? C64_VG + lane - 3
                      : lane == 8 ? C64_T0 : lane == 9 ? C64_C10 : lane == 12 ? C64_ESCALE : lane == 13 ? C64_NORM : -1;
        const int o32 = lane <= 2 ? C32_D0 + lane : lane == 3 ? C32_V1H : lane == 4 ? C32_V2H : lane == 5 ? C32_G12
                      : lane == 6 ? C32_G01 : lane == 7 ? C32_G02 : lane == 8 ? C32_T0 : lane == 9 ? C32_C10
                      : lane == 10 ? C32_TD0 : lane == 11 ? C32_TD1 : lane == 12 ? C32_ESCALE : -1;
        if (o64 >= 0) c64[o64] = x;
        if (lane == 3 || lane == 4) {
            split_ff(x, &c32[o32], &c32[lane == 3 ? C32_V1L : C32_V2L]);
        } else if (o32 >= 0) {
            c32[o32] = (float)x;
        }
    }
}

// ------------------------------------------------------------ lane constants
__device__ __forceinline__ void load_pt32(const float *__restrict__ c, Pt32 &o) {
    o.p0 = c[C32_P0]; o.p1 = c[C32_P1]; o.q0 = c[C32_Q0]; o.q1 = c[C32_Q1]; o.q2 = c[C32_Q2];
    o.T0 = c[C32_T0]; o.c10 = c[C32_C10]; o.smt = c[C32_SMT];
    o.td0 = c[C32_TD0]; o.td1 = c[C32_TD1];
    o.d0 = c[C32_D0]; o.d1 = c[C32_D1]; o.d2 = c[C32_D2];
    o.g01 = c[C32_G01]; o.g02 = c[C32_G02]; o.g12 = c[C32_G12];
    o.v1h = c[C32_V1H]; o.v1l = c[C32_V1L]; o.v2h = c[C32_V2H]; o.v2l = c[C32_V2L];
    o.S0 = c[C32_S0]; o.PI0 = c[C32_PI0]; o.W0 = c[C32_W0]; o.E0 = c[C32_E0];
    o.S1 = c[C32_S1]; o.PI1 = c[C32_PI1]; o.W1 = c[C32_W1]; o.E1 = c[C32_E1];
    o.sd02 = c[C32_SD02]; o.sd01 = c[C32_SD01];
}
__device__ __forceinline__ void load_ch32(const float *__restrict__ c, int ch, Ch32 &o) {
    const int nubar = ch >= 9;
    const int ab = ch - 9 * nubar;
    const float *v = c + C32_CH + 8 * ab;
    const float sg = nubar ? -1.0f : 1.0f;  // antineutrino: U -> conj(U)
    o.X0r = v[0]; o.X0i = sg * v[1]; o.X1r = v[2]; o.X1i = sg * v[3]; o.X2r = v[4]; o.X2i = sg * v[5];
    o.Zr = v[6]; o.Zi = sg * v[7];
    o.ee = (ab == 0) ? 1.0f : 0.0f;
    o.diag = (ab == 0 || ab == 4 || ab == 8) ? 1.0f : 0.0f;
    o.zm = fabsf(o.Zr) + fabsf(o.Zi);
    o.real = ab == 4 || ab == 8;
}
__device__ __forceinline__ void load_pt64(const double *__restrict__ c, Pt64 &o) {
    o.p0 = c[C64_P0]; o.p1 = c[C64_P1]; o.q0 = c[C64_Q0]; o.q1 = c[C64_Q1]; o.q2 = c[C64_Q2];
    o.T0 = c[C64_T0]; o.c10 = c[C64_C10]; o.smt = c[C64_SMT];
    o.S0 = c[C64_SH]; o.PI0 = c[C64_SH + 1]; o.W0 = c[C64_SH + 2]; o.E0 = c[C64_SH + 3];
    o.S1 = c[C64_SH + 4]; o.PI1 = c[C64_SH + 5]; o.W1 = c[C64_SH + 6]; o.E1 = c[C64_SH + 7];
    o.d0 = c[C64_LD]; o.d1 = c[C64_LD + 1]; o.d2 = c[C64_LD + 2];
    o.V1 = c[C64_VG]; o.V2 = c[C64_VG + 1]; o.G12 = c[C64_VG + 2];
}
__device__ __forceinline__ void load_ch64(const double *__restrict__ c, int ch, Ch64 &o) {
    const int nubar = ch >= 9;
    const int ab = ch - 9 * nubar;
    const double *v = c + C64_CH + 6 * ab;
    const double sg = nubar ? -1.0 : 1.0;
    o.Xr = v[0]; o.Xi = sg * v[1]; o.Yr = v[2]; o.Yi = sg * v[3]; o.Zr = v[4]; o.Zi = sg * v[5];
    o.ee = (ab == 0) ? 1.0 : 0.0;
    o.diag = (ab == 0 || ab == 4 || ab == 8) ? 1.0 : 0.0;
}

// The FP64 path's probability of one event for one point, for the FP32
// precisions' events whose error estimate exceeds the tolerance (pc64: the
// point's FP64 constants; ch: channel id; E: E_true).  Out of line, so the FP32
// kernels' main loops keep their registers; it runs for few events.
static __device__ __noinline__ double prob_redo64(const double *__restrict__ pc64, int ch, float E, double kA_rhoye,
                                                  double cLL) {
    Pt64 c;
    Ch64 h;
    load_pt64(pc64, c);
    load_ch64(pc64, ch, h);
    const double Ad = kA_rhoye * (double)E;
    return prob_fp64(c, h, (ch >= 9) ? -Ad : Ad, tau64(cLL, E));
}


// -------------------------------------------------- 128-bit fixed-point bins
// A bin holds sum(w) * 2^F as a two's-complement 128-bit integer (lo, hi).
__device__ __forceinline__ void fx_add(unsigned long long &lo, unsigned long long &hi, unsigned long long l,
                                       unsigned long long h) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(l), "l"(h));
}
__device__ __forceinline__ void fx_add_f64(unsigned long long &lo, unsigned long long &hi, double y) {
    const double fl = floor(y);
    const long long h = __double2ll_rz(fl);
    const unsigned long long l = __double2ull_rz((y - fl) * 18446744073709551616.0);
    fx_add(lo, hi, l, (unsigned long long)h);
}
// Global bins hold kDigits integer columns: a flushed 128-bit value v is split
// into 32-bit digits v = d0 + d1 2^32 + d2 2^64 + d3 2^96 (d0, d1, d2 in
// [0, 2^32), d3 signed) and each digit is added with a fire-and-forget
// reduction.  Column sums are plain integer sums, so the result is exact and
// independent of the flush order, and a column wraps only after 2^32 flushes;
// the finalize kernel recombines the columns.
__device__ __forceinline__ void fx_flush(unsigned long long *p, unsigned long long lo, unsigned long long hi) {
    constexpr unsigned long long M32 = 0xFFFFFFFFull;
    const unsigned long long d0 = lo & M32, d1 = lo >> 32, d2 = hi & M32;
    const long long d3 = (long long)hi >> 32;
    if (d0) atomicAdd(p, d0);
    if (d1) atomicAdd(p + 1, d1);
    if (d2) atomicAdd(p + 2, d2);
    if (d3) atomicAdd(p + 3, (unsigned long long)d3);
}

// The kDigits columns of bin i of an accumulator array (L2 loads: other SMs' reductions).
struct Digits {
    unsigned long long d[kDigits];
};
__device__ __forceinline__ Digits load_digits(const unsigned long long *acc, int64_t i) {
    Digits g;
#pragma unroll
    for (int k = 0; k < kDigits; ++k) g.d[k] = __ldcg(acc + kDigits * i + k);
    return g;
}
__device__ __forceinline__ void clear_digits(unsigned long long *acc, int64_t i) {
#pragma unroll
    for (int k = 0; k < kDigits; ++k) acc[kDigits * i + k] = 0ull;
}

// Value of a bin: the digit columns depend on how runs were split into
// flushes; their combination, the exact 128-bit sum, does not, and only that
// is converted: (hi 2^64 + lo) 2^-F times the point's norm, with m0 = 2^(64-F)
// and m1 = 2^-F (both products exact, so the result does not depend on how the
// sum is contracted).
__device__ __forceinline__ double bin_value(const Digits &g, double m0, double m1, double norm) {
    const unsigned __int128 v = (unsigned __int128)g.d[0] + ((unsigned __int128)g.d[1] << 32) +
                                ((unsigned __int128)g.d[2] << 64) +
                                ((unsigned __int128)(__int128)(long long)g.d[3] << 96);
    const long long hi = (long long)(unsigned long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return ((double)hi * m0 + (double)lo * m1) * norm;
}
// m: the histogram's (2^(64-F), 2^-F, unused, point index)
__device__ __forceinline__ double final_bin(const Digits &g, const double *m, const double *pc64) {
    return bin_value(g, m[0], m[1], pc64[(int64_t)m[3] * C64_STRIDE + C64_NORM]);
}

// Small outputs (one conversion round: up to 256 bins for a block, 128 for a
// warp; larger outputs go to the finalize kernel, launched programmatically):
// the last block or warp of the histogram kernel to finish converts the bins
// instead of a separate launch (or, for the FP32 precisions, the FP64
// recomputation pass launched after it does, which waits for the whole grid
// anyway).  Every thread fences its own flushes before its
// block or warp takes its completion ticket.  The last one runs alone at the
// end of the grid, so it issues the loads of all its bins (digit columns and
// histogram scales, then the points' norms) before it converts any of them.
__device__ __forceinline__ void fused_final(const HistParams &prm) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(prm.counter + 1, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int64_t n = prm.fin_n_hist * (int64_t)prm.nbins;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const Digits g = load_digits(prm.acc, i);
        const double *m = prm.fin_hmeta + 4 * (i / prm.nbins);
        const double m0 = m[0], m1 = m[1];
        const double nm = prm.pc64[(int64_t)m[3] * C64_STRIDE + C64_NORM];
        clear_digits(prm.acc, i);
        prm.fin_out[i] = bin_value(g, m0, m1, nm);
    }
    if (threadIdx.x == 0) {
        prm.counter[0] = 0;
        prm.counter[1] = 0;
    }
}

// The histogram metadata (scales, point index) of a thread's first bin: written
// by the host before any launch, so it can be read before a kernel's
// grid-dependency wait; and, loaded after the wait, that bin's digit columns and
// norm.
struct FinMeta {
    double m0 = 0.0, m1 = 0.0, pt = 0.0, nm = 0.0;
    bool loaded = false;
    Digits d{};
};
// The converting group's threads g = 0 .. G - 1 take bins g, g + G, ... of the output.
__device__ __forceinline__ void fin_meta_load(const HistParams &prm, FinMeta &fm, int g) {
    if (g < prm.fin_n_hist * (int64_t)prm.nbins) {
        const double *m = prm.fin_hmeta + 4 * (g / prm.nbins);
        fm.m0 = m[0];
        fm.m1 = m[1];
        fm.pt = m[3];
    }
}
// After the wait: the bin's digit columns and norm, issued together with the
// caller's other loads (they go unused when the pass has events to recompute).
__device__ __forceinline__ void fin_data_load(const HistParams &prm, FinMeta &fm, int g) {
    if (g < prm.fin_n_hist * (int64_t)prm.nbins) {
        fm.d = load_digits(prm.acc, g);
        fm.nm = prm.pc64[(int64_t)fm.pt * C64_STRIDE + C64_NORM];
    }
    fm.loaded = true;
}
// Converts every bin of the output (kU bins per thread and round) and resets the
// work counters; the group is threads g = 0 .. G - 1 (one warp: G = 32).
__device__ __forceinline__ void convert_bins(const HistParams &prm, int g, int G, const FinMeta *pre) {
    constexpr int kU = 4;
    const int64_t n = prm.fin_n_hist * (int64_t)prm.nbins;
    for (int64_t i0 = 0; i0 < n; i0 += (int64_t)G * kU) {
        Digits d[kU];
        double m0[kU], m1[kU], nm[kU];
        bool norm_in[kU];  // the norm itself (loaded ahead) rather than the point index
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t i = i0 + g + (int64_t)G * k;
            const bool ahead = pre && i0 == 0 && k == 0;  // the thread's first bin, loaded ahead
#pragma unroll
            for (int q = 0; q < kDigits; ++q) d[k].d[q] = 0ull;
            m0[k] = m1[k] = nm[k] = 0.0;
            norm_in[k] = ahead && pre->loaded;
            if (i < n) {
                if (ahead) {
                    m0[k] = pre->m0;
                    m1[k] = pre->m1;
                    nm[k] = pre->loaded ? pre->nm : pre->pt;
                } else {
                    const double *m = prm.fin_hmeta + 4 * (i / prm.nbins);
                    m0[k] = m[0];
                    m1[k] = m[1];
                    nm[k] = m[3];
                }
                d[k] = (ahead && pre->loaded) ? pre->d : load_digits(prm.acc, i);
            }
        }
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (!norm_in[k] && i0 + g + (int64_t)G * k < n) nm[k] = prm.pc64[(int64_t)nm[k] * C64_STRIDE + C64_NORM];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t i = i0 + g + (int64_t)G * k;
            if (i < n) {
                clear_digits(prm.acc, i);
                prm.fin_out[i] = bin_value(d[k], m0[k], m1[k], nm[k]);
            }
        }
    }
    if (g == 0) {
        prm.counter[0] = 0;
        prm.counter[1] = 0;
    }
}
// The last warp's conversion of the fused finalize (four bins per lane per round,
// all loads of a round issued before any conversion), then the counter reset.
__device__ __forceinline__ void convert_bins_warp(const HistParams &prm) { convert_bins(prm, threadIdx.x & 31, 32, nullptr); }
// Per-warp variant for one-point items: warps that finish early exit without
// waiting at a block barrier; the last warp converts four bins per lane per round.
__device__ __forceinline__ void fused_final_warp(const HistParams &prm) {
    const int lane = threadIdx.x & 31;
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = (atomicAdd(prm.counter + 1, 1) == (int)(gridDim.x * (blockDim.x >> 5)) - 1);
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    convert_bins_warp(prm);
}

// Bin one weighted event under the point's energy scale and add it to the lane's
// run-length accumulator (flushing the previous bin when the bin changes).
// FP64: the 128-bit value (lo, hi).
struct RunAcc {
    unsigned long long lo = 0, hi = 0;
    int cur_b = -1;
};
// FP32 precisions: each addend is below 2^63 and a lane's run holds fewer than
// 2^31 events, so the run fits a 96-bit two's-complement sum a0 + a1 2^32 + a2 2^64
// (a2 signed), three 32-bit limbs added with one carry chain.  A negative addend
// enters as its one's complement; neg counts them, the +1 each that completes
// the two's complement, added when the run's value is read.
struct RunAcc32 {
    unsigned a0 = 0, a1 = 0, a2 = 0, neg = 0;
    int cur_b = -1;
};
template <int PREC>
struct AccOf { using T = RunAcc32; };
template <>
struct AccOf<kFP64> { using T = RunAcc; };

// The run's 128-bit value: (lo, hi) with hi the sign extension of a2.
__device__ __forceinline__ void run_value(const RunAcc32 &r, unsigned long long &lo, unsigned long long &hi) {
    const unsigned long long l = ((unsigned long long)r.a1 << 32) | r.a0;
    lo = l + r.neg;
    hi = (unsigned long long)(long long)(int)(r.a2 + (lo < l ? 1u : 0u));
}
__device__ __forceinline__ void run_value(const RunAcc &r, unsigned long long &lo, unsigned long long &hi) {
    lo = r.lo;
    hi = r.hi;
}
__device__ __forceinline__ void run_clear(RunAcc32 &r) { r.a0 = r.a1 = r.a2 = r.neg = 0; }
__device__ __forceinline__ void run_clear(RunAcc &r) { r.lo = r.hi = 0; }
template <class R>
__device__ __forceinline__ void run_flush(const R &r, unsigned long long *accp) {
    unsigned long long lo, hi;
    run_value(r, lo, hi);
    if (r.cur_b >= 0 && (lo | hi)) fx_flush(accp + kDigits * r.cur_b, lo, hi);
}

// The addend of weight w: x = |w| 2^F truncated to an integer (bits below the
// fixed-point LSB 2^-F dropped), returned as its two 32-bit halves, for one or
// two weights.  F = 62 - ceil(log2 max|w_mc|) per sample, so x < 2^63.
// x is formed by two exact power-of-two scalings (2^(F-64), then 2^64; F - 64
// is a normal exponent for every F in [8, 190], and subnormal w scale exactly)
// and split into 32-bit halves with float operations, each exact: the high half
// floor(x 2^-32) and the remainder x - 2^32 floor(x 2^-32) are floats with at
// most 24 significant bits, and both 32-bit conversions truncate toward zero.
// (A 64-bit float-to-integer conversion is an FP64-pipe instruction on this
// GPU; the two 32-bit ones are not.)  sh = F - 150.
template <class V>
__device__ __forceinline__ void fx_halves(V wabs, int sh, V &hf, V &lf) {
    const V x = vmul(vmul(wabs, vb<V>(__int_as_float((sh + 213) << 23))), vb<V>(18446744073709551616.0f));
    hf = vmap(vmul(x, vb<V>(2.3283064365386963e-10f)), [](float v) { return floorf(v); });
    lf = vfma(hf, vb<V>(-4294967296.0f), x);
}
// Adds hi 2^32 + lo to the lane's run, negated when m = 0xffffffff (the weight's
// sign, spread over 32 bits; m = 0: as is), without a branch: the one's
// complement (lo ^ m, hi ^ m, m) goes through the carry chain and r.neg counts
// the missing +1.
__device__ __forceinline__ void fx_add3(RunAcc32 &r, unsigned hi, unsigned lo, unsigned m) {
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(r.a0), "+r"(r.a1), "+r"(r.a2)
        : "r"(lo ^ m), "r"(hi ^ m), "r"(m));
    r.neg -= m;  // +1 for m = 0xffffffff
}
// The sign of w as a 32-bit mask (all ones for a negative w).
__device__ __forceinline__ unsigned sign_mask(float w) { return (unsigned)((int)__float_as_uint(w) >> 31); }
// One event: tb = sf E_reco - lo and u = tb / width (by the reciprocal width)
// decide the bin; (hf, lf) are its addend's halves (zero for an event outside
// the histogram or inactive, which then changes nothing), m its sign mask.
__device__ __forceinline__ void acc_event_u(RunAcc32 &r, unsigned long long *accp, const HistParams &prm, float tb,
                                            float u, float hf, float lf, unsigned m, bool in) {
    const int b = __float2int_rz(u);
    unsigned h = __float2uint_rz(hf), l = __float2uint_rz(lf);
    if (in && !debug_ok(b >= 0 && b < prm.nbins, prm.counter, kDbgBin)) {
        in = false;
        h = l = m = 0u;
    }
    if (in && b != r.cur_b) {
        run_flush(r, accp);
        run_clear(r);
        r.cur_b = b;
    }
    fx_add3(r, h, l, m);
}
__device__ __forceinline__ void acc_event_f32(RunAcc32 &r, unsigned long long *accp, const HistParams &prm, float sf,
                                              float er, float wt, int sh, bool active) {
    const float tb = vsub(vmul(sf, er), prm.lo_f);
    const float u = vmul(tb, prm.inv_f);
    const bool in = active && tb >= 0.0f && u < prm.nb_f;
    float hf, lf;
    fx_halves(in ? fabsf(wt) : 0.0f, sh, hf, lf);
    acc_event_u(r, accp, prm, tb, u, hf, lf, sign_mask(wt), in);
}
// Two events in order (a, then b), their bin and addend arithmetic in one packed
// chain: the same bins and sums as two acc_event_f32 calls.
__device__ __forceinline__ void acc_pair_f32(RunAcc32 &r, unsigned long long *accp, const HistParams &prm, float sf,
                                             float2 er, float2 wt, int sh, bool act_a, bool act_b) {
    const float2 tb = vsub(vmul(vb<float2>(sf), er), vb<float2>(prm.lo_f));
    const float2 u = vmul(tb, vb<float2>(prm.inv_f));
    const bool in_a = act_a && tb.x >= 0.0f && u.x < prm.nb_f;
    const bool in_b = act_b && tb.y >= 0.0f && u.y < prm.nb_f;
    float2 hf, lf;
    fx_halves(make_float2(in_a ? fabsf(wt.x) : 0.0f, in_b ? fabsf(wt.y) : 0.0f), sh, hf, lf);
    acc_event_u(r, accp, prm, tb.x, u.x, hf.x, lf.x, sign_mask(wt.x), in_a);
    acc_event_u(r, accp, prm, tb.y, u.y, hf.y, lf.y, sign_mask(wt.y), in_b);
}
__device__ __forceinline__ void acc_event_f64(RunAcc &r, unsigned long long *accp, const HistParams &prm, float sf,
                                              float er, double wt, double hs, bool active) {
    const float x = __fmul_rn(sf, er);
    const float tb = __fsub_rn(x, prm.lo_f);
    const float u = __fmul_rn(tb, prm.inv_f);
    if (active && tb >= 0.0f && u < prm.nb_f) {
        const int b = __float2int_rz(u);
        if (!debug_ok(b >= 0 && b < prm.nbins, prm.counter, kDbgBin)) return;
        if (b != r.cur_b) {
            if (r.cur_b >= 0 && (r.lo | r.hi)) fx_flush(accp + kDigits * r.cur_b, r.lo, r.hi);
            r.lo = r.hi = 0;
            r.cur_b = b;
        }
        fx_add_f64(r.lo, r.hi, wt * hs);
    }
}
template <class R>
__device__ __forceinline__ void acc_finish(R &r, unsigned long long *accp) {
    run_flush(r, accp);
}
// End of a per-warp work item: lanes that end in the same bin (the lanes hold
// consecutive sorted events, so such lanes are normally contiguous) first sum
// their 128-bit values with shuffles, exactly, and one lane flushes the total.
template <class R>
__device__ __forceinline__ void acc_finish_warp(R &r, unsigned long long *accp) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    unsigned long long lo, hi;
    run_value(r, lo, hi);
    const bool has = r.cur_b >= 0 && (lo | hi);
    const int key = has ? r.cur_b : -1 - lane;
    const unsigned mask = __match_any_sync(0xffffffffu, key);
    const int first = __ffs(mask) - 1;
    const int cnt = __popc(mask);
    const bool contiguous = (mask >> first) == ((cnt == 32) ? 0xffffffffu : ((1u << cnt) - 1u));
    if (!__all_sync(0xffffffffu, contiguous)) {
        acc_finish(r, accp);
        return;
    }
    const int end = first + cnt;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, d);
        const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, d);
        if (lane + d < end) fx_add(lo, hi, l2, h2);
    }
    if (has && lane == first && (lo | hi)) fx_flush(accp + kDigits * r.cur_b, lo, hi);
}

// Counts a work item marked for the FP64 recomputation pass.
__device__ __forceinline__ void mark_redo(const HistParams &prm) { atomicAdd(prm.counter + kRedoCount, 1); }

// FP32 matter term A = +-k_A rho Y_e E and c_L L / (2 pi E) as a float-float
// th + tl, for one or two events (kA: +-k_A rho Y_e per lane), returned as
// (A, th, -tl).  1/E = r0 + rl to ~1e-14: the residual 1 - E r0 of the
// approximate reciprocal is exact in FP32; r0 enters negated (rcp(-E)), which
// negates rl and the whole low part without a packed negation.
template <class V>
__device__ __forceinline__ void event_terms_bulk(const SampleDev &sd, V E, V kA, V &A, V &th, V &ntl) {
    A = vmul(kA, E);
    const V r0n = vmap(E, [](float v) { return rcp_approx(-v); });  // -r0
    const V rln = vmul(r0n, vfma(E, r0n, vb<V>(1.0f)));               // -rl
    th = vmul(vb<V>(-sd.rev_hi), r0n);  // |tl| stays below ulp(th): no renormalisation needed
    ntl = vfma(vb<V>(sd.rev_lo), r0n, vfma(vb<V>(sd.rev_hi), rln, vfma(vb<V>(sd.rev_hi), r0n, th)));
}
__device__ __forceinline__ float kA_lane(const SampleDev &sd, int ch) {
    return (ch >= 9) ? -sd.kA_rhoye_f : sd.kA_rhoye_f;
}
// One event, as (A, th, tl).
__device__ __forceinline__ void event_terms32(const SampleDev &sd, float E, int ch, float &A, float &th, float &tl) {
    float ntl;
    event_terms_bulk(sd, E, kA_lane(sd, ch), A, th, ntl);
    tl = -ntl;
}

// ------------------------------------------------------------ event staging
struct Stage32 {  // one array per field: a lane's two events (j, j + 1) load as packed pairs
    float A[kET];    // signed matter term
    float th[kET];   // c_L L / (2 pi E) float-float: th, -tl
    float ntl[kET];
    float er[kET];   // e_reco
    float w[kET];    // w_mc
    int ch[kET];     // channel
};
struct Stage64 {
    double a[kET];
    double tau[kET];     // c_L L / E as hi + lo (FP32_F64EIG: c_L L / (2 pi E), revolutions per eV^2)
    double tau_lo[kET];
    float2 ew[kET];  // (e_reco, w_mc)
    int ch[kET];
};

__device__ __forceinline__ void stage_one32(Stage32 &s, int j, const SampleDev &sd, float E, float er, float w, int ch) {
    event_terms_bulk(sd, E, kA_lane(sd, ch), s.A[j], s.th[j], s.ntl[j]);
    s.er[j] = er;
    s.w[j] = w;
    s.ch[j] = ch;
}
__device__ __forceinline__ void stage_one64(Stage64 &s, int j, const SampleDev &sd, float E, float er, float w, int ch) {
    const double Ad = sd.kA_rhoye * (double)E;
    s.a[j] = (ch >= 9) ? -Ad : Ad;
    const Tau64 t = tau64(sd.cLL, E);
    s.tau[j] = t.hi;
    s.tau_lo[j] = t.lo;
    s.ew[j] = make_float2(er, w);
    s.ch[j] = ch;
}

// FP32_F64EIG: the FP64 matter term and c_L L / (2 pi E) [revolutions per eV^2]
// from the float-float of event_terms32, as the one-point path forms it (so both
// paths, and the FP64 recomputation, take the same decisions on the same events).
__device__ __forceinline__ void stage_one_mix(Stage64 &s, int j, const SampleDev &sd, float E, float er, float w, int ch) {
    float A, th, tl;
    event_terms32(sd, E, ch, A, th, tl);
    const double Ad = sd.kA_rhoye * (double)E;
    s.a[j] = (ch >= 9) ? -Ad : Ad;
    s.tau[j] = (double)th + (double)tl;
    s.ew[j] = make_float2(er, w);
    s.ch[j] = ch;
}

template <int PREC>
struct StageOf { using T = Stage32; };
template <>
struct StageOf<kFP64> { using T = Stage64; };
template <>
struct StageOf<kMix> { using T = Stage64; };

// Load tile [base, base + nt) of the item into shared memory: one 16-byte event
// record per load, consecutive threads on consecutive events.
template <int PREC>
__device__ __forceinline__ void stage_tile(typename StageOf<PREC>::T &s, const SampleDev &sd, int64_t base, int nt) {
#pragma unroll
    for (int k = 0; k < kET / kNT; ++k) {
        const int j = threadIdx.x + k * kNT;
        if (j < nt) {
            const float4 r = sd.ev[base + j];
            if (PREC == kFP32)
                stage_one32(reinterpret_cast<Stage32 &>(s), j, sd, r.x, r.y, r.z, __float_as_int(r.w));
            else if (PREC == kMix)
                stage_one_mix(reinterpret_cast<Stage64 &>(s), j, sd, r.x, r.y, r.z, __float_as_int(r.w));
            else
                stage_one64(reinterpret_cast<Stage64 &>(s), j, sd, r.x, r.y, r.z, __float_as_int(r.w));
        }
    }
}

// One point per work item (points_per_block = 1): lanes share nothing, so each
// warp takes work items on its own (no block barriers) and each lane reads its
// events straight from global memory -- events ev_begin + lane + 32 k, coalesced
// across the warp -- two per iteration for instruction-level parallelism, with
// the next two prefetched into registers.  The ticket of the warp's next item is
// fetched a whole item ahead, and the sample scalars and point constants are
// reloaded only when the item's sample or point changes.
// pc_inline (FP32 bulk, one point): the point's FP32 constants, read in place
// (a kernel parameter) instead of from the constants table.
template <int PREC>
__device__ __forceinline__ void hist_items_per_warp(const HistParams &prm, const float *pc_inline = nullptr) {
    const int lane = threadIdx.x & 31;
    const int n_warps = (int)(gridDim.x * (blockDim.x >> 5));
    const int gw = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    // The first item of every warp (and, when items are plentiful, the second)
    // is assigned statically, so the grid does not start with one atomic per
    // warp on the same counter; later tickets come from the counter, offset
    // past the static ones.  A second ticket is held ahead only when items are
    // plentiful (a warp holding two tickets of a scarce list would leave other
    // warps idle), and only until the last 2 x n_warps tickets: the list is
    // sorted largest first, so those are its shortest items, and a warp holding
    // one of them ahead when the counter runs out would end the grid up to two
    // items after the first idle warp instead of one.
    const bool ahead = prm.n_items >= 3 * n_warps;
    const int dyn0 = ahead ? 2 * n_warps : n_warps;
    int it = gw, nxt = ahead ? gw + n_warps : 0;
    int cur_sample = -1, cur_point = -1, cur_ch = -1;
    SampleDev sd;
    Pt32 c32;
    Ch32 h32;
    Pt64 c64;
    Ch64 h64;
    const float *pc32 = nullptr;
    const double *pc64 = nullptr;
    float sf = 1.0f;
    // The item in hand: its descriptor and each lane's first two events.
    WorkItem wi{};
    const float4 *ev = nullptr;  // 32-bit offsets within the item (items hold fewer than 2^31 events)
    int end = 0;
    float Ea = 1.0f, ra = 0.0f, wa = 0.0f, Eb = 1.0f, rb = 0.0f, wb = 0.0f;
    int ca = 0, cb = 0;
    auto fetch = [&](int idx) {
        wi = prm.items[idx];
        if (wi.sample != cur_sample) {
            cur_sample = wi.sample;
            sd = prm.samples[wi.sample];
        }
        ev = sd.ev + wi.ev_begin;
        end = debug_ok(wi.ev_begin >= 0 && wi.ev_count >= 0 && wi.ev_begin + wi.ev_count <= sd.n, prm.counter,
                       kDbgItem) ? wi.ev_count : 0;
        Ea = 1.0f; ra = 0.0f; wa = 0.0f; ca = 0;
        Eb = 1.0f; rb = 0.0f; wb = 0.0f; cb = 0;
        if (lane < end) {
            const float4 q = ev[lane];
            Ea = q.x; ra = q.y; wa = q.z; ca = __float_as_int(q.w);
        }
        if (lane + 32 < end) {
            const float4 q = ev[lane + 32];
            Eb = q.x; rb = q.y; wb = q.z; cb = __float_as_int(q.w);
        }
    };
    // The item list, the sample descriptors and the events are never written by
    // a kernel, so the first item is fetched before the grid-dependency wait:
    // under a programmatic dependent launch this overlaps the constants kernel.
    // The first sample's descriptor is loaded beside the first item instead of
    // after it (one dependent memory round trip less at the grid's start; an
    // item of another sample reloads it).
    if (it < prm.n_items) {
        sd = prm.samples[0];
        cur_sample = 0;
        fetch(it);
    }
    grid_dependency_wait();
    while (it < prm.n_items) {
        if (wi.point_base != cur_point) {
            cur_point = wi.point_base;
            cur_ch = -1;
            if (PREC != kFP64) {
                pc32 = pc_inline ? pc_inline : prm.pc32 + (int64_t)wi.point_base * C32_STRIDE;
                load_pt32(pc32, c32);
                sf = pc32[C32_ESCALE];
            }
            if (PREC != kFP32) {
                pc64 = prm.pc64 + (int64_t)wi.point_base * C64_STRIDE;
                load_pt64(pc64, c64);
                sf = (float)pc64[C64_ESCALE];
            }
        }
        unsigned long long *accp = prm.acc + kDigits * wi.acc_base * (int64_t)prm.nbins;
        typename AccOf<PREC>::T r;
        bool redo = false;  // an event of this item is left to the FP64 recomputation (k_redo)
        int e = lane;
        if constexpr (PREC == kFP32) {
            const int sh = sd.frac_bits - 150;
            for (; e < end; e += 64) {
                const bool has_b = e + 32 < end;
                const int en = e + 64;
                float Ena = 1.0f, rna = 0.0f, wna = 0.0f, Enb = 1.0f, rnb = 0.0f, wnb = 0.0f;
                int cna = 0, cnb = 0;
                if (en < end) {
                    const float4 q = ev[en];
                    Ena = q.x; rna = q.y; wna = q.z; cna = __float_as_int(q.w);
                }
                if (en + 32 < end) {
                    const float4 q = ev[en + 32];
                    Enb = q.x; rnb = q.y; wnb = q.z; cnb = __float_as_int(q.w);
                }
                if (ca == cur_ch && (!has_b || cb == cur_ch)) {
                    // both events in one packed chain
                    float2 A, th, ntl;
                    event_terms_bulk(sd, make_float2(Ea, Eb), make_float2(kA_lane(sd, ca), kA_lane(sd, cb)), A, th,
                                     ntl);
                    unsigned x;
                    const float2 P = h32.real ? prob_bulk<true>(c32, h32, A, th, ntl, x)
                                              : prob_bulk<false>(c32, h32, A, th, ntl, x);
                    const bool xa = x & 1u, xb = has_b && (x & 2u);
                    redo = redo || xa || xb;
                    acc_pair_f32(r, accp, prm, sf, make_float2(ra, rb), vmul(P, make_float2(wa, wb)), sh, !xa,
                                 has_b && !xb);
                } else {
                    for (int k = 0; k < 2; ++k) {
                        const float E = k ? Eb : Ea, er = k ? rb : ra, w = k ? wb : wa;
                        const int ch = k ? cb : ca;
                        if (k && !has_b) break;
                        if (ch != cur_ch) {
                            cur_ch = ch;
                            load_ch32(pc32, ch, h32);
                        }
                        float A, th, tl;
                        event_terms32(sd, E, ch, A, th, tl);
                        bool x;
                        const float P = prob_fp32(c32, h32, A, th, tl, x);
                        redo = redo || x;
                        acc_event_f32(r, accp, prm, sf, er, P * w, sh, !x);
                    }
                }
                Ea = Ena; ra = rna; wa = wna; ca = cna;
                Eb = Enb; rb = rnb; wb = wnb; cb = cnb;
            }
        } else if constexpr (PREC == kMix) {
            const int sh = sd.frac_bits - 150;
            for (; e < end; e += 64) {
                const bool has_b = e + 32 < end;
                const int en = e + 64;
                float Ena = 1.0f, rna = 0.0f, wna = 0.0f, Enb = 1.0f, rnb = 0.0f, wnb = 0.0f;
                int cna = 0, cnb = 0;
                if (en < end) {
                    const float4 q = ev[en];
                    Ena = q.x; rna = q.y; wna = q.z; cna = __float_as_int(q.w);
                }
                if (en + 32 < end) {
                    const float4 q = ev[en + 32];
                    Enb = q.x; rnb = q.y; wnb = q.z; cnb = __float_as_int(q.w);
                }
                for (int k = 0; k < 2; ++k) {
                    const float E = k ? Eb : Ea, er = k ? rb : ra, w = k ? wb : wa;
                    const int ch = k ? cb : ca;
                    if (k && !has_b) break;
                    if (ch != cur_ch) {
                        cur_ch = ch;
                        load_ch32(pc32, ch, h32);
                    }
                    float A, th, tl;
                    event_terms32(sd, E, ch, A, th, tl);
                    const double Ad = sd.kA_rhoye * (double)E;
                    bool x;
                    const float P = prob_mix(c32, h32, c64, (ch >= 9) ? -Ad : Ad, (double)th + (double)tl, x);
                    redo = redo || x;
                    acc_event_f32(r, accp, prm, sf, er, P * w, sh, !x);
                }
                Ea = Ena; ra = rna; wa = wna; ca = cna;
                Eb = Enb; rb = rnb; wb = wnb; cb = cnb;
            }
        } else {
            const double hs = sd.hscale_d;
            for (; e < end; e += 64) {
                const bool has_b = e + 32 < end;
                const int en = e + 64;
                float Ena = 1.0f, rna = 0.0f, wna = 0.0f, Enb = 1.0f, rnb = 0.0f, wnb = 0.0f;
                int cna = 0, cnb = 0;
                if (en < end) {
                    const float4 q = ev[en];
                    Ena = q.x; rna = q.y; wna = q.z; cna = __float_as_int(q.w);
                }
                if (en + 32 < end) {
                    const float4 q = ev[en + 32];
                    Enb = q.x; rnb = q.y; wnb = q.z; cnb = __float_as_int(q.w);
                }
                for (int k = 0; k < 2; ++k) {
                    const float E = k ? Eb : Ea, er = k ? rb : ra, w = k ? wb : wa;
                    const int ch = k ? cb : ca;
                    if (k && !has_b) break;
                    if (ch != cur_ch) {
                        cur_ch = ch;
                        load_ch64(pc64, ch, h64);
                    }
                    const double Ad = sd.kA_rhoye * (double)E;
                    const double P = prob_fp64(c64, h64, (ch >= 9) ? -Ad : Ad, tau64(sd.cLL, E));
                    acc_event_f64(r, accp, prm, sf, er, P * (double)w, hs, true);
                }
                Ea = Ena; ra = rna; wa = wna; ca = cna;
                Eb = Enb; rb = rnb; wb = wnb; cb = cnb;
            }
        }
        if constexpr (PREC != kFP64) {
            // mark the item for the FP64 recomputation of its left-out events
            const bool any = __any_sync(0xffffffffu, redo);
            if (any && lane == 0) {
                prm.redo[it] = 1;
                mark_redo(prm);
            }
        }
        // move to the ticket held ahead and fetch the one after it (none, -1,
        // from the last 2 x n_warps tickets on), or (few items, or none held)
        // take the next ticket now; the next item's first events are in flight
        // while this item's runs are closed
        if (ahead) {
            it = __shfl_sync(0xffffffffu, nxt, 0);
            if (it < 0) {
                if (lane == 0) it = atomicAdd(prm.counter, 1) + dyn0;
                it = __shfl_sync(0xffffffffu, it, 0);
            }
            if (lane == 0) nxt = it < prm.n_items - dyn0 ? atomicAdd(prm.counter, 1) + dyn0 : -1;
        } else {
            if (lane == 0) it = atomicAdd(prm.counter, 1) + dyn0;
            it = __shfl_sync(0xffffffffu, it, 0);
        }
        if (it < prm.n_items) fetch(it);
        acc_finish_warp(r, accp);
    }
}

// ----------------------------------------------------------- histogram kernel
// Lane layout for points_per_block PT > 1: PT points x (kNT / PT) event slices.
// Lane (pt, sl) handles point pt of the tile and the tile events sl, sl + S,
// sl + 2S, ... (S = kNT / PT), an increasing subsequence of the sorted events, so
// its bin sequence is monotone within a channel and a register run-length
// accumulator suffices.  Two events are computed per iteration.
// Resident blocks per SM: the 256-point tile fits three blocks (80 registers,
// no spills) and gains from the extra warps; the one-point path needs more
// registers for its two events in flight, and FP64 more still.  The FP32-bulk
// one-point kernel, whose work items are per warp, runs 128-thread blocks, five
// per SM: at 96 registers (a few bytes of spills outside the event loop) they
// hold 20 warps per SM, where two 256-thread blocks of 125 registers hold 16.
template <int PREC, int PT>
constexpr int hist_block_threads() {
    return (PREC == kFP32 && PT == 1) ? 128 : kNT;
}
template <int PREC, int PT>
constexpr int hist_min_blocks() {
    return PREC == kFP64 ? 1 : (PT == 256 ? 3 : ((PREC == kFP32 && PT == 1) ? 4 : 2));
}

template <int PREC, int PT>
__global__ void __launch_bounds__((hist_block_threads<PREC, PT>()), (hist_min_blocks<PREC, PT>()))
    k_hist(const HistParams prm) {
    // a finalize kernel after this one (programmatic launch) may become resident
    // as blocks of this grid retire; it waits for the whole grid
    grid_dependents_launch();
    if constexpr (PT == 1) {
        hist_items_per_warp<PREC>(prm);
        // with an FP64 recomputation pass after it (prm.redo), that kernel converts the bins
        if (prm.fuse_final && !prm.redo) fused_final_warp(prm);
        return;
    } else {
        constexpr int S = kNT / PT;
        __shared__ typename StageOf<PREC>::T stg;
        __shared__ int s_item;
        grid_dependency_wait();
        const int tid = threadIdx.x;
        const int lp = tid % PT;
        const int sl = tid / PT;
        for (;;) {
            __syncthreads();
            if (tid == 0) s_item = atomicAdd(prm.counter, 1);
            __syncthreads();
            const int it = s_item;
            if (it >= prm.n_items) break;
            const WorkItem wi = prm.items[it];
            const SampleDev sd = prm.samples[wi.sample];
            if (!debug_ok(wi.ev_begin >= 0 && wi.ev_count >= 0 && wi.ev_begin + wi.ev_count <= sd.n, prm.counter,
                          kDbgItem))
                continue;
            const bool active = lp < wi.n_pts;
            const int pidx = wi.point_base + (active ? lp : wi.n_pts - 1);
            unsigned long long *accp = prm.acc + kDigits * (wi.acc_base + lp) * (int64_t)prm.nbins;
            typename AccOf<PREC>::T r;
            int cur_ch = -1;
            bool redo = false;  // an event of this item is left to the FP64 recomputation (k_redo)
            if constexpr (PREC == kFP32) {
                const float *pc = prm.pc32 + (int64_t)pidx * C32_STRIDE;
                Pt32 c;
                load_pt32(pc, c);
                Ch32 h;
                const float sf = pc[C32_ESCALE];
                const int sh = sd.frac_bits - 150;
                for (int t0 = 0; t0 < wi.ev_count; t0 += kET) {
                    const int nt = min(kET, wi.ev_count - t0);
                    __syncthreads();
                    stage_tile<PREC>(stg, sd, wi.ev_begin + t0, nt);
                    __syncthreads();
                    const Stage32 &s = reinterpret_cast<const Stage32 &>(stg);
                    // lane sl takes the event pairs (2 sl, 2 sl + 1), (2 (sl + S), ...): an
                    // increasing sequence, so its bins are monotone within a channel
                    for (int j = 2 * sl; j < nt; j += 2 * S) {
                        const bool has_b = j + 1 < nt;  // j + 1 < kET: a stale value past nt is never used
                        const int ca = s.ch[j], cb = has_b ? s.ch[j + 1] : ca;
                        if (ca == cur_ch && cb == cur_ch) {
                            // both events in one packed chain
                            const float2 A = *reinterpret_cast<const float2 *>(s.A + j);
                            const float2 th = *reinterpret_cast<const float2 *>(s.th + j);
                            const float2 ntl = *reinterpret_cast<const float2 *>(s.ntl + j);
                            unsigned x;
                            const float2 P = h.real ? prob_bulk<true>(c, h, A, th, ntl, x)
                                                    : prob_bulk<false>(c, h, A, th, ntl, x);
                            const bool xa = x & 1u, xb = has_b && (x & 2u);
                            redo = redo || (active && (xa || xb));
                            acc_pair_f32(r, accp, prm, sf, *reinterpret_cast<const float2 *>(s.er + j),
                                         vmul(P, *reinterpret_cast<const float2 *>(s.w + j)), sh, active && !xa,
                                         active && has_b && !xb);
                        } else {
                            for (int k = 0; k < 2; ++k) {
                                if (k && !has_b) break;
                                const int jj = j + k;
                                const int ch = k ? cb : ca;
                                if (ch != cur_ch) {
                                    cur_ch = ch;
                                    load_ch32(pc, ch, h);
                                }
                                unsigned x;
                                const float P = h.real ? prob_bulk<true>(c, h, s.A[jj], s.th[jj], s.ntl[jj], x)
                                                       : prob_bulk<false>(c, h, s.A[jj], s.th[jj], s.ntl[jj], x);
                                redo = redo || (active && x);
                                acc_event_f32(r, accp, prm, sf, s.er[jj], vmul(P, s.w[jj]), sh, active && !x);
                            }
                        }
                    }
                }
            } else if constexpr (PREC == kMix) {
                const float *pc = prm.pc32 + (int64_t)pidx * C32_STRIDE;
                Pt32 c;
                load_pt32(pc, c);
                Pt64 c64;
                load_pt64(prm.pc64 + (int64_t)pidx * C64_STRIDE, c64);
                Ch32 h;
                const float sf = pc[C32_ESCALE];
                const int sh = sd.frac_bits - 150;
                for (int t0 = 0; t0 < wi.ev_count; t0 += kET) {
                    const int nt = min(kET, wi.ev_count - t0);
                    __syncthreads();
                    stage_tile<PREC>(stg, sd, wi.ev_begin + t0, nt);
                    __syncthreads();
                    const Stage64 &s = reinterpret_cast<const Stage64 &>(stg);
                    for (int j = sl; j < nt; j += S) {
                        const int ch = s.ch[j];
                        if (ch != cur_ch) {
                            cur_ch = ch;
                            load_ch32(pc, ch, h);
                        }
                        bool x;
                        const float P = prob_mix(c, h, c64, s.a[j], s.tau[j], x);
                        redo = redo || (active && x);
                        const float2 ew = s.ew[j];
                        acc_event_f32(r, accp, prm, sf, ew.x, P * ew.y, sh, active && !x);
                    }
                }
            } else {
                const double *pc = prm.pc64 + (int64_t)pidx * C64_STRIDE;
                Pt64 c;
                load_pt64(pc, c);
                Ch64 h;
                const float sf = (float)pc[C64_ESCALE];
                const double hs = sd.hscale_d;
                for (int t0 = 0; t0 < wi.ev_count; t0 += kET) {
                    const int nt = min(kET, wi.ev_count - t0);
                    __syncthreads();
                    stage_tile<PREC>(stg, sd, wi.ev_begin + t0, nt);
                    __syncthreads();
                    const Stage64 &s = reinterpret_cast<const Stage64 &>(stg);
                    for (int j = sl; j < nt; j += S) {
                        const int ch = s.ch[j];
                        if (ch != cur_ch) {
                            cur_ch = ch;
                            load_ch64(pc, ch, h);
                        }
                        const double P = prob_fp64(c, h, s.a[j], Tau64{s.tau[j], s.tau_lo[j]});
                        const float2 ew = s.ew[j];
                        acc_event_f64(r, accp, prm, sf, ew.x, P * (double)ew.y, hs, active);
                    }
                }
            }
            if constexpr (PREC != kFP64) {
                // mark the item for the FP64 recomputation of its left-out events
                if (__syncthreads_or(redo) && tid == 0) {
                    prm.redo[it] = 1;
                    mark_redo(prm);
                }
            }
            acc_finish(r, accp);
        }
        if (prm.fuse_final && !prm.redo) fused_final(prm);
    }
}

// ------------------------------------------------- FP64 recomputation pass
// The FP32 precisions' histogram kernels leave out every event whose error
// estimate exceeds the tolerance (prob_fp32 / prob_mix) and mark its work item.
// This kernel, launched programmatically after each such histogram kernel,
// returns at once when no item is marked.  Otherwise one warp per marked item
// walks the item's points and events, takes the FP32 path's decision again (the
// same arithmetic on the same inputs gives the same events) and adds the FP64
// weights of the left-out events to the same exact accumulators, so the bins
// do not depend on which kernel added which event.  Its last warp converts the
// bins when the histogram kernel left its fused finalize to it, and resets the
// counters.  The FP64 arithmetic sits here, out of the FP32 kernels' main loops.
// The FP32-bulk one-point histogram kernel of a fit step whose point's constants
// come by value (computed on the host, host_point_consts): no constants kernel
// runs before it.  Block 0 also stores them in row 0 of the constants tables,
// which the FP64 recomputation pass and the finalize read after this grid (and
// later calls find there, as after the constants kernel).
struct PointInline {
    float c32[C32_STRIDE];
    double c64[C64_STRIDE];
};
template <int PREC>
__global__ void __launch_bounds__(kNT, 2) k_redo(const HistParams prm) {
    grid_dependents_launch();  // a finalize kernel after this one may become resident early
    // Four warps of block 0 convert the fused finalize's bins: they read the
    // histograms' metadata before the wait, and after it issue the recomputation
    // count, the digit columns and the norms in one round of loads.
    constexpr int kConvThreads = 128;
    FinMeta fm;
    const bool conv = prm.fuse_final && blockIdx.x == 0 && threadIdx.x < kConvThreads;
    if (conv) fin_meta_load(prm, fm, threadIdx.x);
    grid_dependency_wait();
    if (conv) fin_data_load(prm, fm, threadIdx.x);
    if (__ldcg(prm.counter + kRedoCount) == 0) {
        // nothing to recompute: the conversion the histogram kernel left to this
        // kernel (it also resets the work counters)
        if (conv) convert_bins(prm, threadIdx.x, kConvThreads, &fm);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int n_warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int it = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); it < prm.n_items; it += n_warps) {
        if (!prm.redo[it]) continue;
        const WorkItem wi = prm.items[it];
        const SampleDev &sd = prm.samples[wi.sample];
        if (debug_ok(wi.ev_begin >= 0 && wi.ev_count >= 0 && wi.ev_begin + wi.ev_count <= sd.n, prm.counter,
                     kDbgItem)) {
            const int sh = sd.frac_bits - 150;
            for (int q = 0; q < wi.n_pts; ++q) {
                const float *pc32 = prm.pc32 + (int64_t)(wi.point_base + q) * C32_STRIDE;
                const double *pc64 = prm.pc64 + (int64_t)(wi.point_base + q) * C64_STRIDE;
                Pt32 c;
                load_pt32(pc32, c);
                Pt64 c64;
                if (PREC == kMix) load_pt64(pc64, c64);
                const float sf = pc32[C32_ESCALE];
                unsigned long long *accp = prm.acc + kDigits * (wi.acc_base + q) * (int64_t)prm.nbins;
                RunAcc32 r;
                Ch32 h;
                int cur_ch = -1;
                for (int e = lane; e < wi.ev_count; e += 32) {
                    const float4 rec = sd.ev[wi.ev_begin + e];
                    const int ch = __float_as_int(rec.w);
                    if (ch != cur_ch) {
                        cur_ch = ch;
                        load_ch32(pc32, ch, h);
                    }
                    float A, th, tl;
                    event_terms32(sd, rec.x, ch, A, th, tl);
                    bool x;
                    if (PREC == kFP32) {
                        prob_fp32(c, h, A, th, tl, x);
                    } else {
                        const double Ad = sd.kA_rhoye * (double)rec.x;
                        prob_mix(c, h, c64, (ch >= 9) ? -Ad : Ad, (double)th + (double)tl, x);
                    }
                    if (x) {
                        const float P = (float)prob_redo64(pc64, ch, rec.x, sd.kA_rhoye, sd.cLL);
                        acc_event_f32(r, accp, prm, sf, rec.y, P * rec.z, sh, true);
                    }
                }
                acc_finish(r, accp);
            }
        }
        if (lane == 0) prm.redo[it] = 0;  // cleared for the next launch
    }
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = (atomicAdd(prm.counter + kRedoTicket, 1) == n_warps - 1);
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    if (prm.fuse_final) convert_bins_warp(prm);  // also resets the work and completion counters
    if (lane == 0) {
        prm.counter[kRedoCount] = 0;
        prm.counter[kRedoTicket] = 0;
    }
}

// ------------------------------------------------------- per-event reweight
template <int PREC>
__global__ void __launch_bounds__(256) k_reweight(const ReweightParams r) {
    const SampleDev &sd = r.s;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (PREC == kFP32) {
        const float *pc = r.pc32 + (int64_t)r.point * C32_STRIDE;
        Pt32 c;
        load_pt32(pc, c);
        Ch32 h;
        int cur_ch = -1;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.n; i += stride) {
            const float4 q = sd.ev[i];
            const float E = q.x;
            const int ch = __float_as_int(q.w);
            if (ch != cur_ch) {
                cur_ch = ch;
                load_ch32(pc, ch, h);
            }
            float A, th, tl;
            event_terms32(sd, E, ch, A, th, tl);
            bool x;
            float P = prob_fp32(c, h, A, th, tl, x);
            if (x) P = (float)prob_redo64(r.pc64 + (int64_t)r.point * C64_STRIDE, ch, E, sd.kA_rhoye, sd.cLL);
            const float w = P * q.z;
            const int32_t o = sd.perm[i];
            if (r.out_prob) r.out_prob[o] = (double)P;
            if (r.out_weight) r.out_weight[o] = (double)w * r.norm;
        }
    } else if (PREC == kMix) {
        const float *pc = r.pc32 + (int64_t)r.point * C32_STRIDE;
        Pt32 c;
        load_pt32(pc, c);
        Pt64 c64;
        load_pt64(r.pc64 + (int64_t)r.point * C64_STRIDE, c64);
        Ch32 h;
        int cur_ch = -1;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.n; i += stride) {
            const float4 q = sd.ev[i];
            const float E = q.x;
            const int ch = __float_as_int(q.w);
            if (ch != cur_ch) {
                cur_ch = ch;
                load_ch32(pc, ch, h);
            }
            float A, th, tl;
            event_terms32(sd, E, ch, A, th, tl);
            const double Ad = sd.kA_rhoye * (double)E;
            bool x;
            float P = prob_mix(c, h, c64, (ch >= 9) ? -Ad : Ad, (double)th + (double)tl, x);
            if (x) P = (float)prob_redo64(r.pc64 + (int64_t)r.point * C64_STRIDE, ch, E, sd.kA_rhoye, sd.cLL);
            const float w = P * q.z;
            const int32_t o = sd.perm[i];
            if (r.out_prob) r.out_prob[o] = (double)P;
            if (r.out_weight) r.out_weight[o] = (double)w * r.norm;
        }
    } else {
        const double *pc = r.pc64 + (int64_t)r.point * C64_STRIDE;
        Pt64 c;
        load_pt64(pc, c);
        Ch64 h;
        int cur_ch = -1;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.n; i += stride) {
            const float4 q = sd.ev[i];
            const float E = q.x;
            const int ch = __float_as_int(q.w);
            if (ch != cur_ch) {
                cur_ch = ch;
                load_ch64(pc, ch, h);
            }
            const double Ad = sd.kA_rhoye * (double)E;
            const double P = prob_fp64(c, h, (ch >= 9) ? -Ad : Ad, tau64(sd.cLL, E));
            const double w = P * (double)q.z;
            const int32_t o = sd.perm[i];
            if (r.out_prob) r.out_prob[o] = P;
            if (r.out_weight) r.out_weight[o] = w * r.norm;
        }
    }
}

}  // namespace osc
