// osc_consts_host.cu -- the per-point constants of one parameter point computed
// on the host (Sec. 2.1: parameter-only components are computed once per
// parameter set), for the fit step, whose histogram kernel then takes them by
// value and needs no constants kernel before it.
//
// This is the computation of point_consts_block (osc_kernels.cuh) written out
// serially, operation for operation: the same IEEE-754 double operations (every
// fused multiply-add explicit, as std::fma; no other contraction -- the library
// is built with -ffp-contract=off), the same sine and cosine of delta (Cody-Waite
// reduction by pi/2, Taylor series), the same roundings to float.  Each result is
// therefore bitwise the one the constants kernel writes, which the GPU tests
// check (the fit step against the same point set and histogrammed separately).
#include <cmath>
#include <cstring>

#include "osc_launch.h"

namespace osc {
namespace {

struct C64 {
    double re, im;
};

// sin and cos of x, as the two lanes of sincos_lanes compute them.
void sincos_host(double x, double *sn, double *cs) {
    constexpr double kTwoOverPi = 0.63661977236758134308;
    constexpr double kPio2Hi = 1.5707963267341256;
    constexpr double kPio2Lo = 6.077100506506192e-11;
    const double k = std::rint(x * kTwoOverPi);
    const double r = std::fma(-k, kPio2Lo, std::fma(-k, kPio2Hi, x));
    const double u = r * r;
    double v[2];
    for (int c = 0; c < 2; ++c) {
        double p = c ? 1.0 / 20922789888000.0 : 1.0 / 355687428096000.0;
        p = std::fma(p, u, c ? -1.0 / 87178291200.0 : -1.0 / 1307674368000.0);
        p = std::fma(p, u, c ? 1.0 / 479001600.0 : 1.0 / 6227020800.0);
        p = std::fma(p, u, c ? -1.0 / 3628800.0 : -1.0 / 39916800.0);
        p = std::fma(p, u, c ? 1.0 / 40320.0 : 1.0 / 362880.0);
        p = std::fma(p, u, c ? -1.0 / 720.0 : -1.0 / 5040.0);
        p = std::fma(p, u, c ? 1.0 / 24.0 : 1.0 / 120.0);
        p = std::fma(p, u, c ? -1.0 / 2.0 : -1.0 / 6.0);
        p = std::fma(p, u, 1.0);
        v[c] = c ? p : p * r;
    }
    const int q = (int)(long long)k & 3;
    *sn = q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? -v[0] : -v[1];
    *cs = q == 0 ? v[1] : q == 1 ? -v[0] : q == 2 ? -v[1] : v[0];
}

// PMNS entry U[f][m] (as pmns_entry): t = (s12, c12, s13, c13, s23, c23, sin delta, cos delta).
C64 pmns_host(const double *t, int f, int m) {
    const double s12 = t[0], c12 = t[1], s13 = t[2], s23 = t[4], c23 = t[5], sd = t[6], cd = t[7];
    const double c13 = t[3];
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
    return {std::fma(bs, cd, ax * ay), bs * (g * sd)};
}

// a * m * conj(b) (as cmul_conj)
C64 cmul_conj_host(C64 a, double m, C64 b) {
    return {m * std::fma(a.re, b.re, a.im * b.im), m * std::fma(a.im, b.re, -(a.re * b.im))};
}

void split_ff_host(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

}  // namespace

void host_point_consts(const osc_point &P, float *c32, double *c64) {
    std::memset(c32, 0, sizeof(float) * C32_STRIDE);
    std::memset(c64, 0, sizeof(double) * C64_STRIDE);
    const double dm21 = P.dm21, dm31 = P.dm32 + P.dm21;
    const double T0 = dm21 + dm31;
    const double c10 = dm21 * dm31;
    const bool no = dm31 > 0;
    const double d0 = no ? 0.0 : dm31, d1 = no ? dm21 : 0.0, d2 = no ? dm31 : dm21;

    // warps 0, 1: square roots and sin, cos of delta; U; H0 and H0^2; channel fields
    double t[8];
    t[0] = std::sqrt(P.s2_12);
    t[1] = std::sqrt(1.0 - P.s2_12);
    t[2] = std::sqrt(P.s2_13);
    t[3] = std::sqrt(1.0 - P.s2_13);
    t[4] = std::sqrt(P.s2_23);
    t[5] = std::sqrt(1.0 - P.s2_23);
    sincos_host(P.dcp, &t[6], &t[7]);
    C64 Us[9];
    for (int l = 0; l < 9; ++l) Us[l] = pmns_host(t, l / 3, l % 3);
    double Hs[4][9];
    for (int l = 0; l < 9; ++l) {
        const int b = l / 3, a = l % 3;
        const double m[3] = {0.0, dm21, dm31};
        C64 h = {0, 0}, h2 = {0, 0};
        for (int k = 1; k < 3; ++k) {
            const C64 q = cmul_conj_host(Us[3 * b + k], m[k], Us[3 * a + k]);
            h.re = h.re + q.re;
            h.im = h.im + q.im;
            h2.re = std::fma(q.re, m[k], h2.re);
            h2.im = std::fma(q.im, m[k], h2.im);
        }
        Hs[0][l] = h.re; Hs[1][l] = h.im; Hs[2][l] = h2.re; Hs[3][l] = h2.im;
    }
    for (int l = 0; l < 9; ++l) {
        const int f = l / 3, s = l % 3;
        const int m = no ? s : (s + 2) % 3;
        const C64 u = Us[3 * f + m];
        c32[C32_LU + 2 * l] = (float)u.re;
        c32[C32_LU + 2 * l + 1] = (float)u.im;
        c64[C64_LU + 2 * l] = u.re;
        c64[C64_LU + 2 * l + 1] = u.im;
    }
    for (int w = 0; w < 2; ++w)
        for (int lane = 0; lane < 27; ++lane) {
            const int ch = lane / 3, j = 3 * w + lane % 3;
            const int a = ch / 3, b = ch % 3;
            const int cmp = j < 4 ? j : j - 4;
            const double z = (a == 0 ? Hs[cmp][3 * b] : 0.0) + (b == 0 ? Hs[cmp][a] : 0.0);
            c64[C64_CH + 6 * ch + j] = j < 4 ? Hs[cmp][3 * b + a] : z;
        }
    for (int f = 0; f < 72; ++f) {
        const int ch = f >> 3, j = f & 7, a = ch / 3, b = ch % 3;
        double v;
        if (j < 6) {
            const int l = j >> 1, m = no ? l : (l + 2) % 3;
            const C64 ub = Us[3 * b + m], ua = Us[3 * a + m];
            v = (j & 1) ? std::fma(ub.im, ua.re, -(ub.re * ua.im)) : std::fma(ub.re, ua.re, ub.im * ua.im);
        } else {
            const int cmp = j - 6;
            v = (a == 0 ? Hs[cmp][3 * b] : 0.0) + (b == 0 ? Hs[cmp][a] : 0.0);
        }
        c32[C32_CH + 8 * ch + j] = (float)v;
    }

    // warp 2: shifted-cubic constants of sorted roots 0, 1 and the depressed cubic's coefficients
    const double ze0 = (1.0 - P.s2_12) * (1.0 - P.s2_13), ze1 = P.s2_12 * (1.0 - P.s2_13), ze2 = P.s2_13;
    for (int lane = 0; lane < 2; ++lane) {
        const double z0 = no ? ze0 : ze2, z1 = no ? ze1 : ze0, z2 = no ? ze2 : ze1;
        const double dl = lane ? d1 : d0, dj = lane ? d2 : d1, dk = lane ? d0 : d2;
        const double zl = lane ? z1 : z0, zj = lane ? z2 : z1, zk = lane ? z0 : z2;
        const double aj = dl - dj, ak = dl - dk;
        const int o = lane ? (C32_S1 - C32_S0) : 0;
        const double S = aj + ak, PI = aj * ak, W = std::fma(zl, aj + ak, std::fma(zj, ak, zk * aj)), E = zl * aj * ak;
        c32[C32_S0 + o] = (float)S;
        c32[C32_PI0 + o] = (float)PI;
        c32[C32_W0 + o] = (float)W;
        c32[C32_E0 + o] = (float)E;
        c64[C64_SH + 4 * lane] = S;
        c64[C64_SH + 4 * lane + 1] = PI;
        c64[C64_SH + 4 * lane + 2] = W;
        c64[C64_SH + 4 * lane + 3] = E;
    }
    for (int lane = 0; lane < 5; ++lane) {
        constexpr double k3 = 1.0 / 3.0, k9 = 1.0 / 9.0, k27 = 1.0 / 27.0;
        const double smt = T0 - std::fma(dm21, ze1, dm31 * ze2);
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
        v = std::fma(wst, smt * T0, v);
        v = std::fma(ws, smt, v);
        v = std::fma(wct, c10 * T0, v);
        v = std::fma(wc, c10, v);
        v = std::fma(w1, T0, v);
        v = std::fma(w2, T2, v);
        v = std::fma(w3, T2 * T0, v);
        const int o32 = lane == 0 ? C32_P0 : lane == 1 ? C32_P1 : lane == 2 ? C32_Q0 : lane == 3 ? C32_Q1 : C32_Q2;
        const int o64 = lane == 0 ? C64_P0 : lane == 1 ? C64_P1 : lane == 2 ? C64_Q0 : lane == 3 ? C64_Q1 : C64_Q2;
        c32[o32] = (float)(v * (lane < 2 ? -1.0 / 3.0 : -0.5));
        c64[o64] = v;
        if (lane == 0) {
            c32[C32_SMT] = (float)smt;
            c64[C64_SMT] = smt;
        }
    }

    // warp 3: T0 less one sorted vacuum eigenvalue; the spectrum, its gaps, T0, c1(0),
    // T0 / 3 - d0,1 and the systematics (x = a s - b, as one lane each)
    c32[C32_SD02] = (float)(d0 + d2);
    c32[C32_SD01] = (float)(d0 + d1);
    for (int lane = 0; lane < 14; ++lane) {
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
        const double x = std::fma(a, (lane == 10 || lane == 11) ? 1.0 / 3.0 : 1.0, -b);
        const int o64 = lane <= 2 ? C64_LD + lane : (lane >= 3 && lane <= 5) ? C64_VG + lane - 3
                      : lane == 8 ? C64_T0 : lane == 9 ? C64_C10 : lane == 12 ? C64_ESCALE : lane == 13 ? C64_NORM : -1;
        const int o32 = lane <= 2 ? C32_D0 + lane : lane == 3 ? C32_V1H : lane == 4 ? C32_V2H : lane == 5 ? C32_G12
                      : lane == 6 ? C32_G01 : lane == 7 ? C32_G02 : lane == 8 ? C32_T0 : lane == 9 ? C32_C10
                      : lane == 10 ? C32_TD0 : lane == 11 ? C32_TD1 : lane == 12 ? C32_ESCALE : -1;
        if (o64 >= 0) c64[o64] = x;
        if (lane == 3 || lane == 4) {
            split_ff_host(x, &c32[o32], &c32[lane == 3 ? C32_V1L : C32_V2L]);
        } else if (o32 >= 0) {
            c32[o32] = (float)x;
        }
    }
}

}  // namespace osc
