// osc_math.cuh -- per (event, parameter point) arithmetic of the constant-density
// three-flavour oscillation probability (Sec. 1.1: Eq. (1) and the matter term;
// Sec. 2.1: parameter-only components computed once per parameter set).
//
// Both precisions evaluate the same closed form.  With M = H0 + A Pe the
// flavour-basis Hamiltonian (H0 = U diag(0, dm21, dm31) U^dagger, Pe = e e^T),
// the eigenvalues lambda_l of M are the roots of its characteristic cubic
//   lambda^3 - (T0 + A) lambda^2 + (c1_0 + A s_mt) lambda - A m_ee = 0
// (T0 = tr H0, c1_0 = dm21 dm31, s_mt = H0_mumu + H0_tautau, m_ee the mu-tau
// minor; det H0 = 0), and the propagator is Sylvester's formula
//   S = sum_l exp(-i tau lambda_l) prod_{j != l} (M - lambda_j) / (lambda_l - lambda_j),
// tau = c_L L / E, whose (beta, alpha) entry needs only (M)_{beta alpha} and
// (M^2)_{beta alpha}:  N_l = (M^2)_ba - sigma_l M_ba + pi_l delta_ba with
// sigma_l = lambda_j + lambda_k and pi_l = lambda_j lambda_k.
//
// FP64 path: the matter shifts are refined by FP64 Newton steps on the shifted
// cubics from the FP32 trigonometric seed, and everything else is FP64.
//
// FP32 path (GB300 has ~1/64 of its FP32 rate in FP64): each eigenvalue is
// written as its vacuum value plus a matter shift, lambda_l = d_l + delta_l.
// By the rank-one secular structure of M = U (D + A u u^dagger) U^dagger,
// delta_l solves the shifted cubic
//   delta^3 + (a_j + a_k - A) delta^2 + (a_j a_k - A W_l) delta - A z_l a_j a_k = 0,
// a_j = d_l - d_j, z = |U_e|^2, W_l = z_l (a_j + a_k) + z_j a_k + z_k a_j,
// whose coefficients carry only FP32 rounding relative to delta itself, so one
// FP32 Newton step from a trigonometric FP32 seed gives delta to FP32 relative
// accuracy.  tau delta_l <= tau |A| = c_L L k_A rho Y_e is energy independent
// (<= 0.72 rad for the beam workloads here), so those parts of the phases are
// accurate in FP32; the large vacuum parts tau (d_l - d_0) are formed in
// float-float and reduced exactly in revolutions.  The FP32 amplitude takes the
// Sylvester numerators in the vacuum mass basis (amplitude_bulk), where every
// factor is a vacuum gap minus a matter shift, and bounds its own rounding error
// per event; an event whose bound exceeds the tolerance is recomputed in FP64
// (prob_redo64, osc_kernels.cuh).  The FP32-bulk chain runs on one event or on
// two at once in packed instructions (see the lane notes below).
#pragma once

#include <stdint.h>

namespace osc {

// ------------------------------------------------------------------ FP32 path
// Approximate reciprocal (PTX rcp.approx, about 1 ulp); used only where the
// result is refined or enters a correction term.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------- one or two events at once
// The FP32-bulk chain (acos_third_short, shifts_bulk, phase_rev_bulk,
// amplitude_bulk, prob_bulk) is written once over V = float (one event) or
// V = float2 (two events, one in each half of this GPU's packed add / sub /
// mul / fma.f32x2 instructions, which issue once for both).  Every operation
// is explicitly rounded -- the compiler contracts nothing -- so both forms, and
// every kernel that uses either, give the same bits for an event.  The packed
// instructions take no negated operands, so the chain carries exactly negated
// terms where a negation would otherwise be needed (-1/E, -tl, -(-p/3), -g01).
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as the fused b (-1) + a: one rounding, so the same bits as a subtraction
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// A scalar in every lane.
template <class V>
__device__ __forceinline__ V vb(float x);
template <>
__device__ __forceinline__ float vb<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 vb<float2>(float x) { return make_float2(x, x); }
// Lane access, and lane-wise application of operations that have no packed form.
template <class V>
struct Lanes;
template <>
struct Lanes<float> {
    static constexpr int n = 1;
    static __device__ __forceinline__ float get(float a, int) { return a; }
    static __device__ __forceinline__ void set(float &a, int, float v) { a = v; }
};
template <>
struct Lanes<float2> {
    static constexpr int n = 2;
    static __device__ __forceinline__ float get(float2 a, int i) { return i ? a.y : a.x; }
    static __device__ __forceinline__ void set(float2 &a, int i, float v) { (i ? a.y : a.x) = v; }
};
template <class V, class F>
__device__ __forceinline__ V vmap(V a, F f) {
    V r;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) Lanes<V>::set(r, i, f(Lanes<V>::get(a, i)));
    return r;
}
template <class V>
__device__ __forceinline__ void vsincos(V x, V &s, V &c) {
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) {
        float si, ci;
        __sincosf(Lanes<V>::get(x, i), &si, &ci);
        Lanes<V>::set(s, i, si);
        Lanes<V>::set(c, i, ci);
    }
}

// arccos(x) / 3 on [-1, 1] from Abramowitz & Stegun, Handbook of Mathematical
// Functions, formula 4.4.46: acos(x) = sqrt(1 - x) (a0 + a1 x + ... + a7 x^7)
// for 0 <= x <= 1 with |error| <= 2e-8, and acos(-x) = pi - acos(x); the
// coefficients and pi carry the 1/3 of the cube angle.  Branch-free; it only
// seeds the Newton-refined eigenvalues, which need ~1e-5 relative accuracy.
__device__ __forceinline__ float acos_third(float x) {
    constexpr float k = 1.0f / 3.0f;
    const float ax = fabsf(x);
    float p = -0.0012624911f * k;
    p = fmaf(p, ax, 0.0066700901f * k);
    p = fmaf(p, ax, -0.0170881256f * k);
    p = fmaf(p, ax, 0.0308918810f * k);
    p = fmaf(p, ax, -0.0501743046f * k);
    p = fmaf(p, ax, 0.0889789874f * k);
    p = fmaf(p, ax, -0.2145988016f * k);
    p = fmaf(p, ax, 1.5707963050f * k);
    float sq;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(1.0f - ax));
    const float r = sq * p;
    return x < 0.0f ? 3.14159265358979323846f * k - r : r;
}

// arccos(x) / 3 from Abramowitz & Stegun formula 4.4.45: acos(x) = sqrt(1 - x)
// (a0 + a1 x + a2 x^2 + a3 x^3) for 0 <= x <= 1 with |error| <= 7e-5 rad.  It
// seeds the FP32-bulk shifts only: their Newton step squares the seed's error,
// and its per-event error bound, together with the seed's |cos theta| check,
// sends every event the step would not settle to the FP64 recomputation.  The
// FP64 and FP64-eigen paths, whose Newton polish must reach FP64 accuracy, take
// the seven-term form above.
template <class V>
__device__ __forceinline__ V acos_third_short(V x) {
    constexpr float k = 1.0f / 3.0f;
    // rounding can put |cos theta| just above 1
    const V ax = vmap(x, [](float v) { return fminf(fabsf(v), 1.0f); });
    V p = vfma(vb<V>(-0.0187293f * k), ax, vb<V>(0.0742610f * k));
    p = vfma(p, ax, vb<V>(-0.2121144f * k));
    p = vfma(p, ax, vb<V>(1.5707288f * k));
    const V sq = vmap(vsub(vb<V>(1.0f), ax), [](float v) {
        float q;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(v));
        return q;
    });
    const V r = vmul(sq, p);
    const V rc = vsub(vb<V>(3.14159265358979323846f * k), r);
    V out;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i)
        Lanes<V>::set(out, i, Lanes<V>::get(x, i) < 0.0f ? Lanes<V>::get(rc, i) : Lanes<V>::get(r, i));
    return out;
}

struct Pt32 {
    float p0, p1, q0, q1, q2, T0, c10, smt;  // p*: -p/3, q*: -q/2 of the depressed cubic, in powers of A
    float td0, td1;                          // T0 / 3 - d0, T0 / 3 - d1
    float d0, d1, d2, g01, g02, g12;
    float v1h, v1l, v2h, v2l;
    float S0, PI0, W0, E0, S1, PI1, W1, E1;
    float sd02, sd01;                        // d0 + d2, d0 + d1
};
// One channel (alpha -> beta, nu or nubar) in the vacuum mass basis.
struct Ch32 {
    float X0r, X0i, X1r, X1i, X2r, X2i;  // X_m = U_bm conj(U_am), m a sorted vacuum state
    float Zr, Zi;                        // [alpha = e] H0_be + [beta = e] H0_ea
    float ee;    // 1 for the e -> e channel, else 0
    float diag;  // 1 for alpha == beta, else 0
    float zm;    // |Zr| + |Zi|
    bool real;   // mu -> mu or tau -> tau: X_m real, Z = 0
};

// Approximate reciprocal square root (PTX rsqrt.approx); only seeds use it.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// g and g' of the shifted cubic at dl, for a Newton step (see shifted_newton).
template <class V>
__device__ __forceinline__ void newton_terms(V dl, V A, float S, float PI, float W, float E, V &g, V &gp) {
    const V b = vsub(vb<V>(S), A);
    const V c = vfma(A, vb<V>(-W), vb<V>(PI));
    const V t = vfma(vadd(dl, b), dl, c);
    g = vfma(t, dl, vmul(A, vb<V>(-E)));
    gp = vfma(dl, vfma(vb<V>(2.0f), dl, b), t);
}
template <class V>
__device__ __forceinline__ V shifted_newton(V dl, V A, float S, float PI, float W, float E) {
    // one Newton step on g(delta) = delta^3 + b delta^2 + c delta - e, with
    // t = delta (delta + b) + c:  g = t delta - e,  g' = t + delta (2 delta + b);
    // -e and -1/g' are formed directly (A (-E), rcp(-g'))
    const V b = vsub(vb<V>(S), A);
    const V c = vfma(A, vb<V>(-W), vb<V>(PI));
    const V ne = vmul(A, vb<V>(-E));
    const V t = vfma(vadd(dl, b), dl, c);
    const V g = vfma(t, dl, ne);
    const V gp = vfma(dl, vfma(vb<V>(2.0f), dl, b), t);
    return vfma(g, vmap(gp, [](float v) { return rcp_approx(-v); }), dl);
}

// Phase of root l relative to root 0 in revolutions, reduced to about [-0.62, 0.62]:
// th + tl = c_L L / (2 pi E) (float-float), vh + vl = d_l - d_0, dd = delta_l - delta_0.
__device__ __forceinline__ float phase_rev(float th, float tl, float vh, float vl, float dd) {
    const float ph = th * vh;
    const float e1 = fmaf(th, vh, -ph);  // exact residual of the product
    const float fr = ph - rintf(ph);     // exact
    return fr + fmaf(th, dd, fmaf(th, vl, fmaf(tl, vh, e1)));
}

// Trigonometric FP32 seed of the two lower roots m0 <= m1 of the depressed
// cubic mu^3 + p mu + q (Viete's form with the arccos and cube-angle above),
// from mp3 = -p/3 and qh = -q/2: mu = 2 r cos(theta/3 + 2 pi k/3) with
// r = sqrt(mp3) and cos(theta) = qh / r^3.
// Also returns cos(theta): near +-1 the angle is ill-conditioned (see near_double_pair64).
__device__ __forceinline__ void seed_core32(float mp3, float qh, float &m0, float &m1, float &cth_out) {
    mp3 = fmaxf(mp3, 1e-30f);
    const float ir = rsqrt_approx(mp3);
    const float r = mp3 * ir;
    float cth = qh * ir * ir * ir;
    cth = fminf(fmaxf(cth, -1.0f), 1.0f);
    cth_out = cth;
    const float th3 = acos_third(cth);
    float sn, cs;
    __sincosf(th3, &sn, &cs);
    const float rc = r * cs, rsn = r * sn * 1.7320508075688772f;
    m0 = -rc - rsn;  // smallest root
    m1 = -rc + rsn;  // middle root
}
__device__ __forceinline__ void seed_core32(float mp3, float qh, float &m0, float &m1) {
    float cth;
    seed_core32(mp3, qh, m0, m1, cth);
}
__device__ __forceinline__ void seed_depressed32(float p, float q, float &m0, float &m1, float &cth) {
    seed_core32(p * (-1.0f / 3.0f), -0.5f * q, m0, m1, cth);
}

// The trigonometric seed loses a near-double pair of roots: where two roots of
// mu^3 + p mu + q are close (gap << r = sqrt(-p/3)), cos(theta) is within
// (gap / r)^2 of +-1, and an FP32 rounding of it moves theta, and the pair's
// seeds, by up to r sqrt(2 eps): as much as the gap when the matter term dwarfs
// the vacuum splittings.  Past |cos(theta)| = kNearDouble (seed error / gap up to
// about 1e-4, which two Newton steps take to FP64 rounding) the pair is seeded
// by deflation instead: the isolated root mi (the top one for cos(theta) > 0,
// the bottom one otherwise) is well conditioned, so two Newton steps from its
// FP32 seed fix it in FP64; the pair are the roots of the deflated quadratic
// mu^2 + mi mu + (p + mi^2), whose discriminant -3 mi^2 - 4 p is the squared gap.
// s0, s1: the FP32 seeds of the two lower roots; returns the lower two roots.
constexpr float kNearDouble = 0.999f;
static __device__ __noinline__ double2 near_double_pair64(double p, double q, float cth, float s0, float s1) {
    double mi = cth > 0.0f ? -((double)s0 + (double)s1) : (double)s0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double f = fma(fma(mi, mi, p), mi, q);
        const double fp = fma(3.0 * mi, mi, p);
        mi -= (double)((float)f * rcp_approx((float)fp));
    }
    const double sq = sqrt(fmax(fma(-3.0 * mi, mi, -4.0 * p), 0.0));
    return cth > 0.0f ? make_double2(-0.5 * (mi + sq), 0.5 * (sq - mi)) : make_double2(mi, -0.5 * (mi + sq));
}

// The same seed for the characteristic cubic of one event, from the point's
// pre-scaled coefficients: -p/3 = P0 + P1 A + A^2/9, -q/2 = Q0 + Q1 A + Q2 A^2 + A^3/27.
__device__ __forceinline__ void seed_scaled32(const Pt32 &c, float A, float &m0, float &m1, float &cth) {
    const float mp3 = fmaf(fmaf(A, 1.0f / 9.0f, c.p1), A, c.p0);
    const float qh = fmaf(fmaf(fmaf(A, 1.0f / 27.0f, c.q2), A, c.q1), A, c.q0);
    seed_core32(mp3, qh, m0, m1, cth);
}
__device__ __forceinline__ void seed_scaled32(const Pt32 &c, float A, float &m0, float &m1) {
    float cth;
    seed_scaled32(c, A, m0, m1, cth);
}
// The same seed as (r, t0, t1) with m0 = -r t0 and m1 = -r t1, t0,1 = cos(theta/3)
// +- sqrt(3) sin(theta/3), so that the caller folds the products into its own
// sums (the layered path's shifts; the single-layer FP32-bulk path forms the
// same seed in shifts_bulk with the short arccos).
__device__ __forceinline__ void seed_scaled32_rt(const Pt32 &c, float A, float &r, float &t0, float &t1,
                                                 float &cth) {
    const float mp3 = fmaxf(fmaf(fmaf(A, 1.0f / 9.0f, c.p1), A, c.p0), 1e-30f);
    const float qh = fmaf(fmaf(fmaf(A, 1.0f / 27.0f, c.q2), A, c.q1), A, c.q0);
    const float ir = rsqrt_approx(mp3);
    r = mp3 * ir;
    cth = qh * ir * ir * ir;
    const float th3 = acos_third(fminf(fmaxf(cth, -1.0f), 1.0f));
    float sn, cs;
    __sincosf(th3, &sn, &cs);
    t0 = fmaf(1.7320508075688772f, sn, cs);
    t1 = fmaf(-1.7320508075688772f, sn, cs);
}
// As roots mu of the depressed cubic (lambda = mu + (T0 + A) / 3).
__device__ __forceinline__ void seed_roots32(const Pt32 &c, float A, float &m0, float &m1, float &t3, float &cth) {
    seed_scaled32(c, A, m0, m1, cth);
    t3 = (c.T0 + A) * (1.0f / 3.0f);
}

// |S_ba|^2 from the matter shifts delta_l = lambda_l - d_l, the gaps
// g_ij = lambda_i - lambda_j and the half phases h_l = (phi_l - phi_0) / 2
// relative to root 0 [rad].  The projectors sum to the identity, so
// S = delta_ba + sum_{l=1,2} C_l (e^{-i phi_l} - 1) needs no C_0, and
// e^{-i phi} - 1 = -2 sin(phi/2) (sin(phi/2) + i cos(phi/2)) keeps small phase
// differences accurate; the factor -2 sin(phi_l / 2) is folded into 1/D_l:
// D_1 = (L1 - L0)(L1 - L2) = -g01 g12, D_2 = (L2 - L0)(L2 - L1) = g02 g12, so
// w_l = -2 sin(phi_l / 2) / D_l and S = delta_ba + sum_l N_l w_l (sin + i cos)(phi_l / 2).
//
// Sylvester numerators N_l = [(M - lambda_j)(M - lambda_k)]_ba in the vacuum mass
// basis: M = U (D + A u u^dagger) U^dagger with u = U^dagger e, and U unitary, give
//   N_l = sum_m (d_m - lambda_j)(d_m - lambda_k) X_m + A (Z + [ab = ee] (lambda_l - T0)),
// X_m = U_bm conj(U_am), Z = [a = e] H0_be + [b = e] H0_ea, lambda_l - T0 =
// delta_l - (the other two d's).  Each factor d_m - lambda_j is a vacuum gap
// minus a matter shift, so no term carries the cancellation by dm31 / dm21 of
// the flavour-basis form (M^2)_ba - sigma_l M_ba + pi_l delta_ba.
//
// est: the amplitude's rounding error bound in units of 2^-24, the magnitudes of
// the summed terms of each N_l (and the operands of the A term) times |w_l|.
// REAL: the mu -> mu and tau -> tau channels (X_m real, Z = 0).
// ng01 = -g01 (the packed form has no negated operand; see the lane notes above).
template <bool REAL, class V>
__device__ __forceinline__ V amplitude_bulk(const Pt32 &c, const Ch32 &h, V A, V dl0, V dl1, V dl2, V ng01, V g02,
                                            V g12, V h1, V h2, V &est) {
    V s1, k1, s2, k2;
    vsincos(h1, s1, k1);
    vsincos(h2, s2, k2);
    // 2 / (g01 g02 g12) = -2 / (ng01 g02 g12)
    const V inv2 = vmul(vb<V>(-2.0f), vmap(vmul(vmul(ng01, g02), g12), [](float v) { return rcp_approx(v); }));
    const V w1 = vmul(vmul(g02, s1), inv2), w2 = vmul(vmul(ng01, s2), inv2);
    // a_m = d_m - lambda_0, b_m = d_m - lambda_2, e_m = d_m - lambda_1 (a_0 = -dl0,
    // b_2 = -dl2, e_1 = -dl1), held as na_m = -a_m, nb_m = -b_m, ne0 = -e_0, e2n = -e_2
    const V na1 = vsub(dl0, vb<V>(c.v1h)), na2 = vsub(dl0, vb<V>(c.v2h));
    const V nb0 = vsub(dl2, vb<V>(c.g02)), nb1 = vsub(dl2, vb<V>(c.g12));
    const V ne0 = vsub(dl1, vb<V>(c.g01)), e2n = vadd(vb<V>(c.g12), dl1);
    // root 1 (j, k = 0, 2): p_m = a_m b_m;  root 2 (j, k = 0, 1): q_m = a_m e_m
    const V p0 = vmul(dl0, nb0), p1 = vmul(na1, nb1), p2 = vmul(na2, dl2);
    const V q0 = vmul(dl0, ne0), q1 = vmul(na1, dl1), q2 = vmul(na2, e2n);
    V T1, T2;  // lane-wise: the absolute values fold into the scalar adds
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i) {
        using L = Lanes<V>;
        L::set(T1, i, __fadd_rn(__fadd_rn(fabsf(L::get(p0, i)), fabsf(L::get(p1, i))), fabsf(L::get(p2, i))));
        L::set(T2, i, __fadd_rn(__fadd_rn(fabsf(L::get(q0, i)), fabsf(L::get(q1, i))), fabsf(L::get(q2, i))));
    }
    if (REAL) {
        const V u1 = vmul(vfma(p0, vb<V>(h.X0r), vfma(p1, vb<V>(h.X1r), vmul(p2, vb<V>(h.X2r)))), w1);
        const V u2 = vmul(vfma(q0, vb<V>(h.X0r), vfma(q1, vb<V>(h.X1r), vmul(q2, vb<V>(h.X2r)))), w2);
#pragma unroll
        for (int i = 0; i < Lanes<V>::n; ++i) {
            using L = Lanes<V>;
            L::set(est, i, __fmaf_rn(L::get(T1, i), fabsf(L::get(w1, i)),
                                     __fmul_rn(L::get(T2, i), fabsf(L::get(w2, i)))));
        }
        // S = 1 + sum_l u_l (s_l + i k_l)
        const V Sr = vfma(u1, s1, vfma(u2, s2, vb<V>(1.0f)));
        const V Si = vfma(u1, k1, vmul(u2, k2));
        return vfma(Sr, Sr, vmul(Si, Si));
    } else {
        const V AZi = vmul(A, vb<V>(h.Zi));
        const V t1 = vmul(A, vfma(vb<V>(h.ee), vsub(dl1, vb<V>(c.sd02)), vb<V>(h.Zr)));
        const V t2 = vmul(A, vfma(vb<V>(h.ee), vsub(dl2, vb<V>(c.sd01)), vb<V>(h.Zr)));
        const V n1r = vfma(p0, vb<V>(h.X0r), vfma(p1, vb<V>(h.X1r), vfma(p2, vb<V>(h.X2r), t1)));
        const V n1i = vfma(p0, vb<V>(h.X0i), vfma(p1, vb<V>(h.X1i), vfma(p2, vb<V>(h.X2i), AZi)));
        const V n2r = vfma(q0, vb<V>(h.X0r), vfma(q1, vb<V>(h.X1r), vfma(q2, vb<V>(h.X2r), t2)));
        const V n2i = vfma(q0, vb<V>(h.X0i), vfma(q1, vb<V>(h.X1i), vfma(q2, vb<V>(h.X2i), AZi)));
        const V u1 = vmul(n1r, w1), v1 = vmul(n1i, w1), u2 = vmul(n2r, w2), v2 = vmul(n2i, w2);
#pragma unroll
        for (int i = 0; i < Lanes<V>::n; ++i) {
            using L = Lanes<V>;
            const float aA = fabsf(L::get(A, i));
            const float T1a = __fmaf_rn(
                aA, __fmaf_rn(h.ee, __fadd_rn(fabsf(L::get(dl1, i)), fabsf(c.sd02)), h.zm), L::get(T1, i));
            const float T2a = __fmaf_rn(
                aA, __fmaf_rn(h.ee, __fadd_rn(fabsf(L::get(dl2, i)), fabsf(c.sd01)), h.zm), L::get(T2, i));
            L::set(est, i, __fmaf_rn(T1a, fabsf(L::get(w1, i)), __fmul_rn(T2a, fabsf(L::get(w2, i)))));
        }
        // S = delta_ba + sum_l (u_l + i v_l)(s_l + i k_l)
        const V nv1 = vmul(v1, vb<V>(-1.0f)), nv2 = vmul(v2, vb<V>(-1.0f));
        const V Sr = vfma(u1, s1, vfma(nv1, k1, vfma(u2, s2, vfma(nv2, k2, vb<V>(h.diag)))));
        const V Si = vfma(u1, k1, vfma(v1, s1, vfma(u2, k2, vmul(v2, s2))));
        return vfma(Sr, Sr, vmul(Si, Si));
    }
}
// The same amplitude for one event from g01 (the FP64-eigenvalue variant's FP32 part).
template <bool REAL>
__device__ __forceinline__ float amplitude_mass32(const Pt32 &c, const Ch32 &h, float A, float dl0, float dl1,
                                                  float dl2, float g01, float g02, float g12, float h1, float h2,
                                                  float &est) {
    return amplitude_bulk<REAL, float>(c, h, A, dl0, dl1, dl2, -g01, g02, g12, h1, h2, est);
}

// Matter shifts delta_l = lambda_l - d_l of the three sorted eigenvalues (FP32),
// layered path: trigonometric seed with the eight-term arccos, then one Newton
// step on each lower root's shifted cubic; the top shift follows from the trace
// (sum of shifts = A).
__device__ __forceinline__ void shifts32(const Pt32 &c, float A, float &dl0, float &dl1, float &dl2) {
    float r, t0, t1, cth;
    seed_scaled32_rt(c, A, r, t0, t1, cth);
    // seeds delta_l = (T0 + A) / 3 + m_l - d_l = (A / 3 + (T0 / 3 - d_l)) - r t_l
    dl0 = shifted_newton(fmaf(-r, t0, fmaf(A, 1.0f / 3.0f, c.td0)), A, c.S0, c.PI0, c.W0, c.E0);
    dl1 = shifted_newton(fmaf(-r, t1, fmaf(A, 1.0f / 3.0f, c.td1)), A, c.S1, c.PI1, c.W1, c.E1);
    dl2 = A - dl0 - dl1;
}

// The same shifts for the single-layer FP32-bulk path, one or two events: the
// seed with the four-term arccos (the per-event error bound guards it), formed
// from -(-p/3) = -P0 - P1 A - A^2/9 so that r enters the seeds negated, and
// cos(theta) returned unclamped (the short arccos clamps |x| itself).
template <class V>
__device__ __forceinline__ void shifts_bulk(const Pt32 &c, V A, V &dl0, V &dl1, V &dl2, V &cth) {
    const V nmp3 = vmap(vfma(vfma(A, vb<V>(-1.0f / 9.0f), vb<V>(-c.p1)), A, vb<V>(-c.p0)),
                        [](float v) { return fminf(v, -1e-30f); });
    const V qh = vfma(vfma(vfma(A, vb<V>(1.0f / 27.0f), vb<V>(c.q2)), A, vb<V>(c.q1)), A, vb<V>(c.q0));
    const V ir = vmap(nmp3, [](float v) { return rsqrt_approx(-v); });
    const V nr = vmul(nmp3, ir);  // -r
    cth = vmul(vmul(vmul(qh, ir), ir), ir);
    V sn, cs;
    vsincos(acos_third_short(cth), sn, cs);
    const V t0 = vfma(vb<V>(1.7320508075688772f), sn, cs);
    const V t1 = vfma(vb<V>(-1.7320508075688772f), sn, cs);
    // seeds delta_l = (T0 + A) / 3 + m_l - d_l = (A / 3 + (T0 / 3 - d_l)) - r t_l
    const V s0 = vfma(nr, t0, vfma(A, vb<V>(1.0f / 3.0f), vb<V>(c.td0)));
    const V s1 = vfma(nr, t1, vfma(A, vb<V>(1.0f / 3.0f), vb<V>(c.td1)));
    // one Newton step on each lower root's shifted cubic (as shifted_newton), the
    // two reciprocals -1/g'_0 = g'_1 q and -1/g'_1 = g'_0 q from one approximate
    // q = -1 / (g'_0 g'_1): one reciprocal instead of two (a few ulp; the step's
    // correction needs far less)
    V g0, gp0, g1, gp1;
    newton_terms(s0, A, c.S0, c.PI0, c.W0, c.E0, g0, gp0);
    newton_terms(s1, A, c.S1, c.PI1, c.W1, c.E1, g1, gp1);
    const V q = vmap(vmul(gp0, gp1), [](float v) { return rcp_approx(-v); });
    dl0 = vfma(g0, vmul(gp1, q), s0);
    dl1 = vfma(g1, vmul(gp0, q), s1);
    dl2 = vsub(vsub(A, dl0), dl1);
}

// Phase of root l relative to root 0 in revolutions (as phase_rev), from
// ntl = -tl: with nph = -th vh, th vh - rint(th vh) = rint(nph) - nph exactly.
template <class V>
__device__ __forceinline__ V phase_rev_bulk(V th, V ntl, float vh, float vl, V dd) {
    const V nph = vmul(th, vb<V>(-vh));
    const V e1 = vfma(th, vb<V>(vh), nph);  // exact residual of the product
    const V fr = vsub(vmap(nph, [](float v) { return rintf(v); }), nph);
    return vadd(fr, vfma(th, dd, vfma(th, vb<V>(vl), vfma(ntl, vb<V>(-vh), e1))));
}

// P(alpha -> beta) for one point and one or two events, FP32 bulk.  A: signed
// matter term [eV^2]; (th, -ntl): c_L L / (2 pi E_true) as float-float.  Bit i
// of redo is set when lane i's result may miss the FP32 tolerance: the
// amplitude's error estimate exceeds kFp32EstMax, or the seed's |cos theta|
// exceeds kFp32SeedCos.
template <bool REAL, class V>
__device__ __forceinline__ V prob_bulk(const Pt32 &c, const Ch32 &h, V A, V th, V ntl, unsigned &redo) {
    V dl0, dl1, dl2, cth;
    shifts_bulk(c, A, dl0, dl1, dl2, cth);
    // shift differences relative to root 0, shared by the gaps and the phases
    const V dd1 = vsub(dl1, dl0), dd2 = vsub(dl2, dl0);
    const V ng01 = vsub(dd1, vb<V>(c.g01)), g02 = vsub(vb<V>(c.g02), dd2);
    const V g12 = vadd(vb<V>(c.g12), vsub(dd1, dd2));
    // half phases relative to root 0: pi * revolutions
    const V h1 = vmul(vb<V>(3.14159265358979323846f), phase_rev_bulk(th, ntl, c.v1h, c.v1l, dd1));
    const V h2 = vmul(vb<V>(3.14159265358979323846f), phase_rev_bulk(th, ntl, c.v2h, c.v2l, dd2));
    V est;
    const V P = amplitude_bulk<REAL>(c, h, A, dl0, dl1, dl2, ng01, g02, g12, h1, h2, est);
    redo = 0;
#pragma unroll
    for (int i = 0; i < Lanes<V>::n; ++i)
        if (!(Lanes<V>::get(est, i) <= kFp32EstMax) || fabsf(Lanes<V>::get(cth, i)) > kFp32SeedCos) redo |= 1u << i;
    return P;
}
// One event, from (th, tl).
__device__ __forceinline__ float prob_fp32(const Pt32 &c, const Ch32 &h, float A, float th, float tl, bool &redo) {
    unsigned x;
    const float P = h.real ? prob_bulk<true>(c, h, A, th, -tl, x) : prob_bulk<false>(c, h, A, th, -tl, x);
    redo = x != 0;
    return P;
}

// ------------------------------------------------------------------ FP64 path
// This GPU's FP64 pipe issues one warp instruction per several tens of cycles
// per scheduler, so the FP64 path is bound by its count of FP64 instructions
// and is written to keep that count low: the eigenvalues' matter shifts by FP64
// Newton steps from the FP32 trigonometric seed, reciprocals by Newton-Raphson from the
// approximate PTX reciprocal, sine and cosine of exactly formed phases by
// Cody-Waite reduction and Taylor series, and no Sylvester coefficient for root 0.
struct Pt64 {
    double p0, p1, q0, q1, q2, T0, c10, smt;
    double S0, PI0, W0, E0, S1, PI1, W1, E1;  // shifted cubics of sorted roots 0, 1
    double d0, d1, d2;                        // sorted vacuum eigenvalues
    double V1, V2, G12;                       // d1 - d0, d2 - d0, d1 - d2
};
struct Ch64 {
    double Xr, Xi, Yr, Yi, Zr, Zi, ee, diag;
};

// 1/x for normal x: rcp.approx.ftz.f64 (relative error about 1e-6), then two
// Newton-Raphson steps r <- r + r (1 - x r), each squaring the relative error.
__device__ __forceinline__ double rcp64(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// c_L L / E as an unevaluated sum hi + lo (relative error about 1e-32): hi from
// the reciprocal 1/E, lo from the exact remainder c_L L - hi E.
struct Tau64 {
    double hi, lo;
};
__device__ __forceinline__ Tau64 tau64(double cLL, double E, double iE) {
    const double hi = cLL * iE;
    return {hi, fma(-hi, E, cLL) * iE};
}
__device__ __forceinline__ Tau64 tau64(double cLL, float E) {
    const double Ed = (double)E;
    return tau64(cLL, Ed, rcp64(Ed));
}

// sin and cos of the phase ph + pl [rad] (pl a small correction to ph).  ph is
// reduced by pi/2 in three parts (Cody and Waite; the first two parts have 33
// significant bits, so k times them is exact for |k| < 2^20, i.e. phases below
// 1.6e6 rad), and the Taylor series of sin x / x and cos x through x^16
// (truncation below 4e-18) are evaluated on the remainder x in [-pi/4, pi/4].
__device__ __forceinline__ void sincos_reduce64(double ph, double pl, double *sn, double *cs) {
    const double k = rint(ph * 0.63661977236758134308);  // 2 / pi
    double r = fma(-k, 1.5707963267341256, ph);           // pi/2, first 33 bits: exact
    r = fma(-k, 6.077100506303966e-11, r);                 // next 33 bits
    r = fma(-k, 2.0222662487959506e-21, r);                // remainder of pi/2
    const double x = r + pl;
    const double u = x * x;
    double ps = 1.0 / 355687428096000.0;       // (-1)^j / (2j + 1)!, j = 8 .. 0
    ps = fma(ps, u, -1.0 / 1307674368000.0);
    ps = fma(ps, u, 1.0 / 6227020800.0);
    ps = fma(ps, u, -1.0 / 39916800.0);
    ps = fma(ps, u, 1.0 / 362880.0);
    ps = fma(ps, u, -1.0 / 5040.0);
    ps = fma(ps, u, 1.0 / 120.0);
    ps = fma(ps, u, -1.0 / 6.0);
    ps = fma(ps, u, 1.0);
    double pc = 1.0 / 20922789888000.0;        // (-1)^j / (2j)!, j = 8 .. 0
    pc = fma(pc, u, -1.0 / 87178291200.0);
    pc = fma(pc, u, 1.0 / 479001600.0);
    pc = fma(pc, u, -1.0 / 3628800.0);
    pc = fma(pc, u, 1.0 / 40320.0);
    pc = fma(pc, u, -1.0 / 720.0);
    pc = fma(pc, u, 1.0 / 24.0);
    pc = fma(pc, u, -0.5);
    pc = fma(pc, u, 1.0);
    const double s = ps * x;
    const int iq = (int)k & 3;  // quadrant, two's complement for negative k
    *sn = iq == 0 ? s : iq == 1 ? pc : iq == 2 ? -s : -pc;
    *cs = iq == 0 ? pc : iq == 1 ? -s : iq == 2 ? -pc : s;
}

// sin and cos of the phase tau (V + dd), V a vacuum gap and dd a difference of
// matter shifts: V + dd is formed as an exact sum s + se (Knuth's TwoSum) and the
// product with tau = hi + lo as ph + pl (the rounding error of hi s by an FMA),
// so the phase carries neither the rounding of the gap nor that of the product.
__device__ __forceinline__ void sincos_gap64(const Tau64 &t, double V, double dd, double *sn, double *cs) {
    const double s = V + dd;
    const double bv = s - V;
    const double se = (V - (s - bv)) + (dd - bv);
    const double ph = t.hi * s;
    const double pl = fma(t.hi, s, -ph) + fma(t.hi, se, t.lo * s);
    sincos_reduce64(ph, pl, sn, cs);
}

// One FP64 Newton step on the shifted cubic g(delta) = delta^3 + b delta^2 +
// c delta - e (as in shifted_newton), the correction divided in FP32: every
// step's correction is orders of magnitude below the shift itself.
__device__ __forceinline__ double shifted_step64(double dl, double b, double c, double e) {
    const double t = fma(dl + b, dl, c);
    const double g = fma(t, dl, -e);
    const double gp = fma(dl, fma(2.0, dl, b), t);
    return dl - (double)((float)g * rcp_approx((float)gp));
}

// Matter shifts delta_l = lambda_l - d_l of the sorted eigenvalues in FP64.  The
// FP32 trigonometric seed of the depressed cubic (from p and q rounded to FP32)
// gives each lower eigenvalue to about 1e-10 eV^2; two FP64 Newton steps on that
// root's shifted cubic refine its shift.  The shifted cubic's coefficients
// carry rounding relative to the shift, not to the vacuum eigenvalue, so a small
// matter shift keeps its relative accuracy (the depressed cubic's p alone,
// rounded at ~1e-22 eV^4, would move the roots by ~1e-18 eV^2, 1e-12 rad at
// c_L L / E = 6e5).  The top shift follows from the trace: the shifts sum to A.
__device__ __forceinline__ void shifts64(const Pt64 &c, double A, double &dl0, double &dl1, double &dl2) {
    const double p = fma(fma(A, -1.0 / 3.0, c.p1), A, c.p0);
    const double q = fma(fma(fma(A, -2.0 / 27.0, c.q2), A, c.q1), A, c.q0);
    float s0, s1, cth;
    seed_depressed32((float)p, (float)q, s0, s1, cth);
    double m0 = s0, m1 = s1;
    if (fabsf(cth) > kNearDouble) {
        const double2 m = near_double_pair64(p, q, cth, s0, s1);
        m0 = m.x;
        m1 = m.y;
    }
    const double t3 = (c.T0 + A) * (1.0 / 3.0);
    dl0 = (m0 + t3) - c.d0;
    dl1 = (m1 + t3) - c.d1;
    const double b0 = c.S0 - A, b1 = c.S1 - A;
    const double cc0 = fma(-A, c.W0, c.PI0), cc1 = fma(-A, c.W1, c.PI1);
    const double e0 = A * c.E0, e1 = A * c.E1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        dl0 = shifted_step64(dl0, b0, cc0, e0);
        dl1 = shifted_step64(dl1, b1, cc1, e1);
    }
    dl2 = A - dl0 - dl1;
}

// P(alpha -> beta); A signed matter term [eV^2], tau = c_L L / E_true.  The
// projectors sum to the identity, so S = delta_ba + sum_{l=1,2} C_l (e^{-i phi_l} - 1)
// with phi_l = tau (lambda_l - lambda_0) and C_l = N_l / D_l, D_1 = -g01 g12,
// D_2 = g02 g12 (g_ij = lambda_i - lambda_j, vacuum gap plus shift difference),
// both from one reciprocal.
__device__ __forceinline__ double prob_fp64(const Pt64 &c, const Ch64 &h, double A, const Tau64 &tau) {
    double dl0, dl1, dl2;
    shifts64(c, A, dl0, dl1, dl2);
    const double L1 = c.d1 + dl1, L2 = c.d2 + dl2;
    const double g01 = (dl0 - dl1) - c.V1, g02 = (dl0 - dl2) - c.V2, g12 = c.G12 + (dl1 - dl2);
    const double inv = rcp64(g01 * g02 * g12);
    const double iD1 = -g02 * inv, iD2 = g01 * inv;
    const double TA = c.T0 + A;
    const double c1 = fma(A, c.smt, c.c10);
    const double Kr = fma(A, fma(A, h.ee, h.Zr), h.Yr), Ki = fma(A, h.Zi, h.Yi);
    const double Gr = fma(A, h.ee, h.Xr), Gi = h.Xi;
    // every multiply-add is an explicit fma, so the rounding sequence (and the
    // result, bit for bit) is the same in every kernel that inlines this function
    double sg, pp;
    sg = TA - L1; pp = fma(-L1, sg, c1);
    const double C1r = fma(pp, h.diag, fma(-sg, Gr, Kr)) * iD1, C1i = fma(-sg, Gi, Ki) * iD1;
    sg = TA - L2; pp = fma(-L2, sg, c1);
    const double C2r = fma(pp, h.diag, fma(-sg, Gr, Kr)) * iD2, C2i = fma(-sg, Gi, Ki) * iD2;
    double s1, k1, s2, k2;
    sincos_gap64(tau, c.V1, dl1 - dl0, &s1, &k1);
    sincos_gap64(tau, c.V2, dl2 - dl0, &s2, &k2);
    // e^{-i phi} - 1 = (k - 1) - i s
    const double a1 = k1 - 1.0, a2 = k2 - 1.0;
    const double Sr = fma(C2i, s2, fma(C2r, a2, fma(C1i, s1, fma(C1r, a1, h.diag))));
    const double Si = fma(-C2r, s2, fma(C2i, a2, fma(-C1r, s1, C1i * a1)));
    return fma(Sr, Sr, Si * Si);
}

// The FP64-eigenvalue variant (FP64 for the cubic eigen-solve and the phases,
// FP32 for the amplitude): FP32 seed, one FP64 Newton step per root on the
// depressed cubic, FP64 phase differences tau (mu_l - mu_0) reduced modulo 2 pi
// in FP64, then the same FP32 amplitude.  Ad: signed matter term [eV^2];
// trev = c_L L / (2 pi E) [revolutions per eV^2].
// Depressed-cubic roots for the FP64-eigenvalue variant: FP32 trigonometric
// seed, one FP64 Newton step per lower root (the small correction divided in
// FP32), the top root from the zero sum of the depressed roots.
__device__ __forceinline__ void roots_mix(const Pt32 &c, const Pt64 &c64, double Ad, double &m0, double &m1,
                                          double &m2, double &t3) {
    float s0, s1, t3f, cth;
    seed_roots32(c, (float)Ad, s0, s1, t3f, cth);
    const double p = fma(fma(Ad, -1.0 / 3.0, c64.p1), Ad, c64.p0);
    const double q = fma(fma(fma(Ad, -2.0 / 27.0, c64.q2), Ad, c64.q1), Ad, c64.q0);
    m0 = (double)s0;
    m1 = (double)s1;
    if (fabsf(cth) > kNearDouble) {
        const double2 m = near_double_pair64(p, q, cth, s0, s1);
        m0 = m.x;
        m1 = m.y;
    }
    m0 -= (double)((float)fma(fma(m0, m0, p), m0, q) / (float)fma(3.0 * m0, m0, p));
    m1 -= (double)((float)fma(fma(m1, m1, p), m1, q) / (float)fma(3.0 * m1, m1, p));
    m2 = -m0 - m1;
    t3 = (c64.T0 + Ad) * (1.0 / 3.0);
}

template <bool REAL>
__device__ __forceinline__ float prob_mix(const Pt32 &c, const Ch32 &h, const Pt64 &c64, double Ad, double trev,
                                          bool &redo) {
    const float A = (float)Ad;
    double m0, m1, m2, t3;
    roots_mix(c, c64, Ad, m0, m1, m2, t3);
    // shifts from the FP64 eigenvalues (exact relative to the shift), gaps of the FP64 roots
    const float dl0 = (float)((m0 + t3) - c64.d0), dl1 = (float)((m1 + t3) - c64.d1), dl2 = (float)((m2 + t3) - c64.d2);
    const float g01 = (float)(m0 - m1), g02 = (float)(m0 - m2), g12 = (float)(m1 - m2);
    // phase differences in revolutions, reduced in FP64, then half angles [rad]
    const double r1 = trev * (m1 - m0), r2 = trev * (m2 - m0);
    const float f1 = (float)(r1 - rint(r1)), f2 = (float)(r2 - rint(r2));
    float est;
    const float P = amplitude_mass32<REAL>(c, h, A, dl0, dl1, dl2, g01, g02, g12, 3.14159265358979323846f * f1,
                                           3.14159265358979323846f * f2, est);
    redo = !(est <= kFp32EstMax);
    return P;
}
__device__ __forceinline__ float prob_mix(const Pt32 &c, const Ch32 &h, const Pt64 &c64, double Ad, double trev,
                                          bool &redo) {
    return h.real ? prob_mix<true>(c, h, c64, Ad, trev, redo) : prob_mix<false>(c, h, c64, Ad, trev, redo);
}

}  // namespace osc
