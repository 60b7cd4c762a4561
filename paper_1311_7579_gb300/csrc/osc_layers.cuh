// osc_layers.cuh -- propagation through piecewise-constant matter (a path of
// layers, generalising the constant density of Sec. 1.1).
//
// The amplitude is the product of the layers' constant-density propagators in
// the order of travel.  It is carried as a state vector psi in the vacuum mass
// basis (columns of U in the sorted vacuum order d0 <= d1 <= d2), where every
// layer's Hamiltonian is a rank-one update of the same diagonal matrix:
//   M = D + A w w^dagger,  w_l = conj(U_el)  (antineutrinos: U -> U*, A -> -A).
// Its eigenvectors are known in closed form, v_l proportional to (D - lambda_l)^-1 w,
// so with lambda_l = d_l + delta_l the projectors are P_l = v_l v_l^dagger / |v_l|^2,
//   v_l,i = w_i rt_i,  rt_l = 1,  rt_i = -delta_l / (d_i - d_l - delta_l)  (i != l),
// with every factor formed from the vacuum gaps and the matter shifts, so
// no cancellation happens.  One layer then acts as (up to a global phase)
//   psi <- psi + sum_{l=1,2} (e^{-i (phi_l - phi_0)} - 1) P_l psi
// (projector-sum identity), e^{-i phi} - 1 = -2 sin(phi/2) (sin(phi/2) + i cos(phi/2)).
// psi starts as conj(U_alpha .) and the amplitude is sum_l U_beta l psi_l.
#pragma once

#include "osc_kernels.cuh"

namespace osc {

// U in the sorted vacuum order, conjugated for antineutrinos (U~ = U or U*).
template <typename T>
struct LayU {
    T r[9], i[9];  // entry (f, l) at 3 f + l
};

template <typename T>
__device__ __forceinline__ void load_layu(const T *__restrict__ lu, bool nubar, LayU<T> &u) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        u.r[k] = lu[2 * k];
        u.i[k] = nubar ? -lu[2 * k + 1] : lu[2 * k + 1];
    }
}

template <typename T>
__device__ __forceinline__ T rcp_t(T x);
template <>
__device__ __forceinline__ float rcp_t<float>(float x) {
    return rcp_approx(x);
}
template <>
__device__ __forceinline__ double rcp_t<double>(double x) {
    return rcp64(x);
}

// One layer: psi <- psi + sum_{l=1,2} (e^{-i phi_l} - 1) P_l psi (phases relative
// to root 0).  g01, g02, g12: vacuum gaps d_i - d_j; dl1, dl2: matter shifts of
// roots 1 and 2; (s_l, k_l) = sin, cos of the half phase difference.
template <typename T>
__device__ __forceinline__ void layer_update(T pr[3], T pi[3], const LayU<T> &u, T g01, T g02, T g12, T dl1,
                                             T dl2, T s1, T k1, T s2, T k2) {
    // y_i = conj(w_i) psi_i = U~_ei psi_i and z_i = |w_i|^2
    T yr[3], yi[3], z[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        yr[i] = u.r[i] * pr[i] - u.i[i] * pi[i];
        yi[i] = u.r[i] * pi[i] + u.i[i] * pr[i];
        z[i] = u.r[i] * u.r[i] + u.i[i] * u.i[i];
    }
    // eigenvector weights rt_i of roots 1 and 2 (d2 - d1 = -g12, d1 - d2 = g12)
    const T a10 = -dl1 * rcp_t<T>(g01 - dl1), a12 = dl1 * rcp_t<T>(g12 + dl1);
    const T a20 = -dl2 * rcp_t<T>(g02 - dl2), a21 = -dl2 * rcp_t<T>(g12 - dl2);
    // s_l = v_l^dagger psi (up to the scale of v_l), n_l = |v_l|^2
    const T s1r = a10 * yr[0] + yr[1] + a12 * yr[2], s1i = a10 * yi[0] + yi[1] + a12 * yi[2];
    const T s2r = a20 * yr[0] + a21 * yr[1] + yr[2], s2i = a20 * yi[0] + a21 * yi[1] + yi[2];
    const T n1 = a10 * a10 * z[0] + z[1] + a12 * a12 * z[2];
    const T n2 = a20 * a20 * z[0] + a21 * a21 * z[1] + z[2];
    // kappa_l = s_l (e^{-i phi_l} - 1) / n_l
    const T q1 = T(-2) * s1 * rcp_t<T>(n1), q2 = T(-2) * s2 * rcp_t<T>(n2);
    const T e1r = q1 * s1, e1i = q1 * k1, e2r = q2 * s2, e2i = q2 * k2;
    const T K1r = s1r * e1r - s1i * e1i, K1i = s1r * e1i + s1i * e1r;
    const T K2r = s2r * e2r - s2i * e2i, K2i = s2r * e2i + s2i * e2r;
    // psi_i += w_i (rt_1i kappa_1 + rt_2i kappa_2), w_i = conj(U~_ei)
    const T cr[3] = {a10 * K1r + a20 * K2r, K1r + a21 * K2r, a12 * K1r + K2r};
    const T ci[3] = {a10 * K1i + a20 * K2i, K1i + a21 * K2i, a12 * K1i + K2i};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        pr[i] += u.r[i] * cr[i] + u.i[i] * ci[i];
        pi[i] += u.r[i] * ci[i] - u.i[i] * cr[i];
    }
}

// Entry (f, l) of U~ for a flavour f known only at run time, by selects (an
// indexed register array would go to local memory).
template <typename T>
__device__ __forceinline__ void u_entry(const LayU<T> &u, int f, int l, T &re, T &im) {
    re = (f == 0) ? u.r[l] : (f == 1) ? u.r[3 + l] : u.r[6 + l];
    im = (f == 0) ? u.i[l] : (f == 1) ? u.i[3 + l] : u.i[6 + l];
}

template <typename T>
__device__ __forceinline__ void layer_init(T pr[3], T pi[3], const LayU<T> &u, int alpha) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        T ur, ui;
        u_entry(u, alpha, l, ur, ui);
        pr[l] = ur;
        pi[l] = -ui;
    }
}

template <typename T>
__device__ __forceinline__ T layer_prob(const T pr[3], const T pi[3], const LayU<T> &u, int beta) {
    T ar = 0, ai = 0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        T ur, ui;
        u_entry(u, beta, l, ur, ui);
        ar += ur * pr[l] - ui * pi[l];
        ai += ur * pi[l] + ui * pr[l];
    }
    return ar * ar + ai * ai;
}

// Constants of layer k; a single-layer sample in a layered launch has no layer
// table and uses its own path constants.
__device__ __forceinline__ float4 layer32(const SampleDev &sd, int k) {
    return sd.lay32 ? sd.lay32[k] : make_float4(sd.kA_rhoye_f, sd.rev_hi, sd.rev_lo, 0.0f);
}
__device__ __forceinline__ double2 layer64(const SampleDev &sd, int k) {
    return sd.lay64 ? sd.lay64[k] : make_double2(sd.kA_rhoye, sd.cLL);
}

// P(alpha -> beta) through the sample's layers, FP32 bulk (PREC == kFP32) or with
// the FP64 eigen-solve and phase reduction (PREC == kMix; c64 and d64 used).
template <int PREC>
__device__ __forceinline__ float prob_layers32(const Pt32 &c, const Pt64 &c64, const double *d64, const LayU<float> &u,
                                               const SampleDev &sd, int ch, float E) {
    const int nubar = ch >= 9;
    const int ab = ch - 9 * nubar;
    float pr[3], pi[3];
    layer_init(pr, pi, u, ab / 3);
    const float r0 = rcp_approx(E);
    const float rl = r0 * fmaf(-E, r0, 1.0f);
    for (int k = 0; k < sd.n_layers; ++k) {
        float dl1, dl2, h1, h2;
        if (PREC == kFP32) {
            const float4 ly = layer32(sd, k);
            const float A = nubar ? -(ly.x * E) : ly.x * E;
            const float th = ly.y * r0;
            const float tl = fmaf(ly.y, r0, -th) + fmaf(ly.y, rl, ly.z * r0);
            float dl0;
            shifts32(c, A, dl0, dl1, dl2);
            h1 = 3.14159265358979323846f * phase_rev(th, tl, c.v1h, c.v1l, dl1 - dl0);
            h2 = 3.14159265358979323846f * phase_rev(th, tl, c.v2h, c.v2l, dl2 - dl0);
        } else {
            const double2 ly = layer64(sd, k);
            const double Ad = nubar ? -(ly.x * (double)E) : ly.x * (double)E;
            double m0, m1, m2, t3;
            roots_mix(c, c64, Ad, m0, m1, m2, t3);
            dl1 = (float)((m1 + t3) - d64[1]);
            dl2 = (float)((m2 + t3) - d64[2]);
            const double trev = ly.y * (0.15915494309189533577 / (double)E);
            const double q1 = trev * (m1 - m0), q2 = trev * (m2 - m0);
            h1 = 3.14159265358979323846f * (float)(q1 - rint(q1));
            h2 = 3.14159265358979323846f * (float)(q2 - rint(q2));
        }
        float s1, k1, s2, k2;
        __sincosf(h1, &s1, &k1);
        __sincosf(h2, &s2, &k2);
        layer_update<float>(pr, pi, u, c.g01, c.g02, c.g12, dl1, dl2, s1, k1, s2, k2);
    }
    return layer_prob(pr, pi, u, ab % 3);
}

// P(alpha -> beta) through the sample's layers, all FP64.  d: sorted vacuum eigenvalues.
__device__ __forceinline__ double prob_layers64(const Pt64 &c, const double *d, const LayU<double> &u,
                                                const SampleDev &sd, int ch, float E) {
    const int nubar = ch >= 9;
    const int ab = ch - 9 * nubar;
    double pr[3], pi[3];
    layer_init(pr, pi, u, ab / 3);
    const double Ed = (double)E;
    const double iE = rcp64(Ed);
    for (int k = 0; k < sd.n_layers; ++k) {
        const double2 ly = layer64(sd, k);
        const double A = nubar ? -(ly.x * Ed) : ly.x * Ed;
        double dl0, dl1, dl2;
        shifts64(c, A, dl0, dl1, dl2);
        // half phases c_L L (lambda_l - lambda_0) / (2 E)
        Tau64 ht = tau64(ly.y, Ed, iE);
        ht.hi *= 0.5;
        ht.lo *= 0.5;
        double s1, k1, s2, k2;
        sincos_gap64(ht, c.V1, dl1 - dl0, &s1, &k1);
        sincos_gap64(ht, c.V2, dl2 - dl0, &s2, &k2);
        layer_update<double>(pr, pi, u, d[0] - d[1], d[0] - d[2], d[1] - d[2], dl1, dl2, s1, k1, s2, k2);
    }
    return layer_prob(pr, pi, u, ab % 3);
}

}  // namespace osc
