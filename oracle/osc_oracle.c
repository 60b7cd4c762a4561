/*
 * osc_oracle.c -- plain, slow FP64 CPU oracle for event-by-event three-flavour
 * oscillation reweighting through matter of constant density.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or constant table with the
 * CUDA path: every physical constant below is restated here from its
 * published value.
 *
 * What it computes (the plain definition, not the GPU's algorithm):
 *   Sec. 1.1, Eq. (1): vacuum amplitude  sum_i U*_{alpha i} U_{beta i}
 *       exp(-i m_i^2 L / 2E)   (the printed equation drops the U* factor and the
 *       unit constant; both are restored here, see c_L below).
 *   Sec. 1.1 (matter effects, "calculated as prescribed in [bib1]"): the
 *       flavour-basis Hamiltonian M = U diag(0, dm21, dm31) U^dagger
 *       + diag(A, 0, 0), with A = 2 sqrt(2) G_F N_e E; antineutrinos use U* and -A.
 *   The constant-density propagator S = exp(-i c_L M L / E) is formed from a
 *   cyclic complex-Hermitian Jacobi eigendecomposition M = V Lambda V^dagger,
 *   S = V diag(exp(-i c_L lambda_k L / E)) V^dagger, and P(alpha->beta) = |S_{beta alpha}|^2.
 *   Sec. 1.1.1 (event-by-event reweighting, energy-scale systematic): each event's
 *   weight is P * w_mc * norm; its reconstructed energy, scaled by the point's
 *   energy scale, selects a bin of a histogram over [lo, hi) by a fixed FP32
 *   rounding sequence; bins are plain sums of weights in event-index order.
 *   Sec. 1.1.1 (binned alternative): the probability taken at the centre of the
 *       event's true-energy bin instead of at its own energy.
 *   Layered matter (generalises Sec. 1.1's constant density): the product of
 *       the layers' constant-density propagators in the order of travel.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (contraction off so
 * that the FP32 binning sequence rounds after every operation on every host).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Unit constant of the vacuum phase: lambda[eV^2] * L[km] / E[GeV] -> radians of
 * lambda L / (2E) in natural units; 1e-6 / (2 * hbar c[eV m]),
 * hbar c = 1.973269804e-7 eV m (CODATA 2018). */
#define ORC_HBARC_EV_M 1.973269804e-7
static double orc_c_L(void) { return 1e-6 / (2.0 * ORC_HBARC_EV_M); }

/* Matter potential: A = 2 sqrt(2) G_F N_e E.  With N_e = rho[g/cm^3] Y_e N_A
 * per cm^3, G_F = 1.1663788e-5 GeV^-2 (PDG), N_A = 6.02214076e23 /mol,
 * hbar c = 1.973269804e-5 eV cm, A[eV^2] = k_A * Y_e * rho * E[GeV]. */
static double orc_k_A(void) {
    const double G_F = 1.1663788e-23; /* eV^-2 */
    const double N_A = 6.02214076e23;
    const double hbarc_cm = 1.973269804e-5; /* eV cm */
    double V = sqrt(2.0) * G_F * N_A * hbarc_cm * hbarc_cm * hbarc_cm; /* eV per (rho Ye) */
    return 2.0 * V * 1e9; /* eV^2 per (GeV * rho * Ye) */
}

double orc_const_c_L(void) { return orc_c_L(); }
double orc_const_k_A(void) { return orc_k_A(); }

/* One oscillation-parameter point (all doubles): sin^2 theta12, sin^2 theta13,
 * sin^2 theta23, dm21 [eV^2], dm32 [eV^2] (sign = hierarchy), delta_cp [rad],
 * energy scale applied to E_reco, normalisation applied to the weight. */
typedef struct {
    double s2_12, s2_13, s2_23, dm21, dm32, dcp, escale, norm;
} orc_point;

typedef double complex cplx;

/* PMNS matrix in the PDG parametrisation, U[flavour][mass], flavour order (e, mu, tau). */
void orc_pmns(const orc_point *pt, cplx U[3][3]) {
    double s12 = sqrt(pt->s2_12), c12 = sqrt(1.0 - pt->s2_12);
    double s13 = sqrt(pt->s2_13), c13 = sqrt(1.0 - pt->s2_13);
    double s23 = sqrt(pt->s2_23), c23 = sqrt(1.0 - pt->s2_23);
    cplx eid = cexp(I * pt->dcp);     /* e^{+i delta} */
    cplx emid = cexp(-I * pt->dcp);   /* e^{-i delta} */
    U[0][0] = c12 * c13;
    U[0][1] = s12 * c13;
    U[0][2] = s13 * emid;
    U[1][0] = -s12 * c23 - c12 * s23 * s13 * eid;
    U[1][1] = c12 * c23 - s12 * s23 * s13 * eid;
    U[1][2] = s23 * c13;
    U[2][0] = s12 * s23 - c12 * c23 * s13 * eid;
    U[2][1] = -c12 * s23 - s12 * c23 * s13 * eid;
    U[2][2] = c23 * c13;
}

/* Flavour-basis Hamiltonian (times 2E) in eV^2 for a signed matter term:
 * M = U diag(0, dm21, dm31) U^dagger + diag(A, 0, 0); for antineutrinos U -> U*
 * and A -> -A.  dm31 = dm32 + dm21. */
void orc_hamiltonian(const orc_point *pt, double A_abs, int nubar, cplx M[3][3]) {
    cplx U[3][3];
    orc_pmns(pt, U);
    if (nubar)
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 3; ++i) U[a][i] = conj(U[a][i]);
    double m2[3] = {0.0, pt->dm21, pt->dm32 + pt->dm21};
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0.0;
            for (int i = 0; i < 3; ++i) s += U[b][i] * m2[i] * conj(U[a][i]);
            M[b][a] = s;
        }
    M[0][0] += nubar ? -A_abs : A_abs;
}

static void mat_mul(cplx A[3][3], cplx B[3][3], cplx C[3][3]) {
    cplx T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void mat_adj(cplx A[3][3], cplx B[3][3]) {
    cplx T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = conj(A[j][i]);
    memcpy(B, T, sizeof(T));
}

/* Cyclic Jacobi eigendecomposition of a complex Hermitian 3x3 matrix:
 * M = V diag(lam) V^dagger.  Each step zeroes M[p][q] with G = D R, where
 * D = diag(1, e^{-i phi}) (phi = arg M[p][q]) makes the 2x2 block real and
 * R is the real rotation with tan 2theta = 2|M[p][q]| / (M[q][q] - M[p][p]).
 * Sweeps run until the off-diagonal norm is below 1e-15 of the Frobenius norm.
 * Returns the number of sweeps, or -1 if 100 sweeps did not converge. */
int orc_eigh3(const cplx Min[3][3], double lam[3], cplx V[3][3]) {
    cplx M[3][3];
    memcpy(M, Min, sizeof(M));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) fro += creal(M[i][j] * conj(M[i][j]));
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 3; ++q) off += 2.0 * creal(M[p][q] * conj(M[p][q]));
        off = sqrt(off);
        if (off == 0.0 || off <= 1e-15 * fro) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double r = cabs(M[p][q]);
                if (r == 0.0) continue;
                double phi = carg(M[p][q]);
                double theta = 0.5 * atan2(2.0 * r, creal(M[q][q]) - creal(M[p][p]));
                double c = cos(theta), s = sin(theta);
                cplx G[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                cplx emphi = cexp(-I * phi);
                G[p][p] = c;
                G[p][q] = s;
                G[q][p] = -s * emphi;
                G[q][q] = c * emphi;
                cplx Gh[3][3];
                mat_adj(G, Gh);
                mat_mul(M, G, M);
                mat_mul(Gh, M, M);
                mat_mul(V, G, V);
            }
    }
    for (int i = 0; i < 3; ++i) lam[i] = creal(M[i][i]);
    return sweep < 100 ? sweep : -1;
}

/* S = exp(-i tau M) with tau = c_L L / E, from the eigendecomposition. */
void orc_evolution(const cplx M[3][3], double tau, cplx S[3][3]) {
    double lam[3];
    cplx V[3][3];
    orc_eigh3(M, lam, V);
    cplx ph[3];
    for (int k = 0; k < 3; ++k) ph[k] = cexp(-I * tau * lam[k]);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            cplx s = 0.0;
            for (int k = 0; k < 3; ++k) s += V[b][k] * ph[k] * conj(V[a][k]);
            S[b][a] = s;
        }
}

/* Matter term magnitude for an event: A = k_A * Y_e * rho * E  [eV^2]. */
static double orc_matter_A(double rho, double ye, double E) { return orc_k_A() * ye * rho * E; }

/* All nine probabilities P[beta][alpha] = P(nu_alpha -> nu_beta) at one energy. */
void orc_prob_matrix(const orc_point *pt, double L_km, double rho, double ye, double E_GeV,
                     int nubar, double P[3][3]) {
    cplx M[3][3], S[3][3];
    orc_hamiltonian(pt, orc_matter_A(rho, ye, E_GeV), nubar, M);
    orc_evolution(M, orc_c_L() * L_km / E_GeV, S);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) P[b][a] = creal(S[b][a] * conj(S[b][a]));
}

double orc_prob(const orc_point *pt, double L_km, double rho, double ye, double E_GeV,
                int alpha, int beta, int nubar) {
    double P[3][3];
    orc_prob_matrix(pt, L_km, rho, ye, E_GeV, nubar, P);
    return P[beta][alpha];
}

/* Same, for an explicit (signed-by-nubar) matter term A_abs instead of rho, Y_e. */
void orc_prob_matrix_A(const orc_point *pt, double L_km, double A_abs, double E_GeV, int nubar,
                       double P[3][3]) {
    cplx M[3][3], S[3][3];
    orc_hamiltonian(pt, A_abs, nubar, M);
    orc_evolution(M, orc_c_L() * L_km / E_GeV, S);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) P[b][a] = creal(S[b][a] * conj(S[b][a]));
}

/* Bin of one event under the energy-scale systematic.  The rounding sequence is
 * fixed in FP32: sf = (float)escale, lo_f = (float)lo, inv_f = (float)(nbins/(hi-lo)),
 * x = sf * e_reco, t = x - lo_f, u = t * inv_f; the event is kept iff t >= 0 and
 * u < nbins, and its bin is (int)u.  Returns -1 when dropped (half-open [lo, hi),
 * under- and overflow dropped, nothing clamped). */
int orc_bin(double escale, float e_reco, double lo, double hi, int nbins) {
    float sf = (float)escale;
    float lo_f = (float)lo;
    float inv_f = (float)((double)nbins / (hi - lo));
    float x = sf * e_reco;
    float t = x - lo_f;
    float u = t * inv_f;
    if (!(t >= 0.0f) || !(u < (float)nbins)) return -1;
    return (int)u;
}

/* Event weight (Sec. 1.1.1): probability x MC weight x the point's normalisation. */
static double orc_weight(double p, float w_mc, const orc_point *pt) { return p * (double)w_mc * pt->norm; }

/* Per-event probabilities and weights for one point (Sec. 1.1.1: weight =
 * P(alpha->beta at E_true) * w_mc * norm).  Events are independent; the loop
 * is split over threads, which does not change any result. */
void orc_reweight(int64_t n, const float *e_true, const float *w_mc, const uint8_t *flav_in,
                  const uint8_t *flav_out, const uint8_t *is_nubar, double L_km, double rho,
                  double ye, const orc_point *pt, double *out_prob, double *out_weight) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double p = orc_prob(pt, L_km, rho, ye, (double)e_true[i], flav_in[i], flav_out[i],
                            is_nubar[i]);
        if (out_prob) out_prob[i] = p;
        if (out_weight) out_weight[i] = orc_weight(p, w_mc[i], pt);
    }
}

/* Histogram of given per-event weights: hist[b] = sum over kept events, in
 * event-index order, of weight[i]; bin from orc_bin.  When compensated != 0 the
 * sum uses Neumaier's compensated summation (the "truth" accumulation). */
void orc_hist_from_weights(int64_t n, const float *e_reco, const double *weight, double escale,
                           double lo, double hi, int nbins, int compensated, double *hist) {
    for (int b = 0; b < nbins; ++b) hist[b] = 0.0;
    if (!compensated) {
        for (int64_t i = 0; i < n; ++i) {
            int b = orc_bin(escale, e_reco[i], lo, hi, nbins);
            if (b >= 0) hist[b] += weight[i];
        }
        return;
    }
    for (int b = 0; b < nbins; ++b) {
        double s = 0.0, c = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (orc_bin(escale, e_reco[i], lo, hi, nbins) != b) continue;
            double w = weight[i];
            double t = s + w;
            if (fabs(s) >= fabs(w))
                c += (s - t) + w;
            else
                c += (w - t) + s;
            s = t;
        }
        hist[b] = s + c;
    }
}

/* Event-by-event histograms for n_points points over one sample:
 * out[p][b] for p in [0, n_points).  scratch_w must hold n doubles. */
void orc_histogram(int64_t n, const float *e_true, const float *e_reco, const float *w_mc,
                   const uint8_t *flav_in, const uint8_t *flav_out, const uint8_t *is_nubar,
                   double L_km, double rho, double ye, const orc_point *pts, int n_points,
                   double lo, double hi, int nbins, int compensated, double *scratch_w,
                   double *out) {
    for (int p = 0; p < n_points; ++p) {
        orc_reweight(n, e_true, w_mc, flav_in, flav_out, is_nubar, L_km, rho, ye, &pts[p], 0,
                     scratch_w);
        orc_hist_from_weights(n, e_reco, scratch_w, pts[p].escale, lo, hi, nbins, compensated,
                              out + (int64_t)p * nbins);
    }
}

/* ------------------------------------------------------------- bin centres
 * Sec. 1.1.1 contrasts event-by-event reweighting with the quicker binned
 * method: the oscillation probability is evaluated once per bin of true
 * neutrino energy, at the bin's centre, and applied to every event of that bin
 * (the paper's example is a 25 MeV bin from 0.6 to 0.625 GeV evaluated at its
 * centre).  Here the true-energy bins are t_nbins equal bins over
 * [t_lo, t_hi); an event's bin follows the FP32 rule of orc_bin with unit
 * scale; the centre of bin t is t_lo + (t + 1/2) (t_hi - t_lo) / t_nbins,
 * evaluated in double and then stored in FP32 like an event energy.  Events
 * with E_true outside [t_lo, t_hi) get probability and weight 0. */
float orc_true_centre(double t_lo, double t_hi, int t_nbins, int t) {
    double w = (t_hi - t_lo) / (double)t_nbins;
    double c = t_lo + ((double)t + 0.5) * w;
    return (float)c;
}

void orc_reweight_bin_centre(int64_t n, const float *e_true, const float *w_mc, const uint8_t *flav_in,
                             const uint8_t *flav_out, const uint8_t *is_nubar, double L_km, double rho,
                             double ye, const orc_point *pt, double t_lo, double t_hi, int t_nbins,
                             double *out_prob, double *out_weight) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int t = orc_bin(1.0, e_true[i], t_lo, t_hi, t_nbins);
        double p = 0.0;
        if (t >= 0)
            p = orc_prob(pt, L_km, rho, ye, (double)orc_true_centre(t_lo, t_hi, t_nbins, t), flav_in[i],
                         flav_out[i], is_nubar[i]);
        if (out_prob) out_prob[i] = p;
        if (out_weight) out_weight[i] = orc_weight(p, w_mc[i], pt);
    }
}

/* ------------------------------------------------------- layered matter
 * Sec. 1.1 treats the matter density as constant along the baseline.  The
 * generalisation to a path of n layers (layer k: length L_k [km], density rho_k
 * [g/cm^3], electron fraction ye_k, traversed in the order k = 0, 1, ..., n-1
 * from the source) multiplies the layers' constant-density propagators in the
 * order of travel: S = S_{n-1} ... S_1 S_0 with
 * S_k = exp(-i c_L M(A_k) L_k / E), A_k = k_A ye_k rho_k E, and
 * P(alpha->beta) = |S_{beta alpha}|^2. */
void orc_prob_matrix_layers(const orc_point *pt, int n_layers, const double *L_km, const double *rho,
                            const double *ye, double E_GeV, int nubar, double P[3][3]) {
    cplx S[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int k = 0; k < n_layers; ++k) {
        cplx M[3][3], Sk[3][3];
        orc_hamiltonian(pt, orc_matter_A(rho[k], ye[k], E_GeV), nubar, M);
        orc_evolution(M, orc_c_L() * L_km[k] / E_GeV, Sk);
        mat_mul(Sk, S, S);
    }
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) P[b][a] = creal(S[b][a] * conj(S[b][a]));
}

void orc_prob_matrix_layers_many(const orc_point *pt, int n_layers, const double *L_km, const double *rho,
                                 const double *ye, int64_t n, const double *E_GeV, int nubar, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double P[3][3];
        orc_prob_matrix_layers(pt, n_layers, L_km, rho, ye, E_GeV[i], nubar, P);
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) out[9 * i + 3 * b + a] = P[b][a];
    }
}

/* Per-event probabilities and weights through a layered path (weight as in
 * orc_reweight). */
void orc_reweight_layers(int64_t n, const float *e_true, const float *w_mc, const uint8_t *flav_in,
                         const uint8_t *flav_out, const uint8_t *is_nubar, int n_layers, const double *L_km,
                         const double *rho, const double *ye, const orc_point *pt, double *out_prob,
                         double *out_weight) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double P[3][3];
        orc_prob_matrix_layers(pt, n_layers, L_km, rho, ye, (double)e_true[i], is_nubar[i], P);
        double p = P[flav_out[i]][flav_in[i]];
        if (out_prob) out_prob[i] = p;
        if (out_weight) out_weight[i] = orc_weight(p, w_mc[i], pt);
    }
}

/* Eigen-decomposition exposed for tests: M given as interleaved (re, im) row-major. */
int orc_eigh3_flat(const double *m_reim, double *lam, double *v_reim) {
    cplx M[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = m_reim[2 * (3 * i + j)] + I * m_reim[2 * (3 * i + j) + 1];
    int r = orc_eigh3(M, lam, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            v_reim[2 * (3 * i + j)] = creal(V[i][j]);
            v_reim[2 * (3 * i + j) + 1] = cimag(V[i][j]);
        }
    return r;
}

/* Hamiltonian exposed for tests (interleaved re/im, row-major M[beta][alpha]). */
void orc_hamiltonian_flat(const orc_point *pt, double A_abs, int nubar, double *m_reim) {
    cplx M[3][3];
    orc_hamiltonian(pt, A_abs, nubar, M);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            m_reim[2 * (3 * i + j)] = creal(M[i][j]);
            m_reim[2 * (3 * i + j) + 1] = cimag(M[i][j]);
        }
}

void orc_pmns_flat(const orc_point *pt, double *u_reim) {
    cplx U[3][3];
    orc_pmns(pt, U);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            u_reim[2 * (3 * i + j)] = creal(U[i][j]);
            u_reim[2 * (3 * i + j) + 1] = cimag(U[i][j]);
        }
}

/* Probability matrices for many energies at one point, flat out[n][beta][alpha]. */
void orc_prob_matrix_many(const orc_point *pt, double L_km, double rho, double ye, int64_t n,
                          const double *E_GeV, int nubar, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double P[3][3];
        orc_prob_matrix(pt, L_km, rho, ye, E_GeV[i], nubar, P);
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) out[9 * i + 3 * b + a] = P[b][a];
    }
}

/* Bins for many events (tests of the binning rule). */
void orc_bin_many(int64_t n, const float *e_reco, double escale, double lo, double hi, int nbins,
                  int32_t *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_bin(escale, e_reco[i], lo, hi, nbins);
}

/* Thread count of the OpenMP loops (for timing the oracle on 1 core and on all cores). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
