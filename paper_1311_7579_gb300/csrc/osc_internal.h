// osc_internal.h -- types shared by the host runtime and the CUDA kernels of
// the GB300 oscillation-reweighting library.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/osc.h"

namespace osc {

// Unit constant of the propagation phase: lambda[eV^2] L[km] / E[GeV] -> radians
// of lambda L / (2E); 1e-6 / (2 hbar c), hbar c = 1.973269804e-7 eV m (CODATA 2018).
constexpr double kCL = 1e-6 / (2.0 * 1.973269804e-7);
// Matter term A = kKA * Y_e * rho[g/cm^3] * E[GeV] in eV^2: 2 sqrt(2) G_F N_A (hbar c)^3 * 1e9
// with G_F = 1.1663788e-23 eV^-2 (PDG), N_A = 6.02214076e23, hbar c = 1.973269804e-5 eV cm.
double matter_k_A();

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Channel id of an event: nubar * 9 + alpha * 3 + beta.
__host__ __device__ inline int chan_id(int alpha, int beta, int nubar) { return nubar * 9 + alpha * 3 + beta; }

// ---- per-point constants (written by the constants kernel in FP64) ----------
// FP32 block (floats).  Layout offsets:
enum PC32 : int {
    C32_P0 = 0, C32_P1, C32_Q0, C32_Q1, C32_Q2,  // depressed cubic's -p/3 (P0, P1) and -q/2 (Q0..Q2) in A
    C32_T0, C32_C10, C32_SMT,                    // tr H0, c1(A=0), H0_mumu + H0_tautau
    C32_D0, C32_D1, C32_D2,                      // sorted vacuum eigenvalues (eV^2)
    C32_G01, C32_G02, C32_G12,                   // vacuum gaps d_i - d_j
    C32_V1H, C32_V1L, C32_V2H, C32_V2L,          // (d1 - d0), (d2 - d0) as float-float
    C32_S0, C32_PI0, C32_W0, C32_E0,             // shifted-cubic constants, sorted root 0
    C32_S1, C32_PI1, C32_W1, C32_E1,             // ... sorted root 1
    C32_ESCALE,
    C32_TD0, C32_TD1,                            // T0 / 3 - d0, T0 / 3 - d1
    C32_SD02, C32_SD01,                          // d0 + d2, d0 + d1 (T0 less one sorted vacuum eigenvalue)
    C32_CH = 32,                                 // 9 channels x (X0r, X0i, X1r, X1i, X2r, X2i, Zr, Zi), neutrino:
                                                 // X_m = U_bm conj(U_am) (m a sorted vacuum state),
                                                 // Z = [alpha = e] H0_be + [beta = e] H0_ea
    C32_LU = 104,                                // U[f][l] (re, im), f flavour, l sorted vacuum root, neutrino
    C32_STRIDE = 128                             // floats, 512 B
};
// FP64 block (doubles).
enum PC64 : int {
    C64_P0 = 0, C64_P1, C64_Q0, C64_Q1, C64_Q2, C64_T0, C64_C10, C64_SMT, C64_ESCALE, C64_NORM,
    C64_CH = 16,                                 // 9 channels x (Xr, Xi, Yr, Yi, Zr, Zi), neutrino
    C64_LU = 72,                                 // U[f][l] (re, im) as in the FP32 block
    C64_LD = 90,                                 // sorted vacuum eigenvalues d0 <= d1 <= d2
    C64_SH = 96,                                 // shifted-cubic constants S, PI, W, E of sorted roots 0, 1
    C64_VG = 104,                                // vacuum gaps d1 - d0, d2 - d0, d1 - d2
    C64_STRIDE = 112                             // doubles, 896 B
};

// ---- histogram accumulators -------------------------------------------------
// A bin's exact 128-bit fixed-point sum is held as kDigits integer columns of
// 32-bit digits (u64 each): a flush adds each digit of its 128-bit value, so a
// column absorbs 2^32 flushes before it could wrap -- more than the events of
// any call (n < 2^31), even when every event flushes.
constexpr int kDigits = 4;

// ---- resident sample as seen by a kernel ----------------------------------
struct SampleDev {
    const float4 *ev;         // per event (e_true, e_reco, w_mc, channel id bits), sorted by (channel, e_reco)
    const int32_t *perm;      // sorted position -> caller's event index
    int64_t n;
    double kA_rhoye;          // k_A * rho * Y_e  [eV^2 / GeV]
    double cLL;               // c_L * L           [rad GeV / eV^2]
    float kA_rhoye_f;
    float rev_hi, rev_lo;     // c_L L / (2 pi) as float-float [revolutions GeV / eV^2]
    float hscale_f;           // 2^(F-64): FP32 weight -> fixed-point high word
    double hscale_d;
    int32_t frac_bits;        // F
    int32_t n_layers;         // 1: constant density; > 1: the layer tables below
    const float4 *lay32;      // per layer (k_A rho Y_e, c_L L / (2 pi) hi, lo, 0)
    const double2 *lay64;     // per layer (k_A rho Y_e, c_L L)
};

// One unit of histogram work: a point tile of one sample over an event range.
struct WorkItem {
    int32_t sample;           // index into the launch's SampleDev table
    int32_t point_base;       // first point (row of the constants tables)
    int32_t n_pts;            // points in this tile (<= points per block)
    int32_t ev_count;         // events in this item
    int64_t ev_begin;         // first (sorted) event
    int64_t acc_base;         // first histogram of the tile (histogram index)
};

struct HistParams {
    const WorkItem *items;
    int32_t n_items;
    int32_t nbins;
    const SampleDev *samples;
    const float *pc32;
    const double *pc64;
    unsigned long long *acc;  // fixed-point bins: kDigits integer digit columns per bin
    int32_t *counter;         // dynamic work counter (reset by the finalize kernel)
    float lo_f, inv_f, nb_f;
    // FP32 precisions: per work item, set when an event of the item needs the FP64
    // recomputation (the histogram kernel leaves such events out; k_redo adds them)
    uint8_t *redo;
    // fused finalize (small outputs): the last block converts the bins
    int32_t fuse_final;
    int64_t fin_n_hist;
    const double *fin_hmeta;
    double *fin_out;
};

// Points passed to the constants kernel by value (no host-to-device copy).
constexpr int kPointsByValue = 256;

// Domain of the FP32 paths: the matter term at most kFp32MatterRatio |dm31|.
// Beyond it two eigenvalues in matter form a near-double pair at the scale of
// the eigenvalue cubic, which FP32 constants cannot resolve (errors grow from
// ~1e-4 to O(1) between 1e3 and 3e3); calls with a (point, sample) outside it
// run in FP64.
constexpr double kFp32MatterRatio = 1000.0;
// OSC_FP32_BULK forms the eigenvalue shifts and the phases in FP32.  Their
// rounding, amplified near narrow resonances, grows with the phase the matter
// term adds over the baseline (c_L L k_A rho Y_e, energy independent) and with
// the matter term itself; a call with a (point, sample) whose matter phase
// exceeds kFp32BulkMatterPhase rad or whose largest matter term exceeds
// kFp32BulkMatterRatio |dm31| takes its shifts and phases in FP64
// (OSC_FP32_F64EIG).  Beam baselines stay far inside (1300 km at 2.85 g/cm^3:
// 0.72 rad, and |A| <= 5 |dm31| up to 45 GeV).
constexpr double kFp32BulkMatterPhase = 3.0;
constexpr double kFp32BulkMatterRatio = 10.0;
// Per-event error estimate of the FP32 amplitude (units of the FP32 rounding
// unit 2^-24): an event whose estimate exceeds kFp32EstMax, or (FP32-bulk)
// whose trigonometric seed has |cos theta| above kFp32SeedCos (a near-double
// pair the single Newton step may not resolve), is recomputed in FP64.
// kFp32EstMax = 30 keeps the estimated FP32 error below 30 * 2^-24 * 2 = 3.6e-6
// in P, which with the sine/cosine and phase rounding stays under 1e-5.
constexpr float kFp32EstMax = 30.0f;
constexpr float kFp32SeedCos = 0.9995f;
template <int N>
struct PointsByValueT {
    int32_t n;
    osc_point p[N];
};

struct FinalParams {
    unsigned long long *acc;
    const double *hmeta;      // per histogram: (2^(64-F), 2^-F, unused, point index)
    const double *pc64;       // per-point FP64 constants (norm)
    double *out;
    int64_t n_hist;
    int32_t nbins;
    int32_t *counter;
};

struct ReweightParams {
    SampleDev s;
    int32_t point;
    const float *pc32;
    const double *pc64;
    double norm;
    double *out_prob;         // caller order, may be null
    double *out_weight;
};

constexpr int kMaxLayers = 16;  // layers of a piecewise-constant matter path

// ---- binned (bin-centre) method ---------------------------------------------
constexpr int kChannels = 18;  // channel ids nubar * 9 + alpha * 3 + beta
// One row of the bin-centre probability table: P at every true-bin centre for
// one (sample of the launch, point, channel present in that sample).
struct BcRow {
    int32_t sample, point, chan, pad;
};
struct BcParams {
    HistParams h;             // work items, samples, accumulators, E_reco binning, finalize
    const BcRow *rows;
    int32_t n_rows;
    int32_t t_nbins;          // true-energy bins
    const int32_t *row_map;   // [histogram][channel] -> table row (-1: channel absent)
    double t_lo, t_w;         // first true-bin edge and bin width (t_hi - t_lo) / t_nbins
    float t_lo_f, t_inv_f, t_nb_f;
    float *tab32;             // [n_rows][t_nbins] FP32 / FP32_F64EIG probabilities
    unsigned long long *tabq; // [n_rows][t_nbins] FP64 probabilities as P * 2^63, rounded
};

// Debug builds (OSC_DEBUG_CHECKS): bits of the error word, int kDebugWord of a
// launch's 64-byte counter block, set by a kernel that found an index outside
// its buffers.
enum DebugCode : unsigned { kDbgItem = 1u, kDbgBin = 2u, kDbgRow = 4u, kDbgLayers = 8u };
constexpr int kDebugWord = 15;
// Ints of a launch's counter block used by the FP64 recomputation: the number of
// work items marked for it, and the completion ticket of the redo kernel.
constexpr int kRedoCount = 8;
constexpr int kRedoTicket = 9;

// Precision of a kernel instantiation.
enum Prec { kFP64 = 0, kFP32 = 1, kMix = 2 };  // kMix: FP64 eigen-solve and phases, FP32 amplitude

}  // namespace osc
