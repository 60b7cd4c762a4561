/*
 * osc.h -- C ABI of the GB300 (sm_103a) event-by-event neutrino oscillation
 * reweighting library.
 *
 * The calls follow the paper's statement of the problem (Sec. 2.1 and its code
 * listing): event energies are placed in device memory, the components that
 * depend only on the oscillation parameters are computed once per parameter
 * set, a kernel computes every event's oscillation probability in parallel,
 * and the results come back to the caller.  Unlike the paper, samples stay
 * resident on the device between calls and many parameter points are handled
 * in one launch.
 *
 * Physics (Sec. 1.1, Eq. (1) and the matter term; Sec. 1.1.1 weights):
 *   M = U diag(0, dm21, dm31) U^dagger + diag(A, 0, 0) [eV^2], dm31 = dm32 + dm21,
 *   U the PMNS matrix (PDG parametrisation, U_e3 = s13 e^{-i delta}),
 *   A = k_A * Y_e * rho[g/cm^3] * E_true[GeV], k_A = 2 sqrt(2) G_F N_A (hbar c)^3
 *     = 1.526493e-4 eV^2/GeV per g/cm^3,
 *   antineutrinos: U -> U*, A -> -A,
 *   P(alpha -> beta) = |[exp(-i c_L M L / E_true)]_{beta alpha}|^2,
 *     c_L = 1e-6 / (2 hbar c[eV m]) = 2.533865 (eV^2, km, GeV),
 *   event weight   = P * w_mc * norm,
 *   histogram bin  = FP32 sequence x = (float)escale * e_reco, t = x - (float)lo,
 *                    u = t * (float)(nbins / (hi - lo)); kept iff t >= 0 and
 *                    u < nbins; bin = (int)u  (half-open [lo, hi), no clamping).
 *
 * Conventions
 *   - Ownership: the library owns every device copy it makes (samples, point
 *     table, work lists, accumulators).  The caller owns every output buffer.
 *     No caller pointer is retained after a call returns (except the CUDA
 *     stream given to osc_create, which must outlive the context).
 *   - Errors: every call returns an osc_status.  On error, outputs are left
 *     untouched and osc_last_error() describes the cause.  Invalid input is
 *     rejected on the host before any launch.  A CUDA error poisons the
 *     context: later calls return OSC_E_STATE; running out of device memory
 *     (OSC_E_NOMEM) does not.  Device code never traps.
 *   - Autotuner cache: with OSC_AUTOTUNE_CACHE=<file> set when a context is
 *     created, the launch shapes the autotuner picks are appended to <file> (one
 *     line per GPU model and workload class) and read back by later contexts on
 *     the same GPU model, which then skip tuning.
 *   - Fault injection (tests): with the environment variable
 *     OSC_FAULT_ALLOC_FAIL_AT=k set when a context is created, that context's
 *     k-th device allocation fails as if the device were out of memory.
 *   - Threading: a context is not re-entrant, except osc_submit/osc_wait,
 *     which may be called from any thread while serving runs.
 *   - Determinism: histogram bins are accumulated in exact 128-bit fixed
 *     point, so results are bitwise identical for any tile shape, launch
 *     configuration or scheduling order.
 */
#ifndef OSC_GB300_H
#define OSC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OSC_OK = 0,
    OSC_E_ARG = 1,     /* malformed argument (null pointer, bad enum, bad size) */
    OSC_E_RANGE = 2,   /* value outside the physical / supported range */
    OSC_E_NOMEM = 3,   /* device allocation failed or workspace cap exceeded */
    OSC_E_CUDA = 4,    /* a CUDA call failed; the context is now poisoned */
    OSC_E_STATE = 5,   /* context poisoned, or call not valid in this state */
    OSC_E_TIMEOUT = 6, /* a bounded wait expired */
    OSC_E_BUSY = 7     /* serving queue full */
} osc_status;

/* Precisions.  OSC_FP64 is the plain path.  The two FP32 precisions return, for
 * every event, a probability within |dP| <= 1e-5 of the FP64 definition:
 *   - Per event: the FP32 amplitude (Sylvester numerators in the vacuum mass
 *     basis) bounds its own rounding error; an event whose bound exceeds the
 *     tolerance (narrow resonances: small mixing angles at a level crossing,
 *     eigenvalues nearly degenerate in matter), or whose FP32 eigenvalue seed is
 *     ill-conditioned, is recomputed with the FP64 path's arithmetic.  In a
 *     histogram such events are added by a second pass over the marked work
 *     items; the bins stay exact and deterministic.
 *   - Per call: OSC_FP32_BULK forms the eigenvalue shifts and phases in FP32.  A
 *     call whose points and samples include a pair with the sample's matter
 *     phase c_L L k_A rho Y_e above 3 rad (summed over layers) or its largest
 *     matter term above 10 |dm31| runs as OSC_FP32_F64EIG (shifts and phases in
 *     FP64).  Beam baselines stay far inside: 1300 km at 2.85 g/cm^3 is 0.72 rad,
 *     and |A| <= 5 |dm31| up to 45 GeV there; a 12000 km path through 13 g/cm^3
 *     is 30 rad.
 *   - Per call: both FP32 precisions run wholly in OSC_FP64 where a (point,
 *     sample) pair has a matter term above 1000 |dm31| (with the sample's largest
 *     E_true and densest layer), where two eigenvalues in matter form a
 *     near-double pair that FP32 cannot resolve.  Through layers (osc_set_layers)
 *     OSC_FP32_BULK also needs dm21 >= 5e-3 |dm31| and a matter term at most
 *     100 |dm31|, else it runs in FP64.
 *   The layered kernels do not estimate their error per event: through layers
 *   the tolerance rests on the per-call rules above, measured over random layer
 *   profiles and points across the whole accepted domain.
 * Physical parameters stay far inside every limit: through the Earth's core at
 * 50 GeV, |A| is about 20 |dm31|, and dm21 is about 0.03 |dm31|. */
typedef enum {
    OSC_FP64 = 0,         /* all-FP64 path: closed-form cubic eigenvalues, FP64 amplitude */
    OSC_FP32_BULK = 1,    /* FP32 bulk with FP64-derived per-point constants: eigenvalues as
                             vacuum value + FP32 matter shift, float-float vacuum phases */
    OSC_FP32_F64EIG = 2   /* FP64 cubic eigen-solve and phase reduction, FP32 amplitude */
} osc_precision;

typedef enum { OSC_NU_E = 0, OSC_NU_MU = 1, OSC_NU_TAU = 2 } osc_flavour;

typedef struct osc_ctx osc_ctx;

/* One resident Monte Carlo sample at a fixed baseline and constant density
 * (Sec. 2.1: the per-event energy arrays; Sec. 1.1: L, rho).  All arrays are
 * host pointers of length n, read during osc_load_sample only. */
typedef struct {
    int64_t n;                /* number of events, >= 1 */
    const float *e_true;      /* true neutrino energy [GeV], finite, > 0 */
    const float *e_reco;      /* reconstructed energy [GeV], finite */
    const float *w_mc;        /* Monte Carlo weight, finite */
    const uint8_t *flav_in;   /* initial flavour alpha, osc_flavour */
    const uint8_t *flav_out;  /* final flavour beta, osc_flavour */
    const uint8_t *is_nubar;  /* 0 = neutrino, 1 = antineutrino */
    double baseline_km;       /* L > 0 */
    double density_gcc;       /* rho >= 0 */
    double ye;                /* electron fraction in [0, 1] */
} osc_sample_desc;

/* One oscillation-parameter point plus its systematics (Table 1 fields;
 * Sec. 1.1.1 energy-scale systematic).  sign(dm32) selects the hierarchy. */
typedef struct {
    double s2_12, s2_13, s2_23; /* sin^2 theta_ij in [0, 1] */
    double dm21;                /* eV^2, > 0 */
    double dm32;                /* eV^2, |dm32| > dm21 (non-degenerate vacuum spectrum) */
    double dcp;                 /* rad, |dcp| <= 1e6 */
    double escale;              /* energy scale applied to E_reco before binning, > 0 */
    double norm;                /* weight normalisation, finite */
} osc_point;

/* Library version string (static storage). */
const char *osc_version(void);

/* Create a context on CUDA device `device`.  workspace_cap_bytes bounds all
 * device memory the context allocates (0 = no cap).  cuda_stream is a
 * cudaStream_t to launch on (NULL: the context creates its own). */
osc_status osc_create(int device, size_t workspace_cap_bytes, void *cuda_stream, osc_ctx **out);

/* Stop serving, free every device and host resource of the context. NULL is a no-op. */
void osc_destroy(osc_ctx *ctx);

/* Last error message of the context (static "no context" for NULL). */
const char *osc_last_error(const osc_ctx *ctx);

/* Validate, sort by (channel, E_reco) and copy a sample to the device
 * (Sec. 2.1: host arrays copied to device memory).  The event order seen by
 * osc_reweight outputs is the caller's original order. */
osc_status osc_load_sample(osc_ctx *ctx, const osc_sample_desc *desc, int32_t *sample_id);

/* Free a resident sample (OSC_E_STATE while serving runs). */
osc_status osc_unload_sample(osc_ctx *ctx, int32_t sample_id);

/* Replace the parameter-point table with n_points host points (copied), and
 * compute every point's parameter-only constants on the device in FP64
 * (Sec. 2.1: "components dependent only on the oscillation parameters").
 * n_points in [1, 1<<20]. */
osc_status osc_set_params(osc_ctx *ctx, const osc_point *pts, int32_t n_points);

/* Per-event probability and weight (P * w_mc * norm) for one point of the
 * table, in the caller's event order (Sec. 2.1: result array copied back).
 * out_prob / out_weight: n doubles each, either may be NULL; host pointers if
 * out_on_device == 0 (a page-locked host buffer is written by the kernel
 * directly, a pageable one through a device staging buffer and a copy), device
 * pointers otherwise.  Synchronous. */
osc_status osc_reweight(osc_ctx *ctx, int32_t sample_id, int32_t point, osc_precision prec,
                        double *out_prob, double *out_weight, int out_on_device);

/* Event-by-event binned PDFs (Sec. 1.1.1): out[s][p][b] for s < n_samples,
 * p < n_points (table points point_begin + p), b < nbins, over [lo, hi).
 * All (sample, point, event) work runs in one launch.  out is host memory if
 * out_on_device == 0 (the call then returns when the bins are there; a
 * page-locked host buffer is written by the kernels directly, a pageable one
 * through a device staging buffer and a copy), device memory otherwise (the
 * call returns once the work is enqueued on the context stream). */
osc_status osc_histogram(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                         int32_t point_begin, int32_t n_points, osc_precision prec, double lo,
                         double hi, int32_t nbins, double *out, int out_on_device);

/* One fit step in one call: replaces the point table with the single point *pt
 * (as osc_set_params(ctx, pt, 1)) and computes its histograms (as
 * osc_histogram(ctx, sample_ids, n_samples, 0, 1, prec, lo, hi, nbins, out,
 * out_on_device)); out holds n_samples x nbins doubles.  Same arguments, errors
 * and synchronisation as those two calls; on an error in the point the table is
 * left as it was. */
osc_status osc_histogram_point(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples, const osc_point *pt,
                               osc_precision prec, double lo, double hi, int32_t nbins, double *out,
                               int out_on_device);

/* Exact histograms over several GPUs.  The path shards naturally (Sec. 2.1: one
 * event per thread, every event independent): by parameter points (each rank
 * calls osc_histogram for a slice of the point table; the slices are only
 * gathered) or by events (each rank holds a slice of a sample's events).  For
 * the event split the one exchange step is a sum of partial histograms, and
 * these three calls make it exact, so that the merged bins equal bit for bit
 * those of one osc_histogram call over all events:
 *
 * osc_sample_set_bounds: every rank sets, for its slice of a sample, the bounds
 *   of the whole sample: w_abs_max >= the largest |w_mc| and e_true_max >= the
 *   largest E_true over all ranks' events (an all-reduce of two maxima).  They
 *   fix the fixed-point scale F = 62 - ceil(log2 w_abs_max) (as osc_load_sample
 *   derives it from its own events) and the precision routing (osc_precision),
 *   so every rank sums and routes as one call over all events would.  Each
 *   bound must be at least the slice's own (OSC_E_RANGE otherwise); OSC_E_STATE
 *   while serving runs.  Cached launch plans are dropped.
 * osc_histogram_digits: osc_histogram with the same arguments, except that it
 *   returns each bin's exact fixed-point sum instead of a double: kDigits = 4
 *   uint64 words per bin, digits[((s * n_points + p) * nbins + b) * 4 + q], whose
 *   value is (d0 + d1 2^32 + d2 2^64 + (int64)d3 2^96) 2^-F before the point's
 *   norm.  Word-wise uint64 sums of these arrays over ranks (an all-reduce with
 *   integer wrap-around) are the digits of the exact total, as long as the
 *   ranks' events of a sample number fewer than 2^32 in all.  Host or device
 *   memory as for osc_histogram.
 * osc_histogram_from_digits: converts summed digits to bins exactly as every
 *   histogram call does (each sample's F from the sample, each point's norm
 *   from the current point table): out[s][p][b] for the same sample ids, point
 *   range and nbins as the digits call.  digits and out are both host
 *   (on_device == 0; the call returns when out is written) or both device
 *   memory (on_device == 1; the call returns once the work is enqueued). */
osc_status osc_sample_set_bounds(osc_ctx *ctx, int32_t sample_id, double w_abs_max, double e_true_max);
osc_status osc_histogram_digits(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples, int32_t point_begin,
                                int32_t n_points, osc_precision prec, double lo, double hi, int32_t nbins,
                                uint64_t *digits, int out_on_device);
osc_status osc_histogram_from_digits(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                     int32_t point_begin, int32_t n_points, int32_t nbins, const uint64_t *digits,
                                     double *out, int on_device);

/* Binned ("bin-centre") PDFs: the quicker alternative that Sec. 1.1.1 contrasts
 * with event-by-event reweighting, in which each event's probability is taken
 * at the centre of its true-energy bin instead of at its own E_true (the
 * paper's example: a 25 MeV bin from 0.6 to 0.625 GeV evaluated at its centre).
 *   true-energy bins: t_nbins equal bins over [t_lo, t_hi); an event's bin
 *     follows the histogram binning rule above with escale 1 (t = e_true -
 *     (float)t_lo, u = t * (float)(t_nbins / (t_hi - t_lo)), kept iff t >= 0
 *     and u < t_nbins, bin (int)u); 1 <= t_nbins <= 65536;
 *   centre of true bin k: (float)(t_lo + (k + 0.5) * ((t_hi - t_lo) / t_nbins)),
 *     evaluated in double and rounded to FP32 like an event energy;
 *   events with E_true outside [t_lo, t_hi) contribute nothing;
 *   weight P(centre) * w_mc * norm, binned by E_reco exactly as osc_histogram
 *     does (same out layout and rules, same exact fixed-point accumulation).
 * The probabilities are computed once per (sample, point, channel occurring in
 * the sample, true bin) into a table held by the cached launch plan: 4 bytes per
 * entry for OSC_FP32_BULK and OSC_FP32_F64EIG, 8 for OSC_FP64, counted against
 * the workspace cap (OSC_E_NOMEM beyond it).  out: host memory if
 * out_on_device == 0 (the call returns after the copy), else device memory (the
 * call returns once the work is enqueued on the context stream). */
osc_status osc_histogram_bin_centre(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                    int32_t point_begin, int32_t n_points, osc_precision prec,
                                    double t_lo, double t_hi, int32_t t_nbins, double lo, double hi,
                                    int32_t nbins, double *out, int out_on_device);

/* Piecewise-constant matter along the baseline.  Sec. 1.1 takes the density
 * as constant; this generalises it (the paper has no layered case).  The
 * sample's path becomes n_layers layers traversed in the given order from the
 * source: layer k has length length_km[k] > 0, density density_gcc[k] >= 0
 * [g/cm^3] and electron fraction ye[k] in [0, 1].  Then
 *   P(alpha -> beta) = |[S_{n-1} ... S_1 S_0]_{beta alpha}|^2,
 *   S_k = exp(-i c_L M(A_k) L_k / E_true),  A_k = k_A ye_k rho_k E_true.
 * This replaces the baseline, density and Y_e given at load.
 *   - n_layers == 1 sets a constant-density path, served by the single-layer
 *     kernels.
 *   - 2 <= n_layers <= 16 routes osc_reweight, osc_histogram and
 *     osc_histogram_bin_centre for this sample to the layered kernels.  These
 *     kernels run one point per warp; osc_set_tile does not apply to them.
 * The serving loop runs a batch that holds a layered sample with the layered
 * kernels.  This call returns OSC_E_STATE while serving runs (in-flight batches
 * hold the sample's path).  Arrays are host memory; the call copies them and
 * drops cached launch plans. */
osc_status osc_set_layers(osc_ctx *ctx, int32_t sample_id, int32_t n_layers, const double *length_km,
                          const double *density_gcc, const double *ye);

/* Launch-shape control.  points_per_block in {1, 4, 16, 64, 256}, or 0 to let
 * the autotuner choose per workload class (default); events_per_item a positive
 * multiple of 64, or 0 for the default.  events_per_item also sets the work-item
 * size of osc_histogram_bin_centre; the layered kernels always run one point
 * per warp.  Results never depend on either. */
osc_status osc_set_tile(osc_ctx *ctx, int32_t points_per_block, int32_t events_per_item);

/* Enable (1) / disable (0) CUDA-event timing of each kernel.  Events are
 * recorded on the context stream around every constants, histogram and
 * finalize kernel without any host synchronisation (the histogram step runs as
 * the same CUDA graph, with event-record nodes around its kernels).  osc_last_timing waits for the recorded events and reports the
 * durations (ms) of the most recent kernel of each kind (negative when none);
 * osc_timing_totals waits, returns the launch counts and summed durations of
 * each kind since the last totals call (index 0 constants, 1 histogram,
 * 2 finalize), and resets them. */
osc_status osc_enable_timing(osc_ctx *ctx, int enable);
osc_status osc_last_timing(osc_ctx *ctx, double *k_const_ms, double *k_hist_ms,
                           double *k_final_ms);
osc_status osc_timing_totals(osc_ctx *ctx, int64_t counts[3], double sums_ms[3]);

/* Number of kernels this context has launched so far (graph replays count
 * each kernel node). */
osc_status osc_launch_count(const osc_ctx *ctx, uint64_t *count);

/* Device memory the context holds (samples, point table, plans, accumulators
 * and other buffers), in bytes; the workspace cap applies to this total. */
osc_status osc_workspace_used(const osc_ctx *ctx, size_t *bytes);

/* Block until all work enqueued by the context has finished. */
osc_status osc_sync(osc_ctx *ctx);

/* Continuous-batching serving loop (each request is one MCMC step's reweight,
 * Sec. 2.2).  A scheduler thread inside the library admits queued (sample,
 * point) requests into at most max_slots in-flight slots under the workspace cap
 * and packs them into batches of persistent launches, up to three batches in
 * flight on streams of their own; each request yields one nbins histogram over
 * [lo, hi).  The scheduler learns of a finished batch by polling a flag the
 * batch's last kernel raises in host-mapped memory: while batches are in flight,
 * and for 200 us after the last one, it keeps one host core busy; otherwise it
 * sleeps until a request is submitted. */
osc_status osc_serve_start(osc_ctx *ctx, int32_t max_slots, double lo, double hi, int32_t nbins);
osc_status osc_submit(osc_ctx *ctx, int32_t sample_id, const osc_point *pt, osc_precision prec,
                      uint64_t *ticket);
/* osc_submit validates the point and sample on the calling thread and queues
 * the request (OSC_E_BUSY beyond 2^20 queued requests); the ticket is > 0.
 * osc_wait waits for a ticket's histogram (host buffer of nbins doubles) and
 * releases it; latency_us (may be NULL) receives the submit-to-completion time.
 * timeout_ms < 0 waits forever; OSC_E_TIMEOUT when the time runs out; OSC_E_ARG
 * for a ticket never issued.  osc_serve_stop drops queued requests, lets the
 * in-flight batches finish, and frees the serving buffers. */
osc_status osc_wait(osc_ctx *ctx, uint64_t ticket, double *out_hist, int32_t timeout_ms,
                    double *latency_us);
osc_status osc_serve_stop(osc_ctx *ctx);

/* The FP32 FMA throughput of CUDA device `device` in TFLOP/s (an FMA counts as
 * two flops): the peak against which the FP32 path's roofline is reported (the
 * paper has no counterpart; the vendor's figure assumes the maximum clock).
 * Independent FMA chains run on every SM for about 30 ms in all, timed with CUDA
 * events; the best of five launches is returned.  No clock or power setting is
 * changed.  It allocates a small result buffer of its own, needs no context, and
 * leaves the calling thread's current device as it was.  OSC_E_ARG for a null
 * tflops or an invalid device, OSC_E_CUDA if a CUDA call fails. */
osc_status osc_measure_fp32_peak(int device, double *tflops);

/* One-point histogram that allocates nothing (the paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- for example a host
 * framework that has reserved all device memory for its own allocator, or a
 * fit loop in which an allocation, which may synchronise the device or fail
 * under fragmentation, is not allowed in the middle of a step).
 *
 * Computes the same histogram as osc_histogram for one sample and one point,
 * without a context: d_e_true, d_e_reco, d_w_mc (float) and d_flav_in,
 * d_flav_out, d_is_nubar (uint8) are caller-owned DEVICE arrays of n events in
 * any order (sorted by channel and E_reco is fastest; the bin sums are exact
 * and do not depend on the order); baseline_km, density_gcc, ye as in
 * osc_sample_desc; w_abs_max > 0 bounds |w_mc| and sets the fixed-point scale
 * (F = 62 - ceil(log2 w_abs_max), as osc_load_sample derives it from the
 * sample); *pt is a host point; d_out is a caller-owned DEVICE array of nbins
 * doubles.  Work runs on cuda_stream (NULL = legacy default stream) on the
 * current device, and the call returns after it has finished.
 *
 * Its working memory is one fixed file-scope device array of about 130 KB
 * (point constants, 4 x 4096 accumulator words, a counter and an error flag),
 * held by every GPU that loads this library until the process exits; nbins is
 * therefore limited to 4096, and larger values are rejected with OSC_E_ARG.
 * The accumulators hold 32-bit digit columns, so their bin sums stay exact for
 * any event order up to n = 2^31 - 1.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  The first call on each device resolves the
 * array's device address (cudaGetSymbolAddress), so make that first call before
 * any stream capture.  Every call shares the array: the call clears what must
 * start at zero, and calls that overlap on the GPU (other threads, other
 * streams) race and must not be issued.
 *
 * prec is OSC_FP64, OSC_FP32_BULK or OSC_FP32_F64EIG, with the precision rules
 * above: FP32 events whose error estimate exceeds the tolerance are recomputed
 * in FP64; an OSC_FP32_BULK call whose matter phase exceeds 3 rad runs as
 * OSC_FP32_F64EIG; and since the host does not see the events, the kernel
 * flags any event outside its precision's matter-term limit (10 |dm31| for
 * FP32 bulk, 1000 |dm31| for F64EIG) and the call then runs again in the next
 * precision (FP32 bulk -> FP32_F64EIG -> FP64).
 *
 * Errors: OSC_E_ARG (null pointer, bad precision, n outside [1, 2^31 - 1],
 * nbins outside [1, 4096]), OSC_E_RANGE (invalid scalars or point; or, found
 * on the device, an event with E_true <= 0 or non-finite, non-finite E_reco,
 * |w_mc| > w_abs_max, or a bad flavour -- d_out is then left unwritten),
 * OSC_E_CUDA.  A message goes to err (err_len bytes, may be NULL). */
osc_status osc_histogram_noalloc(const float *d_e_true, const float *d_e_reco, const float *d_w_mc,
                                 const uint8_t *d_flav_in, const uint8_t *d_flav_out,
                                 const uint8_t *d_is_nubar, int64_t n, double baseline_km,
                                 double density_gcc, double ye, double w_abs_max,
                                 const osc_point *pt, osc_precision prec, double lo, double hi,
                                 int32_t nbins, double *d_out, void *cuda_stream, char *err,
                                 size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* OSC_GB300_H */
