// osc_runtime.cu -- host runtime behind the C ABI declared in include/osc.h.
//
// Follows the paper's host pattern (Sec. 2.1 listing: allocate device arrays,
// copy energies, copy the parameter-only components, launch, copy results back)
// with three GB300-first changes: samples are validated, sorted by
// (channel, E_reco) and kept resident; the parameter-only constants are built
// on the device in FP64 for a whole table of points; and one persistent launch
// covers every (sample, point tile, event range) work item of a call.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <numeric>
#include <sstream>

#include "osc_ctx.h"

using namespace osc;

namespace osc {

double matter_k_A() {
    const double G_F = 1.1663788e-23;        // eV^-2
    const double N_A = 6.02214076e23;        // per gram-mole
    const double hbarc_cm = 1.973269804e-5;  // eV cm
    return 2.0 * std::sqrt(2.0) * G_F * N_A * hbarc_cm * hbarc_cm * hbarc_cm * 1e9;
}

osc_status fail(osc_ctx *c, osc_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

osc_status fail_cuda(osc_ctx *c, cudaError_t e, const char *what) {
    std::ostringstream o;
    o << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // not sticky
        return fail(c, OSC_E_NOMEM, o.str());
    }
    c->poisoned = true;
    return fail(c, OSC_E_CUDA, o.str());
}

osc_status dalloc(osc_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->cap && c->used + bytes > c->cap) {
        std::ostringstream o;
        o << "workspace cap exceeded: " << c->used << " + " << bytes << " > " << c->cap << " bytes";
        return fail(c, OSC_E_NOMEM, o.str());
    }
    if (++c->n_allocs == c->fault_alloc_at)
        return fail(c, OSC_E_NOMEM, "injected allocation failure (OSC_FAULT_ALLOC_FAIL_AT)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail_cuda(c, e, "cudaMalloc");
    }
    c->used += bytes;
    c->sizes[*p] = bytes;
    return OSC_OK;
}

void dfree(osc_ctx *c, void *p) {
    if (!p) return;
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->used -= it->second;
        c->sizes.erase(it);
    }
    cudaFree(p);
}

static bool is_fin(double x) { return std::isfinite(x); }

// Debug builds: report (and poison the context on) a kernel's index check that
// failed, once the work has finished.  Release builds do nothing here.
osc_status debug_word_check(osc_ctx *c) {
#ifdef OSC_DEBUG_CHECKS
    unsigned w = 0;
    const cudaError_t e = cudaMemcpy(&w, c->d_counter + kDebugWord, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(c, e, "cudaMemcpy(debug word)");
    if (w) {
        c->poisoned = true;
        std::ostringstream o;
        o << "device index check failed (debug build), code " << w;
        return fail(c, OSC_E_CUDA, o.str());
    }
#else
    (void)c;
#endif
    return OSC_OK;
}

int prec_kind(osc_precision p) { return p == OSC_FP32_BULK ? kFP32 : p == OSC_FP32_F64EIG ? kMix : kFP64; }

// Precisions ordered from the fastest to the most precise.
static int prec_rank(int k) { return k == kFP32 ? 0 : k == kMix ? 1 : 2; }

int pair_prec(const osc_point &p, const Sample *s, int prec) {
    if (prec == kFP64) return kFP64;
    const double dm31 = std::fabs(p.dm32 + p.dm21);
    const double a_max = s->ka_max * (double)s->e_max;
    if (!(a_max <= kFp32MatterRatio * dm31)) return kFP64;
    if (prec == kFP32 && s->dev.n_layers > 1 &&
        !(p.dm21 >= kFp32LayerSolarRatio * dm31 && a_max <= kFp32LayerMatterRatio * dm31))
        return kFP64;
    if (prec == kFP32 && !(s->matter_phase <= kFp32BulkMatterPhase && a_max <= kFp32BulkMatterRatio * dm31))
        return kMix;
    return prec;
}

int call_prec(osc_ctx *c, osc_precision prec, const int32_t *ids, int32_t n_ids, int32_t point_begin,
              int32_t n_points) {
    int pr = prec_kind(prec);
    for (int32_t i = 0; i < n_ids && pr != kFP64; ++i) {
        const Sample *s = c->samples[ids[i]];
        for (int32_t k = point_begin; k < point_begin + n_points; ++k) {
            const int q = pair_prec(c->pts[k], s, pr);
            if (prec_rank(q) > prec_rank(pr)) pr = q;
            if (pr == kFP64) break;
        }
    }
    return pr;
}

osc_status validate_point(osc_ctx *c, const osc_point &p, int i) {
    // the message is formatted only for a rejected point (this runs once per point per call)
    const char *why = nullptr;
    if (!(is_fin(p.s2_12) && is_fin(p.s2_13) && is_fin(p.s2_23) && is_fin(p.dm21) && is_fin(p.dm32) &&
          is_fin(p.dcp) && is_fin(p.escale) && is_fin(p.norm)))
        why = "non-finite field";
    // |U_e1|^2, |U_e2|^2, |U_e3|^2 > 0: no exact level crossing along the matter term
    else if (!(p.s2_12 > 0.0 && p.s2_12 < 1.0)) why = "sin^2 theta12 must be in (0, 1)";
    else if (!(p.s2_13 > 0.0 && p.s2_13 < 1.0)) why = "sin^2 theta13 must be in (0, 1)";
    else if (!(p.s2_23 >= 0.0 && p.s2_23 <= 1.0)) why = "sin^2 theta23 must be in [0, 1]";
    else if (!(p.dm21 > 0.0)) why = "dm21 must be > 0";
    else if (!(std::fabs(p.dm32) > p.dm21)) why = "|dm32| must exceed dm21";
    // the device reduces delta by pi/2 exactly only for |delta| below about 1.6e6
    else if (!(std::fabs(p.dcp) <= 1e6)) why = "|delta_CP| must be <= 1e6 rad";
    else if (!(p.escale > 0.0)) why = "escale must be > 0";
    if (!why) return OSC_OK;
    return fail(c, OSC_E_RANGE, "point " + std::to_string(i) + ": " + why);
}

osc_status ensure_acc(osc_ctx *c, int64_t bins) {
    if (bins <= c->acc_cap_bins) return OSC_OK;
    int64_t want = std::max<int64_t>(bins, 1024);
    void *p;
    osc_status s = dalloc(c, &p, (size_t)want * kDigits * sizeof(unsigned long long));
    if (s) return s;
    cudaError_t e = cudaMemsetAsync(p, 0, (size_t)want * kDigits * sizeof(unsigned long long), c->stream);
    if (e) return fail_cuda(c, e, "cudaMemsetAsync(acc)");
    if (c->d_acc) {
        cudaStreamSynchronize(c->stream);
        dfree(c, c->d_acc);
    }
    c->d_acc = (unsigned long long *)p;
    c->acc_cap_bins = want;
    return OSC_OK;
}

static osc_status ensure_buf(osc_ctx *c, double **buf, int64_t *cap, int64_t n) {
    if (n <= *cap) return OSC_OK;
    void *p;
    osc_status s = dalloc(c, &p, (size_t)n * sizeof(double));
    if (s) return s;
    if (*buf) {
        cudaStreamSynchronize(c->stream);
        dfree(c, *buf);
    }
    *buf = (double *)p;
    *cap = n;
    return OSC_OK;
}

int hist_grid(osc_ctx *c, const void *kernel, int32_t n_items, int threads) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    int g = c->n_sm * per_sm;
    return std::max(1, std::min(g, n_items));
}

// Size of the next one-point work item by guided self-scheduling: full chunks
// while the work left is large, then remaining / (2 x slots) events (a multiple
// of 64, at least 256), so the grid ends on short items while most of the work
// keeps the lower per-item overhead of full chunks.
static int32_t guided_size(int64_t remaining, int32_t chunk, int64_t slots) {
    const int64_t g = remaining / (2 * slots) / 64 * 64;
    return (int32_t)std::max<int64_t>(std::min<int64_t>(chunk, 256), std::min<int64_t>(chunk, g));
}

void build_items(const std::vector<const Sample *> &ss, int32_t point_base, int32_t n_points, int32_t pt,
                 int32_t chunk, int64_t slots, int64_t acc_hist_base, std::vector<WorkItem> &items) {
    const int32_t n_tiles = (n_points + pt - 1) / pt;
    int64_t remaining = 0;
    for (const Sample *s : ss) remaining += s->n * n_tiles;
    for (size_t s = 0; s < ss.size(); ++s)
        for (int32_t t = 0; t < n_tiles; ++t) {
            const int64_t n = ss[s]->n;
            for (int64_t e = 0; e < n;) {
                const int32_t c = (pt == 1 && slots > 0) ? guided_size(remaining, chunk, slots) : chunk;
                WorkItem w;
                w.sample = (int32_t)s;
                w.point_base = point_base + t * pt;
                w.n_pts = std::min(pt, n_points - t * pt);
                w.ev_count = (int32_t)std::min<int64_t>(c, n - e);
                w.ev_begin = e;
                w.acc_base = acc_hist_base + (int64_t)s * n_points + (int64_t)t * pt;
                items.push_back(w);
                e += w.ev_count;
                remaining -= w.ev_count;
            }
        }
    // largest first for the dynamic scheduler
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &a, const WorkItem &b) {
        return (int64_t)a.ev_count * a.n_pts > (int64_t)b.ev_count * b.n_pts;
    });
}

static void fill_hist_params(HistParams &hp, const WorkItem *d_items, int32_t n_items, const SampleDev *d_samples,
                             const float *pc32, const double *pc64, unsigned long long *acc, int32_t *counter,
                             int32_t nbins, double lo, double hi) {
    hp.items = d_items;
    hp.n_items = n_items;
    hp.nbins = nbins;
    hp.samples = d_samples;
    hp.pc32 = pc32;
    hp.pc64 = pc64;
    hp.acc = acc;
    hp.counter = counter;
    hp.lo_f = (float)lo;
    hp.inv_f = (float)((double)nbins / (hi - lo));
    hp.nb_f = (float)nbins;
    hp.redo = nullptr;
    hp.fuse_final = 0;
    hp.fin_n_hist = 0;
    hp.fin_hmeta = nullptr;
    hp.fin_out = nullptr;
}

// Device address of a page-locked host buffer, which the kernels then write
// directly (no staging buffer and copy); null for pageable memory.
static double *pinned_device_ptr(double *host) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? (double *)a.devicePointer : nullptr;
}

// Outputs of one conversion round are converted by the histogram kernel's last
// warp (one-point items: 128 bins) or block (point tiles: 256 bins); larger ones
// by the finalize kernel, whose blocks convert in parallel.
bool fuse_finalize(int64_t n_hist, int32_t nbins, int32_t pt) {
    return n_hist * (int64_t)nbins <= (pt == 1 ? 128 : 256);
}

cudaEvent_t pool_event(osc_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Resolve every pending timed launch (synchronises on the last one).
osc_status drain_timing(osc_ctx *c) {
    if (c->ev_pending.empty()) return OSC_OK;
    cudaError_t e = cudaEventSynchronize(c->ev_pending.back().second.second);
    if (e) return fail_cuda(c, e, "cudaEventSynchronize(timing)");
    for (auto &p : c->ev_pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.second.first, p.second.second);
        c->t_count[p.first] += 1;
        c->t_sum[p.first] += ms;
        if (p.first == 0) c->t_const = ms;
        if (p.first == 1) c->t_hist = ms;
        if (p.first == 2) c->t_final = ms;
        c->ev_pool.push_back(p.second.first);
        c->ev_pool.push_back(p.second.second);
    }
    c->ev_pending.clear();
    return OSC_OK;
}

}  // namespace osc

// ------------------------------------------------------------------ helpers
#define CHECK_CTX(c)                                                                 \
    do {                                                                             \
        if (!(c)) return OSC_E_ARG;                                                  \
        if ((c)->poisoned) return fail((c), OSC_E_STATE, "context poisoned by an earlier CUDA error: " + (c)->err); \
    } while (0)

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #call); \
    } while (0)

static uint32_t float_key(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Stable LSD radix sort of event indices by (channel, E_reco): 37-bit keys, 3 x 13-bit passes.
static void sort_events(int64_t n, const uint8_t *ch, const float *er, std::vector<int32_t> &order) {
    std::vector<uint64_t> key((size_t)n);
    for (int64_t i = 0; i < n; ++i) key[i] = ((uint64_t)ch[i] << 32) | float_key(er[i]);
    std::vector<int32_t> a((size_t)n), b((size_t)n);
    std::iota(a.begin(), a.end(), 0);
    std::vector<int64_t> cnt(1 << 13);
    for (int pass = 0; pass < 3; ++pass) {
        const int sh = 13 * pass;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t i = 0; i < n; ++i) cnt[(key[a[i]] >> sh) & 0x1FFF]++;
        int64_t s = 0;
        for (auto &x : cnt) {
            int64_t t = x;
            x = s;
            s += t;
        }
        for (int64_t i = 0; i < n; ++i) b[cnt[(key[a[i]] >> sh) & 0x1FFF]++] = a[i];
        a.swap(b);
    }
    order.swap(a);
}

// Single-layer path constants of a sample: matter term and phase scale.
static void set_path_consts(SampleDev &sd, double L, double rho, double ye) {
    sd.kA_rhoye = matter_k_A() * rho * ye;
    sd.cLL = kCL * L;
    sd.kA_rhoye_f = (float)sd.kA_rhoye;
    const double rev = kCL * L / kTwoPi;
    sd.rev_hi = (float)rev;
    sd.rev_lo = (float)(rev - (double)sd.rev_hi);
}

static void free_sample(osc_ctx *c, Sample *s) {
    dfree(c, s->ev);
    dfree(c, s->perm);
    dfree(c, s->lay);
    delete s;
}

static void free_plan(osc_ctx *c, Plan *p) {
    if (p->exec_t) cudaGraphExecDestroy(p->exec_t);
    if (p->graph_t) cudaGraphDestroy(p->graph_t);
    if (p->step_exec) cudaGraphExecDestroy(p->step_exec);
    if (p->step_graph) cudaGraphDestroy(p->step_graph);
    dfree(c, p->d_items);
    dfree(c, p->d_samples);
    dfree(c, p->d_hmeta);
    dfree(c, p->d_redo);
    dfree(c, p->d_rows);
    dfree(c, p->d_rowmap);
    dfree(c, p->d_tab);
    delete p;
}

static void drop_plans(osc_ctx *c) {
    if (c->plans.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (Plan *p : c->plans) free_plan(c, p);
    c->plans.clear();
}

// Persisted autotuner results: one line per workload class,
// "<device>/<SMs> <class> <points_per_block> <events_per_item>".  Lines of other
// devices are ignored; unreadable files are treated as empty.
static void load_tuned(osc_ctx *c) {
    if (c->tune_file.empty()) return;
    std::ifstream in(c->tune_file);
    std::string dev, key;
    int32_t pt, chunk;
    while (in >> dev >> key >> pt >> chunk)
        if (dev == c->device_name && (pt == 1 || pt == 4 || pt == 16 || pt == 64 || pt == 256) && chunk > 0 &&
            chunk % 64 == 0)
            c->tuned[key] = {pt, chunk};
}

static void save_tuned(osc_ctx *c, const std::string &key, int32_t pt, int32_t chunk) {
    if (c->tune_file.empty()) return;
    std::ofstream out(c->tune_file, std::ios::app);
    if (out) out << c->device_name << " " << key << " " << pt << " " << chunk << "\n";
}

// ------------------------------------------------------------------ the ABI
extern "C" {

const char *osc_version(void) { return "paper_1311_7579_gb300 0.1 (sm_103a)"; }

const char *osc_last_error(const osc_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

osc_status osc_create(int device, size_t workspace_cap_bytes, void *cuda_stream, osc_ctx **out) {
    if (!out) return OSC_E_ARG;
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || n_dev == 0) {
        cudaGetLastError();
        return OSC_E_CUDA;
    }
    if (device < 0 || device >= n_dev) return OSC_E_ARG;
    osc_ctx *ctx = new osc_ctx();
    ctx->device = device;
    ctx->cap = workspace_cap_bytes;
    if (const char *f = std::getenv("OSC_FAULT_ALLOC_FAIL_AT")) ctx->fault_alloc_at = std::atoll(f);
    if (const char *f = std::getenv("OSC_AUTOTUNE_CACHE")) ctx->tune_file = f;
    e = cudaSetDevice(device);
    if (e) {
        delete ctx;
        return OSC_E_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
    {
        cudaDeviceProp prop{};
        if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) ctx->device_name = prop.name;
        for (char &ch : ctx->device_name)
            if (ch == ' ') ch = '_';
        std::ostringstream o;
        o << ctx->device_name << "/" << ctx->n_sm;
        ctx->device_name = o.str();
    }
    load_tuned(ctx);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e) {
            delete ctx;
            return OSC_E_CUDA;
        }
        ctx->own_stream = true;
    }
    void *p;
    if (dalloc(ctx, &p, 64) != OSC_OK) {
        osc_destroy(ctx);
        return OSC_E_NOMEM;
    }
    ctx->d_counter = (int32_t *)p;
    if (cudaMemsetAsync(p, 0, 64, ctx->stream) || cudaStreamSynchronize(ctx->stream)) {
        osc_destroy(ctx);
        return OSC_E_CUDA;
    }
    *out = ctx;
    return OSC_OK;
}

osc_status osc_serve_stop(osc_ctx *ctx);

void osc_destroy(osc_ctx *ctx) {
    if (!ctx) return;
    if (ctx->serve) osc_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_plans(ctx);
    for (auto &kv : ctx->samples) free_sample(ctx, kv.second);
    ctx->samples.clear();
    dfree(ctx, ctx->d_pts);
    dfree(ctx, ctx->d_pc32);
    dfree(ctx, ctx->d_pc64);
    dfree(ctx, ctx->d_acc);
    dfree(ctx, ctx->d_counter);
    dfree(ctx, ctx->d_out);
    dfree(ctx, ctx->d_rw);
    dfree(ctx, ctx->d_aux);
    for (auto &p : ctx->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

osc_status osc_load_sample(osc_ctx *ctx, const osc_sample_desc *d, int32_t *sample_id) {
    NvtxRange nvtx_range("osc_load_sample");
    CHECK_CTX(ctx);
    if (!d || !sample_id) return fail(ctx, OSC_E_ARG, "null argument");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (d->n < 1 || d->n > (int64_t)INT32_MAX - 8) return fail(ctx, OSC_E_ARG, "n must be in [1, 2^31 - 9]");
    if (!d->e_true || !d->e_reco || !d->w_mc || !d->flav_in || !d->flav_out || !d->is_nubar)
        return fail(ctx, OSC_E_ARG, "null event array");
    if (!(is_fin(d->baseline_km) && d->baseline_km > 0)) return fail(ctx, OSC_E_RANGE, "baseline must be finite and > 0");
    if (!(is_fin(d->density_gcc) && d->density_gcc >= 0)) return fail(ctx, OSC_E_RANGE, "density must be finite and >= 0");
    if (!(d->ye >= 0 && d->ye <= 1)) return fail(ctx, OSC_E_RANGE, "Y_e must be in [0, 1]");
    const int64_t n = d->n;
    double wsum = 0.0, wmax = 0.0;
    uint32_t mask = 0;
    std::vector<uint8_t> ch((size_t)n);
    float e_max = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        const float e = d->e_true[i], r = d->e_reco[i], w = d->w_mc[i];
        e_max = std::max(e_max, e);
        if (!(std::isfinite(e) && e > 0.0f)) {
            std::ostringstream o;
            o << "event " << i << ": E_true must be finite and > 0";
            return fail(ctx, OSC_E_RANGE, o.str());
        }
        if (!std::isfinite(r) || !std::isfinite(w)) {
            std::ostringstream o;
            o << "event " << i << ": non-finite E_reco or w_mc";
            return fail(ctx, OSC_E_RANGE, o.str());
        }
        if (d->flav_in[i] > 2 || d->flav_out[i] > 2 || d->is_nubar[i] > 1) {
            std::ostringstream o;
            o << "event " << i << ": flavour must be 0..2 and is_nubar 0/1";
            return fail(ctx, OSC_E_RANGE, o.str());
        }
        ch[i] = (uint8_t)chan_id(d->flav_in[i], d->flav_out[i], d->is_nubar[i]);
        mask |= 1u << ch[i];
        wsum += std::fabs((double)w);
        wmax = std::max(wmax, std::fabs((double)w));
    }
    if (!(wsum < std::ldexp(1.0, 60))) return fail(ctx, OSC_E_RANGE, "sum of |w_mc| must be < 2^60");
    // Fixed-point fraction bits F: every event weight |P w_mc| <= 1.0001 max|w_mc|
    // becomes one 64-bit addend below 2^63, and bin sums stay far below 2^127.
    int F = 62;
    if (wmax > 0) F = 62 - (int)std::ceil(std::log2(wmax));
    F = std::max(8, std::min(F, 190));

    std::vector<int32_t> order;
    sort_events(n, ch.data(), d->e_reco, order);
    const int64_t n_pad = (n + 3) / 4 * 4 + 4;
    std::vector<float4> rec((size_t)n_pad, make_float4(1.0f, 0.0f, 0.0f, 0.0f));
    for (int64_t k = 0; k < n; ++k) {
        const int32_t i = order[k];
        int32_t cbits = ch[i];
        float cf;
        std::memcpy(&cf, &cbits, 4);
        rec[k] = make_float4(d->e_true[i], d->e_reco[i], d->w_mc[i], cf);
    }
    Sample *s = new Sample();
    s->n = n;
    s->n_pad = n_pad;
    s->L = d->baseline_km;
    s->rho = d->density_gcc;
    s->ye = d->ye;
    s->frac_bits = F;
    s->chan_mask = mask;
    s->e_max = e_max;
    s->w_abs = wmax;
    s->ka_max = matter_k_A() * d->density_gcc * d->ye;
    s->matter_phase = kCL * d->baseline_km * s->ka_max;
    osc_status st = OSC_OK;
    void *p;
    if ((st = dalloc(ctx, &p, n_pad * sizeof(float4))) == OSC_OK) s->ev = (float4 *)p;
    if (!st && (st = dalloc(ctx, &p, n * 4)) == OSC_OK) s->perm = (int32_t *)p;
    if (st) {
        free_sample(ctx, s);
        return st;
    }
    cudaError_t e = cudaMemcpy(s->ev, rec.data(), n_pad * sizeof(float4), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(s->perm, order.data(), n * 4, cudaMemcpyHostToDevice);
    if (e) {
        free_sample(ctx, s);
        return fail_cuda(ctx, e, "cudaMemcpy(sample)");
    }
    SampleDev &sd = s->dev;
    sd.ev = s->ev;
    sd.perm = s->perm;
    sd.n = n;
    set_path_consts(sd, s->L, s->rho, s->ye);
    sd.hscale_d = std::ldexp(1.0, F - 64);
    sd.hscale_f = (float)sd.hscale_d;
    sd.frac_bits = F;
    sd.n_layers = 1;
    sd.lay32 = nullptr;
    sd.lay64 = nullptr;
    s->id = ctx->next_id++;
    ctx->samples[s->id] = s;
    *sample_id = s->id;
    return OSC_OK;
}

osc_status osc_unload_sample(osc_ctx *ctx, int32_t sample_id) {
    CHECK_CTX(ctx);
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    auto it = ctx->samples.find(sample_id);
    if (it == ctx->samples.end()) return fail(ctx, OSC_E_ARG, "unknown sample id");
    if (ctx->serve) return fail(ctx, OSC_E_STATE, "cannot unload a sample while serving runs");
    drop_plans(ctx);  // plans reference the sample's device arrays
    cudaStreamSynchronize(ctx->stream);
    free_sample(ctx, it->second);
    ctx->samples.erase(it);
    return OSC_OK;
}

osc_status osc_set_layers(osc_ctx *ctx, int32_t sample_id, int32_t n_layers, const double *length_km,
                          const double *density_gcc, const double *ye) {
    NvtxRange nvtx_range("osc_set_layers");
    CHECK_CTX(ctx);
    if (!length_km || !density_gcc || !ye) return fail(ctx, OSC_E_ARG, "null argument");
    if (n_layers < 1 || n_layers > kMaxLayers) return fail(ctx, OSC_E_ARG, "n_layers must be in [1, 16]");
    double total = 0.0;
    for (int k = 0; k < n_layers; ++k) {
        if (!(is_fin(length_km[k]) && length_km[k] > 0)) return fail(ctx, OSC_E_RANGE, "layer length must be finite and > 0");
        if (!(is_fin(density_gcc[k]) && density_gcc[k] >= 0)) return fail(ctx, OSC_E_RANGE, "layer density must be finite and >= 0");
        if (!(ye[k] >= 0 && ye[k] <= 1)) return fail(ctx, OSC_E_RANGE, "layer Y_e must be in [0, 1]");
        total += length_km[k];
    }
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    auto it = ctx->samples.find(sample_id);
    if (it == ctx->samples.end()) return fail(ctx, OSC_E_ARG, "unknown sample id");
    if (ctx->serve) return fail(ctx, OSC_E_STATE, "cannot change a sample's path while serving runs");
    Sample *s = it->second;
    void *lay = nullptr;
    double ka_max = 0.0, matter_phase = 0.0;
    for (int k = 0; k < n_layers; ++k) {
        ka_max = std::max(ka_max, matter_k_A() * density_gcc[k] * ye[k]);
        matter_phase += kCL * length_km[k] * matter_k_A() * density_gcc[k] * ye[k];
    }
    if (n_layers > 1) {
        std::vector<float4> l32(n_layers);
        std::vector<double2> l64(n_layers);
        for (int k = 0; k < n_layers; ++k) {
            const double kA = matter_k_A() * density_gcc[k] * ye[k];
            const double rev = kCL * length_km[k] / kTwoPi;
            const float rh = (float)rev;
            l32[k] = make_float4((float)kA, rh, (float)(rev - (double)rh), 0.0f);
            l64[k] = make_double2(kA, kCL * length_km[k]);
        }
        const size_t b32 = n_layers * sizeof(float4);
        osc_status st = dalloc(ctx, &lay, b32 + n_layers * sizeof(double2));
        if (st) return st;
        cudaError_t e = cudaMemcpy(lay, l32.data(), b32, cudaMemcpyHostToDevice);
        if (!e) e = cudaMemcpy((char *)lay + b32, l64.data(), n_layers * sizeof(double2), cudaMemcpyHostToDevice);
        if (e) {
            dfree(ctx, lay);
            return fail_cuda(ctx, e, "cudaMemcpy(layers)");
        }
    }
    drop_plans(ctx);  // plans hold copies of the sample's path constants
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, s->lay);
    s->lay = lay;
    s->ka_max = ka_max;
    s->matter_phase = matter_phase;
    SampleDev &sd = s->dev;
    if (n_layers == 1) {
        s->L = length_km[0];
        s->rho = density_gcc[0];
        s->ye = ye[0];
        set_path_consts(sd, s->L, s->rho, s->ye);
        sd.n_layers = 1;
        sd.lay32 = nullptr;
        sd.lay64 = nullptr;
    } else {
        s->L = total;
        sd.n_layers = n_layers;
        sd.lay32 = (const float4 *)lay;
        sd.lay64 = (const double2 *)((char *)lay + n_layers * sizeof(float4));
    }
    return OSC_OK;
}

// Device room for a point table of n points and its FP32 / FP64 constants.
static osc_status ensure_point_table(osc_ctx *ctx, int32_t n_points) {
    if (n_points <= ctx->pts_cap) return OSC_OK;
    int32_t cap = 1;
    while (cap < n_points) cap <<= 1;
    void *a, *b, *c;
    osc_status s = dalloc(ctx, &a, (size_t)cap * sizeof(osc_point));
    if (s) return s;
    if ((s = dalloc(ctx, &b, (size_t)cap * C32_STRIDE * 4))) {
        dfree(ctx, a);
        return s;
    }
    if ((s = dalloc(ctx, &c, (size_t)cap * C64_STRIDE * 8))) {
        dfree(ctx, a);
        dfree(ctx, b);
        return s;
    }
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, ctx->d_pts);
    dfree(ctx, ctx->d_pc32);
    dfree(ctx, ctx->d_pc64);
    ctx->d_pts = (osc_point *)a;
    ctx->d_pc32 = (float *)b;
    ctx->d_pc64 = (double *)c;
    ctx->pts_cap = cap;
    return OSC_OK;
}

osc_status osc_set_params(osc_ctx *ctx, const osc_point *pts, int32_t n_points) {
    NvtxRange nvtx_range("osc_set_params");
    CHECK_CTX(ctx);
    if (!pts) return fail(ctx, OSC_E_ARG, "null point table");
    if (n_points < 1 || n_points > (1 << 20)) return fail(ctx, OSC_E_ARG, "n_points must be in [1, 2^20]");
    for (int32_t i = 0; i < n_points; ++i) {
        osc_status s = validate_point(ctx, pts[i], i);
        if (s) return s;
    }
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    osc_status s = ensure_point_table(ctx, n_points);
    if (s) return s;
    ctx->pts.assign(pts, pts + n_points);
    // small tables travel as kernel parameters; larger ones through a copy
    const bool by_value = n_points <= kPointsByValue;
    if (!by_value)
        CK(cudaMemcpyAsync(ctx->d_pts, ctx->pts.data(), (size_t)n_points * sizeof(osc_point), cudaMemcpyHostToDevice,
                           ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->timing) {
        e0 = pool_event(ctx);
        e1 = pool_event(ctx);
        CK(cudaEventRecord(e0, ctx->stream));
    }
    if (by_value)
        CK(launch_point_consts_host(ctx->pts.data(), n_points, ctx->d_pc32, ctx->d_pc64, ctx->stream));
    else
        CK(launch_point_consts(ctx->d_pts, n_points, ctx->d_pc32, ctx->d_pc64, ctx->stream));
    ctx->launches += 1;
    if (ctx->timing) {
        CK(cudaEventRecord(e1, ctx->stream));
        ctx->ev_pending.push_back({0, {e0, e1}});
    }
    // The copy source is the context's own host table, and a pageable-source
    // cudaMemcpyAsync has consumed it before returning: no host synchronisation.
    return OSC_OK;
}

osc_status osc_set_tile(osc_ctx *ctx, int32_t points_per_block, int32_t events_per_item) {
    CHECK_CTX(ctx);
    if (points_per_block != 0 && points_per_block != 1 && points_per_block != 4 && points_per_block != 16 &&
        points_per_block != 64 && points_per_block != 256)
        return fail(ctx, OSC_E_ARG, "points_per_block must be 0, 1, 4, 16, 64 or 256");
    if (events_per_item < 0 || (events_per_item % 64) != 0)
        return fail(ctx, OSC_E_ARG, "events_per_item must be 0 or a positive multiple of 64");
    ctx->tile_pt = points_per_block;
    ctx->tile_chunk = events_per_item;
    return OSC_OK;
}

osc_status osc_enable_timing(osc_ctx *ctx, int enable) {
    CHECK_CTX(ctx);
    if (!enable) {
        osc_status st = drain_timing(ctx);
        if (st) return st;
    }
    ctx->timing = enable != 0;
    return OSC_OK;
}

osc_status osc_last_timing(osc_ctx *ctx, double *k_const_ms, double *k_hist_ms, double *k_final_ms) {
    if (!ctx) return OSC_E_ARG;
    osc_status st = drain_timing(ctx);
    if (st) return st;
    if (k_const_ms) *k_const_ms = ctx->t_const;
    if (k_hist_ms) *k_hist_ms = ctx->t_hist;
    if (k_final_ms) *k_final_ms = ctx->t_final;
    return OSC_OK;
}

osc_status osc_timing_totals(osc_ctx *ctx, int64_t counts[3], double sums_ms[3]) {
    if (!ctx || !counts || !sums_ms) return OSC_E_ARG;
    osc_status st = drain_timing(ctx);
    if (st) return st;
    for (int k = 0; k < 3; ++k) {
        counts[k] = ctx->t_count[k];
        sums_ms[k] = ctx->t_sum[k];
        ctx->t_count[k] = 0;
        ctx->t_sum[k] = 0;
    }
    return OSC_OK;
}

osc_status osc_workspace_used(const osc_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return OSC_E_ARG;
    *bytes = ctx->used;
    return OSC_OK;
}

osc_status osc_launch_count(const osc_ctx *ctx, uint64_t *count) {
    if (!ctx || !count) return OSC_E_ARG;
    *count = ctx->launches.load();
    return OSC_OK;
}

osc_status osc_sync(osc_ctx *ctx) {
    CHECK_CTX(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    return debug_word_check(ctx);
}

osc_status osc_reweight(osc_ctx *ctx, int32_t sample_id, int32_t point, osc_precision prec, double *out_prob,
                        double *out_weight, int out_on_device) {
    NvtxRange nvtx_range("osc_reweight");
    CHECK_CTX(ctx);
    if (prec != OSC_FP64 && prec != OSC_FP32_BULK && prec != OSC_FP32_F64EIG)
        return fail(ctx, OSC_E_ARG, "bad precision");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    auto it = ctx->samples.find(sample_id);
    if (it == ctx->samples.end()) return fail(ctx, OSC_E_ARG, "unknown sample id");
    if (point < 0 || point >= (int32_t)ctx->pts.size()) return fail(ctx, OSC_E_ARG, "point index out of range");
    Sample *s = it->second;
    if (!out_prob && !out_weight) return OSC_OK;
    double *dp = out_prob, *dw = out_weight;
    // host outputs: a page-locked buffer is written by the kernel directly, a
    // pageable one through a device staging buffer and a copy
    bool stage_p = false, stage_w = false;
    if (!out_on_device) {
        dp = out_prob ? pinned_device_ptr(out_prob) : nullptr;
        dw = out_weight ? pinned_device_ptr(out_weight) : nullptr;
        stage_p = out_prob && !dp;
        stage_w = out_weight && !dw;
        if (stage_p || stage_w) {
            osc_status st = ensure_buf(ctx, &ctx->d_rw, &ctx->rw_cap, 2 * s->n);
            if (st) return st;
            if (stage_p) dp = ctx->d_rw;
            if (stage_w) dw = ctx->d_rw + s->n;
        }
    }
    ReweightParams rp;
    rp.s = s->dev;
    rp.point = point;
    rp.pc32 = ctx->d_pc32;
    rp.pc64 = ctx->d_pc64;
    rp.norm = ctx->pts[point].norm;
    rp.out_prob = dp;
    rp.out_weight = dw;
    const int pr = call_prec(ctx, prec, &sample_id, 1, point, 1);
    if (s->dev.n_layers > 1)
        CK(launch_reweight_layers(pr, rp, ctx->stream));
    else
        CK(launch_reweight(pr, rp, ctx->stream));
    ctx->launches += 1;
    if (stage_p) CK(cudaMemcpyAsync(out_prob, dp, s->n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (stage_w) CK(cudaMemcpyAsync(out_weight, dw, s->n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return OSC_OK;
}

}  // extern "C"

// ------------------------------------------------------- histogram plans
static std::string tune_key(const std::vector<int32_t> &ids, int32_t n_points, int prec, osc_ctx *ctx) {
    int64_t ev = 0;
    for (int32_t id : ids) ev += ctx->samples[id]->n;
    // workload class: precision, point count (log2 bucket), event count (log2 bucket)
    char k[64];
    std::snprintf(k, sizeof k, "%d:%d:%d", prec, (int)std::ceil(std::log2((double)n_points + 0.5)),
                  (int)std::ceil(std::log2((double)ev + 1)));
    return k;
}

static int32_t default_pt(int32_t n_points) {
    if (n_points >= 192) return 256;
    if (n_points >= 48) return 64;
    if (n_points >= 12) return 16;
    if (n_points >= 3) return 4;
    return 1;
}

static int32_t default_chunk(osc_ctx *ctx, const std::vector<int32_t> &ids, int32_t n_points, int32_t pt, int prec) {
    int64_t ev = 0;
    for (int32_t id : ids) ev += ctx->samples[id]->n;
    const int64_t tiles = (n_points + pt - 1) / pt;
    int per_sm = 1;
    const int threads = hist_threads_for(prec, pt);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hist_kernel_fn(prec, pt), threads, 0);
    per_sm = std::max(per_sm, 1);
    // one point per item: items are taken per warp; otherwise per block
    const int64_t slots = (int64_t)ctx->n_sm * per_sm * (pt == 1 ? threads / 32 : 1);
    const int64_t quantum = (pt == 1) ? 64 : 1024;
    // about 4 items per resident worker
    int64_t c = (ev * tiles + 4 * slots - 1) / (4 * slots);
    c = (c + quantum - 1) / quantum * quantum;
    c = std::max<int64_t>(quantum, std::min<int64_t>(c, 1 << 20));
    return (int32_t)c;
}

// Histogram kernel of an event-by-event or layered plan.
static const void *plan_kernel(const Plan *p) {
    return p->kind == kLayered ? layers_hist_kernel_fn(p->prec) : hist_kernel_fn(p->prec, p->pt);
}
static int plan_threads(const Plan *p) {
    return p->kind == kLayered ? hist_threads() : hist_threads_for(p->prec, p->pt);
}

// Keep at most 16 cached plans: evict the least recently used one.
static void evict_plan_if_full(osc_ctx *ctx) {
    if (ctx->plans.size() < 16) return;
    auto victim = std::min_element(ctx->plans.begin(), ctx->plans.end(),
                                   [](Plan *a, Plan *b) { return a->last_use < b->last_use; });
    cudaStreamSynchronize(ctx->stream);
    free_plan(ctx, *victim);
    ctx->plans.erase(victim);
}

// Per-histogram finalize metadata: (2^(64-F), 2^-F, unused, point index).
static std::vector<double> hist_meta(const std::vector<const Sample *> &ss, int32_t point_begin, int32_t n_points) {
    std::vector<double> hmeta(ss.size() * (size_t)n_points * 4);
    for (size_t s = 0; s < ss.size(); ++s)
        for (int32_t q = 0; q < n_points; ++q) {
            const int64_t h = (int64_t)s * n_points + q;
            const int F = ss[s]->frac_bits;
            hmeta[4 * h] = std::ldexp(1.0, 64 - F);
            hmeta[4 * h + 1] = std::ldexp(1.0, -F);
            hmeta[4 * h + 2] = 0.0;
            hmeta[4 * h + 3] = (double)(point_begin + q);
        }
    return hmeta;
}

static osc_status get_plan(osc_ctx *ctx, const std::vector<int32_t> &ids, int32_t point_begin, int32_t n_points,
                           int prec, int32_t nbins, int32_t pt, int32_t chunk, Plan **out, int kind = kEventByEvent) {
    for (auto it = ctx->plans.begin(); it != ctx->plans.end(); ++it) {
        Plan *p = *it;
        if (p->kind == kind && p->sample_ids == ids && p->point_begin == point_begin &&
            p->n_points == n_points && p->prec == prec && p->nbins == nbins && p->pt == pt && p->chunk == chunk) {
            p->last_use = ++ctx->plan_clock;
            *out = p;
            return OSC_OK;
        }
    }
    evict_plan_if_full(ctx);
    Plan *p = new Plan();
    p->kind = kind;
    p->sample_ids = ids;
    p->point_begin = point_begin;
    p->n_points = n_points;
    p->prec = prec;
    p->nbins = nbins;
    p->pt = pt;
    p->chunk = chunk;
    p->n_hist = (int64_t)ids.size() * n_points;
    std::vector<const Sample *> ss;
    std::vector<SampleDev> sdev;
    for (int32_t id : ids) {
        ss.push_back(ctx->samples[id]);
        sdev.push_back(ctx->samples[id]->dev);
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_kernel(p), plan_threads(p), 0);
    const int64_t slots = (int64_t)ctx->n_sm * std::max(per_sm, 1) * (pt == 1 ? plan_threads(p) / 32 : 1);
    std::vector<WorkItem> items;
    build_items(ss, point_begin, n_points, pt, chunk, slots, 0, items);
    p->n_items = (int32_t)items.size();
    p->grid = hist_grid(ctx, plan_kernel(p), p->n_items, plan_threads(p));
    const std::vector<double> hmeta = hist_meta(ss, point_begin, n_points);
    void *a;
    osc_status st = OSC_OK;
    if ((st = dalloc(ctx, &a, items.size() * sizeof(WorkItem))) == OSC_OK) p->d_items = (WorkItem *)a;
    if (!st && (st = dalloc(ctx, &a, sdev.size() * sizeof(SampleDev))) == OSC_OK) p->d_samples = (SampleDev *)a;
    if (!st && (st = dalloc(ctx, &a, hmeta.size() * sizeof(double))) == OSC_OK) p->d_hmeta = (double *)a;
    // FP32 precisions: one flag per work item for the FP64 recomputation pass (zero between launches)
    const bool redo = kind == kEventByEvent && prec != kFP64;
    if (!st && redo && (st = dalloc(ctx, &a, items.size())) == OSC_OK) p->d_redo = (uint8_t *)a;
    if (st) {
        free_plan(ctx, p);
        return st;
    }
    cudaError_t e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_samples, sdev.data(), sdev.size() * sizeof(SampleDev), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_hmeta, hmeta.data(), hmeta.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (!e && redo) e = cudaMemset(p->d_redo, 0, items.size());
    if (e) {
        free_plan(ctx, p);
        return fail_cuda(ctx, e, "cudaMemcpy(plan)");
    }
    p->last_use = ++ctx->plan_clock;
    ctx->plans.push_back(p);
    *out = p;
    return OSC_OK;
}

// Histogram kernel, then (outputs of more than one conversion round) the
// finalize kernel.  Timing mode runs them as a CUDA graph with event-record
// nodes around each kernel, parameters refreshed per call.
// d_digits (exact sharded histograms): the digit columns go there instead of
// being converted, by direct launches in every mode.
static osc_status run_plan(osc_ctx *ctx, Plan *p, double lo, double hi, double *d_out,
                           unsigned long long *d_digits = nullptr) {
    HistParams hp;
    fill_hist_params(hp, p->d_items, p->n_items, p->d_samples, ctx->d_pc32, ctx->d_pc64, ctx->d_acc, ctx->d_counter,
                     p->nbins, lo, hi);
    hp.redo = p->d_redo;
    FinalParams fp{ctx->d_acc, p->d_hmeta, ctx->d_pc64, d_out, p->n_hist, p->nbins, ctx->d_counter};
    void *hargs[] = {&hp};
    void *fargs[] = {&fp};
    cudaKernelNodeParams kr{};
    if (p->d_redo) {
        kr.func = (void *)redo_kernel_fn(p->prec);
        kr.gridDim = dim3(redo_grid());
        kr.blockDim = dim3(hist_threads());
        kr.kernelParams = hargs;
    }
    cudaKernelNodeParams kh{};
    kh.func = (void *)plan_kernel(p);
    kh.gridDim = dim3(p->grid);
    kh.blockDim = dim3(plan_threads(p));
    kh.kernelParams = hargs;
    cudaKernelNodeParams kf{};
    kf.func = (void *)final_kernel_fn();
    int64_t nfin = p->n_hist * (int64_t)p->nbins;
    int64_t fb = std::min<int64_t>(std::max<int64_t>((nfin + 255) / 256, 1), (int64_t)ctx->n_sm * 8);
    kf.gridDim = dim3((unsigned)fb);
    kf.blockDim = dim3(256);
    kf.kernelParams = fargs;
    const bool fused = !d_digits && fuse_finalize(p->n_hist, p->nbins, p->pt);
    if (fused) {
        hp.fuse_final = 1;
        hp.fin_n_hist = p->n_hist;
        hp.fin_hmeta = p->d_hmeta;
        hp.fin_out = d_out;
    }
    if (!ctx->timing || d_digits) {
        // Direct launches.  The event-by-event histogram kernel goes with
        // programmatic stream serialization: it starts (and fetches its first
        // work) while the constants kernel before it is still running, and waits
        // in griddepcontrol.wait before it reads the constants.  The finalize
        // kernel goes the same way after it: its blocks become resident as the
        // histogram blocks retire and convert as soon as that grid completes.
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(p->grid);
        cfg.blockDim = dim3(plan_threads(p));
        cfg.dynamicSmemBytes = 0;
        cfg.stream = ctx->stream;
        cfg.attrs = at;
        cfg.numAttrs = p->kind == kEventByEvent ? 1 : 0;
        CK(cudaLaunchKernelExC(&cfg, kh.func, hargs));
        // FP32 precisions: the FP64 recomputation pass (returns at once when no event was left out)
        if (p->d_redo) CK(launch_redo_programmatic(p->prec, hp, ctx->stream));
        if (d_digits)
            CK(launch_digits_out_programmatic(fp, d_digits, ctx->stream));
        else if (!fused)
            CK(launch_final_programmatic(fp, ctx->stream));
    } else {
        // timing mode: the same graph with event-record nodes around each kernel,
        // fresh events swapped in per launch (read later without blocking the stream)
        cudaEvent_t ev[4] = {pool_event(ctx), pool_event(ctx), nullptr, nullptr};
        if (!fused) {
            ev[2] = pool_event(ctx);
            ev[3] = pool_event(ctx);
        }
        if (!p->exec_t) {
            CK(cudaGraphCreate(&p->graph_t, 0));
            CK(cudaGraphAddEventRecordNode(&p->t_ev[0], p->graph_t, nullptr, 0, ev[0]));
            CK(cudaGraphAddKernelNode(&p->t_hist_node, p->graph_t, &p->t_ev[0], 1, &kh));
            CK(cudaGraphAddEventRecordNode(&p->t_ev[1], p->graph_t, &p->t_hist_node, 1, ev[1]));
            cudaGraphNode_t tail = p->t_ev[1];
            if (p->d_redo) {
                CK(cudaGraphAddKernelNode(&p->t_redo_node, p->graph_t, &p->t_ev[1], 1, &kr));
                tail = p->t_redo_node;
            }
            if (!fused) {
                CK(cudaGraphAddEventRecordNode(&p->t_ev[2], p->graph_t, &tail, 1, ev[2]));
                CK(cudaGraphAddKernelNode(&p->t_final_node, p->graph_t, &p->t_ev[2], 1, &kf));
                CK(cudaGraphAddEventRecordNode(&p->t_ev[3], p->graph_t, &p->t_final_node, 1, ev[3]));
            }
            CK(cudaGraphInstantiate(&p->exec_t, p->graph_t, 0));
        } else {
            CK(cudaGraphExecKernelNodeSetParams(p->exec_t, p->t_hist_node, &kh));
            if (p->d_redo) CK(cudaGraphExecKernelNodeSetParams(p->exec_t, p->t_redo_node, &kr));
            if (!fused) CK(cudaGraphExecKernelNodeSetParams(p->exec_t, p->t_final_node, &kf));
            for (int k = 0; k < (fused ? 2 : 4); ++k) CK(cudaGraphExecEventRecordNodeSetEvent(p->exec_t, p->t_ev[k], ev[k]));
        }
        CK(cudaGraphLaunch(p->exec_t, ctx->stream));
        ctx->ev_pending.push_back({1, {ev[0], ev[1]}});
        if (!fused) ctx->ev_pending.push_back({2, {ev[2], ev[3]}});
    }
    ctx->launches += (fused ? 1 : 2) + (p->d_redo ? 1 : 0);
    return OSC_OK;
}


// One fit step (osc_histogram_point) as a CUDA graph: the constants kernel of
// the step's point (for FP32 bulk at one point through constant density, the
// constants computed on the host and passed by value to the histogram kernel
// instead), then the histogram kernel, the FP64 recomputation pass
// (FP32 precisions; it returns at once when no event was left out) and the
// finalize kernel (larger outputs), each joined to the one before by a
// programmatic edge, so that a kernel starts while the one before still runs and
// waits in griddepcontrol.wait for its results -- the overlap of the direct
// launches, in one graph launch.  (A conditional node around the pass, set by
// the histogram kernel, measured about 8 us more per step than the pass's early
// return.)  The graph is built once per plan and replayed with its node
// parameters refreshed (the point by value, the output pointer).
static osc_status run_step_graph(osc_ctx *ctx, Plan *p, const osc_point &pt, double lo, double hi, double *d_out) {
    HistParams hp;
    fill_hist_params(hp, p->d_items, p->n_items, p->d_samples, ctx->d_pc32, ctx->d_pc64, ctx->d_acc, ctx->d_counter,
                     p->nbins, lo, hi);
    hp.redo = p->d_redo;
    FinalParams fp{ctx->d_acc, p->d_hmeta, ctx->d_pc64, d_out, p->n_hist, p->nbins, ctx->d_counter};
    const bool fused = fuse_finalize(p->n_hist, p->nbins, p->pt);
    if (fused) {
        hp.fuse_final = 1;
        hp.fin_n_hist = p->n_hist;
        hp.fin_hmeta = p->d_hmeta;
        hp.fin_out = d_out;
    }
    PointsByValueT<1> pv;
    pv.n = 1;
    pv.p[0] = pt;
    float *pc32 = ctx->d_pc32;
    double *pc64 = ctx->d_pc64;
    void *cargs[] = {&pv, &pc32, &pc64};
    void *hargs[] = {&hp};
    void *fargs[] = {&fp};
    // FP32 bulk, one point, constant density: the constants are computed here and
    // passed by value to the histogram kernel (no constants kernel in the graph)
    const bool inl = p->prec == kFP32 && p->pt == 1 && p->kind == kEventByEvent;
    std::vector<unsigned char> pin;
    void *iargs[] = {&hp, nullptr};
    if (inl) {
        pin.resize(point_inline_bytes());
        host_point_consts(pt, reinterpret_cast<float *>(pin.data()),
                          reinterpret_cast<double *>(pin.data() + sizeof(float) * C32_STRIDE));
        iargs[1] = pin.data();
    }
    if (ctx->timing) {
        // timing mode: direct launches with events around the kernels (the
        // constants kernel, where one runs, and the histogram kernel)
        if (!inl) {
            cudaEvent_t c0 = pool_event(ctx), c1 = pool_event(ctx);
            CK(cudaEventRecord(c0, ctx->stream));
            CK(launch_point_consts_host(&pt, 1, ctx->d_pc32, ctx->d_pc64, ctx->stream));
            CK(cudaEventRecord(c1, ctx->stream));
            ctx->ev_pending.push_back({0, {c0, c1}});
        }
        cudaEvent_t h0 = pool_event(ctx), h1 = pool_event(ctx);
        CK(cudaEventRecord(h0, ctx->stream));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(inl ? ctx->n_sm * hist_inline_blocks_per_sm() : p->grid);
        cfg.blockDim = dim3(plan_threads(p));
        cfg.stream = ctx->stream;
        CK(cudaLaunchKernelExC(&cfg, inl ? hist_inline_kernel_fn() : plan_kernel(p), inl ? iargs : hargs));
        CK(cudaEventRecord(h1, ctx->stream));
        ctx->ev_pending.push_back({1, {h0, h1}});
        if (p->d_redo) CK(launch_redo_programmatic(p->prec, hp, ctx->stream));
        if (!fused) {
            cudaEvent_t f0 = pool_event(ctx), f1 = pool_event(ctx);
            CK(cudaEventRecord(f0, ctx->stream));
            CK(launch_final_programmatic(fp, ctx->stream));
            CK(cudaEventRecord(f1, ctx->stream));
            ctx->ev_pending.push_back({2, {f0, f1}});
        }
        ctx->launches += (inl ? 1 : 2) + (p->d_redo ? 1 : 0) + (fused ? 0 : 1);
        return OSC_OK;
    }
    cudaKernelNodeParams kc{}, kh{}, kr{}, kf{};
    kc.func = (void *)point_consts_one_fn();
    kc.gridDim = dim3(1);
    kc.blockDim = dim3(point_consts_threads());
    kc.kernelParams = cargs;
    kh.func = inl ? (void *)hist_inline_kernel_fn() : (void *)plan_kernel(p);
    kh.gridDim = dim3(inl ? ctx->n_sm * hist_inline_blocks_per_sm() : p->grid);
    kh.blockDim = dim3(plan_threads(p));
    kh.kernelParams = inl ? iargs : hargs;
    if (p->step_exec && p->step_fused != fused) {
        cudaGraphExecDestroy(p->step_exec);
        cudaGraphDestroy(p->step_graph);
        p->step_exec = nullptr;
        p->step_graph = nullptr;
    }
    if (!p->step_exec) CK(cudaGraphCreate(&p->step_graph, 0));
    kr.func = p->d_redo ? (void *)redo_kernel_fn(p->prec) : nullptr;
    kr.gridDim = dim3(redo_grid());
    kr.blockDim = dim3(hist_threads());
    kr.kernelParams = hargs;
    kf.func = (void *)final_kernel_fn();
    kf.gridDim = dim3(final_blocks(p->n_hist * (int64_t)p->nbins));
    kf.blockDim = dim3(256);
    kf.kernelParams = fargs;
    if (!p->step_exec) {
        // programmatic edges where the downstream kernel waits in griddepcontrol.wait
        // (every kernel of an event-by-event plan); full completion edges otherwise
        cudaGraphEdgeData ed{};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        const cudaGraphEdgeData *edge = p->kind == kEventByEvent ? &ed : nullptr;
        CK(cudaGraphAddKernelNode(&p->s_hist, p->step_graph, nullptr, 0, &kh));
        if (!inl) {
            CK(cudaGraphAddKernelNode(&p->s_const, p->step_graph, nullptr, 0, &kc));
            CK(cudaGraphAddDependencies(p->step_graph, &p->s_const, &p->s_hist, edge, 1));
        }
        cudaGraphNode_t prev = p->s_hist;
        if (p->d_redo) {
            CK(cudaGraphAddKernelNode(&p->s_redo, p->step_graph, nullptr, 0, &kr));
            CK(cudaGraphAddDependencies(p->step_graph, &prev, &p->s_redo, edge, 1));
            prev = p->s_redo;
        }
        if (!fused) {
            CK(cudaGraphAddKernelNode(&p->s_final, p->step_graph, nullptr, 0, &kf));
            CK(cudaGraphAddDependencies(p->step_graph, &prev, &p->s_final, edge, 1));
        }
        CK(cudaGraphInstantiate(&p->step_exec, p->step_graph, 0));
        p->step_fused = fused;
    } else {
        if (!inl) CK(cudaGraphExecKernelNodeSetParams(p->step_exec, p->s_const, &kc));
        CK(cudaGraphExecKernelNodeSetParams(p->step_exec, p->s_hist, &kh));
        if (p->d_redo) CK(cudaGraphExecKernelNodeSetParams(p->step_exec, p->s_redo, &kr));
        if (!fused) CK(cudaGraphExecKernelNodeSetParams(p->step_exec, p->s_final, &kf));
    }
    CK(cudaGraphLaunch(p->step_exec, ctx->stream));
    ctx->launches += (inl ? 1 : 2) + (p->d_redo ? 1 : 0) + (fused ? 0 : 1);
    return OSC_OK;
}

// Time one candidate tile shape (ms per histogram launch).
static osc_status time_shape(osc_ctx *ctx, const std::vector<int32_t> &ids, int32_t pb, int32_t np, int prec,
                             int32_t nbins, double lo, double hi, int32_t pt, int32_t chunk, double *ms) {
    NvtxRange nvtx_range("autotune candidate");
    Plan *p = nullptr;
    osc_status st = get_plan(ctx, ids, pb, np, prec, nbins, pt, chunk, &p);
    if (st) return st;
    st = ensure_buf(ctx, &ctx->d_out, &ctx->out_cap, p->n_hist * nbins);
    if (st) return st;
    bool tm = ctx->timing;
    ctx->timing = true;
    double best = 1e30;
    for (int r = 0; r < 3; ++r) {
        st = run_plan(ctx, p, lo, hi, ctx->d_out);
        if (!st) st = drain_timing(ctx);
        if (st) break;
        if (r > 0) best = std::min(best, ctx->t_hist);
    }
    ctx->timing = tm;
    *ms = best;
    return st;
}

// osc_histogram, and (digits != null) osc_histogram_digits: the same call with
// the bins' digit columns as its output instead of doubles.
// step_pt (osc_histogram_point): the table holds that one point, whose constants
// the step's CUDA graph computes as its first kernel (or takes by value).
static osc_status histogram_impl(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples, int32_t point_begin,
                                 int32_t n_points, osc_precision prec, double lo, double hi, int32_t nbins,
                                 double *out, uint64_t *digits, int out_on_device, const osc_point *step_pt = nullptr) {
    CHECK_CTX(ctx);
    if (!sample_ids || !(out || digits)) return fail(ctx, OSC_E_ARG, "null argument");
    if (prec != OSC_FP64 && prec != OSC_FP32_BULK && prec != OSC_FP32_F64EIG)
        return fail(ctx, OSC_E_ARG, "bad precision");
    if (n_samples < 1 || n_samples > 4096) return fail(ctx, OSC_E_ARG, "n_samples must be in [1, 4096]");
    if (nbins < 1 || nbins > (1 << 20)) return fail(ctx, OSC_E_ARG, "nbins must be in [1, 2^20]");
    if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo)) return fail(ctx, OSC_E_RANGE, "need finite lo < hi");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (n_points < 1 || point_begin < 0 || (int64_t)point_begin + n_points > (int64_t)ctx->pts.size())
        return fail(ctx, OSC_E_ARG, "point range outside the parameter table");
    std::vector<int32_t> ids(sample_ids, sample_ids + n_samples);
    for (int32_t id : ids)
        if (!ctx->samples.count(id)) return fail(ctx, OSC_E_ARG, "unknown sample id");
    const int pr = call_prec(ctx, prec, ids.data(), n_samples, point_begin, n_points);
    const int64_t bins = (int64_t)n_samples * n_points * nbins;
    osc_status st = ensure_acc(ctx, bins);
    if (st) return st;
    bool layered = false;
    for (int32_t id : ids) layered = layered || ctx->samples[id]->dev.n_layers > 1;
    int32_t pt = ctx->tile_pt, chunk = ctx->tile_chunk;
    if (layered) {
        // one point per warp item; the tile setting applies to the single-layer kernels only
        pt = 1;
        chunk = default_chunk(ctx, ids, n_points, 1, pr);
    } else if (pt == 0) {
        // autotune once per workload class, then reuse
        const std::string key = tune_key(ids, n_points, pr, ctx);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            pt = it->second.first;
            chunk = it->second.second;
        } else {
            // a graph step computes its constants in the graph: the candidates need them now
            if (step_pt) CK(launch_point_consts_host(step_pt, 1, ctx->d_pc32, ctx->d_pc64, ctx->stream));
            int32_t best_pt = default_pt(n_points), best_chunk = 0;
            double best_ms = 1e30;
            const int32_t cands[] = {1, 4, 16, 64, 256};
            for (int32_t c : cands) {
                if (c > n_points && c != 1) continue;  // idle lanes never pay off
                for (int k = 0; k < 3; ++k) {
                    // default item size, a quarter of it (shorter tail), four times it (less overhead)
                    const int32_t q = (c == 1) ? 64 : 1024;
                    const int32_t d0 = default_chunk(ctx, ids, n_points, c, pr);
                    int32_t ch = (k == 0) ? d0 : (k == 1) ? std::max(q, (d0 / 4 + q - 1) / q * q) : d0 * 4;
                    ch = std::min(ch, 1 << 20);
                    if (k == 1 && ch == d0) continue;
                    double ms = 0.0;
                    st = time_shape(ctx, ids, point_begin, n_points, pr, nbins, lo, hi, c, ch, &ms);
                    if (st) return st;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_pt = c;
                        best_chunk = ch;
                    }
                }
            }
            pt = best_pt;
            chunk = best_chunk;
            ctx->tuned[key] = {pt, chunk};
            save_tuned(ctx, key, pt, chunk);
        }
    }
    if (chunk == 0) chunk = default_chunk(ctx, ids, n_points, pt, pr);
    Plan *p = nullptr;
    st = get_plan(ctx, ids, point_begin, n_points, pr, nbins, pt, chunk, &p, layered ? kLayered : kEventByEvent);
    if (st) return st;
    // output: doubles, or kDigits words a bin (the same byte count per word)
    const int64_t words = digits ? bins * kDigits : bins;
    double *host = digits ? (double *)digits : out;
    double *d_out = host;
    bool staged = false;
    if (!out_on_device && !(d_out = pinned_device_ptr(host))) {
        st = ensure_buf(ctx, &ctx->d_out, &ctx->out_cap, words);
        if (st) return st;
        d_out = ctx->d_out;
        staged = true;
    }
    st = digits    ? run_plan(ctx, p, lo, hi, nullptr, (unsigned long long *)d_out)
         : step_pt ? run_step_graph(ctx, p, *step_pt, lo, hi, d_out)
                   : run_plan(ctx, p, lo, hi, d_out);
    if (st) return st;
    if (staged) CK(cudaMemcpyAsync(host, d_out, words * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (!out_on_device) {
        CK(cudaStreamSynchronize(ctx->stream));
        return debug_word_check(ctx);
    }
    return OSC_OK;
}

extern "C" osc_status osc_histogram(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples, int32_t point_begin,
                                    int32_t n_points, osc_precision prec, double lo, double hi, int32_t nbins,
                                    double *out, int out_on_device) {
    NvtxRange nvtx_range("osc_histogram");
    if (!out) return ctx ? fail(ctx, OSC_E_ARG, "null argument") : OSC_E_ARG;
    return histogram_impl(ctx, sample_ids, n_samples, point_begin, n_points, prec, lo, hi, nbins, out, nullptr,
                          out_on_device);
}

// ------------------------------------------------- exact sharded histograms
extern "C" osc_status osc_histogram_digits(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                           int32_t point_begin, int32_t n_points, osc_precision prec, double lo,
                                           double hi, int32_t nbins, uint64_t *digits, int out_on_device) {
    NvtxRange nvtx_range("osc_histogram_digits");
    if (!digits) return ctx ? fail(ctx, OSC_E_ARG, "null argument") : OSC_E_ARG;
    return histogram_impl(ctx, sample_ids, n_samples, point_begin, n_points, prec, lo, hi, nbins, nullptr, digits,
                          out_on_device);
}

extern "C" osc_status osc_histogram_from_digits(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                                int32_t point_begin, int32_t n_points, int32_t nbins,
                                                const uint64_t *digits, double *out, int on_device) {
    NvtxRange nvtx_range("osc_histogram_from_digits");
    CHECK_CTX(ctx);
    if (!sample_ids || !digits || !out) return fail(ctx, OSC_E_ARG, "null argument");
    if (n_samples < 1 || n_samples > 4096) return fail(ctx, OSC_E_ARG, "n_samples must be in [1, 4096]");
    if (nbins < 1 || nbins > (1 << 20)) return fail(ctx, OSC_E_ARG, "nbins must be in [1, 2^20]");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (n_points < 1 || point_begin < 0 || (int64_t)point_begin + n_points > (int64_t)ctx->pts.size())
        return fail(ctx, OSC_E_ARG, "point range outside the parameter table");
    std::vector<const Sample *> ss;
    for (int32_t i = 0; i < n_samples; ++i) {
        auto it = ctx->samples.find(sample_ids[i]);
        if (it == ctx->samples.end()) return fail(ctx, OSC_E_ARG, "unknown sample id");
        ss.push_back(it->second);
    }
    const int64_t bins = (int64_t)n_samples * n_points * nbins;
    const std::vector<double> hmeta = hist_meta(ss, point_begin, n_points);
    // staging: the histograms' metadata, then (host input) the digit columns, then (pageable output) the bins
    const int64_t n_meta = (int64_t)hmeta.size();
    const int64_t n_dig = on_device ? 0 : bins * kDigits;
    double *d_host_out = on_device ? out : pinned_device_ptr(out);
    const int64_t n_stage_out = d_host_out ? 0 : bins;
    osc_status st = ensure_buf(ctx, &ctx->d_aux, &ctx->aux_cap, n_meta + n_dig + n_stage_out);
    if (st) return st;
    double *d_meta = ctx->d_aux;
    const unsigned long long *d_dig = on_device ? (const unsigned long long *)digits
                                                : (const unsigned long long *)(ctx->d_aux + n_meta);
    double *d_out = d_host_out ? d_host_out : ctx->d_aux + n_meta + n_dig;
    CK(cudaMemcpyAsync(d_meta, hmeta.data(), n_meta * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (!on_device) CK(cudaMemcpyAsync((void *)d_dig, digits, n_dig * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_from_digits(d_dig, d_meta, ctx->d_pc64, d_out, bins, nbins, ctx->stream));
    ctx->launches += 1;
    if (!d_host_out) CK(cudaMemcpyAsync(out, d_out, bins * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return OSC_OK;
}

extern "C" osc_status osc_sample_set_bounds(osc_ctx *ctx, int32_t sample_id, double w_abs_max, double e_true_max) {
    NvtxRange nvtx_range("osc_sample_set_bounds");
    CHECK_CTX(ctx);
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    auto it = ctx->samples.find(sample_id);
    if (it == ctx->samples.end()) return fail(ctx, OSC_E_ARG, "unknown sample id");
    if (ctx->serve) return fail(ctx, OSC_E_STATE, "cannot change a sample's bounds while serving runs");
    Sample *s = it->second;
    if (!(std::isfinite(w_abs_max) && w_abs_max >= s->w_abs && w_abs_max > 0 && w_abs_max < 3.0e38))
        return fail(ctx, OSC_E_RANGE, "w_abs_max must be finite, > 0 and at least the sample's own largest |w_mc|");
    if (!(std::isfinite(e_true_max) && e_true_max >= (double)s->e_max && e_true_max < 3.0e38))
        return fail(ctx, OSC_E_RANGE, "e_true_max must be finite and at least the sample's own largest E_true");
    int F = 62 - (int)std::ceil(std::log2(w_abs_max));
    F = std::max(8, std::min(F, 190));
    float e = (float)e_true_max;
    if ((double)e < e_true_max) e = std::nextafter(e, INFINITY);
    drop_plans(ctx);  // plans hold copies of the sample's scale
    s->frac_bits = F;
    s->e_max = e;
    s->dev.frac_bits = F;
    s->dev.hscale_d = std::ldexp(1.0, F - 64);
    s->dev.hscale_f = (float)s->dev.hscale_d;
    return OSC_OK;
}

extern "C" osc_status osc_histogram_point(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                          const osc_point *pt, osc_precision prec, double lo, double hi,
                                          int32_t nbins, double *out, int out_on_device) {
    NvtxRange nvtx_range("osc_histogram_point");
    if (!ctx || !pt || !out || ctx->poisoned) {
        // (the two calls report the argument errors)
        const osc_status s = osc_set_params(ctx, pt, 1);
        if (s) return s;
        return osc_histogram(ctx, sample_ids, n_samples, 0, 1, prec, lo, hi, nbins, out, out_on_device);
    }
    osc_status s = validate_point(ctx, *pt, 0);
    if (s) return s;
    {
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        if ((s = ensure_point_table(ctx, 1))) return s;
        ctx->pts.assign(pt, pt + 1);
    }
    return histogram_impl(ctx, sample_ids, n_samples, 0, 1, prec, lo, hi, nbins, out, nullptr, out_on_device, pt);
}

// ------------------------------------------------------ bin-centre method
// Work items of one point each, event ranges outermost so that the warps
// running at the same time read the same events for different points (L2 reuse).
static void build_items_bc(const std::vector<const Sample *> &ss, int32_t point_base, int32_t n_points,
                           int32_t chunk, std::vector<WorkItem> &items) {
    for (size_t s = 0; s < ss.size(); ++s)
        for (int64_t e = 0; e < ss[s]->n; e += chunk)
            for (int32_t q = 0; q < n_points; ++q) {
                WorkItem w;
                w.sample = (int32_t)s;
                w.point_base = point_base + q;
                w.n_pts = 1;
                w.ev_count = (int32_t)std::min<int64_t>(chunk, ss[s]->n - e);
                w.ev_begin = e;
                w.acc_base = (int64_t)s * n_points + q;
                items.push_back(w);
            }
    std::stable_sort(items.begin(), items.end(),
                     [](const WorkItem &a, const WorkItem &b) { return a.ev_count > b.ev_count; });
}

static osc_status get_bc_plan(osc_ctx *ctx, const std::vector<int32_t> &ids, int32_t point_begin, int32_t n_points,
                              int prec, int32_t nbins, double t_lo, double t_hi, int32_t t_nbins, Plan **out) {
    for (Plan *p : ctx->plans)
        if (p->kind == kBinCentre && p->sample_ids == ids && p->point_begin == point_begin &&
            p->n_points == n_points && p->prec == prec && p->nbins == nbins && p->t_lo == t_lo && p->t_hi == t_hi &&
            p->t_nbins == t_nbins && p->chunk_req == ctx->tile_chunk) {
            p->last_use = ++ctx->plan_clock;
            *out = p;
            return OSC_OK;
        }
    evict_plan_if_full(ctx);
    std::vector<const Sample *> ss;
    std::vector<SampleDev> sdev;
    int64_t ev = 0;
    for (int32_t id : ids) {
        ss.push_back(ctx->samples[id]);
        sdev.push_back(ctx->samples[id]->dev);
        ev += ctx->samples[id]->n;
    }
    // table rows: (sample, point, channel present in the sample)
    const int64_t n_hist = (int64_t)ids.size() * n_points;
    std::vector<BcRow> rows;
    std::vector<int32_t> rowmap((size_t)n_hist * kChannels, -1);
    for (size_t s = 0; s < ss.size(); ++s)
        for (int32_t q = 0; q < n_points; ++q)
            for (int c = 0; c < kChannels; ++c)
                if (ss[s]->chan_mask >> c & 1u) {
                    rowmap[((int64_t)s * n_points + q) * kChannels + c] = (int32_t)rows.size();
                    rows.push_back(BcRow{(int32_t)s, point_begin + q, c, 0});
                }
    const size_t tab_bytes = rows.size() * (size_t)t_nbins * (prec == kFP64 ? 8 : 4);
    // about two items per resident warp (the event stream is uniform work), a
    // multiple of 128 (32 lanes x 4 records); osc_set_tile's events_per_item overrides
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bc_hist_kernel_fn(prec), hist_threads(), 0);
    per_sm = std::max(per_sm, 1);
    const int64_t warps = (int64_t)ctx->n_sm * per_sm * (hist_threads() / 32);
    int64_t chunk = (ev * n_points + 2 * warps - 1) / (2 * warps);
    chunk = std::max<int64_t>(128, std::min<int64_t>((chunk + 127) / 128 * 128, 1 << 20));
    if (ctx->tile_chunk > 0) chunk = ctx->tile_chunk;
    std::vector<WorkItem> items;
    build_items_bc(ss, point_begin, n_points, (int32_t)chunk, items);

    Plan *p = new Plan();
    p->kind = kBinCentre;
    p->sample_ids = ids;
    p->point_begin = point_begin;
    p->n_points = n_points;
    p->prec = prec;
    p->nbins = nbins;
    p->pt = 1;
    p->chunk = (int32_t)chunk;
    p->n_hist = n_hist;
    p->t_lo = t_lo;
    p->t_hi = t_hi;
    p->t_nbins = t_nbins;
    p->chunk_req = ctx->tile_chunk;
    p->n_rows = (int32_t)rows.size();
    p->n_items = (int32_t)items.size();
    p->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->n_sm * per_sm, p->n_items));
    const int64_t tab_n = (int64_t)rows.size() * t_nbins;
    const int64_t tt = bc_table_threads();
    p->table_grid = (int)std::max<int64_t>(1, std::min<int64_t>((tab_n + tt - 1) / tt, (int64_t)ctx->n_sm * 32));
    const std::vector<double> hmeta = hist_meta(ss, point_begin, n_points);
    void *a;
    osc_status st = OSC_OK;
    if ((st = dalloc(ctx, &a, items.size() * sizeof(WorkItem))) == OSC_OK) p->d_items = (WorkItem *)a;
    if (!st && (st = dalloc(ctx, &a, sdev.size() * sizeof(SampleDev))) == OSC_OK) p->d_samples = (SampleDev *)a;
    if (!st && (st = dalloc(ctx, &a, hmeta.size() * sizeof(double))) == OSC_OK) p->d_hmeta = (double *)a;
    if (!st && (st = dalloc(ctx, &a, rows.size() * sizeof(BcRow))) == OSC_OK) p->d_rows = (BcRow *)a;
    if (!st && (st = dalloc(ctx, &a, rowmap.size() * sizeof(int32_t))) == OSC_OK) p->d_rowmap = (int32_t *)a;
    if (!st && (st = dalloc(ctx, &a, tab_bytes)) == OSC_OK) p->d_tab = a;
    if (st) {
        free_plan(ctx, p);
        return st;
    }
    cudaError_t e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_samples, sdev.data(), sdev.size() * sizeof(SampleDev), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_hmeta, hmeta.data(), hmeta.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_rows, rows.data(), rows.size() * sizeof(BcRow), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(p->d_rowmap, rowmap.data(), rowmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e) {
        free_plan(ctx, p);
        return fail_cuda(ctx, e, "cudaMemcpy(bin-centre plan)");
    }
    p->last_use = ++ctx->plan_clock;
    ctx->plans.push_back(p);
    *out = p;
    return OSC_OK;
}

static osc_status run_bc_plan(osc_ctx *ctx, Plan *p, double lo, double hi, double *d_out) {
    BcParams bp;
    fill_hist_params(bp.h, p->d_items, p->n_items, p->d_samples, ctx->d_pc32, ctx->d_pc64, ctx->d_acc,
                     ctx->d_counter, p->nbins, lo, hi);
    bp.rows = p->d_rows;
    bp.n_rows = p->n_rows;
    bp.t_nbins = p->t_nbins;
    bp.row_map = p->d_rowmap;
    bp.t_lo = p->t_lo;
    bp.t_w = (p->t_hi - p->t_lo) / (double)p->t_nbins;
    bp.t_lo_f = (float)p->t_lo;
    bp.t_inv_f = (float)((double)p->t_nbins / (p->t_hi - p->t_lo));
    bp.t_nb_f = (float)p->t_nbins;
    bp.tab32 = p->prec == kFP64 ? nullptr : (float *)p->d_tab;
    bp.tabq = p->prec == kFP64 ? (unsigned long long *)p->d_tab : nullptr;
    FinalParams fp{ctx->d_acc, p->d_hmeta, ctx->d_pc64, d_out, p->n_hist, p->nbins, ctx->d_counter};
    void *targs[] = {&bp};
    void *hargs[] = {&bp};
    // table kernel, then the histogram kernel by programmatic dependent launch
    // (it fetches its first items and events while the table is computed), then
    // the finalize kernel the same way: its blocks are resident when the
    // histogram grid completes, and no block of the histogram kernel waits at a
    // barrier for the block's slowest warp to convert the bins
    CK(cudaLaunchKernel(bc_table_kernel_fn(p->prec), dim3(p->table_grid), dim3(bc_table_threads()), targs, 0,
                        ctx->stream));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(p->grid);
    cfg.blockDim = dim3(hist_threads());
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelExC(&cfg, bc_hist_kernel_fn(p->prec), hargs));
    CK(launch_final_programmatic(fp, ctx->stream));
    ctx->launches += 3;
    return OSC_OK;
}

extern "C" osc_status osc_histogram_bin_centre(osc_ctx *ctx, const int32_t *sample_ids, int32_t n_samples,
                                               int32_t point_begin, int32_t n_points, osc_precision prec,
                                               double t_lo, double t_hi, int32_t t_nbins, double lo, double hi,
                                               int32_t nbins, double *out, int out_on_device) {
    NvtxRange nvtx_range("osc_histogram_bin_centre");
    CHECK_CTX(ctx);
    if (!sample_ids || !out) return fail(ctx, OSC_E_ARG, "null argument");
    if (prec != OSC_FP64 && prec != OSC_FP32_BULK && prec != OSC_FP32_F64EIG)
        return fail(ctx, OSC_E_ARG, "bad precision");
    if (n_samples < 1 || n_samples > 4096) return fail(ctx, OSC_E_ARG, "n_samples must be in [1, 4096]");
    if (nbins < 1 || nbins > (1 << 20)) return fail(ctx, OSC_E_ARG, "nbins must be in [1, 2^20]");
    if (t_nbins < 1 || t_nbins > 65536) return fail(ctx, OSC_E_ARG, "t_nbins must be in [1, 65536]");
    if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo)) return fail(ctx, OSC_E_RANGE, "need finite lo < hi");
    if (!(std::isfinite(t_lo) && std::isfinite(t_hi) && t_hi > t_lo))
        return fail(ctx, OSC_E_RANGE, "need finite t_lo < t_hi");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (n_points < 1 || point_begin < 0 || (int64_t)point_begin + n_points > (int64_t)ctx->pts.size())
        return fail(ctx, OSC_E_ARG, "point range outside the parameter table");
    std::vector<int32_t> ids(sample_ids, sample_ids + n_samples);
    for (int32_t id : ids)
        if (!ctx->samples.count(id)) return fail(ctx, OSC_E_ARG, "unknown sample id");
    const int pr = call_prec(ctx, prec, ids.data(), n_samples, point_begin, n_points);
    const int64_t bins = (int64_t)n_samples * n_points * nbins;
    osc_status st = ensure_acc(ctx, bins);
    if (st) return st;
    Plan *p = nullptr;
    st = get_bc_plan(ctx, ids, point_begin, n_points, pr, nbins, t_lo, t_hi, t_nbins, &p);
    if (st) return st;
    double *d_out = out;
    bool staged = false;
    if (!out_on_device && !(d_out = pinned_device_ptr(out))) {
        st = ensure_buf(ctx, &ctx->d_out, &ctx->out_cap, bins);
        if (st) return st;
        d_out = ctx->d_out;
        staged = true;
    }
    st = run_bc_plan(ctx, p, lo, hi, d_out);
    if (st) return st;
    if (staged) CK(cudaMemcpyAsync(out, d_out, bins * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (!out_on_device) {
        CK(cudaStreamSynchronize(ctx->stream));
        return debug_word_check(ctx);
    }
    return OSC_OK;
}
