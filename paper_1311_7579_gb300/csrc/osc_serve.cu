// osc_serve.cu -- continuous-batching serving loop (one request = one MCMC
// step's reweight of one sample at one parameter point, Sec. 2.2).
//
// A scheduler thread inside the library admits queued (sample, point) requests
// into batches while at most max_slots requests are in flight and a batch slot
// (preallocated device memory, charged to the workspace cap at serve start) is
// free.  Each batch runs on its own stream -- one input copy, constants kernel,
// histogram kernel over (request, event range) work items, finalize kernel that
// writes the bins straight into pinned host memory -- so batches admitted while
// earlier ones run overlap on the device.  The finalize kernel's last block then
// stores the batch's sequence number into a host-mapped flag; the scheduler
// polls the flags of the batches in flight (no stream callback, whose wake-up
// latency would dominate small requests), publishes the results, and osc_wait
// hands each request's histogram back.  While batches are in flight, and for a
// short while after, the scheduler thread spins rather than sleeps.  Bins are
// exact integer sums, so a request's result is bitwise the same alone and in
// any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <sstream>

#include "osc_ctx.h"

using namespace osc;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kBatches = 3;          // batches in flight (one stream each)
constexpr int kMaxItems = 1 << 16;   // work items per batch
constexpr int kFlagTicket = 4;       // int of a batch's counter block used by the finalize kernel's ticket
// the scheduler keeps polling this long after its last batch before it sleeps
constexpr std::chrono::microseconds kIdleSpin(200);

struct Request {
    uint64_t ticket;
    osc_point pt;
    int prec;
    SampleDev sd;
    int32_t frac_bits;
    Clock::time_point t_submit;
};

struct Result {
    std::vector<double> hist;
    double latency_us;
};

// A batch's inputs travel in one copy: the pinned staging block and the device
// block share one layout (points, histogram metadata, sample table, work items),
// and only the used prefix of the item list is copied.
struct StageLayout {
    size_t pts = 0, hmeta = 0, samples = 0, items = 0, bytes = 0;
    explicit StageLayout(size_t slots) {
        auto up = [](size_t x) { return (x + 255) / 256 * 256; };
        hmeta = up(pts + slots * sizeof(osc_point));
        samples = up(hmeta + slots * 4 * sizeof(double));
        items = up(samples + slots * sizeof(SampleDev));
        bytes = items + (size_t)kMaxItems * sizeof(WorkItem);
    }
    StageLayout() = default;
};

struct Batch {
    cudaStream_t stream = nullptr;
    StageLayout lay;
    // device
    char *d_stage = nullptr;
    osc_point *d_pts = nullptr;
    double *d_hmeta = nullptr;
    SampleDev *d_samples = nullptr;
    WorkItem *d_items = nullptr;
    float *d_pc32 = nullptr;
    double *d_pc64 = nullptr;
    unsigned long long *d_acc = nullptr;
    int32_t *d_counter = nullptr;
    uint8_t *d_redo = nullptr;  // FP32 precisions: per work item, marked for the FP64 recomputation pass
    // pinned host memory: staging block (same layout) and the results, which the
    // finalize writes directly (d_out is h_out's device address)
    char *h_stage = nullptr;
    osc_point *h_pts = nullptr;
    double *h_hmeta = nullptr;
    SampleDev *h_samples = nullptr;
    WorkItem *h_items = nullptr;
    double *h_out = nullptr;
    double *d_out = nullptr;
    // completion flag: host-mapped, written by the finalize kernel's last block
    unsigned long long *h_flag = nullptr;
    unsigned long long *d_flag = nullptr;
    unsigned long long seq = 0;  // sequence number of the batch last launched in this slot
    // state
    std::vector<Request> reqs;
    bool busy = false;  // launched and not yet published
};

}  // namespace

struct osc_serve {
    osc_ctx *ctx = nullptr;
    int32_t max_slots = 0, nbins = 0;
    double lo = 0, hi = 0;
    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-ups
    std::condition_variable cv_done;  // waiters
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    int32_t inflight = 0;                 // scheduler thread only
    bool stop = false;                    // under mu
    std::atomic<bool> stop_flag{false};   // the same, for the scheduler's lock-free polling
    std::atomic<int64_t> n_pending{0};    // requests in the pending queue
    std::string thread_error;
    Batch batch[kBatches];
    std::thread th;
};

namespace {

// Publishes a finished batch's histograms, which the finalize wrote into pinned
// host memory, and frees the batch slot (scheduler thread, lock held).
void publish(osc_serve *sv, Batch &b) {
    const auto now = Clock::now();
    for (size_t r = 0; r < b.reqs.size(); ++r) {
        Result res;
        res.hist.assign(b.h_out + r * sv->nbins, b.h_out + (r + 1) * sv->nbins);
        res.latency_us = std::chrono::duration<double, std::micro>(now - b.reqs[r].t_submit).count();
        sv->results[b.reqs[r].ticket] = std::move(res);
    }
    sv->inflight -= (int32_t)b.reqs.size();
    b.reqs.clear();
    b.busy = false;
}

// The batch's completion flag, read with acquire semantics: a value equal to
// the batch's sequence number means every bin of it is in host memory.
bool batch_done(const Batch &b) { return __atomic_load_n(b.h_flag, __ATOMIC_ACQUIRE) == b.seq; }

// Build and enqueue one batch (called by the scheduler thread without the lock).
osc_status launch_batch(osc_serve *sv, Batch &b) {
    NvtxRange nvtx_range("serving batch");
    osc_ctx *ctx = sv->ctx;
    const int n = (int)b.reqs.size();
    const int prec = b.reqs[0].prec;
    // distinct samples, per-request point rows, histogram metadata
    int n_samp = 0;
    std::vector<int> samp_of(n);
    for (int r = 0; r < n; ++r) {
        int s = -1;
        for (int k = 0; k < n_samp; ++k)
            if (b.h_samples[k].ev == b.reqs[r].sd.ev) s = k;
        if (s < 0) {
            s = n_samp++;
            b.h_samples[s] = b.reqs[r].sd;
        }
        samp_of[r] = s;
        b.h_pts[r] = b.reqs[r].pt;
        const int F = b.reqs[r].frac_bits;
        b.h_hmeta[4 * r] = std::ldexp(1.0, 64 - F);
        b.h_hmeta[4 * r + 1] = std::ldexp(1.0, -F);
        b.h_hmeta[4 * r + 2] = 0.0;
        b.h_hmeta[4 * r + 3] = (double)r;
    }
    // one point per item; chunk so that items fill the GPU's warps about four times
    int64_t total = 0;
    for (int r = 0; r < n; ++r) total += b.reqs[r].sd.n;
    const int64_t warps = (int64_t)ctx->n_sm * 2 * (hist_threads() / 32);
    int64_t chunk = std::max<int64_t>((total + 4 * warps - 1) / (4 * warps), 1024);
    chunk = std::max<int64_t>(chunk, (total + kMaxItems - n - 1) / (kMaxItems - n));
    chunk = (chunk + 63) / 64 * 64;
    // Items of layered samples first: a batch that mixes layered and single-layer
    // samples runs each group with its own kernel, so a request's result does not
    // depend on the other requests of its batch.  Within a group, all full chunks
    // come before the shorter tails (largest first, built in one pass, no sort).
    int n_items = 0;
    auto emit = [&](bool layered, bool tails) {
        for (int r = 0; r < n; ++r) {
            if ((b.h_samples[samp_of[r]].n_layers > 1) != layered) continue;
            const int64_t nr = b.reqs[r].sd.n, full_end = nr / chunk * chunk;
            for (int64_t e = tails ? full_end : 0; e < (tails ? nr : full_end); e += chunk) {
                WorkItem &w = b.h_items[n_items++];
                w.sample = samp_of[r];
                w.point_base = r;
                w.n_pts = 1;
                w.ev_count = (int32_t)std::min<int64_t>(chunk, nr - e);
                w.ev_begin = e;
                w.acc_base = r;
            }
        }
    };
    emit(true, false);
    emit(true, true);
    const int n_lay = n_items;
    emit(false, false);
    emit(false, true);
    cudaStream_t st = b.stream;
    cudaError_t e = cudaMemcpyAsync(b.d_stage, b.h_stage, b.lay.items + (size_t)n_items * sizeof(WorkItem),
                                    cudaMemcpyHostToDevice, st);
    if (!e) e = launch_point_consts(b.d_pts, n, b.d_pc32, b.d_pc64, st);
    if (e) return fail_cuda(ctx, e, "serving batch set-up");
    HistParams hp;
    hp.items = b.d_items;
    hp.n_items = n_items;
    hp.nbins = sv->nbins;
    hp.samples = b.d_samples;
    hp.pc32 = b.d_pc32;
    hp.pc64 = b.d_pc64;
    hp.acc = b.d_acc;
    hp.counter = b.d_counter;
    hp.lo_f = (float)sv->lo;
    hp.inv_f = (float)((double)sv->nbins / (sv->hi - sv->lo));
    hp.nb_f = (float)sv->nbins;
    hp.redo = nullptr;
    hp.fuse_final = 0;  // the flag-writing finalize kernel below converts the bins
    hp.fin_n_hist = 0;
    hp.fin_hmeta = nullptr;
    hp.fin_out = nullptr;
    int kernels = 0;
    if (n_lay > 0) {
        // layered items: their own ticket counter, finalized by the last kernel below
        HistParams hl = hp;
        hl.n_items = n_lay;
        if (n_lay < n_items) {
            hl.counter = b.d_counter + 2;
            hl.fuse_final = 0;
            e = cudaMemsetAsync(hl.counter, 0, 2 * sizeof(int32_t), st);
        }
        if (!e) e = launch_hist_layers(prec, hl, hist_grid(ctx, layers_hist_kernel_fn(prec), (n_lay + 7) / 8, hist_threads()),
                                            st);
        ++kernels;
    }
    if (!e && n_lay < n_items) {
        HistParams hs = hp;
        hs.items = b.d_items + n_lay;
        hs.n_items = n_items - n_lay;
        // programmatic launch after the kernel before it (constants or layered histogram)
        if (prec != kFP64) hs.redo = b.d_redo;
        const int thr = hist_threads_for(prec, 1), wpb = thr / 32;
        e = launch_hist_programmatic(prec, 1, hs,
                                     hist_grid(ctx, hist_kernel_fn(prec, 1), (hs.n_items + wpb - 1) / wpb, thr), st);
        ++kernels;
        // FP32 precisions: the FP64 recomputation pass (returns at once when no event was left out)
        if (!e && prec != kFP64) {
            e = launch_redo_programmatic(prec, hs, st);
            ++kernels;
        }
    }
    FinalFlag ff{{b.d_acc, b.d_hmeta, b.d_pc64, b.d_out, (int64_t)n, sv->nbins, b.d_counter}, b.d_flag, b.seq + 1,
                 b.d_counter + kFlagTicket};
    if (!e) e = launch_final_flag(ff, st);
    if (e) return fail_cuda(ctx, e, "serving batch launch");
    ++b.seq;
    ctx->launches += 2 + kernels;
    return OSC_OK;
}

// Fails every batch in flight after a CUDA error (lock held): their requests
// get no result, and osc_wait reports the error.
void fail_inflight(osc_serve *sv, const std::string &what) {
    sv->thread_error = what;
    sv->stop = true;
    sv->stop_flag.store(true);
    for (auto &b : sv->batch) {
        sv->inflight -= (int32_t)b.reqs.size();
        b.reqs.clear();
        b.busy = false;
    }
    sv->cv_done.notify_all();
}

// The scheduler thread.  Batch state (busy, reqs, seq) and the in-flight count
// belong to this thread; the lock guards only what other threads touch: the
// pending queue, the results and the stop state.  Polling reads the completion
// flags and the atomic count of pending requests without the lock, so waiting
// submitters and waiters are never held off by the spinning thread.
void scheduler(osc_serve *sv) {
    cudaSetDevice(sv->ctx->device);
    uint64_t polls = 0;
    Clock::time_point idle_since = Clock::now();
    for (;;) {
        // 1. publish finished batches
        Batch *done[kBatches];
        int n_done = 0;
        bool any_busy = false;
        for (auto &b : sv->batch) {
            if (!b.busy) continue;
            if (batch_done(b))
                done[n_done++] = &b;
            else
                any_busy = true;
        }
        if (n_done) {
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                for (int k = 0; k < n_done; ++k) publish(sv, *done[k]);
            }
            sv->cv_done.notify_all();
            idle_since = Clock::now();
        }
        // every 256 polls of a busy device, ask the streams for errors (a batch
        // whose kernels failed never raises its flag)
        if (any_busy && (++polls & 255u) == 0) {
            for (auto &b : sv->batch) {
                if (!b.busy) continue;
                const cudaError_t e = cudaStreamQuery(b.stream);
                if (e == cudaErrorNotReady) continue;
                std::string what;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    what = std::string("serving batch: ") + cudaGetErrorString(e);
                } else if (!batch_done(b)) {
                    what = "serving batch finished without its completion flag";
                }
                if (!what.empty()) {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    fail_inflight(sv, what);
                    any_busy = false;
                }
                break;
            }
        }
        const bool stopping = sv->stop_flag.load();
        if (stopping && !any_busy) break;
        // 2. admit one batch: a free slot, up to the free request slots, one precision per batch
        Batch *free_b = nullptr;
        for (auto &b : sv->batch)
            if (!b.busy) {
                free_b = &b;
                break;
            }
        if (!stopping && free_b && sv->n_pending.load() > 0 && sv->inflight < sv->max_slots) {
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                const int take_max = sv->max_slots - sv->inflight;
                const int prec = sv->pending.empty() ? 0 : sv->pending.front().prec;
                while ((int)free_b->reqs.size() < take_max && !sv->pending.empty() &&
                       sv->pending.front().prec == prec) {
                    free_b->reqs.push_back(sv->pending.front());
                    sv->pending.pop_front();
                }
                sv->n_pending.fetch_sub((int64_t)free_b->reqs.size());
            }
            if (!free_b->reqs.empty()) {
                sv->inflight += (int32_t)free_b->reqs.size();
                free_b->busy = true;
                const osc_status st = launch_batch(sv, *free_b);
                if (st != OSC_OK) {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    fail_inflight(sv, sv->ctx->err);
                }
                continue;
            }
        }
        // 3. poll while work is in flight or queued, or shortly after the last
        //    batch; otherwise sleep until a request arrives
        if (any_busy || sv->n_pending.load() > 0 || Clock::now() - idle_since < kIdleSpin) {
            std::this_thread::yield();
            continue;
        }
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] { return sv->stop || !sv->pending.empty(); });
        }
        idle_since = Clock::now();
    }
}

void free_serve(osc_ctx *ctx, osc_serve *sv) {
    for (auto &b : sv->batch) {
        if (b.stream) {
            cudaStreamSynchronize(b.stream);
            cudaStreamDestroy(b.stream);
        }
        dfree(ctx, b.d_stage);
        dfree(ctx, b.d_pc32);
        dfree(ctx, b.d_pc64);
        dfree(ctx, b.d_acc);
        dfree(ctx, b.d_redo);
        dfree(ctx, b.d_counter);
        cudaFreeHost(b.h_stage);
        cudaFreeHost(b.h_out);
        cudaFreeHost(b.h_flag);
    }
    delete sv;
}

}  // namespace

extern "C" {

osc_status osc_serve_start(osc_ctx *ctx, int32_t max_slots, double lo, double hi, int32_t nbins) {
    if (!ctx) return OSC_E_ARG;
    if (ctx->poisoned) return fail(ctx, OSC_E_STATE, "context poisoned: " + ctx->err);
    if (ctx->serve) return fail(ctx, OSC_E_STATE, "serving already running");
    if (max_slots < 1 || max_slots > 4096) return fail(ctx, OSC_E_ARG, "max_slots must be in [1, 4096]");
    if (nbins < 1 || nbins > (1 << 16)) return fail(ctx, OSC_E_ARG, "nbins must be in [1, 65536]");
    if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo)) return fail(ctx, OSC_E_RANGE, "need finite lo < hi");
    std::lock_guard<std::mutex> api(ctx->api_mu);
    osc_serve *sv = new osc_serve();
    sv->ctx = ctx;
    sv->max_slots = max_slots;
    sv->lo = lo;
    sv->hi = hi;
    sv->nbins = nbins;
    const size_t S = (size_t)max_slots, B = (size_t)nbins;
    osc_status st = OSC_OK;
    for (auto &b : sv->batch) {
        void *p;
        b.lay = StageLayout(S);
        cudaError_t e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
        if (e) st = fail_cuda(ctx, e, "cudaStreamCreate");
        if (!st && !(st = dalloc(ctx, &p, b.lay.bytes))) b.d_stage = (char *)p;
        if (!st && !(st = dalloc(ctx, &p, S * C32_STRIDE * 4))) b.d_pc32 = (float *)p;
        if (!st && !(st = dalloc(ctx, &p, S * C64_STRIDE * 8))) b.d_pc64 = (double *)p;
        if (!st && !(st = dalloc(ctx, &p, S * B * kDigits * sizeof(unsigned long long)))) b.d_acc = (unsigned long long *)p;
        if (!st && !(st = dalloc(ctx, &p, 64))) b.d_counter = (int32_t *)p;
        if (!st && !(st = dalloc(ctx, &p, kMaxItems))) b.d_redo = (uint8_t *)p;
        if (!st) {
            b.d_pts = (osc_point *)(b.d_stage + b.lay.pts);
            b.d_hmeta = (double *)(b.d_stage + b.lay.hmeta);
            b.d_samples = (SampleDev *)(b.d_stage + b.lay.samples);
            b.d_items = (WorkItem *)(b.d_stage + b.lay.items);
            e = cudaMemsetAsync(b.d_acc, 0, S * B * kDigits * sizeof(unsigned long long), b.stream);
            if (!e) e = cudaMemsetAsync(b.d_counter, 0, 64, b.stream);
            if (!e) e = cudaMemsetAsync(b.d_redo, 0, kMaxItems, b.stream);
            if (!e) e = cudaHostAlloc((void **)&b.h_stage, b.lay.bytes, 0);
            if (!e) e = cudaHostAlloc((void **)&b.h_out, S * B * 8, cudaHostAllocMapped);
            if (!e) e = cudaHostGetDevicePointer((void **)&b.d_out, b.h_out, 0);
            if (!e) e = cudaHostAlloc((void **)&b.h_flag, 64, cudaHostAllocMapped);
            if (!e) {
                *b.h_flag = 0;
                e = cudaHostGetDevicePointer((void **)&b.d_flag, b.h_flag, 0);
            }
            if (!e) e = cudaStreamSynchronize(b.stream);
            if (e) st = fail_cuda(ctx, e, "serving buffers");
        }
        if (!st) {
            b.h_pts = (osc_point *)(b.h_stage + b.lay.pts);
            b.h_hmeta = (double *)(b.h_stage + b.lay.hmeta);
            b.h_samples = (SampleDev *)(b.h_stage + b.lay.samples);
            b.h_items = (WorkItem *)(b.h_stage + b.lay.items);
        }
        if (st) break;
    }
    if (st) {
        free_serve(ctx, sv);
        return st;
    }
    ctx->serve = sv;
    sv->th = std::thread(scheduler, sv);
    return OSC_OK;
}

osc_status osc_submit(osc_ctx *ctx, int32_t sample_id, const osc_point *pt, osc_precision prec, uint64_t *ticket) {
    if (!ctx || !pt || !ticket) return OSC_E_ARG;
    osc_serve *sv = ctx->serve;
    if (!sv) return OSC_E_STATE;
    if (prec != OSC_FP64 && prec != OSC_FP32_BULK && prec != OSC_FP32_F64EIG) return OSC_E_ARG;
    Request r;
    {
        std::lock_guard<std::mutex> api(ctx->api_mu);
        if (validate_point(nullptr, *pt, 0) != OSC_OK) return OSC_E_RANGE;
        auto it = ctx->samples.find(sample_id);
        if (it == ctx->samples.end()) return OSC_E_ARG;
        r.sd = it->second->dev;
        r.frac_bits = it->second->frac_bits;
        r.prec = pair_prec(*pt, it->second, prec_kind(prec));
    }
    r.pt = *pt;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return OSC_E_STATE;
        if (sv->pending.size() >= (size_t)1 << 20) return OSC_E_BUSY;
        r.ticket = sv->next_ticket++;
        r.t_submit = Clock::now();
        sv->pending.push_back(r);
        sv->n_pending.fetch_add(1);
        *ticket = r.ticket;
    }
    sv->cv.notify_all();
    return OSC_OK;
}

osc_status osc_wait(osc_ctx *ctx, uint64_t ticket, double *out_hist, int32_t timeout_ms, double *latency_us) {
    if (!ctx || !out_hist) return OSC_E_ARG;
    osc_serve *sv = ctx->serve;
    if (!sv) return OSC_E_STATE;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (ticket == 0 || ticket >= sv->next_ticket) return OSC_E_ARG;
    auto ready = [&] { return sv->results.count(ticket) > 0 || (sv->stop && !sv->thread_error.empty()); };
    if (timeout_ms < 0)
        sv->cv_done.wait(lk, ready);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return OSC_E_TIMEOUT;
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return OSC_E_CUDA;
    std::memcpy(out_hist, it->second.hist.data(), sizeof(double) * sv->nbins);
    if (latency_us) *latency_us = it->second.latency_us;
    sv->results.erase(it);
    return OSC_OK;
}

osc_status osc_serve_stop(osc_ctx *ctx) {
    if (!ctx) return OSC_E_ARG;
    osc_serve *sv = ctx->serve;
    if (!sv) return OSC_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->stop_flag.store(true);
        sv->n_pending.fetch_sub((int64_t)sv->pending.size());
        sv->pending.clear();
    }
    sv->cv.notify_all();
    if (sv->th.joinable()) sv->th.join();
    sv->cv_done.notify_all();
    const std::string terr = sv->thread_error;
    ctx->serve = nullptr;
    free_serve(ctx, sv);
    if (!terr.empty()) return fail(ctx, OSC_E_CUDA, "serving thread: " + terr);
    return OSC_OK;
}

}  // extern "C"
