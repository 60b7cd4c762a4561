// osc_ctx.h -- the context object behind the C ABI (host runtime internals).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "osc_internal.h"
#include "osc_launch.h"

struct osc_serve;  // serving state (osc_serve.cu)

namespace osc {

struct Sample {
    int32_t id = -1;
    int64_t n = 0, n_pad = 0;
    double L = 0, rho = 0, ye = 0;
    int32_t frac_bits = 96;
    uint32_t chan_mask = 0;  // bit c set when channel id c occurs in the sample
    float e_max = 0.0f;      // largest E_true (or the bound osc_sample_set_bounds set)
    double w_abs = 0.0;      // largest |w_mc|
    double ka_max = 0.0;     // largest k_A rho Y_e over the path's layers (max |A| = ka_max e_max)
    double matter_phase = 0.0;  // sum over the path's layers of c_L L k_A rho Y_e [rad] (energy independent)
    float4 *ev = nullptr;
    int32_t *perm = nullptr;
    void *lay = nullptr;     // layered path: float4[n_layers] then double2[n_layers]
    SampleDev dev{};
};

// A cached launch plan for one histogram call shape.
enum PlanKind { kEventByEvent = 0, kBinCentre = 1, kLayered = 2 };
struct Plan {
    int32_t kind = kEventByEvent;
    std::vector<int32_t> sample_ids;
    int32_t point_begin = 0, n_points = 0, nbins = 0, prec = 0, pt = 0, chunk = 0;
    int64_t n_hist = 0;
    int32_t n_items = 0, grid = 0;
    WorkItem *d_items = nullptr;
    SampleDev *d_samples = nullptr;
    double *d_hmeta = nullptr;
    uint8_t *d_redo = nullptr;  // FP32 precisions: per work item, marked for the FP64 recomputation pass
    // timing mode: the step as a CUDA graph with event-record nodes around each kernel
    cudaGraph_t graph_t = nullptr;
    cudaGraphExec_t exec_t = nullptr;
    cudaGraphNode_t t_hist_node = nullptr, t_redo_node = nullptr, t_final_node = nullptr,
                    t_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // one-point fit step (osc_histogram_point): constants, histogram, FP64
    // recomputation and finalize kernels joined by programmatic edges
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraphNode_t s_const = nullptr, s_hist = nullptr, s_redo = nullptr, s_final = nullptr;
    bool step_fused = false;
    // bin-centre plans: true-energy binning, probability table and its rows
    double t_lo = 0, t_hi = 0;
    int32_t t_nbins = 0, n_rows = 0;
    int32_t chunk_req = 0;  // events_per_item requested by osc_set_tile when the plan was made (0: default)
    BcRow *d_rows = nullptr;
    int32_t *d_rowmap = nullptr;
    void *d_tab = nullptr;
    int32_t table_grid = 0;
    uint64_t last_use = 0;
};

}  // namespace osc

struct osc_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t cap = 0, used = 0;
    // fault injection (tests): the fault_alloc_at-th device allocation fails as
    // if the device were out of memory (0: never)
    int64_t fault_alloc_at = 0, n_allocs = 0;
    std::unordered_map<void *, size_t> sizes;
    std::string err;
    bool poisoned = false;
    std::mutex api_mu;  // serialises ABI calls against the serving thread

    std::map<int32_t, osc::Sample *> samples;
    int32_t next_id = 0;

    std::vector<osc_point> pts;
    osc_point *d_pts = nullptr;
    float *d_pc32 = nullptr;
    double *d_pc64 = nullptr;
    int32_t pts_cap = 0;

    unsigned long long *d_acc = nullptr;
    int64_t acc_cap_bins = 0;
    int32_t *d_counter = nullptr;
    double *d_out = nullptr;
    int64_t out_cap = 0;
    double *d_rw = nullptr;
    int64_t rw_cap = 0;
    double *d_aux = nullptr;  // staging of osc_histogram_from_digits
    int64_t aux_cap = 0;

    std::list<osc::Plan *> plans;
    uint64_t plan_clock = 0;

    bool timing = false;
    double t_const = -1, t_hist = -1, t_final = -1;
    // non-blocking timing: event pairs per kernel kind (0 const, 1 hist, 2 final)
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    int64_t t_count[3] = {0, 0, 0};
    double t_sum[3] = {0, 0, 0};
    std::atomic<uint64_t> launches{0};

    int32_t tile_pt = 0, tile_chunk = 0;
    std::map<std::string, std::pair<int32_t, int32_t>> tuned;
    std::string tune_file;    // autotuner results persisted here (OSC_AUTOTUNE_CACHE), or empty
    std::string device_name;  // part of every persisted key

    osc_serve *serve = nullptr;
};

namespace osc {

// NVTX range over a host-side scope (visible in Nsight timelines; free when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// helpers shared by the runtime and the serving loop
osc_status fail(osc_ctx *c, osc_status s, const std::string &msg);
osc_status fail_cuda(osc_ctx *c, cudaError_t e, const char *what);
osc_status dalloc(osc_ctx *c, void **p, size_t bytes);
void dfree(osc_ctx *c, void *p);
osc_status validate_point(osc_ctx *c, const osc_point &p, int index);
osc_status debug_word_check(osc_ctx *c);
osc_status ensure_acc(osc_ctx *c, int64_t bins);
// grid of the persistent histogram kernel; finalize fusion rule
int hist_grid(osc_ctx *c, const void *kernel, int32_t n_items, int threads);
bool fuse_finalize(int64_t n_hist, int32_t nbins, int32_t pt);
int prec_kind(osc_precision p);
// FP32-bulk through layers also needs dm21 >= kFp32LayerSolarRatio |dm31|: with a
// smaller solar splitting the FP32 seeds of the two solar roots (a near-double
// pair at the cubic's scale) leave shift errors comparable to the vacuum gap,
// which the layer update's eigenvector weights divide by (|dP| reached O(1) at
// 1.2e-4, 1e-4 at 3e-3).  The single-layer Sylvester form stays below 1e-3 there,
// and FP32_F64EIG (FP64 shifts) below 1.2e-5 through layers.
constexpr double kFp32LayerSolarRatio = 5e-3;
// ... and a matter term at most kFp32LayerMatterRatio |dm31|: the layer update meets
// the matter-dominated near-double pair earlier than the single-layer form
// (|dP| 6e-3 to 1e-2 at 300-480 |dm31| through five layers, 8e-4 at 107, 5e-5
// at 49, against at most 7.5e-4 up to 1500 for one layer).
constexpr double kFp32LayerMatterRatio = 100.0;
// The kernel precision of one (point, sample) pair for a requested precision:
// FP64 outside the FP32 precisions' domain (the matter ratio of osc_internal.h
// and, through layers, the two ratios above); OSC_FP32_BULK becomes FP32_F64EIG
// where its FP32 shifts and phases would not hold (the sample's matter phase
// above kFp32BulkMatterPhase or its matter term above kFp32BulkMatterRatio
// |dm31|).  A call runs in the most precise kernel any of its pairs needs.
int pair_prec(const osc_point &p, const Sample *s, int prec);
int call_prec(osc_ctx *c, osc_precision prec, const int32_t *ids, int32_t n_ids, int32_t point_begin,
              int32_t n_points);
cudaEvent_t pool_event(osc_ctx *c);
osc_status drain_timing(osc_ctx *c);
void build_items(const std::vector<const Sample *> &ss, int32_t point_base, int32_t n_points, int32_t pt,
                 int32_t chunk, int64_t slots, int64_t acc_hist_base, std::vector<WorkItem> &items);

}  // namespace osc
