// osc_launch.h -- host-side entry points of the kernel translation units (launch
// helpers and kernel function pointers), used by the runtime and the serving loop.
// Not part of the public ABI.
#pragma once

#include "osc_internal.h"

namespace osc {

cudaError_t launch_point_consts(const osc_point *d_pts, int n, float *pc32, double *pc64, cudaStream_t st);
cudaError_t launch_point_consts_host(const osc_point *h_pts, int n, float *pc32, double *pc64, cudaStream_t st);
cudaError_t launch_hist(int prec, int pt, const HistParams &p, int grid, cudaStream_t st);
cudaError_t launch_hist_programmatic(int prec, int pt, const HistParams &p, int grid, cudaStream_t st);
cudaError_t launch_final(const FinalParams &p, cudaStream_t st);
// The finalize kernel with programmatic stream serialization (after a histogram kernel).
cudaError_t launch_final_programmatic(const FinalParams &p, cudaStream_t st);
int final_blocks(int64_t n_bins);
// Serving: the finalize kernel, launched programmatically, whose last block
// stores seq to *flag (host-mapped memory) after every bin is visible to the
// host; ticket is a device int the kernel leaves at 0.
struct FinalFlag {
    FinalParams f;
    unsigned long long *flag;
    unsigned long long seq;
    int32_t *ticket;
};
cudaError_t launch_final_flag(const FinalFlag &p, cudaStream_t st);
cudaError_t launch_reweight(int prec, const ReweightParams &p, cudaStream_t st);
// Kernel function pointers (for CUDA-graph kernel nodes and occupancy queries).
const void *hist_kernel_fn(int prec, int pt);
const void *bc_table_kernel_fn(int prec);
int bc_table_threads();
const void *bc_hist_kernel_fn(int prec);
const void *layers_hist_kernel_fn(int prec);
cudaError_t launch_reweight_layers(int prec, const ReweightParams &p, cudaStream_t st);
cudaError_t launch_hist_layers(int prec, const HistParams &p, int grid, cudaStream_t st);
const void *final_kernel_fn();
int hist_threads();
// Threads per block of the event-by-event histogram kernel of a precision and
// points-per-block (128 for the FP32-bulk one-point kernel, else hist_threads()).
int hist_threads_for(int prec, int pt);
// FP32 precisions: the FP64 recomputation pass after a histogram kernel (k_redo),
// launched with programmatic stream serialization; its kernel function.
cudaError_t launch_redo_programmatic(int prec, const HistParams &p, cudaStream_t st);
const void *redo_kernel_fn(int prec);
int redo_grid();
// Exact sharded histograms: digit columns out (programmatic, after the
// histogram kernel or its FP64 recomputation pass; clears the accumulators),
// and bins from digit columns.
cudaError_t launch_digits_out_programmatic(const FinalParams &p, unsigned long long *out, cudaStream_t st);
cudaError_t launch_from_digits(const unsigned long long *digits, const double *hmeta, const double *pc64, double *out,
                               int64_t n, int32_t nbins, cudaStream_t st);
// The constants kernel of a one-point table passed by value (a graph node's
// function) and its block size.
const void *point_consts_one_fn();
int point_consts_threads();
// The FP32-bulk one-point histogram kernel of a fit step with the point's
// constants by value (kernel parameters: HistParams, then the C32_STRIDE floats
// and C64_STRIDE doubles of host_point_consts), and that second parameter's size.
const void *hist_inline_kernel_fn();
size_t point_inline_bytes();
int hist_inline_blocks_per_sm();
// The constants of one point computed on the host, bitwise those of the
// constants kernel (the FP32 and FP64 rows of the constants tables).
void host_point_consts(const osc_point &P, float *c32, double *c64);
// Streaming multiprocessors of the current device (queried once per device).
int device_sms();

}  // namespace osc
