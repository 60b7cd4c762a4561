/*
 * osc_abi_test.c -- drives the C ABI of include/osc.h from plain C (no Python).
 *
 *   osc_abi_test nogpu
 *       argument and state checks that need no device: version string, null
 *       arguments, context creation failing cleanly without a GPU.
 *   osc_abi_test gpu <input> <output>
 *       loads the sample in <input>, sets the points in it, and writes the FP64
 *       histograms of every point, the FP64 probabilities of point 0 and the
 *       FP32 histograms to <output>; also checks the error paths of a live
 *       context.  The calling test compares the numbers with the oracle.
 *   osc_abi_test time <input> <k>
 *       loads the sample of <input>, then makes k fit steps (osc_histogram_point
 *       of its first point, FP32-bulk, into a pageable host buffer) after three
 *       untimed ones, and prints the wall time per step [us] (clock_gettime): the
 *       end-to-end cost of the C ABI without any Python in between.
 *
 * Input layout (little endian): int64 n, int32 n_points, int32 nbins,
 * double lo, hi, baseline_km, density_gcc, ye; float e_true[n], e_reco[n],
 * w_mc[n]; uint8 flav_in[n], flav_out[n], is_nubar[n]; double points[n_points][8].
 * Output: double hist64[n_points][nbins], prob64[n], hist32[n_points][nbins].
 * Exit status 0 on success; a message on stderr otherwise.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "osc.h"

#define CHECK(cond, msg)                                        \
    do {                                                        \
        if (!(cond)) {                                          \
            fprintf(stderr, "osc_abi_test: %s\n", (msg));       \
            return 1;                                           \
        }                                                       \
    } while (0)

static int no_gpu(void) {
    osc_ctx *ctx = NULL;
    int32_t sid = 0;
    CHECK(osc_version() && strlen(osc_version()) > 0, "empty version string");
    CHECK(strcmp(osc_last_error(NULL), "no context") == 0, "last_error(NULL)");
    CHECK(osc_load_sample(NULL, NULL, &sid) == OSC_E_ARG, "load_sample(NULL)");
    CHECK(osc_set_params(NULL, NULL, 1) == OSC_E_ARG, "set_params(NULL)");
    CHECK(osc_histogram(NULL, NULL, 1, 0, 1, OSC_FP64, 0.0, 5.0, 10, NULL, 0) == OSC_E_ARG, "histogram(NULL)");
    CHECK(osc_set_layers(NULL, 0, 1, NULL, NULL, NULL) == OSC_E_ARG, "set_layers(NULL)");
    CHECK(osc_create(0, 0, NULL, NULL) == OSC_E_ARG, "create(out = NULL)");
    CHECK(osc_create(0, 0, NULL, &ctx) != OSC_OK && ctx == NULL, "create without a GPU must fail");
    osc_destroy(NULL);
    return 0;
}

static int read_all(const char *path, void **buf, size_t *len) {
    FILE *f = fopen(path, "rb");
    if (!f) return 1;
    fseek(f, 0, SEEK_END);
    *len = (size_t)ftell(f);
    fseek(f, 0, SEEK_SET);
    *buf = malloc(*len);
    const size_t got = *buf ? fread(*buf, 1, *len, f) : 0;
    fclose(f);
    return got != *len;
}

static int gpu(const char *in_path, const char *out_path) {
    void *buf = NULL;
    size_t len = 0;
    CHECK(read_all(in_path, &buf, &len) == 0, "cannot read the input file");
    const char *p = (const char *)buf;
    int64_t n;
    int32_t n_points, nbins;
    double hdr[5];
    memcpy(&n, p, 8);
    memcpy(&n_points, p + 8, 4);
    memcpy(&nbins, p + 12, 4);
    memcpy(hdr, p + 16, sizeof(hdr));
    p += 16 + sizeof(hdr);
    osc_sample_desc d;
    d.n = n;
    d.e_true = (const float *)p;
    d.e_reco = d.e_true + n;
    d.w_mc = d.e_reco + n;
    d.flav_in = (const uint8_t *)(d.w_mc + n);
    d.flav_out = d.flav_in + n;
    d.is_nubar = d.flav_out + n;
    d.baseline_km = hdr[2];
    d.density_gcc = hdr[3];
    d.ye = hdr[4];
    osc_point *pts = (osc_point *)malloc((size_t)n_points * sizeof(osc_point));
    memcpy(pts, d.is_nubar + n, (size_t)n_points * sizeof(osc_point));

    osc_ctx *ctx = NULL;
    CHECK(osc_create(0, 0, NULL, &ctx) == OSC_OK, "create");
    int32_t sid = -1;
    CHECK(osc_load_sample(ctx, &d, &sid) == OSC_OK, osc_last_error(ctx));
    CHECK(osc_set_params(ctx, pts, n_points) == OSC_OK, osc_last_error(ctx));

    const size_t nh = (size_t)n_points * (size_t)nbins;
    double *out = (double *)calloc(2 * nh + (size_t)n, sizeof(double));
    CHECK(osc_histogram(ctx, &sid, 1, 0, n_points, OSC_FP64, hdr[0], hdr[1], nbins, out, 0) == OSC_OK,
          osc_last_error(ctx));
    CHECK(osc_reweight(ctx, sid, 0, OSC_FP64, out + nh, NULL, 0) == OSC_OK, osc_last_error(ctx));
    CHECK(osc_histogram(ctx, &sid, 1, 0, n_points, OSC_FP32_BULK, hdr[0], hdr[1], nbins, out + nh + n, 0) == OSC_OK,
          osc_last_error(ctx));

    /* error paths of a live context: rejected before any launch, context stays usable */
    int32_t bad = sid + 1000;
    CHECK(osc_histogram(ctx, &bad, 1, 0, 1, OSC_FP64, 0.0, 5.0, 10, out, 0) == OSC_E_ARG, "unknown sample id");
    CHECK(strlen(osc_last_error(ctx)) > 0, "error message");
    CHECK(osc_histogram(ctx, &sid, 1, 0, 1, (osc_precision)7, 0.0, 5.0, 10, out, 0) == OSC_E_ARG, "bad precision");
    CHECK(osc_histogram(ctx, &sid, 1, 0, 1, OSC_FP64, 5.0, 5.0, 10, out, 0) == OSC_E_RANGE, "empty range");
    CHECK(osc_histogram(ctx, &sid, 1, n_points, 1, OSC_FP64, 0.0, 5.0, 10, out, 0) == OSC_E_ARG, "point range");
    osc_point bad_pt = pts[0];
    bad_pt.dm21 = -1.0;
    CHECK(osc_set_params(ctx, &bad_pt, 1) == OSC_E_RANGE, "dm21 < 0");
    /* the one-call fit step equals set_params + histogram over point 0, bitwise */
    double *one = (double *)calloc(2 * (size_t)nbins, sizeof(double));
    CHECK(one != NULL, "alloc");
    CHECK(osc_histogram_point(ctx, &sid, 1, &pts[0], OSC_FP64, hdr[0], hdr[1], nbins, one, 0) == OSC_OK,
          osc_last_error(ctx));
    CHECK(memcmp(one, out, (size_t)nbins * sizeof(double)) == 0, "histogram_point != histogram of point 0");
    CHECK(osc_histogram_point(ctx, &sid, 1, &bad_pt, OSC_FP64, hdr[0], hdr[1], nbins, one, 0) == OSC_E_RANGE,
          "histogram_point with dm21 < 0");
    free(one);
    CHECK(osc_sync(ctx) == OSC_OK, "sync");
    uint64_t launches = 0;
    CHECK(osc_launch_count(ctx, &launches) == OSC_OK && launches > 0, "launch count");
    CHECK(osc_unload_sample(ctx, sid) == OSC_OK, "unload");
    CHECK(osc_unload_sample(ctx, sid) == OSC_E_ARG, "double unload");
    osc_destroy(ctx);

    FILE *f = fopen(out_path, "wb");
    CHECK(f != NULL, "cannot write the output file");
    const size_t wrote = fwrite(out, sizeof(double), 2 * nh + (size_t)n, f);
    fclose(f);
    CHECK(wrote == 2 * nh + (size_t)n, "short write");
    free(out);
    free(pts);
    free(buf);
    return 0;
}

static double now_s(void) {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

static int timing(const char *in_path, int k) {
    void *buf = NULL;
    size_t len = 0;
    CHECK(k > 0, "k must be positive");
    CHECK(read_all(in_path, &buf, &len) == 0, "cannot read the input file");
    const char *p = (const char *)buf;
    int64_t n;
    int32_t n_points, nbins;
    double hdr[5];
    memcpy(&n, p, 8);
    memcpy(&n_points, p + 8, 4);
    memcpy(&nbins, p + 12, 4);
    memcpy(hdr, p + 16, sizeof(hdr));
    p += 16 + sizeof(hdr);
    osc_sample_desc d;
    d.n = n;
    d.e_true = (const float *)p;
    d.e_reco = d.e_true + n;
    d.w_mc = d.e_reco + n;
    d.flav_in = (const uint8_t *)(d.w_mc + n);
    d.flav_out = d.flav_in + n;
    d.is_nubar = d.flav_out + n;
    d.baseline_km = hdr[2];
    d.density_gcc = hdr[3];
    d.ye = hdr[4];
    osc_point pt;
    memcpy(&pt, d.is_nubar + n, sizeof(osc_point));
    osc_ctx *ctx = NULL;
    CHECK(osc_create(0, 0, NULL, &ctx) == OSC_OK, "create");
    int32_t sid = -1;
    CHECK(osc_load_sample(ctx, &d, &sid) == OSC_OK, osc_last_error(ctx));
    double *out = (double *)calloc((size_t)nbins, sizeof(double));
    CHECK(out != NULL, "alloc");
    for (int i = 0; i < 3; ++i)
        CHECK(osc_histogram_point(ctx, &sid, 1, &pt, OSC_FP32_BULK, hdr[0], hdr[1], nbins, out, 0) == OSC_OK,
              osc_last_error(ctx));
    const double t0 = now_s();
    for (int i = 0; i < k; ++i)
        CHECK(osc_histogram_point(ctx, &sid, 1, &pt, OSC_FP32_BULK, hdr[0], hdr[1], nbins, out, 0) == OSC_OK,
              osc_last_error(ctx));
    const double dt = now_s() - t0;
    CHECK(out[0] >= 0.0, "histogram");
    printf("{\"steps\": %d, \"us_per_step\": %.3f, \"events\": %lld}\n", k, 1e6 * dt / k, (long long)n);
    free(out);
    osc_destroy(ctx);
    free(buf);
    return 0;
}

int main(int argc, char **argv) {
    if (argc >= 2 && strcmp(argv[1], "nogpu") == 0) return no_gpu();
    if (argc >= 4 && strcmp(argv[1], "gpu") == 0) return gpu(argv[2], argv[3]);
    if (argc >= 4 && strcmp(argv[1], "time") == 0) return timing(argv[2], atoi(argv[3]));
    fprintf(stderr, "usage: osc_abi_test nogpu | gpu <input> <output> | time <input> <k>\n");
    return 2;
}
