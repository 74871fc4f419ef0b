/*
 * A plain C99 consumer of librfd: the ratio-filter path (Eq. 1 per reference, Eqs. 2-3 per
 * template, the trigger reduction of Table II) driven through include/rfd.h alone, with
 * device memory from the CUDA runtime and no Python or PyTorch in the process.
 *
 *   pipeline host                 host-only entry points (no GPU needed)
 *   pipeline run <in> <out>       the whole path on device 0
 *
 * <in> (little-endian, written by the test):
 *   int64  n, n_ref, n_tmpl, K, window, precision, pn_flags, halo
 *   double fs, f_low, threshold, tukey_alpha
 *   double refs[n_ref][5], tmpl[n_tmpl][5]       (m1, m2, chi1, chi2, lambda_tilde)
 *   int32  ref_of[n_tmpl]
 *   double psd[n/2+1]
 *   float  dtilde[n/2+1][2]
 * <out>:
 *   int64  n_cand, n_trig
 *   rfd_trigger trig[n_trig]
 *   int32  lag[n_tmpl]
 *   double sigma[n_tmpl]
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "rfd.h"

#define CHECK(call)                                                                           \
    do {                                                                                      \
        rfd_status st_ = (call);                                                              \
        if (st_ != RFD_OK) {                                                                  \
            fprintf(stderr, "%s:%d %s -> %d (%s): %s\n", __FILE__, __LINE__, #call, (int)st_, \
                    rfd_status_string(st_), rfd_last_error());                                \
            exit(2);                                                                          \
        }                                                                                     \
    } while (0)

#define CUDA(call)                                                                            \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            fprintf(stderr, "%s:%d %s -> %s\n", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            exit(3);                                                                          \
        }                                                                                     \
    } while (0)

static void read_exact(FILE *f, void *p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "short read\n");
        exit(4);
    }
}

static void *host_alloc(size_t bytes) {
    void *p = malloc(bytes ? bytes : 1);
    if (!p) {
        fprintf(stderr, "out of host memory\n");
        exit(5);
    }
    return p;
}

static void *dev_alloc(size_t bytes) {
    void *p = NULL;
    CUDA(cudaMalloc(&p, bytes ? bytes : 1));
    CUDA(cudaMemset(p, 0, bytes ? bytes : 1));
    return p;
}

static int host_only(void) {
    rfd_plan_options o;
    rfd_ctx *ctx = NULL;
    rfd_status st;
    memset(&o, 0x7f, sizeof o);
    rfd_plan_options_default(&o);
    printf("version %d\n", (int)rfd_version());
    printf("qref_ld %lld %lld\n", (long long)rfd_qref_ld(524288, 127), (long long)rfd_qref_ld(1024, 1));
    printf("status %s|%s\n", rfd_status_string(RFD_ERR_OVERFLOW), rfd_status_string(RFD_ERR_TIMEOUT));
    printf("options %d %d %d %d %d %d %d %d %d %d\n", (int)o.tile_nt[0], (int)o.tile_nt[1], (int)o.tile_nt[2],
           (int)o.mix_k, (int)o.grid_ctas, (int)o.long_k, (int)o.fft_k, (int)o.out_len, (int)o.fft_rem,
           (int)o.debug_flags);
    printf("sizes %d %d %d %d\n", (int)sizeof(rfd_candidate), (int)sizeof(rfd_trigger), (int)sizeof(rfd_grid),
           (int)sizeof(rfd_params));
    st = rfd_ctx_create(-1, &ctx);
    printf("ctx_create(-1) %d %s\n", (int)st, ctx == NULL ? "null" : "set");
    return 0;
}

static int run(const char *in_path, const char *out_path) {
    FILE *f = fopen(in_path, "rb");
    int64_t hdr[8];
    double fl[4];
    rfd_grid g;
    rfd_ctx *ctx = NULL;
    rfd_plan *plan = NULL;
    int32_t n_ref, n_tmpl, K, window, precision, halo, j;
    int64_t n, nf, ld, cand_cap, trig_cap, n_cand = 0, n_trig = 0;
    rfd_params *refs, *tmpl;
    int32_t *ref_of, *k_host, *lag_h;
    double *psd_h, *sigma_h;
    float *d_h;
    void *psd_d, *d_d, *href_d, *q_d, *e_d, *taps_d, *lag_d, *sig_d, *cand_d, *cnt_d, *trig_d;
    rfd_trigger *trig_h;
    FILE *o;

    if (!f) {
        perror(in_path);
        return 1;
    }
    read_exact(f, hdr, sizeof hdr);
    read_exact(f, fl, sizeof fl);
    n = hdr[0];
    n_ref = (int32_t)hdr[1];
    n_tmpl = (int32_t)hdr[2];
    K = (int32_t)hdr[3];
    window = (int32_t)hdr[4];
    precision = (int32_t)hdr[5];
    halo = (int32_t)hdr[7];
    nf = n / 2 + 1;
    refs = (rfd_params *)host_alloc(sizeof(rfd_params) * (size_t)n_ref);
    tmpl = (rfd_params *)host_alloc(sizeof(rfd_params) * (size_t)n_tmpl);
    ref_of = (int32_t *)host_alloc(sizeof(int32_t) * (size_t)n_tmpl);
    psd_h = (double *)host_alloc(sizeof(double) * (size_t)nf);
    d_h = (float *)host_alloc(2 * sizeof(float) * (size_t)nf);
    read_exact(f, refs, sizeof(rfd_params) * (size_t)n_ref);
    read_exact(f, tmpl, sizeof(rfd_params) * (size_t)n_tmpl);
    read_exact(f, ref_of, sizeof(int32_t) * (size_t)n_tmpl);
    read_exact(f, psd_h, sizeof(double) * (size_t)nf);
    read_exact(f, d_h, 2 * sizeof(float) * (size_t)nf);
    fclose(f);

    g.fs = fl[0];
    g.n = n;
    g.f_low = fl[1];
    g.pn_flags = (int32_t)hdr[6];
    g.reserved = 0;
    CHECK(rfd_ctx_create(0, &ctx));

    /* Eq. 1 per reference: templates, then the matched filter into the split q_ref planes */
    ld = rfd_qref_ld(n, halo);
    psd_d = dev_alloc(sizeof(double) * (size_t)nf);
    d_d = dev_alloc(2 * sizeof(float) * (size_t)nf);
    href_d = dev_alloc(2 * sizeof(float) * (size_t)nf * (size_t)n_ref);
    q_d = dev_alloc((size_t)n_ref * 8 * (size_t)ld);
    e_d = dev_alloc(sizeof(int32_t) * (size_t)n_ref);
    CUDA(cudaMemcpy(psd_d, psd_h, sizeof(double) * (size_t)nf, cudaMemcpyHostToDevice));
    CUDA(cudaMemcpy(d_d, d_h, 2 * sizeof(float) * (size_t)nf, cudaMemcpyHostToDevice));
    CHECK(rfd_gen_templates(ctx, &g, refs, n_ref, href_d, NULL));
    CHECK(rfd_filter_reference(ctx, &g, d_d, (const double *)psd_d, href_d, n_ref, halo, precision, q_d,
                               (int32_t *)e_d, NULL));

    /* Sec. V: taps, lags and sigma_eff per template */
    k_host = (int32_t *)host_alloc(sizeof(int32_t) * (size_t)n_tmpl);
    for (j = 0; j < n_tmpl; ++j) k_host[j] = K;
    taps_d = dev_alloc(2 * sizeof(float) * (size_t)n_tmpl * (size_t)K);
    lag_d = dev_alloc(sizeof(int32_t) * (size_t)n_tmpl);
    sig_d = dev_alloc(sizeof(double) * (size_t)n_tmpl);
    CHECK(rfd_make_taps(ctx, &g, (const double *)psd_d, refs, n_ref, tmpl, ref_of, n_tmpl, k_host, NULL, 0, 0.999,
                        K, fl[3], taps_d, NULL, (int32_t *)lag_d, (double *)sig_d, NULL, NULL));

    /* Eq. 3 and the trigger reduction */
    CHECK(rfd_plan_create(ctx, &g, n_ref, n_tmpl, ref_of, k_host, precision, window, (float)fl[2], halo, &plan));
    CHECK(rfd_plan_set_taps(plan, taps_d, K, (const int32_t *)lag_d, (const double *)sig_d, NULL));
    cand_cap = (int64_t)1 << 20;
    trig_cap = (int64_t)1 << 18;
    cand_d = dev_alloc(sizeof(rfd_candidate) * (size_t)cand_cap);
    cnt_d = dev_alloc(sizeof(int64_t));
    trig_d = dev_alloc(sizeof(rfd_trigger) * (size_t)trig_cap);
    CHECK(rfd_ratio_filter_batch(plan, q_d, (const int32_t *)e_d, (rfd_candidate *)cand_d, cand_cap,
                                 (int64_t *)cnt_d, NULL));
    CHECK(rfd_find_triggers(ctx, n_tmpl, (const rfd_candidate *)cand_d, (const int64_t *)cnt_d, cand_cap,
                            (rfd_trigger *)trig_d, trig_cap, &n_trig, NULL));
    CUDA(cudaMemcpy(&n_cand, cnt_d, sizeof(int64_t), cudaMemcpyDeviceToHost));
    trig_h = (rfd_trigger *)host_alloc(sizeof(rfd_trigger) * (size_t)n_trig);
    lag_h = (int32_t *)host_alloc(sizeof(int32_t) * (size_t)n_tmpl);
    sigma_h = (double *)host_alloc(sizeof(double) * (size_t)n_tmpl);
    CUDA(cudaMemcpy(trig_h, trig_d, sizeof(rfd_trigger) * (size_t)n_trig, cudaMemcpyDeviceToHost));
    CUDA(cudaMemcpy(lag_h, lag_d, sizeof(int32_t) * (size_t)n_tmpl, cudaMemcpyDeviceToHost));
    CUDA(cudaMemcpy(sigma_h, sig_d, sizeof(double) * (size_t)n_tmpl, cudaMemcpyDeviceToHost));

    o = fopen(out_path, "wb");
    if (!o) {
        perror(out_path);
        return 1;
    }
    fwrite(&n_cand, sizeof n_cand, 1, o);
    fwrite(&n_trig, sizeof n_trig, 1, o);
    fwrite(trig_h, sizeof(rfd_trigger), (size_t)n_trig, o);
    fwrite(lag_h, sizeof(int32_t), (size_t)n_tmpl, o);
    fwrite(sigma_h, sizeof(double), (size_t)n_tmpl, o);
    fclose(o);

    rfd_plan_destroy(plan);
    rfd_ctx_destroy(ctx);
    CUDA(cudaFree(psd_d));
    CUDA(cudaFree(d_d));
    CUDA(cudaFree(href_d));
    CUDA(cudaFree(q_d));
    CUDA(cudaFree(e_d));
    CUDA(cudaFree(taps_d));
    CUDA(cudaFree(lag_d));
    CUDA(cudaFree(sig_d));
    CUDA(cudaFree(cand_d));
    CUDA(cudaFree(cnt_d));
    CUDA(cudaFree(trig_d));
    free(refs);
    free(tmpl);
    free(ref_of);
    free(psd_h);
    free(d_h);
    free(k_host);
    free(trig_h);
    free(lag_h);
    free(sigma_h);
    printf("ok %lld candidates, %lld triggers\n", (long long)n_cand, (long long)n_trig);
    return 0;
}

int main(int argc, char **argv) {
    if (argc == 2 && strcmp(argv[1], "host") == 0) return host_only();
    if (argc == 4 && strcmp(argv[1], "run") == 0) return run(argv[2], argv[3]);
    fprintf(stderr, "usage: %s host | run <in> <out>\n", argv[0]);
    return 1;
}
