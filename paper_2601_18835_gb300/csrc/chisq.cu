// Sub-band chi^2 signal-consistency test through the ratio filter (Sec. VI): the reference's
// band is split into p sub-bands of equal reference SNR, the data are matched-filtered per
// sub-band once per reference, and a template's sub-band SNRs at a trigger are the ratio FIR of
// Eq. 3 applied to the reference's sub-band series:
//   z_b(t) = (1/sigma_eff) sum_k rho[k] q_r,b[(t - s - k) mod n],  z = sum_b z_b,
//   u_b = sigma_b^2 / sigma_eff^2 (sigma_b^2 = sum_{k in b} w_k |A_k|^2, the effective
//   template's power in the band), chi^2 = sum_b |z_b - u_b z|^2 / u_b  (2 (p - 1) dof).
// Band edges: w_k = 4 df |h_r,k|^2 / S_k on the reference band; e_b is one past the first bin at
// which the running sum (FP64, in k order from k_lo) reaches b W / p, W = the total.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace rfd {
namespace {

__global__ void k_band_edges(const PNParams *__restrict__ refs, const double *__restrict__ psd, double df,
                             int64_t k_lo, int32_t p, int32_t *__restrict__ edges) {
    if (threadIdx.x != 0) return;
    const int r = blockIdx.x;
    const int64_t k_hi = refs[r].k_hi;
    double W = 0.0;
    for (int64_t k = k_lo; k <= k_hi; ++k) {
        const double amp = pow((double)k * df, -7.0 / 6.0);
        W += 4.0 * df * (amp * amp) / psd[k];
    }
    int32_t *e = edges + (int64_t)r * (p + 1);
    e[0] = (int32_t)k_lo;
    e[p] = (int32_t)(k_hi + 1);
    double run = 0.0;
    int b = 1;
    for (int64_t k = k_lo; k <= k_hi && b < p; ++k) {
        const double amp = pow((double)k * df, -7.0 / 6.0);
        run += 4.0 * df * (amp * amp) / psd[k];
        while (b < p && run >= b * W / p) e[b++] = (int32_t)(k + 1);
    }
    while (b < p) e[b++] = (int32_t)(k_hi + 1);
}

// c[r p + b][k] = 4 df d conj(h_r) / S on the bins of band b, zero elsewhere (FP32, as the
// full-band reference filter forms it).
__global__ void __launch_bounds__(256) k_band_spectrum(const float2 *__restrict__ d, const double *__restrict__ psd,
                                                       const float2 *__restrict__ h, int64_t h_stride, double df,
                                                       int64_t n, const int32_t *__restrict__ edges, int32_t p,
                                                       int64_t row0, float2 *__restrict__ c) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = row0 + blockIdx.y;
    const int64_t r = row / p, b = row - r * p;
    const int32_t *e = edges + r * (p + 1);
    float2 out = make_float2(0.f, 0.f);
    if (k >= e[b] && k < e[b + 1]) {
        const float2 hv = h[r * h_stride + k];
        const float w = (float)(4.0 * df) / (float)psd[k];
        const float2 dv = d[k];
        out = make_float2(w * (dv.x * hv.x + dv.y * hv.y), w * (dv.y * hv.x - dv.x * hv.y));
    }
    c[(int64_t)blockIdx.y * n + k] = out;
}

__global__ void k_band_finalize(const float2 *__restrict__ q, int64_t n, int64_t ld, int64_t keep,
                                float2 *__restrict__ out) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= ld) return;
    const int64_t r = blockIdx.y;
    out[r * ld + m] = (m < keep) ? q[r * n + (m & (n - 1))] : make_float2(0.f, 0.f);
}

// Row b of `a`: the taps of template j[b] placed at (s + k) mod n, zero elsewhere.
__global__ void k_place_rows(const float2 *__restrict__ taps, int32_t k_stride, const int32_t *__restrict__ kk,
                             const int32_t *__restrict__ lag, int64_t j0, int64_t n, float2 *__restrict__ a) {
    const int64_t b = blockIdx.x, j = j0 + b;
    const int K = kk[j];
    const int64_t s = lag[j];
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        a[b * n + (((s + k) % n) + n) % n] = taps[j * k_stride + k];
}

__device__ __forceinline__ double bsum(double v, double *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    return t;
}

// u[j][b] = sum_{k in b} w_k |A_k|^2 / sum over all bands (A = forward transform of the placed taps).
__global__ void __launch_bounds__(256) k_band_shares(const float2 *__restrict__ A, int64_t n,
                                                     const int32_t *__restrict__ edges, int32_t p,
                                                     const int32_t *__restrict__ ref_of, const double *__restrict__ psd,
                                                     double df, int64_t j0, float *__restrict__ u) {
    __shared__ double sm[8];
    __shared__ double pw[64];
    const int64_t b = blockIdx.x, j = j0 + b;
    const int32_t *e = edges + (int64_t)ref_of[j] * (p + 1);
    double tot = 0.0;
    for (int q = 0; q < p; ++q) {
        double part = 0.0;
        for (int64_t k = e[q] + threadIdx.x; k < e[q + 1]; k += blockDim.x) {
            const double amp = pow((double)k * df, -7.0 / 6.0);
            const float2 a = A[b * n + k];
            part += 4.0 * df * (amp * amp) / psd[k] * ((double)a.x * a.x + (double)a.y * a.y);
        }
        const double v = bsum(part, sm);
        if (threadIdx.x == 0) pw[q] = v;
        tot += v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < p; q += blockDim.x) u[j * p + q] = tot > 0.0 ? (float)(pw[q] / tot) : 0.f;
}

// One block per trigger: the p sub-band ratio FIRs at the trigger's sample and chi^2.
__global__ void __launch_bounds__(128) k_subband_chi2(const float2 *__restrict__ qb, int64_t ld, int64_t n,
                                                      int32_t p, const float2 *__restrict__ taps, int32_t k_stride,
                                                      const int32_t *__restrict__ kk, const int32_t *__restrict__ lag,
                                                      const double *__restrict__ sigma, const float *__restrict__ u,
                                                      const int32_t *__restrict__ ref_of,
                                                      const rfd_trigger *__restrict__ trig, float *__restrict__ chi2,
                                                      float2 *__restrict__ zb_out) {
    __shared__ double sm[8];
    __shared__ double zr[64], zi[64];
    const int64_t i = blockIdx.x;
    const rfd_trigger T = trig[i];
    const int64_t j = T.j;
    const int K = kk[j];
    const int64_t s = lag[j];
    const int64_t r = ref_of[j];
    const double inv = sigma[j] > 0.0 ? 1.0 / sigma[j] : 0.0;
    for (int b = 0; b < p; ++b) {
        const float2 *q = qb + (r * p + b) * ld;
        double ar = 0.0, ai = 0.0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const float2 t = taps[j * k_stride + k];
            const float2 v = q[((((int64_t)T.t - s - k) % n) + n) % n];
            ar += (double)t.x * v.x - (double)t.y * v.y;
            ai += (double)t.x * v.y + (double)t.y * v.x;
        }
        ar = bsum(ar, sm);
        ai = bsum(ai, sm);
        if (threadIdx.x == 0) {
            zr[b] = ar * inv;
            zi[b] = ai * inv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Zr = 0.0, Zi = 0.0;
        for (int b = 0; b < p; ++b) {
            Zr += zr[b];
            Zi += zi[b];
        }
        double c = 0.0;
        for (int b = 0; b < p; ++b) {
            const double ub = u[j * p + b];
            if (ub > 0.0) {
                const double dr = zr[b] - ub * Zr, di = zi[b] - ub * Zi;
                c += (dr * dr + di * di) / ub;
            }
        }
        chi2[i] = (float)c;
    }
    if (zb_out)
        for (int b = threadIdx.x; b < p; b += blockDim.x) zb_out[i * p + b] = make_float2((float)zr[b], (float)zi[b]);
}

}  // namespace
}  // namespace rfd

struct rfd_subband {
    rfd_ctx *ctx = nullptr;
    rfd::Grid grid{};
    int32_t R = 0, p = 0;
    std::vector<rfd::PNParams> refs;
    std::vector<int32_t> edges;        // [R][p + 1]
    rfd::DevBuf d_edges, d_refs, d_ref_of, d_work;
    rfd::DevBuf w1, w2, w3;            // own FFT scratch (not the context's shared slots)
};

using namespace rfd;

extern "C" {

void rfd_subband_destroy(rfd_subband *S) {
    if (!S) return;
    release(S->d_edges);
    release(S->d_refs);
    release(S->d_ref_of);
    release(S->d_work);
    release(S->w1);
    release(S->w2);
    release(S->w3);
    delete S;
}

rfd_status rfd_subband_create(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev, const rfd_params *refs_host,
                              int32_t n_ref, int32_t p, rfd_subband **out) {
    RFD_REQUIRE(ctx && grid && psd_dev && refs_host && out, RFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1, RFD_ERR_SHAPE, "n_ref must be >= 1");
    RFD_REQUIRE(p >= 2 && p <= 64, RFD_ERR_ARG, "p=%d must be in [2, 64]", p);
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    rfd_subband *S = new rfd_subband();
    S->ctx = ctx;
    S->grid = g;
    S->R = n_ref;
    S->p = p;
    rfd_status st = RFD_OK;
    do {
        if ((st = make_pn_vec(g, refs_host, n_ref, &S->refs))) break;
        for (int32_t r = 0; r < n_ref && st == RFD_OK; ++r)
            if (S->refs[r].k_hi - g.k_lo + 1 < p) {
                set_error("reference %d has fewer band bins than sub-bands", r);
                st = RFD_ERR_ARG;
            }
        if (st) break;
        if ((st = ensure(S->d_refs, n_ref * sizeof(PNParams))) ||
            (st = ensure(S->d_edges, (size_t)n_ref * (p + 1) * sizeof(int32_t))))
            break;
        cudaError_t e = cudaMemcpy(S->d_refs.p, S->refs.data(), n_ref * sizeof(PNParams), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        k_band_edges<<<(unsigned)n_ref, 32>>>((const PNParams *)S->d_refs.p, psd_dev, g.df, g.k_lo, p,
                                              (int32_t *)S->d_edges.p);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("band edges failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        count_launch();
        S->edges.resize((size_t)n_ref * (p + 1));
        if ((e = cudaMemcpy(S->edges.data(), S->d_edges.p, S->edges.size() * 4, cudaMemcpyDeviceToHost)) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
        }
    } while (0);
    if (st) {
        rfd_subband_destroy(S);
        return st;
    }
    *out = S;
    return RFD_OK;
}

rfd_status rfd_subband_edges(const rfd_subband *S, int32_t *edges_host) {
    RFD_REQUIRE(S && edges_host, RFD_ERR_ARG, "NULL argument");
    std::copy(S->edges.begin(), S->edges.end(), edges_host);
    return RFD_OK;
}

rfd_status rfd_subband_filter_reference(rfd_subband *S, const void *dtilde_dev, const double *psd_dev,
                                        const void *href_dev, int32_t halo, void *qband_dev, void *stream) {
    RFD_REQUIRE(S && dtilde_dev && psd_dev && href_dev && qband_dev, RFD_ERR_ARG, "NULL argument");
    const Grid &g = S->grid;
    RFD_REQUIRE(halo >= 0 && halo < g.n, RFD_ERR_SHAPE, "halo=%d must be in [0, n)", halo);
    RFD_TRY_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    rfd_ctx *ctx = S->ctx;
    const int64_t n = g.n, ld = rfd_qref_ld(n, halo), rows = (int64_t)S->R * S->p;
    int64_t B = std::max<int64_t>(1, ((int64_t)1 << 30) / (n * (int64_t)sizeof(float2)));
    B = std::min<int64_t>(std::min<int64_t>(B, rows), 65535);
    RFD_TRY(ensure(S->w1, B * n * sizeof(float2)));
    RFD_TRY(ensure(S->w2, B * n * sizeof(float2)));
    RFD_TRY(ensure(S->w3, B * n * sizeof(float2)));
    float2 *c = (float2 *)S->w1.p, *q = (float2 *)S->w2.p;
    for (int64_t r0 = 0; r0 < rows; r0 += B) {
        const int64_t nb = std::min<int64_t>(B, rows - r0);
        k_band_spectrum<<<dim3((unsigned)(n / 256), (unsigned)nb), 256, 0, s>>>(
            (const float2 *)dtilde_dev, psd_dev, (const float2 *)href_dev, g.nf, g.df, n,
            (const int32_t *)S->d_edges.p, S->p, r0, c);
        RFD_LAUNCH_CHECK();
        RFD_TRY(fft_c2c<float>(ctx, n, nb, c, n, q, n, (float2 *)S->w3.p, true, s));
        k_band_finalize<<<dim3((unsigned)((ld + 255) / 256), (unsigned)nb), 256, 0, s>>>(q, n, ld, n + halo,
                                                                                       (float2 *)qband_dev + r0 * ld);
        RFD_LAUNCH_CHECK();
    }
    return RFD_OK;
}

rfd_status rfd_subband_shares(rfd_subband *S, const double *psd_dev, const void *taps_dev, int32_t k_stride,
                              const int32_t *k_dev, const int32_t *lag_dev, const int32_t *ref_of_host, int32_t n_tmpl,
                              float *u_dev, void *stream) {
    RFD_REQUIRE(S && psd_dev && taps_dev && k_dev && lag_dev && ref_of_host && u_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n_tmpl >= 0 && k_stride >= 1, RFD_ERR_SHAPE, "bad shape");
    if (n_tmpl == 0) return RFD_OK;
    for (int32_t j = 0; j < n_tmpl; ++j)
        RFD_REQUIRE(ref_of_host[j] >= 0 && ref_of_host[j] < S->R, RFD_ERR_ARG, "ref_of[%d]=%d out of range", j,
                    ref_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    rfd_ctx *ctx = S->ctx;
    const Grid &g = S->grid;
    const int64_t n = g.n;
    RFD_TRY(ensure(S->d_ref_of, (size_t)n_tmpl * 4));
    RFD_TRY_CUDA(cudaMemcpyAsync(S->d_ref_of.p, ref_of_host, (size_t)n_tmpl * 4, cudaMemcpyHostToDevice, s));
    int64_t B = std::max<int64_t>(1, ((int64_t)1 << 30) / (n * (int64_t)sizeof(float2)));
    B = std::min<int64_t>(B, n_tmpl);
    RFD_TRY(ensure(S->w1, B * n * sizeof(float2)));
    RFD_TRY(ensure(S->w2, B * n * sizeof(float2)));
    RFD_TRY(ensure(S->w3, B * n * sizeof(float2)));
    float2 *a = (float2 *)S->w1.p, *A = (float2 *)S->w2.p;
    for (int64_t j0 = 0; j0 < n_tmpl; j0 += B) {
        const int64_t nb = std::min<int64_t>(B, n_tmpl - j0);
        RFD_TRY_CUDA(cudaMemsetAsync(a, 0, nb * n * sizeof(float2), s));
        k_place_rows<<<(unsigned)nb, 128, 0, s>>>((const float2 *)taps_dev, k_stride, k_dev, lag_dev, j0, n, a);
        RFD_LAUNCH_CHECK();
        RFD_TRY(fft_c2c<float>(ctx, n, nb, a, n, A, n, (float2 *)S->w3.p, false, s));
        k_band_shares<<<(unsigned)nb, 256, 0, s>>>(A, n, (const int32_t *)S->d_edges.p, S->p,
                                                   (const int32_t *)S->d_ref_of.p, psd_dev, g.df, j0, u_dev);
        RFD_LAUNCH_CHECK();
    }
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return RFD_OK;
}

rfd_status rfd_subband_chi2(rfd_subband *S, const void *qband_dev, int32_t halo, const void *taps_dev,
                            int32_t k_stride, const int32_t *k_dev, const int32_t *lag_dev, const double *sigma_dev,
                            const float *u_dev, const int32_t *ref_of_host, int32_t n_tmpl,
                            const rfd_trigger *trig_dev, int64_t n_trig, float *chi2_dev, void *zb_dev, void *stream) {
    RFD_REQUIRE(S && qband_dev && taps_dev && k_dev && lag_dev && sigma_dev && u_dev && ref_of_host && chi2_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n_trig >= 0 && n_tmpl >= 1, RFD_ERR_SHAPE, "bad shape");
    if (n_trig == 0) return RFD_OK;
    RFD_REQUIRE(trig_dev, RFD_ERR_ARG, "NULL triggers");
    for (int32_t j = 0; j < n_tmpl; ++j)
        RFD_REQUIRE(ref_of_host[j] >= 0 && ref_of_host[j] < S->R, RFD_ERR_ARG, "ref_of[%d]=%d out of range", j,
                    ref_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(ensure(S->d_ref_of, (size_t)n_tmpl * 4));
    RFD_TRY_CUDA(cudaMemcpyAsync(S->d_ref_of.p, ref_of_host, (size_t)n_tmpl * 4, cudaMemcpyHostToDevice, s));
    const int64_t ld = rfd_qref_ld(S->grid.n, halo);
    k_subband_chi2<<<(unsigned)n_trig, 128, 0, s>>>((const float2 *)qband_dev, ld, S->grid.n, S->p,
                                                    (const float2 *)taps_dev, k_stride, k_dev, lag_dev, sigma_dev,
                                                    u_dev, (const int32_t *)S->d_ref_of.p, trig_dev, chi2_dev,
                                                    (float2 *)zb_dev);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return RFD_OK;
}

}  // extern "C"
