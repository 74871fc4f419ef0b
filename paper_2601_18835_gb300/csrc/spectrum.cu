// Templates (FP64 TaylorF2 phase), the matched-filter spectrum of Eq. 1, the reference
// series of Eq. 3 (filter_reference) and the FINDCHIRP comparison path.
#include <cmath>

#include "epilogue.cuh"
#include "internal.cuh"

namespace rfd {

namespace {

// h(f_k) = f^(-7/6) exp(-i Psi(f_k)) inside the template's band, 0 elsewhere; FP64 phase.
__global__ void k_gen_templates(const PNParams *__restrict__ pn, int flags, double df, int64_t nf,
                                int64_t k_lo, float2 *__restrict__ h) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const int64_t row = blockIdx.y;
    const PNParams p = pn[row];
    float2 out = make_float2(0.f, 0.f);
    if (k >= k_lo && k <= p.k_hi) {
        const double f = (double)k * df;
        const double psi = pn_phase(f, p, flags);
        double s, c;
        sincos(psi, &s, &c);
        const double amp = pow(f, -7.0 / 6.0);
        out = make_float2((float)(amp * c), (float)(-amp * s));
    }
    h[row * nf + k] = out;
}

// Block-wide FP64 sum in a fixed order (deterministic); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sm[i];
    __syncthreads();
    return r;
}

// Block-wide FP32 sum in a fixed order; result valid in thread 0.
__device__ __forceinline__ float block_sum_f(float v, float *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sm[i];
    __syncthreads();
    return r;
}

// c[row][k] = 4 df d[k] conj(h_row[k]) / S[k] for k <= n/2 from a stored template row (zero
// outside its band), 0 for k > n/2: the discretised integrand of Eq. 1, in FP32.  Per block,
// partial sums of |c|^2 and of 4 df |h|^2 / S (sigma^2 of the row's template); the partials
// are summed in FP64 in a fixed order afterwards, so the result is deterministic.
__global__ void __launch_bounds__(256) k_spectrum_stored(
    const float2 *__restrict__ d, const double *__restrict__ psd, const float2 *__restrict__ h,
    int64_t h_stride, double df, int64_t n, float2 *__restrict__ c, int64_t c_stride,
    double *__restrict__ part_c, double *__restrict__ part_s) {
    __shared__ float sm[8];
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = blockIdx.y;
    float cr = 0.f, ci = 0.f, sg = 0.f;
    if (k <= n / 2) {
        const float2 hv = h[row * h_stride + k];
        if (hv.x != 0.f || hv.y != 0.f) {
            const float w = (float)(4.0 * df) / (float)psd[k];
            const float2 dv = d[k];
            // d conj(h) = (dr hr + di hi) + i (di hr - dr hi)
            cr = w * (dv.x * hv.x + dv.y * hv.y);
            ci = w * (dv.y * hv.x - dv.x * hv.y);
            sg = w * (hv.x * hv.x + hv.y * hv.y);
        }
    }
    c[row * c_stride + k] = make_float2(cr, ci);
    const float pc = block_sum_f(cr * cr + ci * ci, sm);
    const float ps = block_sum_f(sg, sm);
    if (threadIdx.x == 0) {
        part_c[row * gridDim.x + blockIdx.x] = (double)pc;
        part_s[row * gridDim.x + blockIdx.x] = (double)ps;
    }
}

// out[row] = sum of the row's partials, in index order.
__global__ void k_sum_rows(const double *__restrict__ part, int64_t nparts, double *__restrict__ out) {
    __shared__ double sm[8];
    const int64_t row = blockIdx.x;
    double v = 0.0;
    // each thread sums a contiguous chunk, then a fixed-order block reduction
    const int64_t per = (nparts + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(nparts, b + per);
    for (int64_t i = b; i < e; ++i) v += part[row * nparts + i];
    v = block_sum(v, sm);
    if (threadIdx.x == 0) out[row] = v;
}

// Largest |Re q| or |Im q| of each reference's series (float bits of a non-negative value
// order like the values, so an integer maximum is exact); qmax zeroed beforehand.
__global__ void k_qmax(const float2 *__restrict__ q, int64_t n, uint32_t *__restrict__ qmax) {
    const int64_t r = blockIdx.y;
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = q[r * n + i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&qmax[r], __float_as_uint(m));
}

// Per-reference power-of-two scale: the rms of q is sqrt(sum_k |c_k|^2) for the unnormalised
// inverse transform; e_r puts it near 2^8 so the fp16 hi part keeps >= 8 bits of headroom, and
// no lower than needed to keep the largest component of the series at or below 2^14 (fp16's
// largest finite value is 65504), so that a very loud sample (a glitch or a strong signal,
// more than 64 times the rms) cannot overflow the hi part.
__global__ void k_qscale(const double *__restrict__ pow_c, const uint32_t *__restrict__ qmax, int n_ref,
                         int precision, int32_t *__restrict__ e) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ref) return;
    int v = 0;
    if (precision != RFD_PREC_FP32 && pow_c[r] > 0.0) {
        const double rms = sqrt(pow_c[r]);
        v = (int)nearbyint(8.0 - log2(rms));
        const double mx = (double)__uint_as_float(qmax[r]);
        if (mx > 0.0) v = min(v, (int)floor(14.0 - log2(mx)));
        v = max(-120, min(120, v));
    }
    e[r] = v;
}

__global__ void k_finalize_fp32(const float2 *__restrict__ q, int64_t n, int64_t ld, int64_t keep,
                                float2 *__restrict__ out) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= ld) return;
    const int64_t r = blockIdx.y;
    out[r * ld + m] = (m < keep) ? q[r * n + (m & (n - 1))] : make_float2(0.f, 0.f);
}

template <typename H>
__device__ __forceinline__ H to_h(float x);
template <>
__device__ __forceinline__ __half to_h<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_h<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float from_h(__half x) { return __half2float(x); }
__device__ __forceinline__ float from_h(__nv_bfloat16 x) { return __bfloat162float(x); }

// hi = round(x 2^e), lo = round(x 2^e - hi), separately for Re and Im; planes
// (re_hi, im_hi, re_lo, im_lo) of ld elements each, wrap halo, zero padding.
template <typename H>
__global__ void k_finalize_split(const float2 *__restrict__ q, int64_t n, int64_t ld, int64_t keep,
                                 const int32_t *__restrict__ e, H *__restrict__ out) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= ld) return;
    const int64_t r = blockIdx.y;
    H rh = to_h<H>(0.f), ih = rh, rl = rh, il = rh;
    if (m < keep) {
        const float2 x = q[r * n + (m & (n - 1))];
        const float xr = ldexpf(x.x, e[r]), xi = ldexpf(x.y, e[r]);
        rh = to_h<H>(xr);
        ih = to_h<H>(xi);
        rl = to_h<H>(xr - from_h(rh));
        il = to_h<H>(xi - from_h(ih));
    }
    H *base = out + (4 * r) * ld;
    base[m] = rh;
    base[ld + m] = ih;
    base[2 * ld + m] = rl;
    base[3 * ld + m] = il;
}

// FINDCHIRP weights, k < n/2: GW[k] = (Re G, Im G, Wt, 0) with Wt = 4 df / S and G = Wt d on the
// data band [k_lo, n/2), 0 elsewhere.
__global__ void k_fc_weights(const float2 *__restrict__ d, const double *__restrict__ psd, double df, int64_t k_lo,
                             int64_t half, float4 *__restrict__ GW) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= half) return;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= k_lo) {
        const float w = (float)(4.0 * df) / (float)psd[k];
        const float2 dv = d[k];
        out = make_float4(w * dv.x, w * dv.y, w, 0.f);
    }
    GW[k] = out;
}

}  // namespace

rfd_status gen_templates_impl(rfd_ctx *ctx, const Grid &g, const std::vector<PNParams> &pn,
                              float2 *h, cudaStream_t s) {
    const int64_t rows = (int64_t)pn.size();
    if (rows == 0) return RFD_OK;
    RFD_TRY(ensure(ctx->ws[0], rows * sizeof(PNParams)));
    RFD_TRY_CUDA(cudaMemcpyAsync(ctx->ws[0].p, pn.data(), rows * sizeof(PNParams),
                                 cudaMemcpyHostToDevice, s));
    for (int64_t r0 = 0; r0 < rows; r0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(65535, rows - r0);
        dim3 grid((unsigned)((g.nf + 255) / 256), gy);
        k_gen_templates<<<grid, 256, 0, s>>>((const PNParams *)ctx->ws[0].p + r0, g.pn_flags, g.df,
                                             g.nf, g.k_lo, h + r0 * g.nf);
        RFD_LAUNCH_CHECK();
    }
    // the parameter upload must finish before ws[0] can be reused by a later call
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return RFD_OK;
}

// Workspace slots: ws[1] spectrum c, ws[2] FFT output, ws[3] FFT tmp, ws[4] partials,
// ws[5] per-row sums.
rfd_status filter_reference_impl(rfd_ctx *ctx, const Grid &g, const float2 *d, const double *psd,
                                 const float2 *href, int64_t R, int32_t halo, int32_t precision,
                                 void *qref, int32_t *qscale, cudaStream_t s) {
    const int64_t n = g.n, ld = rfd_qref_ld(n, halo);
    const unsigned nblk = (unsigned)(n / 256);
    RFD_TRY(ensure(ctx->ws[1], R * n * sizeof(float2)));
    RFD_TRY(ensure(ctx->ws[2], R * n * sizeof(float2)));
    RFD_TRY(ensure(ctx->ws[3], R * n * sizeof(float2)));
    RFD_TRY(ensure(ctx->ws[4], 2 * R * nblk * sizeof(double)));
    RFD_TRY(ensure(ctx->ws[5], 2 * R * sizeof(double) + R * sizeof(uint32_t)));
    float2 *c = (float2 *)ctx->ws[1].p;
    double *part = (double *)ctx->ws[4].p;
    double *sums = (double *)ctx->ws[5].p;
    uint32_t *qmax = (uint32_t *)(sums + 2 * R);
    for (int64_t r0 = 0; r0 < R; r0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(65535, R - r0);
        k_spectrum_stored<<<dim3(nblk, gy), 256, 0, s>>>(d, psd, href + r0 * g.nf, g.nf, g.df, n, c + r0 * n, n,
                                                         part + r0 * nblk, part + R * nblk + r0 * nblk);
        RFD_LAUNCH_CHECK();
    }
    k_sum_rows<<<(unsigned)R, 256, 0, s>>>(part, nblk, sums);
    RFD_LAUNCH_CHECK();
    float2 *q = (float2 *)ctx->ws[2].p;
    RFD_TRY(fft_c2c<float>(ctx, n, R, c, n, q, n, (float2 *)ctx->ws[3].p, true, s));
    if (precision != RFD_PREC_FP32) {
        RFD_TRY_CUDA(cudaMemsetAsync(qmax, 0, R * sizeof(uint32_t), s));
        for (int64_t r0 = 0; r0 < R; r0 += 65535) {
            const unsigned gy = (unsigned)std::min<int64_t>(65535, R - r0);
            k_qmax<<<dim3((unsigned)std::min<int64_t>(64, (n + 255) / 256), gy), 256, 0, s>>>(q + r0 * n, n,
                                                                                            qmax + r0);
            RFD_LAUNCH_CHECK();
        }
    }
    k_qscale<<<(unsigned)((R + 127) / 128), 128, 0, s>>>(sums, qmax, (int)R, precision, qscale);
    RFD_LAUNCH_CHECK();
    const int64_t keep = n + halo;
    for (int64_t r0 = 0; r0 < R; r0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(65535, R - r0);
        dim3 grid((unsigned)((ld + 255) / 256), gy);
        if (precision == RFD_PREC_FP32) {
            k_finalize_fp32<<<grid, 256, 0, s>>>(q + r0 * n, n, ld, keep, (float2 *)qref + r0 * ld);
        } else if (precision == RFD_PREC_FP16X3) {
            k_finalize_split<__half><<<grid, 256, 0, s>>>(q + r0 * n, n, ld, keep, qscale + r0,
                                                          (__half *)qref + 4 * r0 * ld);
        } else {
            k_finalize_split<__nv_bfloat16><<<grid, 256, 0, s>>>(
                q + r0 * n, n, ld, keep, qscale + r0, (__nv_bfloat16 *)qref + 4 * r0 * ld);
        }
        RFD_LAUNCH_CHECK();
    }
    return RFD_OK;
}

// FINDCHIRP over all templates in batches from stored templates, two fused kernels per batch
// (fft.cu: findchirp_fused); candidates as in the ratio-filter epilogue.  Batches keep the
// intermediate array near 64 MB so that it stays in the 126 MB L2 between the passes.
rfd_status findchirp_impl(rfd_ctx *ctx, const Grid &g, const float2 *d, const double *psd, const float2 *h,
                          int64_t J, int32_t W, float thr, rfd_candidate *cand, int64_t cap, int64_t *count,
                          cudaStream_t s) {
    const int64_t n = g.n, half = n / 2;
    const int64_t B = std::max<int64_t>(1, std::min<int64_t>(J, ((int64_t)64 << 20) / (n * (int64_t)sizeof(float2))));
    RFD_TRY(ensure(ctx->ws[1], (size_t)half * sizeof(float4)));
    RFD_TRY(ensure(ctx->ws[2], (size_t)B * n * sizeof(float2)));
    RFD_TRY(ensure(ctx->ws[4], (size_t)B * 2048 * sizeof(double)));
    RFD_TRY(ensure(ctx->ws[5], (size_t)B * sizeof(double)));
    float4 *GW = (float4 *)ctx->ws[1].p;
    RFD_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
    k_fc_weights<<<(unsigned)((half + 255) / 256), 256, 0, s>>>(d, psd, g.df, g.k_lo, half, GW);
    RFD_LAUNCH_CHECK();
    for (int64_t j0 = 0; j0 < J; j0 += B) {
        const int64_t b = std::min<int64_t>(B, J - j0);
        RFD_TRY(findchirp_fused(ctx, n, b, GW, h + j0 * g.nf, g.nf, (int32_t)j0, thr, W, (float2 *)ctx->ws[2].p,
                                (double *)ctx->ws[4].p, (double *)ctx->ws[5].p, cand, cap, count, s));
    }
    return RFD_OK;
}

}  // namespace rfd
