// make_taps: ratio-filter taps, lags, sigma_eff and tap match (Eq. 2, Eq. 3, Sec. V,
// Eqs. 5-6), all in FP64 on the device.
//
// Per batch of templates:
//   1. G = conj(h_j / h_r) from the FP64 phase difference in the reference band (0 above the
//      template's cutoff), linear magnitude / shortest-arc phase fill on the out-of-band arc;
//   2. g = IDFT_n(G) (FP64 Stockham; the 1/n is applied when the taps are cut);
//   3. E[s] = sum_k w[k]^2 |g[(s+k) mod n]|^2 for every s, its maximum, then the tie rule
//      (within 1e-9 of the maximum; closest to s = -K/2, then smaller s);
//   4. rho[k] = w[k] g[(s+k) mod n] / n;
//   5. sigma_eff^2 = sum_{a,b} rho[a] conj(rho[b]) C_r[b-a] (C_r from one FP64 IDFT per
//      reference of 4 df |h_r|^2 / S);
//   6. optionally the match of h_eff = h_r conj(DFT(placed taps)) with h_j.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace rfd {

namespace {

struct TapJob {          // one template of the current batch
    PNParams tj;         // template
    PNParams tr;         // its reference
    int32_t K;
    int32_t ref;
    double ma, pa, mb, dp;   // fill end points
};

__device__ __forceinline__ double tukey_w(int k, int K, double alpha) {
    if (K == 1 || alpha <= 0.0) return 1.0;
    if (alpha >= 1.0) return 0.5 * (1.0 - cos(2.0 * kPi * (double)k / (double)(K - 1)));
    const double width = alpha * (double)(K - 1) / 2.0;
    const double x = (double)k;
    if (x < width) return 0.5 * (1.0 + cos(kPi * (x / width - 1.0)));
    if (x > (double)(K - 1) - width) return 0.5 * (1.0 + cos(kPi * (x / width - 2.0 / alpha + 1.0)));
    return 1.0;
}

// fill end points G[k_hi_r] and G[k_lo]
__global__ void k_fill_ends(TapJob *jobs, int nb, int flags, double df, int64_t k_lo) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    TapJob &J = jobs[b];
    const int64_t k_hi = J.tr.k_hi;
    const int64_t k_top = min(k_hi, J.tj.k_hi);
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    if (k_top >= k_lo) {
        double s, c;
        const double fl = (double)k_lo * df;
        sincos(pn_phase(fl, J.tj, flags) - pn_phase(fl, J.tr, flags), &s, &c);
        br = c;
        bi = s;
        if (k_top == k_hi) {
            const double fh = (double)k_hi * df;
            sincos(pn_phase(fh, J.tj, flags) - pn_phase(fh, J.tr, flags), &s, &c);
            ar = c;
            ai = s;
        }
    }
    J.ma = hypot(ar, ai);
    J.mb = hypot(br, bi);
    J.pa = atan2(ai, ar);
    const double pb = atan2(bi, br);
    double dp = pb - J.pa;
    dp -= 2.0 * kPi * floor((dp + kPi) / (2.0 * kPi));
    J.dp = dp;
}

__global__ void __launch_bounds__(256) k_ratio_spectrum(const TapJob *__restrict__ jobs, int flags,
                                                        double df, int64_t n, int64_t k_lo,
                                                        double2 *__restrict__ G) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = blockIdx.y;
    const TapJob &J = jobs[b];
    const int64_t k_hi = J.tr.k_hi;
    const int64_t k_top = min(k_hi, J.tj.k_hi);
    double2 out;
    if (k >= k_lo && k <= k_hi) {
        if (k <= k_top) {
            const double f = (double)k * df;
            double s, c;
            sincos(pn_phase(f, J.tj, flags) - pn_phase(f, J.tr, flags), &s, &c);
            out = make_double2(c, s);
        } else {
            out = make_double2(0.0, 0.0);
        }
    } else {
        const int64_t L = n - (k_hi - k_lo + 1);
        const int64_t i = (k - k_hi + n) % n;        // 1 .. L along the arc
        const double s = (double)i / (double)(L + 1);
        const double mag = (1.0 - s) * J.ma + s * J.mb;
        double sn, cs;
        sincos(J.pa + s * J.dp, &sn, &cs);
        out = make_double2(mag * cs, mag * sn);
    }
    G[(int64_t)b * n + k] = out;
}

// E[s] for s = i - n/2, i in [0, n); 256 consecutive s per block; per-template maximum.
__global__ void __launch_bounds__(256) k_window_energy(const TapJob *__restrict__ jobs,
                                                       const double2 *__restrict__ g, int64_t n,
                                                       double alpha, double *__restrict__ E,
                                                       unsigned long long *__restrict__ emax) {
    extern __shared__ double sh[];
    const int b = blockIdx.y;
    const int K = jobs[b].K;
    double *w2 = sh;                 // [K]
    double *e = sh + K;              // [256 + K - 1]
    const int64_t i0 = (int64_t)blockIdx.x * 256;
    const int64_t s0 = i0 - n / 2;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double w = tukey_w(k, K, alpha);
        w2[k] = w * w;
    }
    const double2 *gb = g + (int64_t)b * n;
    for (int t = threadIdx.x; t < 256 + K - 1; t += blockDim.x) {
        const int64_t m = ((s0 + t) % n + n) % n;
        const double2 v = gb[m];
        e[t] = v.x * v.x + v.y * v.y;
    }
    __syncthreads();
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += w2[k] * e[threadIdx.x + k];
    E[(int64_t)b * n + i0 + threadIdx.x] = acc;
    // block max (E >= 0, so the bit patterns order like the values)
    unsigned long long bits = (unsigned long long)__double_as_longlong(acc);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&emax[b], bits);
}

__global__ void __launch_bounds__(256) k_lag_select(const TapJob *__restrict__ jobs,
                                                    const double *__restrict__ E, int64_t n,
                                                    const unsigned long long *__restrict__ emax,
                                                    unsigned long long *__restrict__ lagkey) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = blockIdx.y;
    const double em = __longlong_as_double((long long)emax[b]);
    if (E[(int64_t)b * n + i] >= em * (1.0 - 1e-9)) {
        const int64_t s = i - n / 2;
        const int64_t K = jobs[b].K;
        const int64_t d = s + K / 2 < 0 ? -(s + K / 2) : s + K / 2;
        const unsigned long long key = ((unsigned long long)d << 32) | (unsigned long long)i;
        atomicMin(&lagkey[b], key);
    }
}

// rho[k] = w[k] g[(s+k) mod n] / n; also the placed-taps row for the match FFT.
__global__ void k_place(const TapJob *__restrict__ jobs, const double2 *__restrict__ g, int64_t n,
                        double alpha, const unsigned long long *__restrict__ lagkey, int32_t j0,
                        int32_t k_stride, double2 *__restrict__ rho64, float2 *__restrict__ taps,
                        int32_t *__restrict__ lag, double2 *__restrict__ placed) {
    const int b = blockIdx.x;
    const int K = jobs[b].K;
    const int64_t s = (int64_t)(lagkey[b] & 0xffffffffull) - n / 2;
    if (threadIdx.x == 0) lag[j0 + b] = (int32_t)s;
    const double inv_n = 1.0 / (double)n;
    for (int k = threadIdx.x; k < k_stride; k += blockDim.x) {
        double2 r = make_double2(0.0, 0.0);
        if (k < K) {
            const int64_t m = ((s + k) % n + n) % n;
            const double w = tukey_w(k, K, alpha);
            const double2 v = g[(int64_t)b * n + m];
            r = make_double2(w * (v.x * inv_n), w * (v.y * inv_n));
            if (placed) placed[(int64_t)b * n + m] = r;
        }
        rho64[(int64_t)b * k_stride + k] = r;
        taps[(int64_t)(j0 + b) * k_stride + k] = make_float2((float)r.x, (float)r.y);
    }
}

__device__ __forceinline__ double block_sum_d(double v, double *sm) {
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

// 4 df |h_r|^2 / S on the reference band, as complex rows for the C_r transform.
__global__ void k_ref_weight(const PNParams *__restrict__ refs, const double *__restrict__ psd,
                             double df, int64_t n, int64_t k_lo, double2 *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int r = blockIdx.y;
    double v = 0.0;
    if (k >= k_lo && k <= refs[r].k_hi) {
        const double f = (double)k * df;
        const double amp = pow(f, -7.0 / 6.0);
        v = 4.0 * df * (amp * amp) / psd[k];
    }
    out[(int64_t)r * n + k] = make_double2(v, 0.0);
}

// Cc[r][l + kmax - 1] = C_r[l] for |l| < kmax, from the full inverse transform rows.
__global__ void k_compact_C(const double2 *__restrict__ full, int64_t n, int32_t kmax,
                            double2 *__restrict__ Cc) {
    const int r = blockIdx.x;
    const int32_t width = 2 * kmax - 1;
    for (int32_t i = threadIdx.x; i < width; i += blockDim.x) {
        const int64_t l = (int64_t)i - (kmax - 1);
        Cc[(int64_t)r * width + i] = full[(int64_t)r * n + ((l % n) + n) % n];
    }
}

// sigma_eff^2 = Re sum_a rho[a] sum_b conj(rho[b]) C[b - a] (Eq. 6 over the taps).
__global__ void __launch_bounds__(256) k_sigma_eff(const TapJob *__restrict__ jobs,
                                                   const double2 *__restrict__ rho64,
                                                   int32_t k_stride, const double2 *__restrict__ Cc,
                                                   int32_t kmax, int32_t j0,
                                                   double *__restrict__ sigma) {
    __shared__ double sm[8];
    extern __shared__ double2 rs[];
    const int b = blockIdx.x;
    const int K = jobs[b].K;
    const double2 *Cr = Cc + (int64_t)jobs[b].ref * (2 * kmax - 1) + (kmax - 1);
    for (int k = threadIdx.x; k < K; k += blockDim.x) rs[k] = rho64[(int64_t)b * k_stride + k];
    __syncthreads();
    double part = 0.0;
    for (int a = threadIdx.x; a < K; a += blockDim.x) {
        double ir = 0.0, ii = 0.0;
        for (int bb = 0; bb < K; ++bb) {
            const double2 c = Cr[bb - a];
            const double2 r = rs[bb];
            // conj(r) * c
            ir += r.x * c.x + r.y * c.y;
            ii += r.x * c.y - r.y * c.x;
        }
        const double2 ra = rs[a];
        part += ra.x * ir - ra.y * ii;
    }
    const double tot = block_sum_d(part, sm);
    if (threadIdx.x == 0) sigma[j0 + b] = sqrt(tot);
}

// Per-block partial sums of <h_j, h_eff>, |h_j|^2, |h_eff|^2 (all / S), k in [0, n/2].
__global__ void __launch_bounds__(256) k_match_partial(const TapJob *__restrict__ jobs, int flags,
                                                       const double *__restrict__ psd, double df,
                                                       int64_t n, int64_t k_lo,
                                                       const double2 *__restrict__ A,
                                                       double *__restrict__ part) {
    __shared__ double sm[8];
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const TapJob &J = jobs[b];
    double ir = 0.0, ii = 0.0, sj = 0.0, se = 0.0;
    if (k <= n / 2 && k >= k_lo) {
        const double f = (double)k * df;
        const double amp = pow(f, -7.0 / 6.0);
        const double S = psd[k];
        double hjr = 0.0, hji = 0.0, her = 0.0, hei = 0.0;
        if (k <= J.tj.k_hi) {
            double s, c;
            sincos(pn_phase(f, J.tj, flags), &s, &c);
            hjr = amp * c;
            hji = -amp * s;
        }
        if (k <= J.tr.k_hi) {
            double s, c;
            sincos(pn_phase(f, J.tr, flags), &s, &c);
            const double hrr = amp * c, hri = -amp * s;
            const double2 a = A[(int64_t)b * n + k];
            // h_eff = h_r conj(A)
            her = hrr * a.x + hri * a.y;
            hei = hri * a.x - hrr * a.y;
        }
        // conj(h_j) h_eff / S
        ir = (hjr * her + hji * hei) / S;
        ii = (hjr * hei - hji * her) / S;
        sj = (hjr * hjr + hji * hji) / S;
        se = (her * her + hei * hei) / S;
    }
    const int64_t nb = gridDim.x;
    const double v0 = block_sum_d(ir, sm), v1 = block_sum_d(ii, sm);
    const double v2 = block_sum_d(sj, sm), v3 = block_sum_d(se, sm);
    if (threadIdx.x == 0) {
        double *p = part + ((int64_t)b * 4) * nb;
        p[blockIdx.x] = v0;
        p[nb + blockIdx.x] = v1;
        p[2 * nb + blockIdx.x] = v2;
        p[3 * nb + blockIdx.x] = v3;
    }
}

__global__ void k_match_final(const double *__restrict__ part, int64_t nb, int32_t j0,
                              double *__restrict__ match) {
    __shared__ double sm[8];
    const int b = blockIdx.x;
    double v[4];
    for (int q = 0; q < 4; ++q) {
        const double *p = part + ((int64_t)b * 4 + q) * nb;
        const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
        const int64_t lo = threadIdx.x * per, hi = min(nb, lo + per);
        double a = 0.0;
        for (int64_t i = lo; i < hi; ++i) a += p[i];
        v[q] = block_sum_d(a, sm);
    }
    if (threadIdx.x == 0) match[j0 + b] = hypot(v[0], v[1]) / sqrt(v[2] * v[3]);
}

}  // namespace

// Workspace slots: ws[6] jobs, ws[7] G / placed taps, ws[8] g / A, ws[9] FFT tmp, ws[10] E,
// ws[11] per-template scalars (emax, lagkey) + rho64 + C_r rows + match partials.
rfd_status make_taps_impl(rfd_ctx *ctx, const Grid &g, const double *psd,
                          const std::vector<PNParams> &refs, const std::vector<PNParams> &tmpl,
                          const std::vector<int32_t> &ref_of, const std::vector<int32_t> &K,
                          int32_t k_stride, double alpha, float2 *taps, int32_t *lag,
                          double *sigma, double *match, cudaStream_t s) {
    const int64_t n = g.n;
    const int64_t J = (int64_t)tmpl.size(), R = (int64_t)refs.size();
    int64_t B = std::max<int64_t>(1, ((int64_t)2 << 30) / (n * 56));
    B = std::min<int64_t>(std::min<int64_t>(B, J), 4096);
    const int64_t nb_match = (n / 2 + 1 + 255) / 256;
    // C_r rows (complex, n each) live after the per-batch scalars in ws[11]
    const size_t off_lagkey = B * sizeof(unsigned long long);
    const size_t off_rho = 2 * off_lagkey;
    int kmax = 0;
    for (int64_t i = 0; i < J; ++i) kmax = std::max(kmax, K[i]);
    const size_t off_C = off_rho + (size_t)B * k_stride * sizeof(double2);
    const size_t off_part = off_C + (size_t)R * (2 * kmax - 1) * sizeof(double2);
    const size_t ws11 = off_part + (size_t)B * 4 * nb_match * sizeof(double);
    RFD_TRY(ensure(ctx->ws[6], B * sizeof(TapJob)));
    RFD_TRY(ensure(ctx->ws[7], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[8], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[9], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[10], B * n * sizeof(double)));
    RFD_TRY(ensure(ctx->ws[11], ws11));
    RFD_TRY(ensure(ctx->ws[0], R * sizeof(PNParams)));
    char *base11 = (char *)ctx->ws[11].p;
    unsigned long long *emax = (unsigned long long *)base11;
    unsigned long long *lagkey = (unsigned long long *)(base11 + off_lagkey);
    double2 *rho64 = (double2 *)(base11 + off_rho);
    double2 *C = (double2 *)(base11 + off_C);
    double *part = (double *)(base11 + off_part);
    double2 *Gb = (double2 *)ctx->ws[7].p, *gb = (double2 *)ctx->ws[8].p, *tmp = (double2 *)ctx->ws[9].p;
    double *E = (double *)ctx->ws[10].p;

    // C_r[l] = sum_k 4 df |h_r|^2/S exp(+2 pi i k l / n): one inverse FFT per reference
    RFD_TRY_CUDA(cudaMemcpyAsync(ctx->ws[0].p, refs.data(), R * sizeof(PNParams),
                                 cudaMemcpyHostToDevice, s));
    k_ref_weight<<<dim3((unsigned)((n + 255) / 256), (unsigned)R), 256, 0, s>>>(
        (const PNParams *)ctx->ws[0].p, psd, g.df, n, g.k_lo, gb);
    RFD_LAUNCH_CHECK();
    RFD_TRY(fft_c2c<double>(ctx, n, R, gb, n, Gb, n, tmp, true, s));
    k_compact_C<<<(unsigned)R, 256, 0, s>>>(Gb, n, kmax, C);
    RFD_LAUNCH_CHECK();

    std::vector<TapJob> jobs(B);
    for (int64_t j0 = 0; j0 < J; j0 += B) {
        const int64_t nbt = std::min<int64_t>(B, J - j0);
        int kb = 0;
        for (int64_t b = 0; b < nbt; ++b) {
            TapJob &jb = jobs[b];
            jb = TapJob{};
            jb.tj = tmpl[j0 + b];
            jb.ref = ref_of[j0 + b];
            jb.tr = refs[jb.ref];
            jb.K = K[j0 + b];
            kb = std::max(kb, jb.K);
        }
        TapJob *dj = (TapJob *)ctx->ws[6].p;
        RFD_TRY_CUDA(cudaMemcpyAsync(dj, jobs.data(), nbt * sizeof(TapJob), cudaMemcpyHostToDevice, s));
        k_fill_ends<<<(unsigned)((nbt + 127) / 128), 128, 0, s>>>(dj, (int)nbt, g.pn_flags, g.df, g.k_lo);
        RFD_LAUNCH_CHECK();
        k_ratio_spectrum<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, g.pn_flags, g.df,
                                                                               n, g.k_lo, Gb);
        RFD_LAUNCH_CHECK();
        RFD_TRY(fft_c2c<double>(ctx, n, nbt, Gb, n, gb, n, tmp, true, s));
        RFD_TRY_CUDA(cudaMemsetAsync(emax, 0, nbt * sizeof(unsigned long long), s));
        RFD_TRY_CUDA(cudaMemsetAsync(lagkey, 0xff, nbt * sizeof(unsigned long long), s));
        const size_t shm = (size_t)(kb + 256 + kb) * sizeof(double);
        k_window_energy<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, shm, s>>>(dj, gb, n, alpha, E, emax);
        RFD_LAUNCH_CHECK();
        k_lag_select<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, E, n, emax, lagkey);
        RFD_LAUNCH_CHECK();
        if (match) RFD_TRY_CUDA(cudaMemsetAsync(Gb, 0, nbt * n * sizeof(double2), s));
        k_place<<<(unsigned)nbt, 256, 0, s>>>(dj, gb, n, alpha, lagkey, (int32_t)j0, k_stride, rho64,
                                              taps, lag, match ? Gb : nullptr);
        RFD_LAUNCH_CHECK();
        k_sigma_eff<<<(unsigned)nbt, 256, (size_t)kb * sizeof(double2), s>>>(dj, rho64, k_stride, C,
                                                                           kmax, (int32_t)j0, sigma);
        RFD_LAUNCH_CHECK();
        if (match) {
            RFD_TRY(fft_c2c<double>(ctx, n, nbt, Gb, n, gb, n, tmp, false, s));
            k_match_partial<<<dim3((unsigned)nb_match, (unsigned)nbt), 256, 0, s>>>(
                dj, g.pn_flags, psd, g.df, n, g.k_lo, gb, part);
            RFD_LAUNCH_CHECK();
            k_match_final<<<(unsigned)nbt, 256, 0, s>>>(part, nb_match, (int32_t)j0, match);
            RFD_LAUNCH_CHECK();
        }
        // the job table is rewritten by the next batch
        RFD_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return RFD_OK;
}

}  // namespace rfd
