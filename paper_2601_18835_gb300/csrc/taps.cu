// make_taps: ratio-filter taps, lags, sigma_eff and tap match (Eq. 2, Eq. 3, Sec. V,
// Eqs. 5-6), all in FP64 on the device.
//
// Per batch of templates:
//   1. G = conj(h_j / h_r) from the FP64 phase difference in the reference band (0 above the
//      template's cutoff), linear magnitude / shortest-arc phase fill on the out-of-band arc;
//   2. g = IDFT_n(G) (FP64 Stockham; the 1/n is applied when the taps are cut);
//   3. K (when bucketed): the smallest bucket b whose best circular window of b samples holds
//      `frac` of sum |g|^2 (prefix sums of |g|^2, FP64);
//      lag: the maximiser of E[s] = sum_k w[k]^2 |g[(s+k) mod n]|^2 with the tie rule (within
//      1e-9 of the maximum; closest to s = -K/2, then smaller s).  Since w^2 <= 1,
//      E[s] <= U[s] = sum_k |g[(s+k) mod n]|^2, so E is evaluated exactly only where U reaches
//      E at the argmax of U (minus a rounding allowance): the same maximiser as an exhaustive
//      search, at O(n + candidates K) instead of O(n K);
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

// P[b][i] = sum_{m < i} |g_b[m]|^2, i = 0 .. n, one block per template (fixed-order scan).
__global__ void __launch_bounds__(1024) k_energy_prefix(const double2 *__restrict__ g, int64_t n,
                                                        double *__restrict__ P) {
    __shared__ double part[1024];
    const int b = blockIdx.x;
    const double2 *gb = g + (int64_t)b * n;
    double *Pb = P + (int64_t)b * (n + 1);
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = min(n, (int64_t)threadIdx.x * per), hi = min(n, lo + per);
    double acc = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
        const double2 v = gb[i];
        acc += v.x * v.x + v.y * v.y;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const double v = part[t];
            part[t] = run;
            run += v;
        }
        Pb[n] = run;
    }
    __syncthreads();
    double run = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        Pb[i] = run;
        const double2 v = gb[i];
        run += v.x * v.x + v.y * v.y;
    }
}

// sum of |g|^2 over the circular window [m, m + L), from the prefix sums
__device__ __forceinline__ double window_sum(const double *__restrict__ P, int64_t n, int64_t m, int64_t L) {
    return (m + L <= n) ? P[m + L] - P[m] : (P[n] - P[m]) + P[m + L - n];
}

// per template and bucket: the best window energy over all starts (max of bit patterns)
__global__ void __launch_bounds__(256) k_bucket_max(const double *__restrict__ P, int64_t n,
                                                    const int32_t *__restrict__ buckets, int nb,
                                                    unsigned long long *__restrict__ bmax) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const double *Pb = P + (int64_t)b * (n + 1);
    for (int i = 0; i < nb; ++i) {
        unsigned long long bits = 0ull;
        if (m < n) bits = (unsigned long long)__double_as_longlong(fmax(0.0, window_sum(Pb, n, m, buckets[i])));
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
            bits = other > bits ? other : bits;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&bmax[(int64_t)b * nb + i], bits);
    }
}

// K_j = the smallest bucket whose best window holds frac of the energy (else the largest)
__global__ void k_bucket_pick(TapJob *jobs, int nbt, const double *__restrict__ P, int64_t n,
                              const int32_t *__restrict__ buckets, int nb, double frac,
                              const unsigned long long *__restrict__ bmax, int32_t j0,
                              int32_t *__restrict__ k_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbt) return;
    const double total = P[(int64_t)b * (n + 1) + n];
    int K = buckets[nb - 1];
    for (int i = 0; i < nb; ++i)
        if (__longlong_as_double((long long)bmax[(int64_t)b * nb + i]) >= frac * total) {
            K = buckets[i];
            break;
        }
    jobs[b].K = K;
    if (k_out) k_out[j0 + b] = K;
}

// U[s] = window_sum over K for every start; per-template maximum (bit patterns)
__global__ void __launch_bounds__(256) k_umax(const TapJob *__restrict__ jobs, const double *__restrict__ P,
                                              int64_t n, unsigned long long *__restrict__ umax) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    unsigned long long bits = 0ull;
    if (m < n) bits = (unsigned long long)__double_as_longlong(fmax(0.0, window_sum(P + (int64_t)b * (n + 1), n, m, jobs[b].K)));
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&umax[b], bits);
}

// the smallest start m whose U equals the maximum
__global__ void __launch_bounds__(256) k_uargmax(const TapJob *__restrict__ jobs, const double *__restrict__ P,
                                                 int64_t n, const unsigned long long *__restrict__ umax,
                                                 unsigned long long *__restrict__ uarg) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (m >= n) return;
    const double u = fmax(0.0, window_sum(P + (int64_t)b * (n + 1), n, m, jobs[b].K));
    if ((unsigned long long)__double_as_longlong(u) == umax[b]) atomicMin(&uarg[b], (unsigned long long)m);
}

__device__ __forceinline__ double exact_energy(const double2 *__restrict__ gb, int64_t n, int64_t m, int K,
                                               double alpha) {
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        const double w = tukey_w(k, K, alpha);
        int64_t idx = m + k;
        if (idx >= n) idx -= n;
        const double2 v = gb[idx];
        acc += (w * w) * (v.x * v.x + v.y * v.y);
    }
    return acc;
}

// bound[b] = E at the argmax of U (a lower bound on the maximum of E), one thread per template
__global__ void k_bound(const TapJob *__restrict__ jobs, const double2 *__restrict__ g, int64_t n, double alpha,
                        int nbt, const unsigned long long *__restrict__ uarg, double *__restrict__ bound) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbt) return;
    const int64_t m0 = uarg[b] < (unsigned long long)n ? (int64_t)uarg[b] : 0;
    bound[b] = exact_energy(g + (int64_t)b * n, n, m0, jobs[b].K, alpha);
}

// E[i] (i = s + n/2) exactly where U[s mod n] can reach the bound, -1 elsewhere; maximum.
__global__ void __launch_bounds__(256) k_candidates(const TapJob *__restrict__ jobs, const double2 *__restrict__ g,
                                                    const double *__restrict__ P, int64_t n, double alpha,
                                                    const double *__restrict__ bound,
                                                    double *__restrict__ E,
                                                    unsigned long long *__restrict__ emax) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= n) return;
    const int K = jobs[b].K;
    const double *Pb = P + (int64_t)b * (n + 1);
    const double2 *gb = g + (int64_t)b * n;
    // allowance for the rounding of the prefix sums against the direct sums
    const double tau = bound[b] * (1.0 - 1e-9) - 1e-6 * Pb[n];
    const int64_t m = (i - n / 2 + n) % n;
    double e = -1.0;
    if (window_sum(Pb, n, m, K) >= tau) {
        e = exact_energy(gb, n, m, K, alpha);
        atomicMax(&emax[b], (unsigned long long)__double_as_longlong(e));
    }
    E[(int64_t)b * n + i] = e;
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
// ------------------------------------------------------------------ chi^2-fitted taps (Sec. V.A)
// w G on the reference band (w = 4 df |h_r|^2 / S, the reference's SNR density), zero elsewhere
// and above n/2, in place: its inverse transform read at the lag window is the right-hand side
// of the fit's normal equations.
__global__ void __launch_bounds__(256) k_weight_spectrum(const TapJob *__restrict__ jobs,
                                                         const double *__restrict__ psd, double df, int64_t n,
                                                         int64_t k_lo, double2 *__restrict__ G) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = blockIdx.y;
    const int64_t k_hi = jobs[b].tr.k_hi;
    double2 *gk = G + (int64_t)b * n + k;
    if (k >= k_lo && k <= k_hi) {
        const double f = (double)k * df;
        const double amp = pow(f, -7.0 / 6.0);
        const double w = 4.0 * df * (amp * amp) / psd[k];
        *gk = make_double2(w * gk->x, w * gk->y);
    } else {
        *gk = make_double2(0.0, 0.0);
    }
}

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv_d(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Block-wide sum of three complex values (256 threads); every thread gets the totals.
__device__ __forceinline__ void block_sum3(double2 &a, double2 &b, double2 &c, double *red) {
    double v[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
#pragma unroll
    for (int q = 0; q < 6; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) red[(threadIdx.x >> 5) * 6 + q] = v[q];
    __syncthreads();
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
        for (int q = 0; q < 6; ++q) t[q] += red[w * 6 + q];
    a = make_double2(t[0], t[1]);
    b = make_double2(t[2], t[3]);
    c = make_double2(t[4], t[5]);
}

// The ridge-regularised normal equations sum_m (C_r[n-m] + lam delta) rho_m = b_n, n < K,
// solved by the Levinson recursion (forward / backward vectors of the Hermitian Toeplitz
// matrix, O(K^2)), one block per template, FP64.  b_n = bw[(s + n) mod N] (bw: the inverse
// transform of w G).  Writes the taps (FP64 and FP32), the lag and rho^H b (for the match).
__global__ void __launch_bounds__(256) k_fit_levinson(const TapJob *__restrict__ jobs,
                                                      const double2 *__restrict__ bw, int64_t n,
                                                      const double2 *__restrict__ Cc, int32_t kmax, double eps,
                                                      const unsigned long long *__restrict__ lagkey,
                                                      int32_t j0, int32_t k_stride, double2 *__restrict__ rho64,
                                                      float2 *__restrict__ taps, int32_t *__restrict__ lag,
                                                      double2 *__restrict__ bdot) {
    extern __shared__ double2 lv[];
    __shared__ double red[8 * 6];
    const int b = blockIdx.x;
    const int K = jobs[b].K;
    double2 *c = lv, *y = lv + kmax, *f = lv + 2 * kmax, *g = lv + 3 * kmax, *x = lv + 4 * kmax;
    const double2 *Cr = Cc + (int64_t)jobs[b].ref * (2 * kmax - 1) + (kmax - 1);   // Cr[l], |l| < kmax
    const int64_t s = (int64_t)(lagkey[b] & 0xffffffffull) - n / 2;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        c[i] = Cr[i];
        y[i] = bw[(int64_t)b * n + (((s + i) % n) + n) % n];
        f[i] = g[i] = x[i] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c[0].x += eps * c[0].x;
        const double2 inv = cdiv_d(make_double2(1.0, 0.0), c[0]);
        f[0] = g[0] = inv;
        x[0] = cmul_d(y[0], inv);
    }
    __syncthreads();
    for (int m = 1; m < K; ++m) {
        // errors of the extended vectors: ef = sum_i T[m][i] f_i, eb = sum_i T[0][i+1] g_i,
        // ex = sum_i T[m][i] x_i with T[a][b] = C[a - b], C[-l] = conj(C[l])
        double2 ef = make_double2(0.0, 0.0), eb = ef, ex = ef;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double2 cm = c[m - i], ci = c[i + 1];
            const double2 fi = f[i], gi = g[i], xi = x[i];
            ef.x += cm.x * fi.x - cm.y * fi.y;
            ef.y += cm.x * fi.y + cm.y * fi.x;
            eb.x += ci.x * gi.x + ci.y * gi.y;          // conj(c[i+1]) g_i
            eb.y += ci.x * gi.y - ci.y * gi.x;
            ex.x += cm.x * xi.x - cm.y * xi.y;
            ex.y += cm.x * xi.y + cm.y * xi.x;
        }
        block_sum3(ef, eb, ex, red);
        const double2 d = make_double2(1.0 - (ef.x * eb.x - ef.y * eb.y), -(ef.x * eb.y + ef.y * eb.x));
        const double2 a1 = cdiv_d(make_double2(1.0, 0.0), d), af = cdiv_d(ef, d), ab = cdiv_d(eb, d);
        // new f_i = a1 [f;0]_i - af [0;g]_i,  new g_i = a1 [0;g]_i - ab [f;0]_i  (K <= 512)
        double2 nf[2], ng[2];
        int cnt = 0;
        for (int i = threadIdx.x; i <= m && cnt < 2; i += blockDim.x, ++cnt) {
            const double2 fo = i < m ? f[i] : make_double2(0.0, 0.0);
            const double2 go = i >= 1 ? g[i - 1] : make_double2(0.0, 0.0);
            const double2 t1 = cmul_d(a1, fo), t2 = cmul_d(af, go), t3 = cmul_d(a1, go), t4 = cmul_d(ab, fo);
            nf[cnt] = make_double2(t1.x - t2.x, t1.y - t2.y);
            ng[cnt] = make_double2(t3.x - t4.x, t3.y - t4.y);
        }
        __syncthreads();
        const double2 e = make_double2(y[m].x - ex.x, y[m].y - ex.y);
        cnt = 0;
        for (int i = threadIdx.x; i <= m && cnt < 2; i += blockDim.x, ++cnt) {
            f[i] = nf[cnt];
            g[i] = ng[cnt];
            const double2 xo = i < m ? x[i] : make_double2(0.0, 0.0);
            const double2 u = cmul_d(e, ng[cnt]);
            x[i] = make_double2(xo.x + u.x, xo.y + u.y);
        }
        __syncthreads();
    }
    // taps, rho^H b
    double2 p = make_double2(0.0, 0.0), z0 = p, z1 = p;
    for (int i = threadIdx.x; i < k_stride; i += blockDim.x) {
        const double2 r = i < K ? x[i] : make_double2(0.0, 0.0);
        rho64[(int64_t)b * k_stride + i] = r;
        taps[(int64_t)(j0 + b) * k_stride + i] = make_float2((float)r.x, (float)r.y);
        if (i < K) {
            p.x += r.x * y[i].x + r.y * y[i].y;      // conj(rho_i) b_i
            p.y += r.x * y[i].y - r.y * y[i].x;
        }
    }
    block_sum3(p, z0, z1, red);
    if (threadIdx.x == 0) {
        lag[j0 + b] = (int32_t)s;
        bdot[b] = p;
    }
}

// sigma_j^2 = 4 df sum |h_j|^2 / S over the template's band, and the fitted taps' match
// |rho^H b| / (sigma_eff sigma_j) (sigma_eff = sqrt(rho^H C_r rho), from k_sigma_eff).
__global__ void __launch_bounds__(256) k_fit_match(const TapJob *__restrict__ jobs, const double *__restrict__ psd,
                                                   double df, int64_t n, int64_t k_lo,
                                                   const double2 *__restrict__ bdot, const double *__restrict__ sigma,
                                                   int32_t j0, double *__restrict__ match) {
    __shared__ double sm[8];
    const int b = blockIdx.x;
    const int64_t k_hi = min(jobs[b].tj.k_hi, n / 2);
    double part = 0.0;
    for (int64_t k = k_lo + threadIdx.x; k <= k_hi; k += blockDim.x) {
        const double f = (double)k * df;
        part += pow(f, -7.0 / 3.0) / psd[k];
    }
    const double tot = block_sum_d(part, sm) * 4.0 * df;
    if (threadIdx.x == 0) {
        const double2 p = bdot[b];
        const double se = sigma[j0 + b];
        match[j0 + b] = (se > 0.0 && tot > 0.0) ? sqrt(p.x * p.x + p.y * p.y) / (se * sqrt(tot)) : 0.0;
    }
}

// C_r[l] = sum_k 4 df |h_r|^2/S exp(+2 pi i k l / n) for |l| < kmax, one inverse FFT per
// reference (Eq. 6 on the sample grid): C[r][l + kmax - 1], complex128.  refs_dev: PNParams[R].
// Scratch: ws[7], ws[8], ws[9] (R n complex128 each).
rfd_status ref_autocorr_impl(rfd_ctx *ctx, const Grid &g, const double *psd, const PNParams *refs_dev, int64_t R,
                             int32_t kmax, double2 *C, cudaStream_t s) {
    const int64_t n = g.n;
    RFD_TRY(ensure(ctx->ws[7], R * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[8], R * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[9], R * n * sizeof(double2)));
    double2 *Gb = (double2 *)ctx->ws[7].p, *gb = (double2 *)ctx->ws[8].p, *tmp = (double2 *)ctx->ws[9].p;
    k_ref_weight<<<dim3((unsigned)((n + 255) / 256), (unsigned)R), 256, 0, s>>>(refs_dev, psd, g.df, n, g.k_lo, gb);
    RFD_LAUNCH_CHECK();
    RFD_TRY(fft_c2c<double>(ctx, n, R, gb, n, Gb, n, tmp, true, s));
    k_compact_C<<<(unsigned)R, 256, 0, s>>>(Gb, n, kmax, C);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

rfd_status make_taps_impl(rfd_ctx *ctx, const Grid &g, const double *psd,
                          const std::vector<PNParams> &refs, const std::vector<PNParams> &tmpl,
                          const std::vector<int32_t> &ref_of, const std::vector<int32_t> &K,
                          const std::vector<int32_t> &buckets, const std::vector<int32_t> &lag_in,
                          double energy_frac, int32_t k_stride, double alpha, float2 *taps, int32_t *k_out,
                          int32_t *lag, double *sigma, double *match, cudaStream_t s, double fit_eps) {
    const bool fixed_lag = !lag_in.empty();
    const bool fitted = fit_eps > 0.0;
    const int64_t n = g.n;
    const int64_t J = (int64_t)tmpl.size(), R = (int64_t)refs.size();
    const bool bucketed = K.empty();
    const int nbk = (int)buckets.size();
    int64_t B = std::max<int64_t>(1, ((int64_t)2 << 30) / (n * 64));
    B = std::min<int64_t>(std::min<int64_t>(B, J), 4096);
    const int64_t nb_match = (n / 2 + 1 + 255) / 256;
    int kmax = 0;
    if (bucketed)
        for (int b : buckets) kmax = std::max(kmax, b);
    else
        for (int64_t i = 0; i < J; ++i) kmax = std::max(kmax, K[i]);
    // per-batch scalars, taps in FP64, compact C_r rows and match partials share ws[11]
    const size_t u64b = (size_t)B * sizeof(unsigned long long);
    const size_t off_lagkey = u64b, off_umax = 2 * u64b, off_uarg = 3 * u64b, off_bmax = 4 * u64b;
    const size_t off_bk = off_bmax + (size_t)B * std::max(nbk, 1) * sizeof(unsigned long long);
    const size_t off_rho = (off_bk + (size_t)std::max(nbk, 1) * sizeof(int32_t) + 15) / 16 * 16;
    const size_t off_C = off_rho + (size_t)B * k_stride * sizeof(double2);
    const size_t off_part = off_C + (size_t)R * (2 * kmax - 1) * sizeof(double2);
    const size_t off_bdot = off_part + (size_t)B * 4 * nb_match * sizeof(double);
    const size_t ws11 = off_bdot + (size_t)B * sizeof(double2);
    RFD_TRY(ensure(ctx->ws[6], B * sizeof(TapJob)));
    RFD_TRY(ensure(ctx->ws[7], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[8], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[9], std::max(B, R) * n * sizeof(double2)));
    RFD_TRY(ensure(ctx->ws[10], B * n * sizeof(double)));
    RFD_TRY(ensure(ctx->ws[15], B * (n + 1) * sizeof(double)));
    RFD_TRY(ensure(ctx->ws[11], ws11));
    RFD_TRY(ensure(ctx->ws[0], R * sizeof(PNParams)));
    char *base11 = (char *)ctx->ws[11].p;
    unsigned long long *emax = (unsigned long long *)base11;
    unsigned long long *lagkey = (unsigned long long *)(base11 + off_lagkey);
    unsigned long long *umax = (unsigned long long *)(base11 + off_umax);
    unsigned long long *uarg = (unsigned long long *)(base11 + off_uarg);
    unsigned long long *bmax = (unsigned long long *)(base11 + off_bmax);
    int32_t *d_buckets = (int32_t *)(base11 + off_bk);
    double2 *rho64 = (double2 *)(base11 + off_rho);
    double2 *C = (double2 *)(base11 + off_C);
    double *part = (double *)(base11 + off_part);
    double2 *bdot = (double2 *)(base11 + off_bdot);
    double *E = (double *)ctx->ws[10].p;
    double *Pbuf = (double *)ctx->ws[15].p;
    if (bucketed)
        RFD_TRY_CUDA(cudaMemcpyAsync(d_buckets, buckets.data(), nbk * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    // C_r[l] = sum_k 4 df |h_r|^2/S exp(+2 pi i k l / n): one inverse FFT per reference
    RFD_TRY_CUDA(cudaMemcpyAsync(ctx->ws[0].p, refs.data(), R * sizeof(PNParams),
                                 cudaMemcpyHostToDevice, s));
    RFD_TRY(ref_autocorr_impl(ctx, g, psd, (const PNParams *)ctx->ws[0].p, R, kmax, C, s));
    double2 *Gb = (double2 *)ctx->ws[7].p, *gb = (double2 *)ctx->ws[8].p, *tmp = (double2 *)ctx->ws[9].p;
    std::vector<unsigned long long> lk;

    std::vector<TapJob> jobs(B);
    for (int64_t j0 = 0; j0 < J; j0 += B) {
        const int64_t nbt = std::min<int64_t>(B, J - j0);
        for (int64_t b = 0; b < nbt; ++b) {
            TapJob &jb = jobs[b];
            jb = TapJob{};
            jb.tj = tmpl[j0 + b];
            jb.ref = ref_of[j0 + b];
            jb.tr = refs[jb.ref];
            jb.K = bucketed ? kmax : K[j0 + b];      // bucketed: chosen on the device below
        }
        TapJob *dj = (TapJob *)ctx->ws[6].p;
        RFD_TRY_CUDA(cudaMemcpyAsync(dj, jobs.data(), nbt * sizeof(TapJob), cudaMemcpyHostToDevice, s));
        k_fill_ends<<<(unsigned)((nbt + 127) / 128), 128, 0, s>>>(dj, (int)nbt, g.pn_flags, g.df, g.k_lo);
        RFD_LAUNCH_CHECK();
        k_ratio_spectrum<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, g.pn_flags, g.df,
                                                                               n, g.k_lo, Gb);
        RFD_LAUNCH_CHECK();
        RFD_TRY(fft_c2c<double>(ctx, n, nbt, Gb, n, gb, n, tmp, true, s));
        if (fixed_lag) {
            // lags given by the caller: the placement key holds s + n/2 in its low bits
            lk.resize(nbt);
            for (int64_t b = 0; b < nbt; ++b) lk[b] = (unsigned long long)((int64_t)lag_in[j0 + b] + n / 2);
            RFD_TRY_CUDA(cudaMemcpyAsync(lagkey, lk.data(), nbt * sizeof(unsigned long long),
                                         cudaMemcpyHostToDevice, s));
            if (k_out)
                RFD_TRY_CUDA(cudaMemcpyAsync(k_out + j0, K.data() + j0, nbt * sizeof(int32_t),
                                             cudaMemcpyHostToDevice, s));
        } else {
        // energy prefix sums, optional K bucket, pruned exact lag search
        k_energy_prefix<<<(unsigned)nbt, 1024, 0, s>>>(gb, n, Pbuf);
        RFD_LAUNCH_CHECK();
        if (bucketed) {
            RFD_TRY_CUDA(cudaMemsetAsync(bmax, 0, nbt * nbk * sizeof(unsigned long long), s));
            k_bucket_max<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(Pbuf, n, d_buckets, nbk, bmax);
            RFD_LAUNCH_CHECK();
            k_bucket_pick<<<(unsigned)((nbt + 127) / 128), 128, 0, s>>>(dj, (int)nbt, Pbuf, n, d_buckets, nbk,
                                                                        energy_frac, bmax, (int32_t)j0, k_out);
            RFD_LAUNCH_CHECK();
        } else if (k_out) {
            RFD_TRY_CUDA(cudaMemcpyAsync(k_out + j0, K.data() + j0, nbt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        }
        RFD_TRY_CUDA(cudaMemsetAsync(emax, 0, nbt * sizeof(unsigned long long), s));
        RFD_TRY_CUDA(cudaMemsetAsync(lagkey, 0xff, nbt * sizeof(unsigned long long), s));
        RFD_TRY_CUDA(cudaMemsetAsync(umax, 0, nbt * sizeof(unsigned long long), s));
        RFD_TRY_CUDA(cudaMemsetAsync(uarg, 0xff, nbt * sizeof(unsigned long long), s));
        k_umax<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, Pbuf, n, umax);
        RFD_LAUNCH_CHECK();
        k_uargmax<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, Pbuf, n, umax, uarg);
        RFD_LAUNCH_CHECK();
        k_bound<<<(unsigned)((nbt + 127) / 128), 128, 0, s>>>(dj, gb, n, alpha, (int)nbt, uarg, (double *)umax);
        RFD_LAUNCH_CHECK();
        k_candidates<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, gb, Pbuf, n, alpha,
                                                                             (const double *)umax, E, emax);
        RFD_LAUNCH_CHECK();
        k_lag_select<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, E, n, emax, lagkey);
        RFD_LAUNCH_CHECK();
        }
        if (fitted) {
            // Sec. V.A: taps fitted to the ratio in the reference's SNR-weighted band, ridge eps
            k_weight_spectrum<<<dim3((unsigned)(n / 256), (unsigned)nbt), 256, 0, s>>>(dj, psd, g.df, n, g.k_lo,
                                                                                      Gb);
            RFD_LAUNCH_CHECK();
            RFD_TRY(fft_c2c<double>(ctx, n, nbt, Gb, n, gb, n, tmp, true, s));
            k_fit_levinson<<<(unsigned)nbt, 256, (size_t)5 * kmax * sizeof(double2), s>>>(
                dj, gb, n, C, kmax, fit_eps, lagkey, (int32_t)j0, k_stride, rho64, taps, lag, bdot);
            RFD_LAUNCH_CHECK();
        } else {
            if (match) RFD_TRY_CUDA(cudaMemsetAsync(Gb, 0, nbt * n * sizeof(double2), s));
            k_place<<<(unsigned)nbt, 256, 0, s>>>(dj, gb, n, alpha, lagkey, (int32_t)j0, k_stride, rho64,
                                                  taps, lag, match ? Gb : nullptr);
            RFD_LAUNCH_CHECK();
        }
        k_sigma_eff<<<(unsigned)nbt, 256, (size_t)kmax * sizeof(double2), s>>>(dj, rho64, k_stride, C,
                                                                           kmax, (int32_t)j0, sigma);
        RFD_LAUNCH_CHECK();
        if (fitted && match) {
            k_fit_match<<<(unsigned)nbt, 256, 0, s>>>(dj, psd, g.df, n, g.k_lo, bdot, sigma, (int32_t)j0, match);
            RFD_LAUNCH_CHECK();
        } else if (match) {
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

namespace {
__global__ void k_scatter_fit_rows(const float2 *__restrict__ st, const int32_t *__restrict__ sl,
                                   const double *__restrict__ ss, const double *__restrict__ sm,
                                   const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int32_t K,
                                   int32_t k_stride, float2 *__restrict__ taps, int32_t *__restrict__ lag,
                                   double *__restrict__ sigma, double *__restrict__ match, int32_t *__restrict__ k_out) {
    const int64_t i = src[blockIdx.x], j = dst[blockIdx.x];
    for (int k = threadIdx.x; k < k_stride; k += blockDim.x) taps[j * k_stride + k] = st[i * k_stride + k];
    if (threadIdx.x == 0) {
        lag[j] = sl[i];
        sigma[j] = ss[i];
        match[j] = sm[i];
        if (k_out) k_out[j] = K;
    }
}
}  // namespace

// Sec. V.A's dynamic tap count: every template is fitted at the smallest bucket whose fitted
// match reaches `target` (the largest bucket otherwise).  One fit pass per bucket over the
// templates still pending.
rfd_status make_taps_fit_dynamic(rfd_ctx *ctx, const Grid &g, const double *psd, const std::vector<PNParams> &refs,
                                 const std::vector<PNParams> &tmpl, const std::vector<int32_t> &ref_of,
                                 const std::vector<int32_t> &buckets, double target, double eps, int32_t k_stride,
                                 double alpha, float2 *taps, int32_t *k_out, int32_t *lag, double *sigma,
                                 double *match, cudaStream_t s) {
    const int64_t J = (int64_t)tmpl.size();
    std::vector<int32_t> pending(J);
    for (int64_t j = 0; j < J; ++j) pending[j] = (int32_t)j;
    std::vector<int32_t> sorted(buckets);
    std::sort(sorted.begin(), sorted.end());
    DevBuf buf;
    rfd_status st = RFD_OK;
    for (size_t bi = 0; bi < sorted.size() && !pending.empty() && st == RFD_OK; ++bi) {
        const int32_t K = sorted[bi];
        const int64_t np = (int64_t)pending.size();
        auto up = [](size_t x) { return (x + 255) / 256 * 256; };
        const size_t bt = up((size_t)np * k_stride * sizeof(float2));
        if ((st = ensure(buf, bt + up(np * 4) * 2 + up(np * 8) * 2)) != RFD_OK) break;
        char *base = (char *)buf.p;
        float2 *t_taps = (float2 *)base;
        int32_t *t_lag = (int32_t *)(base + bt);
        int32_t *t_idx = (int32_t *)(base + bt + up(np * 4));
        double *t_sig = (double *)(base + bt + 2 * up(np * 4));
        double *t_match = (double *)(base + bt + 2 * up(np * 4) + up(np * 8));
        std::vector<PNParams> sub(np);
        std::vector<int32_t> sub_ref(np), sub_k(np, K);
        for (int64_t i = 0; i < np; ++i) {
            sub[i] = tmpl[pending[i]];
            sub_ref[i] = ref_of[pending[i]];
        }
        if ((st = make_taps_impl(ctx, g, psd, refs, sub, sub_ref, sub_k, {}, {}, 1.0, k_stride, alpha, t_taps,
                                 nullptr, t_lag, t_sig, t_match, s, eps)) != RFD_OK)
            break;
        std::vector<double> hm(np);
        cudaError_t e = cudaMemcpyAsync(hm.data(), t_match, np * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("reading the fitted matches failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        const bool last = bi + 1 == sorted.size();
        std::vector<int32_t> take_src, take_dst, still;
        for (int64_t i = 0; i < np; ++i) {
            if (last || hm[i] >= target) {
                take_src.push_back((int32_t)i);
                take_dst.push_back(pending[i]);
            } else {
                still.push_back(pending[i]);
            }
        }
        if (!take_src.empty()) {
            // compact the accepted rows to the front of the scratch, then scatter them into place
            const int64_t na = (int64_t)take_src.size();
            std::vector<int32_t> dst(na);
            for (int64_t i = 0; i < na; ++i) dst[i] = take_dst[i];
            // the scatter reads row take_src[i]: pass the source rows through an index remap
            std::vector<int32_t> src_rows(take_src);
            DevBuf ib;
            if ((st = ensure(ib, (size_t)na * 8)) != RFD_OK) break;
            int32_t *d_src = (int32_t *)ib.p, *d_dst = d_src + na;
            if ((e = cudaMemcpyAsync(d_src, src_rows.data(), na * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(d_dst, dst.data(), na * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
                (void)cudaGetLastError();
                set_error("cudaMemcpyAsync failed: %s", cudaGetErrorString(e));
                st = RFD_ERR_CUDA;
                release(ib);
                break;
            }
            k_scatter_fit_rows<<<(unsigned)na, 128, 0, s>>>(t_taps, t_lag, t_sig, t_match, d_src, d_dst, K, k_stride,
                                                            taps, lag, sigma, match, k_out);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            release(ib);
            if (e != cudaSuccess) {
                set_error("scattering the fitted taps failed: %s", cudaGetErrorString(e));
                st = RFD_ERR_CUDA;
                break;
            }
            count_launch();
        }
        pending.swap(still);
    }
    release(buf);
    return st;
}

}  // namespace rfd
