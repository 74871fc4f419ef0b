// Hand-written Stockham FFT (FP32 and FP64) for the matched filter of Eq. 1, the reference
// series of Eq. 3 and the FP64 tap design of Sec. V.
//
// Stockham auto-sort: each pass p with radix R reads element j + r L/R (r < R), applies the
// twiddles exp(+-2 pi i r (j mod Ns) / (Ns R)), does an R-point DFT in registers and writes
// to (j - j mod Ns) R + (j mod Ns) + r Ns, where Ns is the product of the radices of the
// earlier passes.  No bit reversal is needed.  Radix-16 passes, preceded by one radix-2, -4
// or -8 pass when log2 L is not a multiple of 4.  The R-point DFT is an unrolled radix-2
// decimation-in-time network over the 16th roots of unity; twiddles come from tables of
// exp(+2 pi i m / L) built once per length with FP64 sincospi.
//
// Two passes over memory (four-step form) for 2^12 <= n <= 2^22 (FP32) or 2^20 (FP64): with
// n = N1 N2, input index n1 N2 + n2 and output index k1 + N1 k2,
//   X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) [ w_N^(n2 k1) sum_n1 x[n1 N2 + n2] w_N1^(n1 k1) ].
// Kernel A takes C adjacent columns n2 per block (global accesses C elements wide), does the
// length-N1 transforms and applies w_N^(n2 k1); kernel B takes C rows k1 per block, does the
// length-N2 transforms and writes X, again C elements wide.  Inside a block the first radix
// pass reads global memory directly (every load of a thread issued at once), middle passes
// run in place in a padded shared-memory tile, and the last pass writes global memory.
// Other lengths take one kernel per Stockham pass over global memory.
#include "epilogue.cuh"
#include "fft_reg.cuh"
#include "internal.cuh"

namespace rfd {

namespace {

__global__ void k_twiddle64(double2 *w, int64_t n) {
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    w[m] = make_double2(c, s);
}

__global__ void k_twiddle32(const double2 *w64, float2 *w32, int64_t n) {
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    w32[m] = make_float2((float)w64[m].x, (float)w64[m].y);
}

template <typename T, int R, bool INV>
__global__ void __launch_bounds__(256) k_stockham(const typename Cplx<T>::type *__restrict__ in,
                                                  int64_t in_stride,
                                                  typename Cplx<T>::type *__restrict__ out,
                                                  int64_t out_stride,
                                                  const typename Cplx<T>::type *__restrict__ tw,
                                                  int64_t n, int64_t ns, int64_t batch0) {
    using T2 = typename Cplx<T>::type;
    const int64_t nr = n / R;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nr) return;
    const int64_t b = batch0 + blockIdx.y;
    const T2 *src = in + b * in_stride;
    T2 *dst = out + b * out_stride;
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * nr];
    const int64_t k = j & (ns - 1);
    if (ns > 1) {
        const int64_t step = n / (ns * R);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const T2 w = tw[r * k * step];
            v[r] = INV ? cmul(v[r], w) : cmulc(v[r], w);
        }
    }
    dft_reg<T, R, INV>(v);
    const int64_t idx = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[idx + r * ns] = v[r];
}

// ------------------------------------------------------------------ two-pass (four-step) form
// A block holds C short transforms of length L = 2^logL in shared memory, column-major, with
// one pad element per 16 and two per column: element i of column c at c LP + i + (i >> 4),
// LP = L + L/16 + 2.  The per-16 pad makes the radix-16 scatter of the first pass (stride 16)
// conflict-free; the per-column pad does the same for the loads and stores that walk across
// columns (C adjacent elements of global memory per row).
__host__ __device__ constexpr int tile_ld(int L) { return L + L / 16 + 2; }
__device__ __forceinline__ int tile_pos(int c, int i, int LP) { return c * LP + i + (i >> 4); }

// Stage twiddles of a length-L Stockham transform, the passes in order (first the radix-2, -4
// or -8 pass when logL is not a multiple of 4, then radix-16): pass p with radix R after
// ns = product of the earlier radices holds w_(ns R)^(r k) at base_p + (r - 1) ns + k,
// r = 1 .. R-1, k < ns.  The counts add up to L - 1.
template <typename T2>
__global__ void k_stage_twiddles(const double2 *__restrict__ wL, T2 *__restrict__ out, int logL) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int L = 1 << logL;
    if (e >= L - 1) return;
    const int first = logL & 3;
    const int np = (first ? 1 : 0) + logL / 4;
    int ns = 1, base = 0;
    for (int p = 0; p < np; ++p) {
        const int R = (p == 0 && first) ? (1 << first) : 16;
        const int cnt = (R - 1) * ns;
        if (e < base + cnt) {
            const int r = (e - base) / ns + 1, k = (e - base) % ns;
            const double2 w = wL[r * k * (L / (ns * R))];
            out[e] = T2{(decltype(T2::x))w.x, (decltype(T2::x))w.y};
            return;
        }
        base += cnt;
        ns *= R;
    }
}

// Butterfly bt of a radix-R pass over C columns of length L: column c and index j < L/R.
// CFAST puts adjacent threads on adjacent columns (global accesses C elements wide when the
// columns are adjacent in memory); otherwise on adjacent j within a column.
template <bool CFAST>
__device__ __forceinline__ void butterfly_of(int bt, int loglr, int logC, int &c, int &j) {
    if (CFAST) {
        c = bt & ((1 << logC) - 1);
        j = bt >> logC;
    } else {
        c = bt >> loglr;
        j = bt & ((1 << loglr) - 1);
    }
}

template <int R>
struct Log2R {
    static constexpr int v = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
};

// First pass (ns = 1, no twiddles): element i of column c read from g[i g_ld + c g_cs], all
// EPT loads of a thread issued before any use; results to the tile at j R + r.
template <typename T, int R, int EPT, bool INV, bool CFAST>
__device__ __forceinline__ void first_pass(typename Cplx<T>::type *S, int logL, int LP, int logC,
                                           const typename Cplx<T>::type *__restrict__ g, int64_t g_ld,
                                           int64_t g_cs) {
    using T2 = typename Cplx<T>::type;
    constexpr int NB = EPT / R, LOGR = Log2R<R>::v;
    const int loglr = logL - LOGR, lr = 1 << loglr;
    T2 v[NB][R];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<CFAST>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = g[(int64_t)(j + r * lr) * g_ld + c * g_cs];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<CFAST>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
        dft_reg<T, R, INV>(v[q]);
#pragma unroll
        for (int r = 0; r < R; ++r) S[tile_pos(c, (j << LOGR) + r, LP)] = v[q][r];
    }
}

// A middle pass in place over the tile: every thread reads its EPT elements, the block waits,
// then writes.  stw: this pass's stage twiddles.
template <typename T, int R, int EPT, bool INV>
__device__ __forceinline__ void mid_pass(typename Cplx<T>::type *S, int logL, int LP, int ns,
                                         const typename Cplx<T>::type *stw) {
    using T2 = typename Cplx<T>::type;
    constexpr int NB = EPT / R, LOGR = Log2R<R>::v;
    const int loglr = logL - LOGR, lr = 1 << loglr;
    T2 v[NB][R];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<false>(threadIdx.x + q * blockDim.x, loglr, 0, c, j);
        const int k = j & (ns - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = S[tile_pos(c, j + r * lr, LP)];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const T2 w = stw[(r - 1) * ns + k];
            v[q][r] = INV ? cmul(v[q][r], w) : cmulc(v[q][r], w);
        }
        dft_reg<T, R, INV>(v[q]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<false>(threadIdx.x + q * blockDim.x, loglr, 0, c, j);
        const int k = j & (ns - 1);
        const int idx = ((j - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) S[tile_pos(c, idx + r * ns, LP)] = v[q][r];
    }
    __syncthreads();
}

// Last pass (ns = L/R, so k = j and the outputs of butterfly j are j + r ns): tile to
// g[k g_ld + c] (adjacent columns adjacent in memory).  OUTER: each output (c, k) is also
// multiplied by w_N^((c0 + c) k) = hi[m >> sh] lo[m & (2^sh - 1)], m = (c0 + c) k.
template <typename T, int R, int EPT, bool INV, bool OUTER>
__device__ __forceinline__ void last_pass(const typename Cplx<T>::type *S, int logL, int LP, int logC,
                                          const typename Cplx<T>::type *stw, typename Cplx<T>::type *__restrict__ g,
                                          int64_t g_ld, int c0, int sh, const typename Cplx<T>::type *lo,
                                          const typename Cplx<T>::type *hi) {
    using T2 = typename Cplx<T>::type;
    constexpr int NB = EPT / R, LOGR = Log2R<R>::v;
    const int loglr = logL - LOGR, ns = 1 << loglr;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<true>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = S[tile_pos(c, j + r * ns, LP)];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const T2 w = stw[(r - 1) * ns + j];
            v[r] = INV ? cmul(v[r], w) : cmulc(v[r], w);
        }
        dft_reg<T, R, INV>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = j + r * ns;
            T2 o = v[r];
            if (OUTER) {
                const int m = (c0 + c) * k;
                const T2 w = cmul(hi[m >> sh], lo[m & ((1 << sh) - 1)]);
                o = INV ? cmul(o, w) : cmulc(o, w);
            }
            g[(int64_t)k * g_ld + c] = o;
        }
    }
}

// The middle passes of a block's transforms, after a first pass of radix R0 (whose output is
// in the tile); returns the last pass's stage twiddles.
template <typename T, int EPT, bool INV>
__device__ __forceinline__ const typename Cplx<T>::type *mid_passes(typename Cplx<T>::type *S, int logL, int LP,
                                                                   const typename Cplx<T>::type *stw, int R0) {
    stw += R0 - 1;
    int ns = R0;
    const int npass = ((logL & 3) ? 1 : 0) + logL / 4;
    for (int p = 1; p + 1 < npass; ++p) {
        mid_pass<T, 16, EPT, INV>(S, logL, LP, ns, stw);
        stw += 15 * ns;
        ns *= 16;
    }
    return stw;
}

// The C transforms of a block, global to global: first pass from g_in, middle passes in the
// tile, last pass to g_out.  logL >= 6, so there are two or three passes.
template <typename T, int EPT, bool INV, bool IN_CFAST, bool OUTER>
__device__ __forceinline__ void block_fft(typename Cplx<T>::type *S, int logL, int logC,
                                          const typename Cplx<T>::type *stw,
                                          const typename Cplx<T>::type *__restrict__ g_in, int64_t in_ld,
                                          int64_t in_cs, typename Cplx<T>::type *__restrict__ g_out,
                                          int64_t out_ld, int c0, int sh, const typename Cplx<T>::type *lo,
                                          const typename Cplx<T>::type *hi) {
    const int LP = tile_ld(1 << logL);
    const int first = logL & 3;
    const int R0 = first ? (1 << first) : 16;
    if (R0 == 2) first_pass<T, 2, EPT, INV, IN_CFAST>(S, logL, LP, logC, g_in, in_ld, in_cs);
    else if (R0 == 4) first_pass<T, 4, EPT, INV, IN_CFAST>(S, logL, LP, logC, g_in, in_ld, in_cs);
    else if (R0 == 8) first_pass<T, 8, EPT, INV, IN_CFAST>(S, logL, LP, logC, g_in, in_ld, in_cs);
    else first_pass<T, 16, EPT, INV, IN_CFAST>(S, logL, LP, logC, g_in, in_ld, in_cs);
    __syncthreads();                 // also covers the tables the caller copied
    stw = mid_passes<T, EPT, INV>(S, logL, LP, stw, R0);
    last_pass<T, 16, EPT, INV, OUTER>(S, logL, LP, logC, stw, g_out, out_ld, c0, sh, lo, hi);
}

template <typename T2>
__device__ __forceinline__ void copy_table(T2 *dst, const T2 *__restrict__ src, int cnt) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = src[i];
}

// Pass A: columns n2 in [c0, c0 + C) of x viewed as [N1][N2] (n = n1 N2 + n2); length-N1
// transforms over n1, times w_N^(n2 k1); y[k1 N2 + n2].  Threads: N1 C / EPT.
template <typename T, int EPT, bool INV>
__global__ void __launch_bounds__(512) k_fft_cols(const typename Cplx<T>::type *__restrict__ x, int64_t x_stride,
                                                  typename Cplx<T>::type *__restrict__ y, int64_t y_stride,
                                                  int logN1, int logN2, int logC, int sh,
                                                  const typename Cplx<T>::type *__restrict__ stage,
                                                  const typename Cplx<T>::type *__restrict__ tw_lo,
                                                  const typename Cplx<T>::type *__restrict__ tw_hi, int64_t batch0) {
    using T2 = typename Cplx<T>::type;
    extern __shared__ __align__(16) uint8_t fsm[];
    const int N1 = 1 << logN1, N2 = 1 << logN2, C = 1 << logC;
    const int nlo = 1 << sh, nhi = 1 << (logN1 + logN2 - sh);
    T2 *S = (T2 *)fsm;
    T2 *stw = S + C * tile_ld(N1);
    T2 *lo = stw + N1;
    T2 *hi = lo + nlo;
    copy_table(stw, stage, N1 - 1);
    copy_table(lo, tw_lo, nlo);
    copy_table(hi, tw_hi, nhi);
    const int64_t b = batch0 + blockIdx.y;
    const int c0 = blockIdx.x * C;
    block_fft<T, EPT, INV, true, true>(S, logN1, logC, stw, x + b * x_stride + c0, N2, 1, y + b * y_stride + c0, N2,
                                       c0, sh, lo, hi);
}

// Pass B: rows k1 in [r0, r0 + C) of y ([N1][N2]); length-N2 transforms over n2;
// X[k1 + N1 k2].  Threads: N2 C / EPT.
template <typename T, int EPT, bool INV>
__global__ void __launch_bounds__(512) k_fft_rows(const typename Cplx<T>::type *__restrict__ y, int64_t y_stride,
                                                  typename Cplx<T>::type *__restrict__ out, int64_t out_stride,
                                                  int logN1, int logN2, int logC,
                                                  const typename Cplx<T>::type *__restrict__ stage, int64_t batch0) {
    using T2 = typename Cplx<T>::type;
    extern __shared__ __align__(16) uint8_t fsm[];
    const int N1 = 1 << logN1, N2 = 1 << logN2, C = 1 << logC;
    T2 *S = (T2 *)fsm;
    T2 *stw = S + C * tile_ld(N2);
    copy_table(stw, stage, N2 - 1);
    const int64_t b = batch0 + blockIdx.y;
    const int r0 = blockIdx.x * C;
    block_fft<T, EPT, INV, false, false>(S, logN2, logC, stw, y + b * y_stride + (int64_t)r0 * N2, 1, N2,
                                         out + b * out_stride + r0, N1, 0, 0, nullptr, nullptr);
}

// ------------------------------------------------------------------ fused FINDCHIRP (Eq. 1)
// The inverse transform of c_j[k] = G[k] conj(h_j[k]) (G = 4 df d / S, zero outside the data
// band and for k >= n/2), z_j = q_j / sigma_j, in the two passes above with the pointwise
// product folded into pass A's first radix pass (elements with k >= n/2 are zero and never
// loaded) and the |z|^2 threshold / window maximum folded into pass B's last radix pass (q is
// never written).  Pass A also forms each block's share of sigma_j^2 = sum_k Wt[k] |h_j[k]|^2
// (Wt = 4 df / S), summed per template in a fixed order afterwards.

// First pass of pass A (ns = 1): element n1 = j + r lr of column c is k = n1 N2 + c0 + c, and
// k < n/2 exactly when r < R/2 (j < lr = N1 / R), so the upper half of every butterfly is zero
// and never loaded.  GW[k] = (Re G, Im G, Wt, 0).  Every load of the thread is issued before
// any product is formed.
template <int R, int EPT>
__device__ __forceinline__ void fc_first_pass(float2 *S, int logL, int LP, int logC, const float4 *__restrict__ GW,
                                              const float2 *__restrict__ h, int64_t N2, int c0, float &psum) {
    constexpr int NB = EPT / R, LOGR = Log2R<R>::v, RH = R / 2;
    const int loglr = logL - LOGR, lr = 1 << loglr;
    float2 hv[NB][RH];
    float4 gw[NB][RH];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<true>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int64_t k = (int64_t)(j + r * lr) * N2 + c0 + c;
            hv[q][r] = h[k];
            gw[q][r] = GW[k];
        }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<true>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < RH) {
                const float2 x = hv[q][r];
                const float4 g = gw[q][r];
                psum += g.z * (x.x * x.x + x.y * x.y);
                v[r] = make_float2(g.x * x.x + g.y * x.y, g.y * x.x - g.x * x.y);   // g conj(h)
            } else {
                v[r] = make_float2(0.f, 0.f);
            }
        }
        dft_reg<float, R, true>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) S[tile_pos(c, (j << LOGR) + r, LP)] = v[r];
    }
}

// Pass A of FINDCHIRP: template b's spectrum formed on the fly; y[k1 N2 + n2]; sigma^2 partials.
template <int EPT>
__global__ void __launch_bounds__(256) k_fc_cols(const float4 *__restrict__ GW,
                                                 const float2 *__restrict__ h, int64_t nf, float2 *__restrict__ y,
                                                 int logN1, int logN2, int logC, int sh,
                                                 const float2 *__restrict__ stage, const float2 *__restrict__ tw_lo,
                                                 const float2 *__restrict__ tw_hi, double *__restrict__ part) {
    extern __shared__ __align__(16) uint8_t fsm[];
    __shared__ float red[16];
    const int N1 = 1 << logN1, N2 = 1 << logN2, C = 1 << logC;
    const int nlo = 1 << sh, nhi = 1 << (logN1 + logN2 - sh);
    float2 *S = (float2 *)fsm;
    float2 *stw = S + C * tile_ld(N1);
    float2 *lo = stw + N1;
    float2 *hi = lo + nlo;
    copy_table(stw, stage, N1 - 1);
    copy_table(lo, tw_lo, nlo);
    copy_table(hi, tw_hi, nhi);
    const int64_t b = blockIdx.y;
    const int c0 = blockIdx.x * C;
    const int64_t n = (int64_t)N1 * N2;
    const int LP = tile_ld(N1);
    const int R0 = (logN1 & 3) ? (1 << (logN1 & 3)) : 16;
    float psum = 0.f;
    const float2 *hb = h + b * nf;
    if (R0 == 2) fc_first_pass<2, EPT>(S, logN1, LP, logC, GW, hb, N2, c0, psum);
    else if (R0 == 4) fc_first_pass<4, EPT>(S, logN1, LP, logC, GW, hb, N2, c0, psum);
    else if (R0 == 8) fc_first_pass<8, EPT>(S, logN1, LP, logC, GW, hb, N2, c0, psum);
    else fc_first_pass<16, EPT>(S, logN1, LP, logC, GW, hb, N2, c0, psum);
    __syncthreads();
    const float2 *st = mid_passes<float, EPT, true>(S, logN1, LP, stw, R0);
    last_pass<float, 16, EPT, true, true>(S, logN1, LP, logC, st, y + b * n + c0, N2, c0, sh, lo, hi);
    // the block's share of sigma^2, fixed order
    for (int o = 16; o > 0; o >>= 1) psum += __shfl_down_sync(0xffffffffu, psum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = psum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)red[w];
        part[b * gridDim.x + blockIdx.x] = t;
    }
}

// Pass B of FINDCHIRP: rows k1 of y; the last radix pass hands every output q[k1 + N1 k2]
// straight to the trigger epilogue (z = q / sigma, |z|^2 > thr, one candidate per window and
// warp), lanes on adjacent k1.
template <int EPT>
__global__ void __launch_bounds__(256) k_fc_rows(const float2 *__restrict__ y, int logN1, int logN2, int logC,
                                                 const float2 *__restrict__ stage, const double *__restrict__ sig2,
                                                 int32_t j0, float thr, uint32_t W, rfd_candidate *__restrict__ cand,
                                                 int64_t cap, unsigned long long *__restrict__ count) {
    extern __shared__ __align__(16) uint8_t fsm[];
    const int N1 = 1 << logN1, N2 = 1 << logN2, C = 1 << logC;
    float2 *S = (float2 *)fsm;
    float2 *stw = S + C * tile_ld(N2);
    copy_table(stw, stage, N2 - 1);
    const int64_t b = blockIdx.y;
    const int r0 = blockIdx.x * C;
    const int64_t n = (int64_t)N1 * N2;
    const int LP = tile_ld(N2);
    const float2 *g = y + b * n + (int64_t)r0 * N2;
    const int R0 = (logN2 & 3) ? (1 << (logN2 & 3)) : 16;
    if (R0 == 2) first_pass<float, 2, EPT, true, false>(S, logN2, LP, logC, g, 1, N2);
    else if (R0 == 4) first_pass<float, 4, EPT, true, false>(S, logN2, LP, logC, g, 1, N2);
    else if (R0 == 8) first_pass<float, 8, EPT, true, false>(S, logN2, LP, logC, g, 1, N2);
    else first_pass<float, 16, EPT, true, false>(S, logN2, LP, logC, g, 1, N2);
    __syncthreads();
    const float2 *st = mid_passes<float, EPT, true>(S, logN2, LP, stw, R0);
    // last pass (ns = N2 / 16, k = j): outputs j + r ns of column c are q[r0 + c + N1 (j + r ns)]
    const float inv = (float)(1.0 / sqrt(sig2[b]));
    constexpr int NB = EPT / 16;
    const int loglr = logN2 - 4, ns = 1 << loglr;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        int c, j;
        butterfly_of<true>(threadIdx.x + q * blockDim.x, loglr, logC, c, j);
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = S[tile_pos(c, j + r * ns, LP)];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], st[(r - 1) * ns + j]);
        dft_reg<float, 16, true>(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const uint32_t t = (uint32_t)(r0 + c) + (uint32_t)N1 * (uint32_t)(j + r * ns);
            emit_window_max(true, (uint32_t)(j0 + b), t, v[r].x * inv, v[r].y * inv, thr, W, cand, cap, count);
        }
    }
}

// sig2[row] = the row's pass-A partials summed in a fixed order: one warp per row, lane l sums
// the partials l, l + 32, ..., then a fixed shuffle tree.
__global__ void k_fc_sum(const double *__restrict__ part, int64_t nparts, double *__restrict__ sig2) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int64_t i = lane; i < nparts; i += 32) t += part[blockIdx.x * nparts + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sig2[blockIdx.x] = t;
}

template <typename T>
rfd_status get_twiddles(rfd_ctx *ctx, int64_t n, const typename Cplx<T>::type **out,
                        cudaStream_t s);

template <>
rfd_status get_twiddles<double>(rfd_ctx *ctx, int64_t n, const double2 **out, cudaStream_t s) {
    auto it = ctx->tw64.find(n);
    if (it == ctx->tw64.end()) {
        void *p = nullptr;
        RFD_TRY_CUDA(cudaMalloc(&p, n * sizeof(double2)));
        k_twiddle64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double2 *)p, n);
        RFD_LAUNCH_CHECK();
        it = ctx->tw64.emplace(n, p).first;
    }
    *out = (const double2 *)it->second;
    return RFD_OK;
}

template <>
rfd_status get_twiddles<float>(rfd_ctx *ctx, int64_t n, const float2 **out, cudaStream_t s) {
    auto it = ctx->tw32.find(n);
    if (it == ctx->tw32.end()) {
        const double2 *w64 = nullptr;
        RFD_TRY(get_twiddles<double>(ctx, n, &w64, s));
        void *p = nullptr;
        RFD_TRY_CUDA(cudaMalloc(&p, n * sizeof(float2)));
        k_twiddle32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w64, (float2 *)p, n);
        RFD_LAUNCH_CHECK();
        it = ctx->tw32.emplace(n, p).first;
    }
    *out = (const float2 *)it->second;
    return RFD_OK;
}

// Stage twiddles of a length-2^logL transform in T (cached per logL).
template <typename T>
rfd_status get_stage_twiddles(rfd_ctx *ctx, int logL, const typename Cplx<T>::type **out, cudaStream_t s) {
    using T2 = typename Cplx<T>::type;
    auto &cache = sizeof(T2) == 8 ? ctx->stw32 : ctx->stw64;
    auto it = cache.find(logL);
    if (it == cache.end()) {
        const int64_t L = int64_t(1) << logL;
        const double2 *wL = nullptr;
        RFD_TRY(get_twiddles<double>(ctx, L, &wL, s));
        void *p = nullptr;
        RFD_TRY_CUDA(cudaMalloc(&p, L * sizeof(T2)));
        k_stage_twiddles<T2><<<(unsigned)((L + 255) / 256), 256, 0, s>>>(wL, (T2 *)p, logL);
        RFD_LAUNCH_CHECK();
        it = cache.emplace(logL, p).first;
    }
    *out = (const T2 *)it->second;
    return RFD_OK;
}

}  // namespace

rfd_status fft_stage_twiddles32(rfd_ctx *ctx, int logL, const float2 **out, cudaStream_t s) {
    return get_stage_twiddles<float>(ctx, logL, out, s);
}

template <typename T>
rfd_status fft_c2c(rfd_ctx *ctx, int64_t n, int64_t batch, const typename Cplx<T>::type *in,
                   int64_t in_stride, typename Cplx<T>::type *out, int64_t out_stride,
                   typename Cplx<T>::type *tmp, bool inverse, cudaStream_t s) {
    using T2 = typename Cplx<T>::type;
    RFD_REQUIRE(n >= 4 && (n & (n - 1)) == 0, RFD_ERR_SHAPE, "fft: n=%lld is not a power of two >= 4",
                (long long)n);
    if (batch <= 0) return RFD_OK;
    const T2 *tw = nullptr;
    RFD_TRY(get_twiddles<T>(ctx, n, &tw, s));
    int log2n = 0;
    while ((int64_t(1) << log2n) < n) ++log2n;
    const int max_two_pass = sizeof(T2) == 8 ? 22 : 20;   // shared-memory tile limit (FP32 / FP64)
    if (log2n >= 12 && log2n <= max_two_pass) {
        constexpr int EPT = sizeof(T2) == 8 ? 32 : 16;         // elements per thread
        const int log_min_el = sizeof(T2) == 8 ? 13 : 12;      // >= 64 KB of data per block
        const int log_min_c = sizeof(T2) == 8 ? 3 : 2;         // >= 64 B runs in global memory
        const int logN1 = (log2n + 1) / 2, logN2 = log2n - logN1;
        const int N1 = 1 << logN1, N2 = 1 << logN2;
        auto pick_c = [&](int logL, int logOther) {
            return std::min(std::max(log_min_c, log_min_el - logL), logOther);
        };
        const int logCA = pick_c(logN1, logN2), logCB = pick_c(logN2, logN1);
        const int sh = (log2n + 1) / 2;                         // outer twiddle split: 2^sh low entries
        const unsigned thA = (unsigned)((N1 << logCA) / EPT), thB = (unsigned)((N2 << logCB) / EPT);
        const size_t shA = ((size_t)(tile_ld(N1) << logCA) + N1 + ((size_t)1 << sh) + ((size_t)1 << (log2n - sh))) * sizeof(T2);
        const size_t shB = ((size_t)(tile_ld(N2) << logCB) + N2) * sizeof(T2);
        const T2 *stA = nullptr, *stB = nullptr, *hi = nullptr;
        RFD_TRY(get_stage_twiddles<T>(ctx, logN1, &stA, s));
        RFD_TRY(get_stage_twiddles<T>(ctx, logN2, &stB, s));
        RFD_TRY(get_twiddles<T>(ctx, n >> sh, &hi, s));
        // set once per device and T, so that calls inside a stream capture make no other runtime call
        static bool attr_set[64] = {};
        const int dev = ctx->device < 64 ? ctx->device : 63;
        if (!attr_set[dev]) {
            const int mx = 200 * 1024;
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_fft_cols<T, EPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_fft_rows<T, EPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_fft_cols<T, EPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_fft_rows<T, EPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            attr_set[dev] = true;
        }
        // the whole batch in one launch per pass (chunking the batch so that the intermediate
        // stays in L2 measured slower: the short grids lose more to wave tails)
        for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
            const unsigned gy = (unsigned)std::min<int64_t>(65535, batch - b0);
            const dim3 gA((unsigned)(N2 >> logCA), gy), gB((unsigned)(N1 >> logCB), gy);
            if (inverse) {
                k_fft_cols<T, EPT, true><<<gA, thA, shA, s>>>(in + b0 * in_stride, in_stride, tmp, n, logN1, logN2, logCA, sh, stA, tw, hi, 0);
                RFD_LAUNCH_CHECK();
                k_fft_rows<T, EPT, true><<<gB, thB, shB, s>>>(tmp, n, out + b0 * out_stride, out_stride, logN1, logN2, logCB, stB, 0);
                RFD_LAUNCH_CHECK();
            } else {
                k_fft_cols<T, EPT, false><<<gA, thA, shA, s>>>(in + b0 * in_stride, in_stride, tmp, n, logN1, logN2, logCA, sh, stA, tw, hi, 0);
                RFD_LAUNCH_CHECK();
                k_fft_rows<T, EPT, false><<<gB, thB, shB, s>>>(tmp, n, out + b0 * out_stride, out_stride, logN1, logN2, logCB, stB, 0);
                RFD_LAUNCH_CHECK();
            }
        }
        return RFD_OK;
    }
    std::vector<int> radix;
    if (log2n % 4) radix.push_back(1 << (log2n % 4));
    for (int i = 0; i < log2n / 4; ++i) radix.push_back(16);
    const int P = (int)radix.size();
    int64_t ns = 1;
    const T2 *src = in;
    int64_t src_stride = in_stride;
    for (int p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p) % 2) == 0;
        T2 *dst = to_out ? out : tmp;
        const int64_t dst_stride = to_out ? out_stride : n;
        const int R = radix[p];
        const int64_t nr = n / R;
        const unsigned gx = (unsigned)((nr + 255) / 256);
        for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
            const unsigned gy = (unsigned)std::min<int64_t>(65535, batch - b0);
            dim3 grid(gx, gy);
#define RFD_PASS(RR)                                                                                       \
    do {                                                                                                   \
        if (inverse)                                                                                       \
            k_stockham<T, RR, true><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0);  \
        else                                                                                               \
            k_stockham<T, RR, false><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0); \
    } while (0)
            if (R == 2) RFD_PASS(2);
            else if (R == 4) RFD_PASS(4);
            else if (R == 8) RFD_PASS(8);
            else RFD_PASS(16);
#undef RFD_PASS
            RFD_LAUNCH_CHECK();
        }
        ns *= R;
        src = dst;
        src_stride = dst_stride;
    }
    return RFD_OK;
}

// FINDCHIRP over templates h (complex64 [J][nf]) with the weights GW (length n/2): pass A
// into tmp (J n complex64), sigma^2 per template, pass B with the trigger epilogue.  n must be
// in [2^12, 2^22].
rfd_status findchirp_fused(rfd_ctx *ctx, int64_t n, int64_t J, const float4 *GW, const float2 *h,
                           int64_t nf, int32_t j0, float thr, int32_t W, float2 *tmp, double *part,
                           double *sig2, rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s) {
    int log2n = 0;
    while ((int64_t(1) << log2n) < n) ++log2n;
    RFD_REQUIRE(log2n >= 12 && log2n <= 22, RFD_ERR_SHAPE, "findchirp: n=%lld outside [2^12, 2^22]", (long long)n);
    constexpr int EPT = 32;
    const int logN1 = (log2n + 1) / 2, logN2 = log2n - logN1;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    auto pick_c = [&](int logL, int logOther) { return std::min(std::max(2, 12 - logL), logOther); };
    const int logCA = pick_c(logN1, logN2), logCB = pick_c(logN2, logN1);
    const int sh = (log2n + 1) / 2;
    const unsigned thA = (unsigned)((N1 << logCA) / EPT), thB = (unsigned)((N2 << logCB) / EPT);
    const size_t shA = ((size_t)(tile_ld(N1) << logCA) + N1 + ((size_t)1 << sh) + ((size_t)1 << (log2n - sh))) *
                       sizeof(float2);
    const size_t shB = ((size_t)(tile_ld(N2) << logCB) + N2) * sizeof(float2);
    const float2 *tw = nullptr, *stA = nullptr, *stB = nullptr, *hi = nullptr;
    RFD_TRY(get_twiddles<float>(ctx, n, &tw, s));
    RFD_TRY(get_stage_twiddles<float>(ctx, logN1, &stA, s));
    RFD_TRY(get_stage_twiddles<float>(ctx, logN2, &stB, s));
    RFD_TRY(get_twiddles<float>(ctx, n >> sh, &hi, s));
    static bool attr_set[64] = {};
    const int dev = ctx->device < 64 ? ctx->device : 63;
    if (!attr_set[dev]) {
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_fc_cols<EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_fc_rows<EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set[dev] = true;
    }
    for (int64_t b0 = 0; b0 < J; b0 += 65535) {
        const int64_t nb = std::min<int64_t>(65535, J - b0);
        const dim3 gA((unsigned)(N2 >> logCA), (unsigned)nb), gB((unsigned)(N1 >> logCB), (unsigned)nb);
        k_fc_cols<EPT><<<gA, thA, shA, s>>>(GW, h + b0 * nf, nf, tmp, logN1, logN2, logCA, sh, stA, tw, hi, part);
        RFD_LAUNCH_CHECK();
        k_fc_sum<<<(unsigned)nb, 32, 0, s>>>(part, (int64_t)gA.x, sig2);
        RFD_LAUNCH_CHECK();
        k_fc_rows<EPT><<<gB, thB, shB, s>>>(tmp, logN1, logN2, logCB, stB, sig2, (int32_t)(j0 + b0), thr, (uint32_t)W,
                                            cand, cap, (unsigned long long *)count);
        RFD_LAUNCH_CHECK();
    }
    return RFD_OK;
}

template rfd_status fft_c2c<float>(rfd_ctx *, int64_t, int64_t, const float2 *, int64_t, float2 *,
                                   int64_t, float2 *, bool, cudaStream_t);
template rfd_status fft_c2c<double>(rfd_ctx *, int64_t, int64_t, const double2 *, int64_t,
                                    double2 *, int64_t, double2 *, bool, cudaStream_t);

}  // namespace rfd
