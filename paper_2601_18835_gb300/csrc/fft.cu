// Hand-written Stockham FFT (FP32 and FP64) for the matched filter of Eq. 1, the reference
// series of Eq. 3 and the FP64 tap design of Sec. V.
//
// Stockham auto-sort: each pass p with radix R reads element j + r n/R (r < R), applies the
// twiddles exp(+-2 pi i r (j mod Ns) / (Ns R)), does an R-point DFT in registers and writes
// to (j - j mod Ns) R + (j mod Ns) + r Ns, where Ns is the product of the radices of the
// earlier passes.  No bit reversal is needed.  Radix-16 passes, preceded by one radix-2, -4
// or -8 pass when log2 n is not a multiple of 4 (n = 2^19: 5 passes over memory).  The
// R-point DFT is an unrolled radix-2 decimation-in-time network over the 16th roots of
// unity; the pass twiddles come from a table w[m] = exp(+2 pi i m / n) built once per n with
// FP64 sincospi.
#include "internal.cuh"

namespace rfd {

namespace {

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T2>
__device__ __forceinline__ T2 cmulc(T2 a, T2 b) {   // a * conj(b)
    return T2{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

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

// cos and sin of 2 pi t / 16, t = 0 .. 15 (exact values of the 16th roots of unity)
__device__ __constant__ double kRoot16[16][2] = {
    {1.0, 0.0},
    {0.92387953251128675613, 0.38268343236508977173},
    {0.70710678118654752440, 0.70710678118654752440},
    {0.38268343236508977173, 0.92387953251128675613},
    {0.0, 1.0},
    {-0.38268343236508977173, 0.92387953251128675613},
    {-0.70710678118654752440, 0.70710678118654752440},
    {-0.92387953251128675613, 0.38268343236508977173},
    {-1.0, 0.0},
    {-0.92387953251128675613, -0.38268343236508977173},
    {-0.70710678118654752440, -0.70710678118654752440},
    {-0.38268343236508977173, -0.92387953251128675613},
    {0.0, -1.0},
    {0.38268343236508977173, -0.92387953251128675613},
    {0.70710678118654752440, -0.70710678118654752440},
    {0.92387953251128675613, -0.38268343236508977173}};

__host__ __device__ constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}

// y[k] = sum_r v[r] exp(sign 2 pi i r k / R), in place, R = 2, 4, 8 or 16.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(typename Cplx<T>::type (&v)[R]) {
    using T2 = typename Cplx<T>::type;
    constexpr int L = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
    T2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[bitrev(r, L)] = v[r];
#pragma unroll
    for (int m = 2; m <= R; m <<= 1) {
        const int half = m >> 1;
#pragma unroll
        for (int g = 0; g < R; g += m) {
#pragma unroll
            for (int t = 0; t < half; ++t) {
                const int e = t * (16 / m);                       // exp(2 pi i t / m) = root16^e
                const T wr = (T)kRoot16[e][0];
                const T wi = INV ? (T)kRoot16[e][1] : -(T)kRoot16[e][1];
                const T2 x = a[g + t], y = a[g + t + half];
                const T2 yw = T2{y.x * wr - y.y * wi, y.x * wi + y.y * wr};
                a[g + t] = T2{x.x + yw.x, x.y + yw.y};
                a[g + t + half] = T2{x.x - yw.x, x.y - yw.y};
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[r];
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

}  // namespace

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

template rfd_status fft_c2c<float>(rfd_ctx *, int64_t, int64_t, const float2 *, int64_t, float2 *,
                                   int64_t, float2 *, bool, cudaStream_t);
template rfd_status fft_c2c<double>(rfd_ctx *, int64_t, int64_t, const double2 *, int64_t,
                                    double2 *, int64_t, double2 *, bool, cudaStream_t);

}  // namespace rfd
