// Hand-written Stockham FFT (FP32 and FP64) for the matched filter of Eq. 1, the reference
// series of Eq. 3 and the FP64 tap design of Sec. V.
//
// Stockham auto-sort: each pass p with radix R reads element j + r n/R (r < R), applies the
// twiddles exp(+-2 pi i r (j mod Ns) / (Ns R)), does a radix-R butterfly in registers and
// writes to (j - j mod Ns) R + (j mod Ns) + r Ns, where Ns is the product of the radices of
// the earlier passes.  No bit reversal is needed.  A radix-2 pass is used first when log2 n
// is odd, then radix-4 passes.  Twiddles come from a table w[m] = exp(+2 pi i m / n) built
// once per n with FP64 sincospi.
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
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return T2{a.x + b.x, a.y + b.y}; }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return T2{a.x - b.x, a.y - b.y}; }

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
    if (R == 2) {
        const T2 a = v[0], c = v[1];
        v[0] = cadd(a, c);
        v[1] = csub(a, c);
    } else {
        const T2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        const T2 a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        // multiply d by +i (inverse) or -i (forward)
        const T2 a3 = INV ? T2{-d.y, d.x} : T2{d.y, -d.x};
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
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
    if (log2n & 1) radix.push_back(2);
    for (int i = 0; i < log2n / 2; ++i) radix.push_back(4);
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
            if (R == 2) {
                if (inverse)
                    k_stockham<T, 2, true><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0);
                else
                    k_stockham<T, 2, false><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0);
            } else {
                if (inverse)
                    k_stockham<T, 4, true><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0);
                else
                    k_stockham<T, 4, false><<<grid, 256, 0, s>>>(src, src_stride, dst, dst_stride, tw, n, ns, b0);
            }
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
