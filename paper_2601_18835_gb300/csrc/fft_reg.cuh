// Register-level pieces of the Stockham transforms (fft.cu, rf_fft.cu): complex products and
// the R-point DFT (R = 2, 4, 8, 16) as an unrolled radix-2 decimation-in-time network over the
// exact 16th roots of unity.
#pragma once
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

// cos and sin of 2 pi e / 16 for e = 0 .. 7 (the roots a radix-2 stage of an R <= 16 DFT
// uses), as compile-time constants so that they fold into the instructions.
__host__ __device__ constexpr double cos16(int e) {
    return e == 0 ? 1.0
         : e == 1 ? 0.92387953251128675613
         : e == 2 ? 0.70710678118654752440
         : e == 3 ? 0.38268343236508977173
         : e == 4 ? 0.0
         : e == 5 ? -0.38268343236508977173
         : e == 6 ? -0.70710678118654752440
                  : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int e) {
    return e == 0 ? 0.0
         : e == 1 ? 0.38268343236508977173
         : e == 2 ? 0.70710678118654752440
         : e == 3 ? 0.92387953251128675613
         : e == 4 ? 1.0
         : e == 5 ? 0.92387953251128675613
         : e == 6 ? 0.70710678118654752440
                  : 0.38268343236508977173;
}

__host__ __device__ constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}

// The R-point DFT is written as compile-time recursion (stages, then butterflies), so every
// array index and every root is a constant and the arrays stay in registers; the same network
// as loops can leave indices to run time in a large kernel and put the arrays in local memory.

// a[bitrev(i)] = v[i] for i = I .. R-1
template <int R, int I>
struct BitrevCopy {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&a)[R], const T2 (&v)[R]) {
        constexpr int L = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
        constexpr int d = bitrev(I, L);
        a[d] = v[I];
        BitrevCopy<R, I + 1>::run(a, v);
    }
};
template <int R>
struct BitrevCopy<R, R> {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&)[R], const T2 (&)[R]) {}
};

// One radix-2 butterfly (x, y) <- (x + w y, x - w y), w = root16^E (inverse) or its conjugate.
// In single precision each (re, im) operation is one packed FP32 instruction (sm_100 and
// later): the FP32 pipe does the same work, but in half the issue slots, which is what binds
// the register transforms.  With ys = (y.im, y.re):
//   E = 0:  x + y, x - y;
//   E = 4:  x + s ys, x - s ys with s = (-1, 1) (inverse) or (1, -1);
//   else:   x + (wr, wr) y + (-wi, wi) ys, x - (wr, wr) y - (-wi, wi) ys.
template <typename T, bool INV, int E, typename T2>
__device__ __forceinline__ void bfly(T2 &x, T2 &y) {
    if constexpr (sizeof(T) == 4) {
        const float2 xo = x;
        if constexpr (E == 0) {
            x = __fadd2_rn(xo, y);
            y = __ffma2_rn(y, make_float2(-1.f, -1.f), xo);
        } else if constexpr (E == 4) {
            const float2 ys = make_float2(y.y, y.x);
            x = __ffma2_rn(ys, INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f), xo);
            y = __ffma2_rn(ys, INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), xo);
        } else {
            constexpr float wr = (float)cos16(E);
            constexpr float wi = INV ? (float)sin16(E) : -(float)sin16(E);
            const float2 ys = make_float2(y.y, y.x);
            x = __ffma2_rn(make_float2(wr, wr), y, __ffma2_rn(make_float2(-wi, wi), ys, xo));
            y = __ffma2_rn(make_float2(-wr, -wr), y, __ffma2_rn(make_float2(wi, -wi), ys, xo));
        }
    } else {
        T2 yw;
        if constexpr (E == 0) {
            yw = y;
        } else if constexpr (E == 4) {                       // times +i (inverse) or -i
            yw = INV ? T2{-y.y, y.x} : T2{y.y, -y.x};
        } else {
            constexpr T wr = (T)cos16(E);
            constexpr T wi = INV ? (T)sin16(E) : -(T)sin16(E);
            yw = T2{y.x * wr - y.y * wi, y.x * wi + y.y * wr};
        }
        const T2 xo = x;
        x = T2{xo.x + yw.x, xo.y + yw.y};
        y = T2{xo.x - yw.x, xo.y - yw.y};
    }
}

// Butterflies I .. R/2-1 of the stage with span M: butterfly I pairs g + t and g + t + M/2,
// g = (I / (M/2)) M, t = I mod (M/2), with the root exp(2 pi i t / M) = root16^(16 t / M).
template <typename T, int R, bool INV, int M, int I>
struct DitStage {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&a)[R]) {
        constexpr int half = M / 2, g = (I / half) * M, t = I % half;
        bfly<T, INV, t * (16 / M)>(a[g + t], a[g + t + half]);
        DitStage<T, R, INV, M, I + 1>::run(a);
    }
};
template <typename T, int R, bool INV, int M>
struct DitStage<T, R, INV, M, R / 2> {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&)[R]) {}
};

template <typename T, int R, bool INV, int M>
struct DitStages {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&a)[R]) {
        DitStage<T, R, INV, M, 0>::run(a);
        DitStages<T, R, INV, 2 * M>::run(a);
    }
};
template <typename T, int R, bool INV>
struct DitStages<T, R, INV, 2 * R> {
    template <typename T2>
    __device__ __forceinline__ static void run(T2 (&)[R]) {}
};

// y[k] = sum_r v[r] exp(sign 2 pi i r k / R), in place, R = 2, 4, 8 or 16 (radix-2
// decimation in time: bit-reversed input order, stages of span 2, 4, .., R).
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(typename Cplx<T>::type (&v)[R]) {
    using T2 = typename Cplx<T>::type;
    T2 a[R];
    BitrevCopy<R, 0>::run(a, v);
    DitStages<T, R, INV, 2>::run(a);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[r];
}

}  // namespace
}  // namespace rfd
