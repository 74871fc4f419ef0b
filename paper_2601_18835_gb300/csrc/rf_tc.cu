// Tensor-core ratio filter (Eq. 3) with the fused trigger epilogue, sm_103a (tcgen05 + TMEM).
//
// For the templates of one tile (same reference, NT of them: 128 when K <= 128, 64 when
// K <= 256, 32 when K <= 512) and one item of 128 output positions u0 .. u0+127:
//   Y[a, u] = sum_k P[a, k] q[u + k],  P = reversed taps scaled by 2^e_a, q scaled by 2^e_r,
// with hi/lo splits of both operands (three products hi*hi + hi*lo + lo*hi) and FP32
// accumulation in tensor memory.  The complex product uses the real block form arranged so
// that every MMA is one instruction of N = 2 NT (a tcgen05.mma costs about the same for any
// N <= 256, so wide N is what keeps the tensor pipe full):
//   D = [Re Y | -Im Y] (N = 2 NT columns),
//   D += Qr_h [Pr;-Pi]_h^T + Qr_h [Pr;-Pi]_l^T + Qr_l [Pr;-Pi]_h^T
//      + (-Qi)_h [Pi;Pr]_h^T + (-Qi)_h [Pi;Pr]_l^T + (-Qi)_l [Pi;Pr]_h^T.
// The taps image holds the rows [Pi; Pr; -Pi] once, so [Pi;Pr] and [Pr;-Pi] are its rows
// 0..2NT-1 and NT..3NT-1 (two descriptors into one image).
//
// A (the Hankel operand A[u, k] = q[u0 + u + k], M = 128 rows = TMEM lanes, planes Qr_h,
// -Qi_h, Qr_l, -Qi_l) is written into tensor memory by four builder warps with tcgen05.st,
// 16 taps per stage (8 stages), so the Toeplitz expansion never goes through shared memory.
// B (the tile's taps) stays in shared memory in the K-major 128-byte swizzle layout,
// bulk-copied once per tile change from the image rfd_plan_set_taps pre-swizzles.  One CTA
// per SM walks a contiguous, cost-balanced range of (tile, time block) items.  Roles: warp 0
// bulk copies, warp 1 issues the MMAs (and owns the TMEM allocation), warps 4-7 build A,
// warps 8-15 drain the accumulator and run the epilogue.  Every wait is bounded.  Every bulk
// copy completes on a barrier that only the producer arms, and before the CTA ends the producer
// waits (bounded) for the last phase it armed on each: no copy is still landing in shared
// memory when the CTA exits, also after a wait has given up.
#include "epilogue.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kM = 128;           // output positions per item (MMA M, TMEM lanes)
constexpr int kStages = 8;        // A stages in TMEM, 32 columns each
constexpr int kThreads = 512;
constexpr int kEpiWarps = 8;      // two per TMEM lane group, each half of the templates
constexpr uint32_t kACol = 256;   // first TMEM column of the A stages (D uses 0 .. 2 NT - 1)
constexpr uint32_t kSpin = 1u << 22;
constexpr uint32_t kSpinStall = 1u << 12;        // RFD_DEBUG_STALL_TAPS: give up quickly

enum {
    kBarTapsFull = 0,
    kBarTapsEmpty = 1,
    kBarQFull = 2,     // 2
    kBarQEmpty = 4,    // 2
    kBarAFull = 6,     // kStages
    kBarAEmpty = 14,   // kStages
    kBarDFull = 22,
    kBarDEmpty = 23,
    kBarDone = 24,
    kNumBars = 25
};

struct TcArgs {
    const TcTile *tiles;
    const int64_t *ranges;      // [gridDim.x + 1] item ranges
    int64_t n_tt;               // time blocks per tile = window length / 128
    const int64_t *u_begin;     // first output position of the window (device), or NULL
    const uint8_t *taps;        // operand images
    const uint16_t *q;          // q planes (fp16 or bf16 bits)
    int64_t ld;
    const int32_t *qscale;
    const int32_t *perm;
    const int32_t *off;
    const float *scale;
    int64_t n;
    float thr;
    uint32_t W;
    rfd_candidate *cand;
    int64_t cap;
    unsigned long long *count;
    uint32_t taps_cap;          // bytes of the taps region
    uint32_t win;               // elements per q window plane
    uint32_t spin;              // polls before a wait gives up
    uint32_t stall;             // RFD_DEBUG_STALL_TAPS: never copy the taps (tests the abort path)
};

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile uint32_t *abort_flag,
                                         unsigned long long *count, uint32_t spin) {
    for (uint32_t i = 0; i < spin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1u;
    atomicOr(count, 1ull << 62);   // reported as RFD_ERR_TIMEOUT by find_triggers
    return false;
}

template <int BF16>
__global__ void __launch_bounds__(kThreads, 1) k_rf_tc(const TcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *s_taps = sm;
    uint16_t *s_q = (uint16_t *)(sm + A.taps_cap);
    uint64_t *bars = (uint64_t *)(sm + A.taps_cap + 2u * 4u * A.win * 2u);
    uint32_t *s_misc = (uint32_t *)(bars + kNumBars);
    volatile uint32_t *abort_flag = &s_misc[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t it0 = A.ranges[blockIdx.x], it1 = A.ranges[blockIdx.x + 1];
    const int64_t ubase = window_base(A.u_begin, A.n);
    const uint32_t bar0 = smem_u32(bars);
#define BAR(i) (bar0 + 8u * (uint32_t)(i))

    if (threadIdx.x == 0) {
        mbar_init(BAR(kBarTapsFull), 1);
        mbar_init(BAR(kBarTapsEmpty), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(BAR(kBarQFull + b), 1);
            mbar_init(BAR(kBarQEmpty + b), 4);
        }
        mbar_init(BAR(kBarDFull), 1);
        mbar_init(BAR(kBarDEmpty), kEpiWarps);
        for (int s = 0; s < kStages; ++s) {
            mbar_init(BAR(kBarAFull + s), 4);
            mbar_init(BAR(kBarAEmpty + s), 1);
        }
        mbar_init(BAR(kBarDone), 1);
        s_misc[1] = 0u;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(smem_u32(&s_misc[0]), 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_misc[0];

    if (warp == 0) {
        // ------------------------------------------------------------ producer (bulk copies)
        if (lane == 0) {
            uint32_t tchg = 0, li = 0;
            uint32_t taps_armed = 0u, q_armed[2] = {0u, 0u};   // phases armed (for the final drain)
            int64_t prev = -1;
            for (int64_t it = it0; it < it1; ++it, ++li) {
                const int64_t ti = it / A.n_tt, tt = it - ti * A.n_tt;
                const TcTile T = A.tiles[ti];
                if (ti != prev) {
                    if (!wait_bar(BAR(kBarTapsEmpty), (tchg & 1u) ^ 1u, abort_flag, A.count, A.spin)) break;
                    if (!A.stall) {                // stalled: the taps barrier never completes
                        mbar_arrive_expect_tx(BAR(kBarTapsFull), (uint32_t)T.taps_bytes);
                        ++taps_armed;
                        for (uint32_t o = 0; o < (uint32_t)T.taps_bytes; o += 32768u) {
                            const uint32_t len = min(32768u, (uint32_t)T.taps_bytes - o);
                            bulk_g2s(smem_u32(s_taps) + o, A.taps + T.taps_off + o, len, BAR(kBarTapsFull));
                        }
                    }
                    ++tchg;
                    prev = ti;
                }
                const uint32_t qb = li & 1u, use = li >> 1;
                if (!wait_bar(BAR(kBarQEmpty + qb), (use & 1u) ^ 1u, abort_flag, A.count, A.spin)) break;
                const uint32_t wbytes = (uint32_t)(kM + T.kpad) * 2u;
                mbar_arrive_expect_tx(BAR(kBarQFull + qb), 4u * wbytes);
                ++q_armed[qb];
                for (int p = 0; p < 4; ++p) {
                    const uint16_t *src = A.q + (int64_t)(4 * T.ref + p) * A.ld + wrap_pos(ubase, tt * kM, A.n);
                    bulk_g2s(smem_u32(s_q + (qb * 4 + p) * A.win), src, wbytes, BAR(kBarQFull + qb));
                }
            }
            // drain: the last phase armed on each copy barrier has completed before this thread
            // reaches the CTA's final barrier (bounded, like every wait)
            const uint32_t bars3[3] = {BAR(kBarTapsFull), BAR(kBarQFull), BAR(kBarQFull + 1)};
            const uint32_t armed[3] = {taps_armed, q_armed[0], q_armed[1]};
            for (int k = 0; k < 3; ++k) {
                if (armed[k] == 0u) continue;
                uint32_t i = 0;
                while (i < kSpin && !mbar_try_wait(bars3[k], (armed[k] - 1u) & 1u)) ++i;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t tchg = 0, li = 0, ka = 0;
            int64_t prev = -1;
            const uint32_t taps_addr = smem_u32(s_taps);
            for (int64_t it = it0; it < it1; ++it, ++li) {
                const int64_t ti = it / A.n_tt;
                const TcTile T = A.tiles[ti];
                if (ti != prev) {
                    if (!wait_bar(BAR(kBarTapsFull), tchg & 1u, abort_flag, A.count, A.spin)) break;
                    ++tchg;
                    prev = ti;
                }
                if (!wait_bar(BAR(kBarDEmpty), (li & 1u) ^ 1u, abort_flag, A.count, A.spin)) break;
                fence_after();
                const uint32_t nt = (uint32_t)T.nt;
                const uint32_t d = tmem;
                const uint32_t idn = idesc_f16(128, 2 * nt, BF16, 0);
                const uint32_t chunk_bytes = 3u * nt * 128u;
                bool ok = true;
                for (int s = 0; s < T.nk16; ++s, ++ka) {
                    const uint32_t st = ka % kStages, r = ka / kStages;
                    if (!wait_bar(BAR(kBarAFull + st), r & 1u, abort_flag, A.count, A.spin)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t c = (uint32_t)s >> 2, o = ((uint32_t)s & 3u) * 32u;
                    const uint32_t bh = taps_addr + c * chunk_bytes + o;
                    const uint32_t bl = taps_addr + ((uint32_t)T.nch + c) * chunk_bytes + o;
                    const uint64_t B2h = desc_sw128(bh), B2l = desc_sw128(bl);                    // [Pi; Pr]
                    const uint64_t B1h = desc_sw128(bh + nt * 128u), B1l = desc_sw128(bl + nt * 128u);  // [Pr; -Pi]
                    const uint32_t a_qr_h = tmem + kACol + st * 32u;
                    const uint32_t a_qi_h = a_qr_h + 8u, a_qr_l = a_qr_h + 16u, a_qi_l = a_qr_h + 24u;
                    mma_ts(d, a_qr_h, B1h, idn, s > 0 ? 1u : 0u);
                    mma_ts(d, a_qr_h, B1l, idn, 1u);
                    mma_ts(d, a_qr_l, B1h, idn, 1u);
                    mma_ts(d, a_qi_h, B2h, idn, 1u);
                    mma_ts(d, a_qi_h, B2l, idn, 1u);
                    mma_ts(d, a_qi_l, B2h, idn, 1u);
                    mma_commit(BAR(kBarAEmpty + st));
                }
                if (!ok) break;
                mma_commit(BAR(kBarDFull));
                const bool last_of_tile = (it + 1 == it1) || ((it + 1) / A.n_tt != ti);
                if (last_of_tile) mma_commit(BAR(kBarTapsEmpty));
            }
            // every MMA this thread issued has completed before TMEM is released
            mma_commit(BAR(kBarDone));
            for (uint32_t i = 0; i < kSpin && !mbar_try_wait(BAR(kBarDone), 0); ++i) {
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------------------ Hankel builders -> TMEM
        const uint32_t lg = (uint32_t)warp & 3u;
        const uint32_t row = lg * 32u + (uint32_t)lane;
        const uint32_t tlane = (lg * 32u) << 16;
        uint32_t li = 0, ka = 0;
        for (int64_t it = it0; it < it1; ++it, ++li) {
            const int64_t ti = it / A.n_tt;
            const int nk16 = A.tiles[ti].nk16;
            const uint32_t qb = li & 1u, use = li >> 1;
            bool ok = wait_bar(BAR(kBarQFull + qb), use & 1u, abort_flag, A.count, A.spin);
            if (!__all_sync(0xffffffffu, ok)) break;
            const uint32_t *W0 = (const uint32_t *)(s_q + (qb * 4 + 0) * A.win);
            const uint32_t *W1 = (const uint32_t *)(s_q + (qb * 4 + 1) * A.win);
            const uint32_t *W2 = (const uint32_t *)(s_q + (qb * 4 + 2) * A.win);
            const uint32_t *W3 = (const uint32_t *)(s_q + (qb * 4 + 3) * A.win);
            for (int s = 0; s < nk16; ++s, ++ka) {
                const uint32_t st = ka % kStages, r = ka / kStages;
                ok = wait_bar(BAR(kBarAEmpty + st), (r & 1u) ^ 1u, abort_flag, A.count, A.spin);
                if (!__all_sync(0xffffffffu, ok)) break;
                const uint32_t e0 = row + (uint32_t)s * 16u, w0 = e0 >> 1, sh = (e0 & 1u) * 16u;
                uint32_t v[32];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const uint32_t *Wp = p == 0 ? W0 : (p == 1 ? W1 : (p == 2 ? W2 : W3));
                    uint32_t prev = Wp[w0];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t nx = Wp[w0 + i + 1];
                        // the Qi planes (1, 3) go in negated: flip both halves' sign bits
                        v[p * 8 + i] = __funnelshift_r(prev, nx, sh) ^ ((p & 1) ? 0x80008000u : 0u);
                        prev = nx;
                    }
                }
                tmem_st32(tmem + tlane + kACol + st * 32u, v);
                tmem_st_wait();
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(BAR(kBarAFull + st));
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(BAR(kBarQEmpty + qb));
        }
    } else if (warp >= 8 && warp < 8 + kEpiWarps) {
        // ------------------------------------------------------------ epilogue
        const uint32_t lg = (uint32_t)warp & 3u;
        const int half = (warp - 8) >> 2;                 // which half of the tile's templates
        const uint32_t row = lg * 32u + (uint32_t)lane;
        const uint32_t tlane = (lg * 32u) << 16;
        uint32_t li = 0;
        for (int64_t it = it0; it < it1; ++it, ++li) {
            const int64_t ti = it / A.n_tt, tt = it - ti * A.n_tt;
            const TcTile T = A.tiles[ti];
            const bool ok = wait_bar(BAR(kBarDFull), li & 1u, abort_flag, A.count, A.spin);
            if (!__all_sync(0xffffffffu, ok)) break;
            fence_after();
            const float esc = ldexpf(1.0f, -A.qscale[T.ref]);
            const int64_t u = wrap_pos(ubase, tt * kM, A.n) + row;
            const int per = T.nt >> 1;                    // templates per half (multiple of 8)
            const int a_begin = half * per, a_end = a_begin + per;
            if (per < 32 && half == 1) {
                // nothing to drain for this warp when the tile is narrow
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(BAR(kBarDEmpty));
                continue;
            }
            const int step = per < 32 ? 2 * per : 32;     // narrow tiles: one warp takes all
            const int lo = per < 32 ? 0 : a_begin, hi = per < 32 ? T.nt : a_end;
            for (int a0 = lo; a0 < hi; a0 += 32) {
                const int my_a = a0 + lane;
                const bool my_valid = my_a < T.count && my_a < hi;
                const int64_t my_slot = (int64_t)T.first + (my_valid ? my_a : 0);
                const float my_sc = my_valid ? A.scale[my_slot] * esc : 0.f;
                // screen factor: |z|^2 = |D|^2 sc^2 against thr lowered by 2^-10 (far above the
                // few-ulp difference to the exact |z|^2 below); 0 for an invalid template
                const float my_inv = my_valid ? (my_sc * my_sc) / (A.thr * (1.0f - 0.0009765625f)) : 0.f;
                uint32_t re[32], im[32];
                tmem_ld32(tmem + tlane + (uint32_t)a0, re);
                tmem_ld32(tmem + tlane + (uint32_t)(T.nt + a0), im);
                tmem_ld_wait();
                if (a0 + 32 >= hi) {
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(BAR(kBarDEmpty));
                }
                // screen the 32 templates of this sample, two per packed FP32 instruction: the
                // largest |D|^2 sc^2 / thr' (a NaN from an invalid template or thr = 0 with
                // |D| = 0 is ignored by the max; such a sample cannot trigger)
                float smax = 0.f;
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float2 r2 = make_float2(__uint_as_float(re[i]), __uint_as_float(re[i + 1]));
                    const float2 i2 = make_float2(__uint_as_float(im[i]), __uint_as_float(im[i + 1]));
                    const float2 f2 = make_float2(__shfl_sync(0xffffffffu, my_inv, i), __shfl_sync(0xffffffffu, my_inv, i + 1));
                    const float2 s2 = __fmul2_rn(__ffma2_rn(r2, r2, __fmul2_rn(i2, i2)), f2);
                    smax = fmaxf(smax, fmaxf(s2.x, s2.y));
                }
                if (!__any_sync(0xffffffffu, smax > 1.0f)) continue;
                // rare: z and |z|^2 exactly as the emitter forms them; one vote for the whole chunk
                uint32_t hit = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float sc = __shfl_sync(0xffffffffu, my_sc, i);
                    const float zr = __fmul_rn(__uint_as_float(re[i]), sc);
                    const float zi = -__fmul_rn(__uint_as_float(im[i]), sc);   // D holds -Im
                    re[i] = __float_as_uint(zr);
                    im[i] = __float_as_uint(zi);
                    const float p = __fadd_rn(__fmul_rn(zr, zr), __fmul_rn(zi, zi));
                    hit |= (p > A.thr ? 1u : 0u) << i;
                }
                if (__any_sync(0xffffffffu, hit != 0u)) {
                    const int32_t my_j = my_valid ? A.perm[my_slot] : 0;
                    const int32_t my_o = my_valid ? A.off[my_slot] : 0;
                    const uint32_t any_bits = __reduce_or_sync(0xffffffffu, hit);
#pragma unroll 1
                    for (int i = 0; i < 32; ++i) {
                        if (!((any_bits >> i) & 1u)) continue;          // warp-uniform
                        const int32_t j = __shfl_sync(0xffffffffu, my_j, i);
                        const int32_t o = __shfl_sync(0xffffffffu, my_o, i);
                        const bool valid = a0 + i < T.count && a0 + i < hi;
                        const uint32_t t = (uint32_t)((u + o) & (A.n - 1));
                        float zr = 0.f, zi = 0.f;
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            if (q == i) {
                                zr = __uint_as_float(re[q]);
                                zi = __uint_as_float(im[q]);
                            }
                        emit_window_max(valid, (uint32_t)j, t, zr, zi, A.thr, A.W, A.cand, A.cap, A.count);
                    }
                }
            }
            (void)step;
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
#undef BAR
}

// ------------------------------------------------------------------ taps packing
template <typename H>
__device__ __forceinline__ uint16_t h_bits(H x);
template <>
__device__ __forceinline__ uint16_t h_bits<__half>(__half x) { return __half_as_ushort(x); }
template <>
__device__ __forceinline__ uint16_t h_bits<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat16_as_ushort(x); }
template <typename H>
__device__ __forceinline__ H to_h(float x);
template <>
__device__ __forceinline__ __half to_h<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_h<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float from_h(__half x) { return __half2float(x); }
__device__ __forceinline__ float from_h(__nv_bfloat16 x) { return __bfloat162float(x); }

// One block per tile: per-template power-of-two scale (max |component| * 2^e < 2^8), then the
// B-operand image: [hl][chunk][row][128 B] with rows [Pi (NT); Pr (NT); -Pi (NT)]; element e
// of a chunk holds reversed tap k = 64 chunk + e, 16-byte units XOR-swizzled by row % 8.
// Also the per-slot lag offset and normalisation.
template <typename H>
__global__ void __launch_bounds__(256) k_pack_tc(const TcTile *__restrict__ tiles, const float2 *__restrict__ taps,
                                                 int32_t k_stride, const int32_t *__restrict__ perm,
                                                 const int32_t *__restrict__ kslot, const int32_t *__restrict__ lag,
                                                 const double *__restrict__ sigma, int64_t n,
                                                 uint8_t *__restrict__ out, int32_t *__restrict__ off,
                                                 float *__restrict__ scale) {
    __shared__ int s_exp[128];
    __shared__ int s_j[128], s_k[128];
    const TcTile T = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = warp; a < T.nt; a += (int)(blockDim.x >> 5)) {
        float mx = 0.f;
        int j = 0, K = 0;
        if (a < T.count) {
            j = perm[T.first + a];
            K = kslot[T.first + a];
            for (int k = lane; k < K; k += 32) {
                const float2 v = taps[(int64_t)j * k_stride + k];
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int e = 0;
            if (mx > 0.f) {
                int ex;
                frexpf(mx, &ex);      // mx < 2^ex
                e = 8 - ex;
            }
            s_exp[a] = e;
            s_j[a] = j;
            s_k[a] = K;
        }
    }
    __syncthreads();
    const int rows = 3 * T.nt;
    const int64_t total = (int64_t)2 * T.nch * rows * 64;
    uint8_t *img = out + T.taps_off;
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int e = (int)(idx & 63);
        const int64_t r1 = idx >> 6;
        const int row = (int)(r1 % rows);
        const int64_t r2 = r1 / rows;
        const int c = (int)(r2 % T.nch);
        const int hl = (int)(r2 / T.nch);
        const int a = row % T.nt, part = row / T.nt;   // 0: Pi, 1: Pr, 2: -Pi
        const int k = 64 * c + e;
        uint16_t bits = 0;
        if (a < T.count && k < s_k[a]) {
            const float2 v = taps[(int64_t)s_j[a] * k_stride + (s_k[a] - 1 - k)];
            const float comp = part == 1 ? v.x : (part == 0 ? v.y : -v.y);
            const float x = ldexpf(comp, s_exp[a]);
            const H hi = to_h<H>(x);
            bits = hl ? h_bits<H>(to_h<H>(x - from_h(hi))) : h_bits<H>(hi);
        }
        const int64_t rowbase = ((int64_t)(hl * T.nch + c) * rows + row) * 128;
        *(uint16_t *)(img + rowbase + ((((e >> 3) ^ (row & 7)) << 4)) + (e & 7) * 2) = bits;
    }
    for (int a = threadIdx.x; a < T.count; a += blockDim.x) {
        const int64_t slot = (int64_t)T.first + a;
        const int j = s_j[a], K = s_k[a];
        off[slot] = (int32_t)((((int64_t)lag[j] + K - 1) % n + n) % n);
        const double sg = sigma[j];
        scale[slot] = sg > 0.0 ? (float)(ldexp(1.0, -s_exp[a]) / sg) : 0.f;
    }
}

}  // namespace

size_t tc_smem_bytes(uint32_t taps_cap, uint32_t win) {
    return 1024 + (size_t)taps_cap + 2u * 4u * win * 2u + kNumBars * 8 + 16;
}

rfd_status tc_pack(rfd_plan *plan, const float2 *taps, int32_t k_stride, const int32_t *lag,
                   const double *sigma, cudaStream_t s) {
    const unsigned ntiles = (unsigned)plan->tc_tiles.size();
    if (ntiles == 0) return RFD_OK;
    if (plan->precision == RFD_PREC_FP16X3)
        k_pack_tc<__half><<<ntiles, 256, 0, s>>>((const TcTile *)plan->d_tiles.p, taps, k_stride,
                                                  (const int32_t *)plan->d_perm.p, (const int32_t *)plan->d_kslot.p,
                                                  lag, sigma, plan->grid.n, (uint8_t *)plan->d_taps.p,
                                                  (int32_t *)plan->d_off.p, (float *)plan->d_scale.p);
    else
        k_pack_tc<__nv_bfloat16><<<ntiles, 256, 0, s>>>(
            (const TcTile *)plan->d_tiles.p, taps, k_stride, (const int32_t *)plan->d_perm.p,
            (const int32_t *)plan->d_kslot.p, lag, sigma, plan->grid.n, (uint8_t *)plan->d_taps.p,
            (int32_t *)plan->d_off.p, (float *)plan->d_scale.p);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

rfd_status tc_launch(const rfd_plan *plan, const void *q, const int32_t *qscale, const int64_t *u_begin,
                     rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s) {
    if (plan->tc_tiles.empty()) return RFD_OK;
    TcArgs a;
    a.tiles = (const TcTile *)plan->d_tiles.p;
    a.ranges = (const int64_t *)plan->d_ranges.p;
    a.n_tt = plan->out_len / kM;
    a.u_begin = u_begin;
    a.taps = (const uint8_t *)plan->d_taps.p;
    a.q = (const uint16_t *)q;
    a.ld = plan->ld;
    a.qscale = qscale;
    a.perm = (const int32_t *)plan->d_perm.p;
    a.off = (const int32_t *)plan->d_off.p;
    a.scale = (const float *)plan->d_scale.p;
    a.n = plan->grid.n;
    a.thr = plan->threshold;
    a.W = (uint32_t)plan->window;
    a.cand = cand;
    a.cap = cap;
    a.count = (unsigned long long *)count;
    a.taps_cap = plan->tc_taps_cap;
    a.win = plan->tc_win;
    a.stall = (plan->debug_flags & RFD_DEBUG_STALL_TAPS) ? 1u : 0u;
    a.spin = a.stall ? kSpinStall : kSpin;
    // at least 120 KB so that exactly one CTA (and one 512-column TMEM allocation) fits per SM
    const size_t shm = std::max<size_t>(tc_smem_bytes(a.taps_cap, a.win), 120 * 1024);
    const unsigned grid = (unsigned)plan->tc_grid;
    // the attribute is set once per device and size, so that launches inside a stream capture
    // make no other runtime calls
    static size_t smem_set[64][2] = {};
    const int dev = plan->ctx->device < 64 ? plan->ctx->device : 63;
    const int bf = plan->precision == RFD_PREC_FP16X3 ? 0 : 1;
    if (shm > smem_set[dev][bf]) {
        if (bf == 0)
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_rf_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        else
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_rf_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        smem_set[dev][bf] = shm;
    }
    if (bf == 0)
        k_rf_tc<0><<<grid, kThreads, shm, s>>>(a);
    else
        k_rf_tc<1><<<grid, kThreads, shm, s>>>(a);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

int tc_rows_per_item() { return kM; }

}  // namespace rfd
