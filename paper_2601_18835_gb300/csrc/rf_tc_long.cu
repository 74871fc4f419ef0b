// Tensor-core ratio filter with templates on the MMA's M side and time on its N side (the
// default for K > 64; full-width MMAs for any K <= 512), sm_103a.
//
// For a tile of 64 templates of one reference and one item of 256 output positions
// u0 .. u0+255:
//   D[row, u] = sum_k A[row, k] q[u0 + u + k]      (Eq. 3 with P = reversed, scaled taps)
// with rows 0..63 the real parts and rows 64..127 the imaginary parts of the 64 templates:
//   D = [Pr; Pi] Qr^T + [-Pi; Pr] Qi^T,
// each as three products hi*hi + hi*lo + lo*hi of the FP16 (BF16) splits, FP32 accumulation in
// tensor memory.  The taps image holds the rows [-Pi; Pr; Pi] once, so the two A operands are
// its rows 0..127 and 64..191; every MMA is M = 128, N = 256, K = 16 (full rate).
//
// The time operand B[u, k] = q[u0 + u + k] is a Hankel matrix.  It is not materialised:
// shared memory holds Y[r] = q[u0 + r .. u0 + r + 7] (16 bytes per row, an eight-fold copy of
// the q window) and the MMA reads it through a K-major, non-swizzled descriptor whose
// K-direction and N-direction strides are both 128 bytes, so that element (u, k) lands on
// Y[u + k - k mod 8][k mod 8] = q[u0 + u + k].  The taps (A) stream through shared memory in
// 64-tap chunks by bulk copies; two accumulators in tensor memory let the epilogue drain one
// item while the MMAs fill the next.
//
// Roles: warp 0 bulk copies (taps chunks and each item's q window), lane 0 of warp 1 issues
// the MMAs (warp 1 owns the TMEM allocation), warps 4-7 expand the q window into Y
// (consecutive lanes on consecutive rows: conflict-free), warps 8-15 drain: a warp of lane
// quarter 2/3 (imaginary rows) and the warp of quarter 0/1 (real rows, same templates) swap
// half of each 32-column chunk through shared memory, and each forms z, |z|^2 and the
// per-window maxima of its 16 columns.  The MMA thread waits once per item, on a barrier of
// the item's buffer that the epilogue (accumulator free), the builders (Y built) and the
// producer (first taps chunk landed) all arrive on.  The tensor pipe queues only a few MMAs
// ahead of the issuing thread, so any hand-off that thread has to make between MMAs idles the
// pipe; a tile of at most two 64-tap chunks (K <= 128) therefore stays resident in the two
// stages, copied at its first item, with no per-chunk hand-off at all; longer taps stream
// through the stages, each chunk released by a commit of the MMAs that read it.  At a tile
// change the producer overwrites a stage only after a commit the MMA thread makes when it
// leaves the previous tile, and it arrives on an item's go barrier only once the go phase of
// the item two back (the same barrier) has completed.  Every wait is bounded.  Each bulk
// copy completes on a barrier that only the producer arms (the first chunk of an item on a
// barrier of its own, which the producer waits on before it arrives on the item's barrier),
// so before the CTA ends the producer can wait for the last phase it armed on each of them:
// no copy is still landing in shared memory when the CTA exits, also after a wait has given
// up.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kN = 256;                 // output positions per item (MMA N)
constexpr int kNT = 64;                 // templates per tile
constexpr int kThreads = 512;
constexpr int kAStages = 2;
constexpr uint32_t kChunkImg = 3u * kNT * 128u;      // one 64-tap chunk, hi or lo: 24 KB
constexpr uint32_t kChunkBytes = 2u * kChunkImg;     // hi + lo: 48 KB
constexpr uint32_t kSpin = 1u << 22;
constexpr uint32_t kSpinStall = 1u << 12;            // RFD_DEBUG_STALL_TAPS: give up quickly
constexpr int kXPitch = 20;     // floats per lane of an exchange buffer: 16 used, 16-byte rows, no bank conflicts

enum {
    kBarAFull = 0,      // kAStages
    kBarAEmpty = 2,     // kAStages
    kBarGo = 4,         // 2: accumulator free + Y built + chunk 0 staged, per item buffer
    kBarDFull = 6,      // 2
    kBarQFull = 8,      // 2
    kBarQEmpty = 10,    // 2
    kBarDone = 12,
    kBarT0 = 13,        // 2: the first taps chunk of an item, per item buffer (producer only)
    kBarTile = 15,      // every MMA before a tile change has completed (one phase per change)
    kNumBars = 16
};

struct TlArgs {
    const TcTile *tiles;
    const int64_t *ranges;      // [gridDim.x + 1] item ranges
    int64_t n_tb;               // time blocks per tile = window length / 256
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
    uint32_t ystride;           // bytes per Y plane
    uint32_t qwin;              // halfs per q-window plane
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

// Shared-memory descriptor of the Hankel operand: K-major, no swizzle, LBO = SBO = 128 B.
__device__ __forceinline__ uint64_t desc_hankel(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void named_sync(uint32_t id, uint32_t threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Appends one candidate (thread-level; every float compare is on the p formed by the caller).
__device__ __forceinline__ void emit_one(uint32_t j, uint32_t w, uint32_t pbits, uint32_t t, float zr, float zi,
                                         rfd_candidate *__restrict__ cand, int64_t cap,
                                         unsigned long long *__restrict__ count) {
    const unsigned long long idx = atomicAdd(count, 1ull);
    if ((int64_t)idx < cap) {
        rfd_candidate c;
        c.key = ((uint64_t)pbits << 32) | (uint64_t)(0xffffffffu - t);
        c.j = j;
        c.w = w;
        c.zr = zr;
        c.zi = zi;
        cand[idx] = c;
    }
}

template <int BF16>
__global__ void __launch_bounds__(kThreads, 1) k_rf_tc_long(const TlArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *s_a = sm;                                              // kAStages x 48 KB
    uint8_t *s_y = sm + kAStages * kChunkBytes;                     // 2 buffers x 4 planes
    uint16_t *s_qw = (uint16_t *)(s_y + 2u * 4u * A.ystride);       // 2 buffers x 4 planes
    float *s_x = (float *)(s_qw + 2u * 4u * A.qwin);                // 4 pairs x 2 x 32 x kXPitch
    uint64_t *bars = (uint64_t *)(s_x + 4 * 2 * 32 * kXPitch);
    uint32_t *s_misc = (uint32_t *)(bars + kNumBars);
    volatile uint32_t *abort_flag = &s_misc[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t it0 = A.ranges[blockIdx.x], it1 = A.ranges[blockIdx.x + 1];
    const int64_t ubase = window_base(A.u_begin, A.n);
    const uint32_t bar0 = smem_u32(bars);
#define BAR(i) (bar0 + 8u * (uint32_t)(i))

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAStages; ++s) {
            mbar_init(BAR(kBarAFull + s), 1);
            mbar_init(BAR(kBarAEmpty + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            // one phase per use of item buffer b: 8 epilogue warps (the accumulator is free),
            // 4 builder warps (Y is built), the producer (chunk 0 of the taps, with its bytes)
            mbar_init(BAR(kBarGo + b), 8 + 4 + 1);
            mbar_init(BAR(kBarDFull + b), 1);
            mbar_init(BAR(kBarQFull + b), 1);
            mbar_init(BAR(kBarQEmpty + b), 4);
            mbar_init(BAR(kBarT0 + b), 1);
        }
        mbar_init(BAR(kBarDone), 1);
        mbar_init(BAR(kBarTile), 1);
        s_misc[1] = 0u;
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(smem_u32(&s_misc[0]), 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_misc[0];

    if (warp == 0) {
        // ------------------------------------------------------------ producer: taps chunks
        if (lane == 0) {
            uint32_t ka = 0, li = 0, ntc = 0;     // ka: streamed chunks so far; ntc: tile changes
            static_assert(kAStages == 2, "two A stages");
            // phases armed so far on each barrier the copies complete on (for the final drain)
            uint32_t q_armed[2] = {0u, 0u}, a_armed[2] = {0u, 0u}, t0_armed[2] = {0u, 0u};
            int64_t ti = it0 / A.n_tb, tb = it0 - ti * A.n_tb, prev = -1;
            TcTile T{};
            for (int64_t it = it0; it < it1; ++it, ++li, tb = (tb + 1 == A.n_tb) ? 0 : tb + 1, ti += (tb == 0)) {
                const bool first = ti != prev;    // the first item of a tile (tiles never recur in a range)
                if (first) {
                    T = A.tiles[ti];
                    prev = ti;
                }
                // this item's q window, 256 + kpad samples of each plane
                const uint32_t qb = li & 1u, use = li >> 1;
                if (!wait_bar(BAR(kBarQEmpty + qb), (use & 1u) ^ 1u, abort_flag, A.count, A.spin)) break;
                const uint32_t wbytes = (uint32_t)(kN + T.kpad) * 2u;
                mbar_arrive_expect_tx(BAR(kBarQFull + qb), 4u * wbytes);
                ++q_armed[qb];
                for (int p = 0; p < 4; ++p)
                    bulk_g2s(smem_u32(s_qw + (qb * 4u + (uint32_t)p) * A.qwin),
                             A.q + (int64_t)(4 * T.ref + p) * A.ld + wrap_pos(ubase, tb * kN, A.n), wbytes,
                             BAR(kBarQFull + qb));
                if (A.stall) continue;            // no taps: the item's go barrier never completes
                const uint32_t ib = li & 1u;
                // a new tile: every MMA before it has completed before a copy overwrites a stage
                // (the MMA issuer commits once after the last item of each tile it leaves)
                if (first && li > 0u) {
                    if (!wait_bar(BAR(kBarTile), ntc & 1u, abort_flag, A.count, A.spin)) break;
                    ++ntc;
                }
                // the go phase of item li - 2 (same barrier) has completed before this item's
                // arrival below, so the arrivals of two items never meet in one phase
                if (li >= 2u && !wait_bar(BAR(kBarGo + ib), ((li >> 1) & 1u) ^ 1u, abort_flag, A.count, A.spin))
                    break;
                bool ok = true;
                if (T.nch <= kAStages) {
                    // resident tile (K <= 128): chunk c stays in stage c for all of the tile's items,
                    // copied at its first item (chunk 0 on the item's transaction barrier, chunk 1
                    // on stage 1's); no per-chunk hand-off afterwards
                    if (first) {
                        for (int c = 0; c < T.nch; ++c) {
                            const uint32_t full = c == 0 ? BAR(kBarT0 + ib) : BAR(kBarAFull + 1);
                            mbar_arrive_expect_tx(full, kChunkBytes);
                            const uint8_t *src = A.taps + T.taps_off + (int64_t)c * kChunkBytes;
                            bulk_g2s(smem_u32(s_a + (uint32_t)c * kChunkBytes), src, kChunkImg, full);
                            bulk_g2s(smem_u32(s_a + (uint32_t)c * kChunkBytes) + kChunkImg, src + kChunkImg, kChunkImg,
                                     full);
                            if (c > 0) ++a_armed[1];
                        }
                        const uint32_t par = t0_armed[ib]++ & 1u;
                        if (!wait_bar(BAR(kBarT0 + ib), par, abort_flag, A.count, A.spin)) break;
                    }
                    mbar_arrive(BAR(kBarGo + ib));
                    continue;
                }
                // streamed tile: chunks cycle through the stages, each released by the MMAs' commit
                for (int c = 0; c < T.nch; ++c, ++ka) {
                    const uint32_t st = ka % kAStages, r = ka / kAStages;
                    if (!wait_bar(BAR(kBarAEmpty + st), (r & 1u) ^ 1u, abort_flag, A.count, A.spin)) {
                        ok = false;
                        break;
                    }
                    // chunk 0 completes on the item's own transaction barrier, later chunks on the stage's
                    const uint32_t full = c == 0 ? BAR(kBarT0 + ib) : BAR(kBarAFull + st);
                    mbar_arrive_expect_tx(full, kChunkBytes);
                    const uint8_t *src = A.taps + T.taps_off + (int64_t)c * kChunkBytes;
                    bulk_g2s(smem_u32(s_a + st * kChunkBytes), src, kChunkImg, full);
                    bulk_g2s(smem_u32(s_a + st * kChunkBytes) + kChunkImg, src + kChunkImg, kChunkImg, full);
                    if (c == 0) {
                        // landed, then the producer's share of the item's go barrier
                        const uint32_t par = t0_armed[ib]++ & 1u;
                        if (!wait_bar(BAR(kBarT0 + ib), par, abort_flag, A.count, A.spin)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive(BAR(kBarGo + ib));
                    } else {
                        ++a_armed[st];
                    }
                }
                if (!ok) break;
            }
            // drain: the last phase armed on each copy barrier has completed (every copy landed)
            // before this thread reaches the CTA's final barrier; bounded, like every wait
            for (int b = 0; b < 2; ++b) {
                const uint32_t bars3[3] = {BAR(kBarQFull + b), BAR(kBarAFull + b), BAR(kBarT0 + b)};
                const uint32_t armed[3] = {q_armed[b], a_armed[b], t0_armed[b]};
                for (int k = 0; k < 3; ++k) {
                    if (armed[k] == 0u) continue;
                    uint32_t i = 0;
                    while (i < kSpin && !mbar_try_wait(bars3[k], (armed[k] - 1u) & 1u)) ++i;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t ka = 0, li = 0, uf0 = 0, uf1 = 0;      // ka: streamed chunks so far
            const uint32_t idn = idesc_f16(128, kN, BF16, 0);
            const uint32_t a_base = smem_u32(s_a), y_base = smem_u32(s_y);
            const uint64_t yp = (uint64_t)(A.ystride >> 4);   // one Y plane in descriptor units
            int64_t ti = it0 / A.n_tb, tb = it0 - ti * A.n_tb, prev = -1;
            TcTile T{};
            bool go_seen = false;                 // the go barrier of this item was already waited on
            for (int64_t it = it0; it < it1; ++it, ++li, tb = (tb + 1 == A.n_tb) ? 0 : tb + 1, ti += (tb == 0)) {
                const bool first = ti != prev;
                if (first) {
                    prev = ti;
                    T = A.tiles[ti];
                }
                const bool resident = T.nch <= kAStages;
                const uint32_t acc = li & 1u, yb = li & 1u, use = li >> 1;
                // one wait: the accumulator is free, Y is built and chunk 0 of the taps is staged
                if (!go_seen && !wait_bar(BAR(kBarGo + acc), use & 1u, abort_flag, A.count, A.spin)) break;
                go_seen = false;
                fence_after();
                const uint32_t d = tmem + acc * (uint32_t)kN;
                const uint32_t y0 = y_base + yb * 4u * A.ystride;
                bool ok = true;
                for (int c = 0; c < T.nch; ++c) {
                    // a resident tile's chunk c sits in stage c (chunk 1 waited on at the tile's
                    // first item only); a streamed chunk in stage ka mod 2
                    const uint32_t st = resident ? (uint32_t)c : ka % kAStages;
                    if (c > 0 && (!resident || first)) {
                        const uint32_t uf = st == 0u ? uf0++ : uf1++;
                        if (!wait_bar(BAR(kBarAFull + st), uf & 1u, abort_flag, A.count, A.spin)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                    }
                    // descriptors of the chunk's first 16-tap step; a later step adds a constant
                    // to the 14-bit start-address field (no carry: shared memory < 256 KB)
                    const uint32_t ah = a_base + st * kChunkBytes, al = ah + kChunkImg;
                    const uint64_t dA2h = desc_sw128(ah), dA2l = desc_sw128(al);                              // [-Pi; Pr]
                    const uint64_t dA1h = desc_sw128(ah + kNT * 128u), dA1l = desc_sw128(al + kNT * 128u);  // [Pr; Pi]
                    const uint64_t dQ = desc_hankel(y0 + (uint32_t)(64 * c) * 16u);
                    const int s_end = min(4, T.nk16 - 4 * c);
                    for (int s = 0; s < s_end; ++s) {
                        if (c == T.nch - 1 && s == s_end - 1 && it + 1 < it1 && tb + 1 < A.n_tb) {
                            // the next item's go barrier, waited on while this item's earlier
                            // MMAs still run (deadlock-free: it needs only work issued before;
                            // not across a tile change, where the producer waits for this
                            // item's MMAs before it arrives for the next one)
                            const uint32_t nli = li + 1u;
                            if (!wait_bar(BAR(kBarGo + (nli & 1u)), (nli >> 1) & 1u, abort_flag, A.count, A.spin)) {
                                ok = false;
                                break;
                            }
                            go_seen = true;
                        }
                        const uint64_t o = (uint64_t)(2 * s);            // 32 B along K in the taps rows
                        const uint64_t A2h = dA2h + o, A2l = dA2l + o, A1h = dA1h + o, A1l = dA1l + o;
                        const uint64_t Qrh = dQ + (uint64_t)(16 * s);    // 16 Y rows of 16 B
                        const uint64_t Qih = Qrh + yp, Qrl = Qrh + 2u * yp, Qil = Qrh + 3u * yp;
                        const uint32_t acc0 = (c == 0 && s == 0) ? 0u : 1u;
                        // the products and their order match the other kernel's (q_h p_h, q_h p_l,
                        // q_l p_h per plane), so both give bit-identical sums
                        mma_ss(d, A1h, Qrh, idn, acc0);
                        mma_ss(d, A1l, Qrh, idn, 1u);
                        mma_ss(d, A1h, Qrl, idn, 1u);
                        mma_ss(d, A2h, Qih, idn, 1u);
                        mma_ss(d, A2l, Qih, idn, 1u);
                        mma_ss(d, A2h, Qil, idn, 1u);
                    }
                    if (!ok) break;
                    if (!resident) {
                        mma_commit(BAR(kBarAEmpty + st));   // the stage may take the next chunk
                        ++ka;
                    }
                }
                if (!ok) break;
                // one commit: the accumulator is full and Y buffer yb (= acc) is free again
                mma_commit(BAR(kBarDFull + acc));
                // leaving the tile: the producer may overwrite the stages once these complete
                if (tb + 1 == A.n_tb && it + 1 < it1) mma_commit(BAR(kBarTile));
            }
            // every MMA this thread issued has completed before TMEM is released
            mma_commit(BAR(kBarDone));
            for (uint32_t i = 0; i < kSpin && !mbar_try_wait(BAR(kBarDone), 0); ++i) {
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------------------ Y builders
        const int bt = (warp - 4) * 32 + lane;          // 0..127
        uint32_t li = 0;
        int kpad = 0;
        int64_t ti = it0 / A.n_tb, tb = it0 - ti * A.n_tb, prev = -1;
        for (int64_t it = it0; it < it1; ++it, ++li, tb = (tb + 1 == A.n_tb) ? 0 : tb + 1, ti += (tb == 0)) {
            if (ti != prev) {
                prev = ti;
                kpad = A.tiles[ti].kpad;
            }
            const uint32_t b2 = li & 1u, use = li >> 1;
            // Y buffer b2 is free once the MMAs of the item two back completed (its accumulator is full)
            bool ok = wait_bar(BAR(kBarDFull + b2), (use & 1u) ^ 1u, abort_flag, A.count, A.spin);
            ok = ok && wait_bar(BAR(kBarQFull + b2), use & 1u, abort_flag, A.count, A.spin);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int rows = kN - 8 + kpad;             // Y rows 0 .. 248 + kpad - 1
            uint8_t *y0 = s_y + b2 * 4u * A.ystride;
#pragma unroll 1
            for (int p = 0; p < 4; ++p) {
                const uint32_t *W = (const uint32_t *)(s_qw + (b2 * 4u + (uint32_t)p) * A.qwin);
                uint4 *Y = (uint4 *)(y0 + p * A.ystride);
                for (int r = bt; r < rows; r += 128) {
                    // Y[r] = q[r .. r+7]: four aligned words, shifted by one half when r is odd
                    const int w0 = r >> 1;
                    const uint32_t x0 = W[w0], x1 = W[w0 + 1], x2 = W[w0 + 2], x3 = W[w0 + 3];
                    uint4 v;
                    if (r & 1) {
                        const uint32_t x4 = W[w0 + 4];
                        v = make_uint4(__funnelshift_r(x0, x1, 16), __funnelshift_r(x1, x2, 16),
                                       __funnelshift_r(x2, x3, 16), __funnelshift_r(x3, x4, 16));
                    } else {
                        v = make_uint4(x0, x1, x2, x3);
                    }
                    Y[r] = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(BAR(kBarGo + b2));
                mbar_arrive(BAR(kBarQEmpty + b2));
            }
        }
    } else if (warp >= 8) {
        // ------------------------------------------------------------ epilogue (pairs)
        const uint32_t lq = (uint32_t)warp & 3u;             // TMEM lane quarter
        const int half = (warp - 8) >> 2;                    // which 128 of the 256 columns
        const bool is_re = lq < 2u;
        const int pair = (int)(lq & 1u) + 2 * half;
        // Xs: what this warp hands over (Re of columns 16..31, or Im of columns 0..15); Xr: what it gets
        float *Xs = s_x + (pair * 2 + (is_re ? 0 : 1)) * 32 * kXPitch + lane * kXPitch;
        const float *Xr = s_x + (pair * 2 + (is_re ? 1 : 0)) * 32 * kXPitch + lane * kXPitch;
        const uint32_t tlane = (lq * 32u) << 16;
        uint32_t li = 0;
        bool valid = false;
        float sc = 0.f, thr_raw = 0.f;
        int32_t j = 0, o = 0;
        int64_t ti = it0 / A.n_tb, tb = it0 - ti * A.n_tb, prev = -1;
        // One 32-column chunk of a warp's lane quarter (v: columns c0 .. c0 + 31 of its rows).  The
        // real-row warp (RE) keeps columns 0..15 and hands 16..31 over, the imaginary-row warp the
        // reverse; both then screen their 16 samples.  A warp-uniform branch picks the variant, so
        // every register index is static (a runtime index would put v in local memory).
        auto chunk = [&](auto re_tag, const uint32_t (&v)[32], uint32_t c0) {
            constexpr bool RE = decltype(re_tag)::value;
            float re[16], im[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int b0 = RE ? 16 + 4 * q : 4 * q;
                reinterpret_cast<float4 *>(Xs)[q] = make_float4(__uint_as_float(v[b0]), __uint_as_float(v[b0 + 1]),
                                                               __uint_as_float(v[b0 + 2]), __uint_as_float(v[b0 + 3]));
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (RE)
                    re[i] = __uint_as_float(v[i]);
                else
                    im[i] = __uint_as_float(v[16 + i]);
            }
            named_sync(1u + (uint32_t)pair, 64u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = reinterpret_cast<const float4 *>(Xr)[q];
                float *dst = RE ? im : re;
                dst[4 * q] = f.x;
                dst[4 * q + 1] = f.y;
                dst[4 * q + 2] = f.z;
                dst[4 * q + 3] = f.w;
            }
            named_sync(5u + (uint32_t)pair, 64u);     // both buffers read: free for the next chunk
            if (!valid) return;
            // screen: the largest unscaled |D|^2 of the 16 samples, two samples per packed FP32
            // instruction (the same fma(re, re, im * im) per sample as the exact test below)
            float pmax = 0.f;
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float2 r2 = make_float2(re[i], re[i + 1]), i2 = make_float2(im[i], im[i + 1]);
                const float2 p2 = __ffma2_rn(r2, r2, __fmul2_rn(i2, i2));
                pmax = fmaxf(pmax, fmaxf(p2.x, p2.y));
            }
            if (!(pmax > thr_raw)) return;
            // rare: the samples above the screen, then the running maximum of each window along
            // u, one candidate per (window, run of samples); ties keep the earlier t
            uint32_t hit = 0u;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float p_raw = fmaf(re[i], re[i], im[i] * im[i]);
                hit |= (p_raw > thr_raw ? 1u : 0u) << i;
            }
            uint32_t bw = 0xffffffffu, bp = 0u, bt = 0u;
            float bzr = 0.f, bzi = 0.f;
            const int64_t u0 = wrap_pos(ubase, tb * kN, A.n) + c0 + (RE ? 0 : 16);
#pragma unroll 1
            for (int i = 0; i < 16; ++i) {
                if (!((hit >> i) & 1u)) continue;
                float zr = 0.f, zim = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q == i) {
                        zr = __fmul_rn(re[q], sc);
                        zim = __fmul_rn(im[q], sc);
                    }
                // z and |z|^2 exactly as the other kernel forms them
                const float p = __fadd_rn(__fmul_rn(zr, zr), __fmul_rn(zim, zim));
                if (!(p > A.thr)) continue;
                const uint32_t t = (uint32_t)((u0 + i + o) & (A.n - 1));
                const uint32_t w = t / A.W;
                if (w != bw) {
                    if (bw != 0xffffffffu) emit_one((uint32_t)j, bw, bp, bt, bzr, bzi, A.cand, A.cap, A.count);
                    bw = w;
                    bp = 0u;
                }
                const uint32_t pb = __float_as_uint(p);
                if (pb > bp || (pb == bp && t < bt)) {
                    bp = pb;
                    bt = t;
                    bzr = zr;
                    bzi = zim;
                }
            }
            if (bw != 0xffffffffu) emit_one((uint32_t)j, bw, bp, bt, bzr, bzi, A.cand, A.cap, A.count);
        };
        // both accumulators start free: this warp's share of the first phase of each go barrier
        if (lane == 0) {
            mbar_arrive(BAR(kBarGo + 0));
            mbar_arrive(BAR(kBarGo + 1));
        }
        for (int64_t it = it0; it < it1; ++it, ++li, tb = (tb + 1 == A.n_tb) ? 0 : tb + 1, ti += (tb == 0)) {
            if (ti != prev) {
                // this lane's template: a = 32 (quarter & 1) + lane, the same in both warps of the pair
                prev = ti;
                const TcTile T = A.tiles[ti];
                const int a = 32 * (int)(lq & 1u) + lane;
                const int64_t slot = (int64_t)T.first + (a < T.count ? a : 0);
                sc = a < T.count ? A.scale[slot] * ldexpf(1.0f, -A.qscale[T.ref]) : 0.f;
                valid = a < T.count && sc > 0.f;
                j = valid ? A.perm[slot] : 0;
                o = valid ? A.off[slot] : 0;
                // screen on the unscaled |D|^2 against thr / sc^2 lowered by 2^-10 (far above the
                // few-ulp difference to the scaled |z|^2); every hit is re-tested exactly below
                thr_raw = valid ? A.thr / (sc * sc) * (1.0f - 0.0009765625f) : 0.f;
            }
            const uint32_t acc = li & 1u, use = li >> 1;
            const bool ok = wait_bar(BAR(kBarDFull + acc), use & 1u, abort_flag, A.count, A.spin);
            if (!__all_sync(0xffffffffu, ok)) break;
            fence_after();
            for (int cc = 0; cc < 4; ++cc) {
                const uint32_t c0 = (uint32_t)(half * 128 + cc * 32);
                uint32_t v[32];
                tmem_ld32(tmem + tlane + acc * (uint32_t)kN + c0, v);
                tmem_ld_wait();
                if (cc == 3) {
                    // the accumulator is free for the item two ahead
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(BAR(kBarGo + acc));
                }
                if (is_re)
                    chunk(std::true_type{}, v, c0);
                else
                    chunk(std::false_type{}, v, c0);
            }
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
template <typename H> __device__ __forceinline__ uint16_t hbits(H x);
template <> __device__ __forceinline__ uint16_t hbits<__half>(__half x) { return __half_as_ushort(x); }
template <> __device__ __forceinline__ uint16_t hbits<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat16_as_ushort(x); }
template <typename H> __device__ __forceinline__ H toh(float x);
template <> __device__ __forceinline__ __half toh<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 toh<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float fromh(__half x) { return __half2float(x); }
__device__ __forceinline__ float fromh(__nv_bfloat16 x) { return __bfloat162float(x); }

// One block per tile: per-template power-of-two scale (max |component| * 2^e < 2^8), then the
// A-operand image [chunk][hl][row][128 B], rows [-Pi (64); Pr (64); Pi (64)]; element e of
// chunk c holds reversed tap k = 64 c + e, 16-byte units XOR-swizzled by row % 8.  Also the
// per-slot lag offset and normalisation.
template <typename H>
__global__ void __launch_bounds__(256) k_pack_tl(const TcTile *__restrict__ tiles, const float2 *__restrict__ taps,
                                                 int32_t k_stride, const int32_t *__restrict__ perm,
                                                 const int32_t *__restrict__ kslot, const int32_t *__restrict__ lag,
                                                 const double *__restrict__ sigma, int64_t n,
                                                 uint8_t *__restrict__ out, int32_t *__restrict__ off,
                                                 float *__restrict__ scale) {
    __shared__ int s_exp[kNT], s_j[kNT], s_k[kNT];
    const TcTile T = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = warp; a < kNT; a += (int)(blockDim.x >> 5)) {
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
                frexpf(mx, &ex);
                e = 8 - ex;
            }
            s_exp[a] = e;
            s_j[a] = j;
            s_k[a] = K;
        }
    }
    __syncthreads();
    const int rows = 3 * kNT;
    const int64_t total = (int64_t)T.nch * 2 * rows * 64;
    uint8_t *img = out + T.taps_off;
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int e = (int)(idx & 63);
        const int64_t r1 = idx >> 6;
        const int row = (int)(r1 % rows);
        const int64_t r2 = r1 / rows;
        const int hl = (int)(r2 & 1);
        const int c = (int)(r2 >> 1);
        const int a = row % kNT, part = row / kNT;     // 0: -Pi, 1: Pr, 2: Pi
        const int k = 64 * c + e;
        uint16_t bits = 0;
        if (a < T.count && k < s_k[a]) {
            const float2 v = taps[(int64_t)s_j[a] * k_stride + (s_k[a] - 1 - k)];
            const float comp = part == 1 ? v.x : (part == 2 ? v.y : -v.y);
            const float x = ldexpf(comp, s_exp[a]);
            const H hi = toh<H>(x);
            bits = hl ? hbits<H>(toh<H>(x - fromh(hi))) : hbits<H>(hi);
        }
        const int64_t rowbase = ((int64_t)(c * 2 + hl) * rows + row) * 128;
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

uint32_t tl_ystride(int32_t kpad_max) { return (uint32_t)(kN - 8 + kpad_max) * 16u; }
uint32_t tl_qwin(int32_t kpad_max) { return (uint32_t)(kN + kpad_max); }

size_t tl_smem_bytes(uint32_t ystride, uint32_t qwin) {
    return 1024 + (size_t)kAStages * kChunkBytes + 2u * 4u * ystride + 2u * 4u * qwin * 2u + 4 * 2 * 32 * kXPitch * 4 +
           kNumBars * 8 + 16;
}

int tl_rows_per_item() { return kN; }
int tl_tile_templates() { return kNT; }

rfd_status tl_pack(rfd_plan *plan, const float2 *taps, int32_t k_stride, const int32_t *lag, const double *sigma,
                   cudaStream_t s) {
    const unsigned ntiles = (unsigned)plan->tl_tiles.size();
    if (ntiles == 0) return RFD_OK;
    if (plan->precision == RFD_PREC_FP16X3)
        k_pack_tl<__half><<<ntiles, 256, 0, s>>>((const TcTile *)plan->d_tl_tiles.p, taps, k_stride,
                                                  (const int32_t *)plan->d_perm.p, (const int32_t *)plan->d_kslot.p,
                                                  lag, sigma, plan->grid.n, (uint8_t *)plan->d_tl_taps.p,
                                                  (int32_t *)plan->d_off.p, (float *)plan->d_scale.p);
    else
        k_pack_tl<__nv_bfloat16><<<ntiles, 256, 0, s>>>(
            (const TcTile *)plan->d_tl_tiles.p, taps, k_stride, (const int32_t *)plan->d_perm.p,
            (const int32_t *)plan->d_kslot.p, lag, sigma, plan->grid.n, (uint8_t *)plan->d_tl_taps.p,
            (int32_t *)plan->d_off.p, (float *)plan->d_scale.p);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

rfd_status tl_launch(const rfd_plan *plan, const void *q, const int32_t *qscale, const int64_t *u_begin,
                     rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s) {
    if (plan->tl_tiles.empty()) return RFD_OK;
    TlArgs a;
    a.tiles = (const TcTile *)plan->d_tl_tiles.p;
    a.ranges = (const int64_t *)plan->d_tl_ranges.p;
    a.n_tb = plan->out_len / kN;
    a.u_begin = u_begin;
    a.taps = (const uint8_t *)plan->d_tl_taps.p;
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
    a.ystride = plan->tl_ystride;
    a.qwin = plan->tl_qwin;
    a.stall = (plan->debug_flags & RFD_DEBUG_STALL_TAPS) ? 1u : 0u;
    a.spin = a.stall ? kSpinStall : kSpin;
    const size_t shm = tl_smem_bytes(a.ystride, a.qwin);
    const unsigned grid = (unsigned)plan->tl_grid;
    static size_t smem_set[64][2] = {};
    const int dev = plan->ctx->device < 64 ? plan->ctx->device : 63;
    const int bf = plan->precision == RFD_PREC_FP16X3 ? 0 : 1;
    if (shm > smem_set[dev][bf]) {
        if (bf == 0)
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_rf_tc_long<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        else
            RFD_TRY_CUDA(cudaFuncSetAttribute(k_rf_tc_long<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        smem_set[dev][bf] = shm;
    }
    if (bf == 0)
        k_rf_tc_long<0><<<grid, kThreads, shm, s>>>(a);
    else
        k_rf_tc_long<1><<<grid, kThreads, shm, s>>>(a);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

}  // namespace rfd
