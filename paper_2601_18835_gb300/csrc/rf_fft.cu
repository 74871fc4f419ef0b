// Block-FFT (overlap-save) realisation of the ratio filter (Eq. 3) on CUDA cores, the form in
// which the paper applies its short FIR (Sec. III, Table II: FFT blocks of about 2048
// samples), with the fused trigger epilogue.
//
// With off_j = (s_j + K_j - 1) mod n, the FIR of Eq. 3 reads
//   z_j[(u + off_j) mod n] = sum_{m < K_j} c_j[m] q_r[(u + m) mod n],
//   c_j[m] = rho_j[K_j - 1 - m] / sigma_eff,j.
// Output positions u are cut into blocks of L = M - K_max + 1 (M = 2048, K_max the largest K
// on this path); block b starts at u_0 = b L and sees x_b[i] = q_r[(u_0 + i) mod n], i < M.
// For l < L no product wraps around the block, so
//   z_j[(u_0 + l + off_j) mod n] = sum_k X_b[k] P_j[k] exp(+2 pi i k l / M),
//   X_b[k] = sum_i x_b[i] exp(-2 pi i k i / M)      (per reference and block, every segment),
//   P_j[k] = (1/M) sum_m c_j[m] exp(+2 pi i k m / M) (per template, when the taps are set).
// A CTA holds three 128-thread groups, one block b each.  The templates of a tile stream
// through a two-buffer ring in shared memory (bulk copies completing on mbarriers; a buffer is
// refilled once every group has released it, so the groups never wait for one another as a
// whole); every group multiplies its X_b, kept in registers, by P_j, runs the inverse
// transform (Stockham passes of radix 8, 16, 16 through two padded tiles, twiddles in
// registers) and screens |z|^2.
#include "epilogue.cuh"
#include "fft_reg.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace rfd {

namespace {

constexpr int kM = 2048;                     // block transform length
constexpr int kGT = 128;                     // threads per block transform, 16 elements each
constexpr int kGroups = 4;                   // block transforms per CTA of the spectra kernel
constexpr int kThreads = kGT * kGroups;
constexpr int kFGroups = 3;                  // block transforms per CTA of the filter kernel
constexpr int kFThreads = kGT * kFGroups;    // (384 threads: room for both twiddle rows in registers)
constexpr int kTileLd = kM + kM / 16 + 2;    // padded shared-memory tile (one pad per 16)
constexpr int kTileTemplates = 64;           // templates per tile (one reference)

__device__ __forceinline__ int tpos(int i) { return i + (i >> 4); }


__device__ __forceinline__ void group_bar(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kGT) : "memory");
}

// Length-2048 transform by one 128-thread group: thread t holds elements t + 128 r (r < 16) in
// v on entry and on exit (natural order).  Passes: radix 8 (ns = 1) into tile A, radix 16
// (ns = 8) from A into B, radix 16 (ns = 128) from B into registers.  w2, w3: this thread's
// twiddles of the last two passes (load_twiddles), held in registers across transforms.  Every thread of the group calls this; bar is the
// group's named barrier.  Two calls in a row are safe: a thread writes A again only after
// every thread of the group passed the barrier that follows its reads of A, and likewise B.
// Thread-major, XOR-swizzled rows of 16 complex values: value r of row i is float2 index
// 16 i + 2 ((r / 2) ^ (i & 7)) + (r & 1), so that eight threads reading the 16-byte chunk c of
// eight consecutive rows hit eight different bank groups.
__device__ __forceinline__ int swz(int i, int c) { return 16 * i + 2 * (c ^ (i & 7)); }

// Reads row i (16 values) with eight 16-byte loads.
__device__ __forceinline__ void load_row16(float2 (&w)[16], const float2 *base, int i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float4 q = *reinterpret_cast<const float4 *>(base + swz(i, c));
        w[2 * c] = make_float2(q.x, q.y);
        w[2 * c + 1] = make_float2(q.z, q.w);
    }
}

// Twiddles of the last two passes in the swizzled row layout: rows k < 8 (pass 2, value r =
// w_128^(r k)) then rows t < 128 (pass 3, value r = w_2048^(r t)); value 0 of each row is 1.
// Built from the stage table (7 + 120 + 1920 entries) by the whole CTA.
constexpr int kTwRows = 8 + kGT;
__device__ __forceinline__ void build_twiddles(float2 *tw, const float2 *__restrict__ stage) {
    for (int e = threadIdx.x; e < kTwRows * 16; e += blockDim.x) {
        const int i = e >> 4, r = e & 15;
        float2 w = make_float2(1.f, 0.f);
        if (r > 0) w = i < 8 ? stage[7 + (r - 1) * 8 + i] : stage[127 + (r - 1) * kGT + (i - 8)];
        tw[swz(i, r >> 1) + (r & 1)] = w;
    }
}

template <bool INV>
__device__ __forceinline__ void group_fft(float2 (&v)[16], float2 *A, float2 *B, const float2 (&w2)[16],
                                          const float2 (&w3)[16], int t, int bar) {
    {
        float2 a[8], b[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            a[r] = v[2 * r];          // butterfly j = t: elements t + 256 r
            b[r] = v[2 * r + 1];      // butterfly j = t + 128
        }
        dft_reg<float, 8, INV>(a);
        dft_reg<float, 8, INV>(b);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            A[tpos(8 * t + r)] = a[r];
            A[tpos(8 * (t + kGT) + r)] = b[r];
        }
    }
    group_bar(bar);
    {
        const int k = t & 7;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = A[tpos(t + kGT * r)];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = INV ? cmul(v[r], w2[r]) : cmulc(v[r], w2[r]);
        dft_reg<float, 16, INV>(v);
        const int idx = ((t - k) << 4) + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) B[tpos(idx + 8 * r)] = v[r];
    }
    group_bar(bar);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = B[tpos(t + kGT * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = INV ? cmul(v[r], w3[r]) : cmulc(v[r], w3[r]);
    dft_reg<float, 16, INV>(v);
}

// Thread t's twiddle rows: pass 2 (row t mod 8) and pass 3 (row 8 + t) of the table.
__device__ __forceinline__ void load_twiddles(float2 (&w2)[16], float2 (&w3)[16], const float2 *tw, int t) {
    load_row16(w2, tw, t & 7);
    load_row16(w3, tw, 8 + t);
}

// q_r[m] as FP32 from the stored reference series (complex64, or the four hi/lo planes of
// the split precisions with hi + lo = q 2^e_r).
template <int PREC>
__device__ __forceinline__ float2 load_q(const void *__restrict__ q, int r, int64_t ld, int64_t m, float sc) {
    if (PREC == RFD_PREC_FP32) return ((const float2 *)q)[(int64_t)r * ld + m];
    const uint16_t *h = (const uint16_t *)q;
    const int64_t base = (int64_t)4 * r * ld + m;
    float v[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint16_t u = h[base + p * ld];
        v[p] = PREC == RFD_PREC_FP16X3 ? __half2float(__ushort_as_half(u)) : __bfloat162float(__ushort_as_bfloat16(u));
    }
    return make_float2((v[0] + v[2]) * sc, (v[1] + v[3]) * sc);
}

// X[r][b][k] for the references in refs (blockIdx.y) and blocks b = 4 blockIdx.x + group.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_block_spectra(const void *__restrict__ q,
                                                            const int32_t *__restrict__ qscale, int64_t ld,
                                                            int64_t n, int32_t L, int32_t nb,
                                                            const int32_t *__restrict__ refs,
                                                            float2 *__restrict__ X,
                                                            const float2 *__restrict__ stw_g,
                                                            const int64_t *__restrict__ u_begin) {
    extern __shared__ __align__(16) uint8_t sm[];
    float2 *tw = (float2 *)sm;                  // [kTwRows][16] swizzled twiddle rows
    float2 *tl = tw + kTwRows * 16;
    const int g = threadIdx.x / kGT, t = threadIdx.x % kGT;
    float2 *TA = tl + (2 * g) * kTileLd, *TB = TA + kTileLd;
    build_twiddles(tw, stw_g);
    __syncthreads();
    const int r = refs[blockIdx.y];
    const int b = blockIdx.x * kGroups + g;
    const bool bvalid = b < nb;                         // uniform within the group
    const int64_t u0 = window_base(u_begin, n) + (int64_t)(bvalid ? b : 0) * L;
    const float sc = PREC == RFD_PREC_FP32 ? 1.f : ldexpf(1.f, -qscale[r]);
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = load_q<PREC>(q, r, ld, (u0 + t + kGT * i) & (n - 1), sc);
    float2 w2[16], w3[16];
    load_twiddles(w2, w3, tw, t);
    group_fft<false>(v, TA, TB, w2, w3, t, 1 + g);
    if (bvalid) {
        float2 *dst = X + ((int64_t)r * nb + b) * kM;
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[t + kGT * i] = v[i];
    }
}

struct RfFftArgs {
    const FftTile *tiles;
    const int64_t *ranges;      // item ranges per CTA; item = tile * nbg + block group
    int32_t nbg, nb, L;
    int64_t out_len;            // outputs of the window
    const int64_t *u_begin;     // first output position of the window (device), or NULL
    const float2 *X, *stw;
    const float2 *P;            // [slot - slot0][kM], row layout of swz (row t holds k = t + 128 r)
    int64_t slot0;              // first block-FFT slot
    const int32_t *perm, *off;
    int64_t n;
    float thr;
    uint32_t W;
    rfd_candidate *cand;
    int64_t cap;
    unsigned long long *count;
};

constexpr uint32_t kFSpin = 1u << 22;

// Bounded wait on an mbarrier phase.  A wait that gives up raises the CTA's abort flag and
// bit 62 of the candidate count (reported as RFD_ERR_TIMEOUT by find_triggers); every later
// wait then returns at once, so every thread keeps the same control flow (the group barriers
// stay matched) and the kernel ends.
__device__ __forceinline__ void ring_wait(uint32_t bar, uint32_t parity, volatile uint32_t *abort_flag,
                                          unsigned long long *count) {
    for (uint32_t i = 0; i < kFSpin; ++i) {
        if (tc::mbar_try_wait(bar, parity) || *abort_flag) return;
    }
    *abort_flag = 1u;
    atomicOr(count, 1ull << 62);
}

__global__ void __launch_bounds__(kFThreads, 1) k_rf_fft(const RfFftArgs a) {
    extern __shared__ __align__(16) uint8_t sm[];
    float2 *tw = (float2 *)sm;                  // [kTwRows][16] swizzled twiddle rows
    float2 *Ps = tw + kTwRows * 16;             // [2][kM] template spectra ring
    float2 *tl = Ps + 2 * kM;                   // [kFGroups][2][kTileLd]
    uint64_t *bars = (uint64_t *)(tl + 2 * kFGroups * kTileLd);   // full[2], empty[2]
    volatile uint32_t *abort_flag = (volatile uint32_t *)(bars + 4);
    const int g = threadIdx.x / kGT, t = threadIdx.x % kGT;
    float2 *TA = tl + (2 * g) * kTileLd, *TB = TA + kTileLd;
    const uint32_t full0 = tc::smem_u32(bars), empty0 = full0 + 16u;
    if (threadIdx.x == 0) {
        tc::mbar_init(full0, 1);
        tc::mbar_init(full0 + 8u, 1);
        tc::mbar_init(empty0, kFGroups);
        tc::mbar_init(empty0 + 8u, kFGroups);
        *abort_flag = 0u;
        tc::mbar_fence_init();
    }
    build_twiddles(tw, a.stw);
    __syncthreads();
    float2 w2[16], w3[16];
    load_twiddles(w2, w3, tw, t);
    const int64_t it0 = a.ranges[blockIdx.x], it1 = a.ranges[blockIdx.x + 1];
    const int64_t ubase = window_base(a.u_begin, a.n);
    uint32_t tq = 0;                            // templates this CTA has started (ring position)
    uint32_t last0 = 0xffffffffu, last1 = 0xffffffffu;   // thread 0: last template copied per buffer
    for (int64_t it = it0; it < it1; ++it) {
        const int64_t ti = it / a.nbg;
        const int bg = (int)(it - ti * a.nbg);
        const FftTile tile = a.tiles[ti];
        const int b = bg * kFGroups + g;
        const bool bvalid = b < a.nb;
        const int64_t u0 = ubase + (int64_t)b * a.L;
        // outputs l of this block inside the window: l < lim
        const int64_t rest = a.out_len - (int64_t)b * a.L;
        const int lim = bvalid ? (int)(rest < a.L ? rest : a.L) : 0;
        const float2 *Xb = a.X + ((int64_t)tile.ref * a.nb + (bvalid ? b : 0)) * kM;
        float2 x[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = Xb[t + kGT * r];
        const float2 *Pt = a.P + (tile.first - a.slot0) * kM;
        for (int q = 0; q < tile.count; ++q, ++tq) {
            // template spectra stream through a ring of two buffers (template tq in buffer
            // tq & 1): thread 0 copies the item's first template, and each next one, once
            // every group has released the buffer's previous template; the groups do not
            // wait for one another
            if (threadIdx.x == 0) {
                for (int k = (q == 0 ? 0 : 1); k < 2; ++k) {
                    const uint32_t t2 = tq + (uint32_t)k;
                    if (q + k >= tile.count) break;
                    const uint32_t b2 = t2 & 1u;
                    ring_wait(empty0 + 8u * b2, ((t2 >> 1) & 1u) ^ 1u, abort_flag, a.count);
                    tc::mbar_arrive_expect_tx(full0 + 8u * b2, (uint32_t)(kM * sizeof(float2)));
                    tc::bulk_g2s(tc::smem_u32(Ps + b2 * kM), Pt + (int64_t)(q + k) * kM,
                                 (uint32_t)(kM * sizeof(float2)), full0 + 8u * b2);
                    if (b2 == 0u)
                        last0 = t2;
                    else
                        last1 = t2;
                }
            }
            const uint32_t bq = tq & 1u;
            ring_wait(full0 + 8u * bq, (tq >> 1) & 1u, abort_flag, a.count);
            float2 v[16];
            load_row16(v, Ps + bq * kM, t);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = cmul(x[r], v[r]);
            group_fft<true>(v, TA, TB, w2, w3, t, 1 + g);
            // the group's reads of the buffer precede its first barrier inside group_fft
            if (t == 0) tc::mbar_arrive(empty0 + 8u * bq);
            // epilogue: v[r] = z at u = u0 + t + 128 r
            // screen on the largest |z|^2 of the thread (invalid outputs included: a false
            // alarm only costs the exact pass below, which drops them)
            float pmax = 0.f;
#pragma unroll
            for (int r = 0; r < 16; ++r)
                pmax = fmaxf(pmax, __fadd_rn(__fmul_rn(v[r].x, v[r].x), __fmul_rn(v[r].y, v[r].y)));
            if (__any_sync(0xffffffffu, pmax > a.thr)) {
                const int64_t slot = tile.first + q;
                const int32_t j = a.perm[slot];
                const int32_t o = a.off[slot];
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int l = t + kGT * r;
                    const bool valid = l < lim;
                    const uint32_t tt = (uint32_t)((u0 + l + o) & (a.n - 1));
                    emit_window_max(valid, (uint32_t)j, tt, v[r].x, v[r].y, a.thr, a.W, a.cand, a.cap, a.count);
                }
            }
        }
    }
    // no copy may still be landing when the CTA ends (after a wait that gave up, the groups no
    // longer consume them): thread 0 waits, bounded, for the last copy into each buffer; in
    // normal operation these phases completed long ago
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < kFSpin && last0 != 0xffffffffu && !tc::mbar_try_wait(full0, (last0 >> 1) & 1u); ++i) {
        }
        for (uint32_t i = 0; i < kFSpin && last1 != 0xffffffffu &&
                             !tc::mbar_try_wait(full0 + 8u, (last1 >> 1) & 1u); ++i) {
        }
    }
}

// P_j for block-FFT slots slot0 + s_off + blockIdx.x (one 128-thread block each; P holds the
// block-FFT slots only, from slot0) and off_j.
__global__ void __launch_bounds__(kGT) k_taps_spectra(const float2 *__restrict__ taps, int32_t k_stride,
                                                      const int32_t *__restrict__ perm,
                                                      const int32_t *__restrict__ kslot,
                                                      const int32_t *__restrict__ lag,
                                                      const double *__restrict__ sigma, int64_t n, int64_t slot0,
                                                      int64_t s_off, float2 *__restrict__ P, int32_t *__restrict__ off,
                                                      const float2 *__restrict__ stw) {
    extern __shared__ __align__(16) uint8_t sm[];
    float2 *tw = (float2 *)sm;
    float2 *tiles = tw + kTwRows * 16;
    build_twiddles(tw, stw);
    __syncthreads();
    const int64_t local = s_off + blockIdx.x;
    const int64_t slot = slot0 + local;
    const int t = threadIdx.x;
    const int32_t j = perm[slot], K = kslot[slot];
    const double s = sigma[j];
    // a window with no weight has sigma_eff = 0: zero spectrum, no triggers
    const double inv = s > 0.0 ? 1.0 / (s * (double)kM) : 0.0;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int m = t + kGT * r;
        if (m < K) {
            const float2 c = taps[(int64_t)j * k_stride + (K - 1 - m)];
            v[r] = make_float2((float)((double)c.x * inv), (float)((double)c.y * inv));
        } else {
            v[r] = make_float2(0.f, 0.f);
        }
    }
    float2 w2[16], w3[16];
    load_twiddles(w2, w3, tw, t);
    group_fft<true>(v, tiles, tiles + kTileLd, w2, w3, t, 1);
    float2 *dst = P + local * kM;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4 *>(dst + swz(t, c)) = make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
    if (t == 0) off[slot] = (int32_t)((((int64_t)lag[j] + K - 1) % n + n) % n);
}

constexpr size_t kSmemSpectra = (size_t)(kTwRows * 16 + 2 * kGroups * kTileLd) * sizeof(float2);
constexpr size_t kSmemFilter = (size_t)(kTwRows * 16 + 2 * kM + 2 * kFGroups * kTileLd) * sizeof(float2) + 64;
constexpr size_t kSmemTaps = (size_t)(kTwRows * 16 + 2 * kTileLd) * sizeof(float2);

}  // namespace

int fft_fir_block_len() { return kM; }
int fft_fir_tile_templates() { return kTileTemplates; }
int fft_fir_blocks_per_cta() { return kFGroups; }

rfd_status fft_pack(rfd_plan *plan, const float2 *taps, int32_t k_stride, const int32_t *lag, const double *sigma,
                    cudaStream_t s) {
    if (plan->fft_nslots == 0) return RFD_OK;
    static bool attr_set[64] = {};                      // once per device
    const int dev = plan->ctx->device < 64 ? plan->ctx->device : 63;
    if (!attr_set[dev]) {
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_taps_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTaps));
        attr_set[dev] = true;
    }
    for (int64_t s0 = 0; s0 < plan->fft_nslots; s0 += 65535) {
        const unsigned nblk = (unsigned)std::min<int64_t>(65535, plan->fft_nslots - s0);
        k_taps_spectra<<<nblk, kGT, kSmemTaps, s>>>(taps, k_stride, (const int32_t *)plan->d_perm.p,
                                             (const int32_t *)plan->d_kslot.p, lag, sigma, plan->grid.n,
                                             plan->fft_slot0, s0, (float2 *)plan->d_fft_P.p,
                                             (int32_t *)plan->d_off.p, plan->fft_stw);
        RFD_LAUNCH_CHECK();
    }
    return RFD_OK;
}

rfd_status fft_launch(const rfd_plan *plan, const void *q, const int32_t *qscale, const int64_t *u_begin,
                      rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s) {
    if (plan->fft_tiles.empty()) return RFD_OK;
    static bool attr_set[64] = {};                      // once per device (none inside a capture)
    const int dev = plan->ctx->device < 64 ? plan->ctx->device : 63;
    if (!attr_set[dev]) {
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_block_spectra<RFD_PREC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSmemSpectra));
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_block_spectra<RFD_PREC_FP16X3>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSpectra));
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_block_spectra<RFD_PREC_BF16X3>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemSpectra));
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_rf_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFilter));
        attr_set[dev] = true;
    }
    const dim3 gs((unsigned)((plan->fft_nb + kGroups - 1) / kGroups), (unsigned)plan->fft_refs.size());
    const int32_t *refs = (const int32_t *)plan->d_fft_refs.p;
    float2 *X = (float2 *)plan->d_fft_X.p;
    if (plan->precision == RFD_PREC_FP32)
        k_block_spectra<RFD_PREC_FP32><<<gs, kThreads, kSmemSpectra, s>>>(q, qscale, plan->ld, plan->grid.n,
                                                                            plan->fft_L, plan->fft_nb, refs, X,
                                                                            plan->fft_stw, u_begin);
    else if (plan->precision == RFD_PREC_FP16X3)
        k_block_spectra<RFD_PREC_FP16X3><<<gs, kThreads, kSmemSpectra, s>>>(q, qscale, plan->ld, plan->grid.n,
                                                                              plan->fft_L, plan->fft_nb, refs, X,
                                                                              plan->fft_stw, u_begin);
    else
        k_block_spectra<RFD_PREC_BF16X3><<<gs, kThreads, kSmemSpectra, s>>>(q, qscale, plan->ld, plan->grid.n,
                                                                              plan->fft_L, plan->fft_nb, refs, X,
                                                                              plan->fft_stw, u_begin);
    RFD_LAUNCH_CHECK();
    RfFftArgs a;
    a.tiles = (const FftTile *)plan->d_fft_tiles.p;
    a.ranges = (const int64_t *)plan->d_fft_ranges.p;
    a.nbg = plan->fft_nbg;
    a.nb = plan->fft_nb;
    a.L = plan->fft_L;
    a.out_len = plan->out_len;
    a.u_begin = u_begin;
    a.X = X;
    a.P = (const float2 *)plan->d_fft_P.p;
    a.slot0 = plan->fft_slot0;
    a.stw = plan->fft_stw;
    a.perm = (const int32_t *)plan->d_perm.p;
    a.off = (const int32_t *)plan->d_off.p;
    a.n = plan->grid.n;
    a.thr = plan->threshold;
    a.W = (uint32_t)plan->window;
    a.cand = cand;
    a.cap = cap;
    a.count = (unsigned long long *)count;
    k_rf_fft<<<(unsigned)plan->fft_grid, kFThreads, kSmemFilter, s>>>(a);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

}  // namespace rfd
