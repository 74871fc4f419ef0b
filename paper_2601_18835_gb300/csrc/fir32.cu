// FP32 CUDA-core ratio filter (Eq. 3) with the fused trigger epilogue.
//
// One CTA = one tile of JT templates sharing a reference x TT consecutive output positions u.
// The q_ref window [u0, u0 + TT + K - 1) and the tile's reversed taps P[j][k] = rho_j[K-1-k]
// are staged in shared memory; thread (tg, ts) accumulates Y[j, u] = sum_k P[j][k] q[u + k]
// for 4 templates x 8 positions u = u0 + ts + 64 i.  The true sample is
// t = (u + s_j + K_j - 1) mod n; z = Y / sigma_eff.
#include "epilogue.cuh"
#include "internal.cuh"

namespace rfd {

namespace {

constexpr int kJT = 16;    // templates per tile
constexpr int kTT = 512;   // output positions per CTA
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fir32(
    const RfdTile *__restrict__ tiles, const float2 *__restrict__ q, int64_t ld,
    const float2 *__restrict__ taps, int32_t k_stride, const int32_t *__restrict__ perm,
    const int32_t *__restrict__ off, const float *__restrict__ scale, int64_t n, float thr,
    uint32_t W, rfd_candidate *__restrict__ cand, int64_t cap,
    unsigned long long *__restrict__ count, const int64_t *__restrict__ u_begin) {
    extern __shared__ float2 sm[];
    const RfdTile tile = tiles[blockIdx.y];
    const int K = tile.k_tile;
    const int64_t u0 = wrap_pos(window_base(u_begin, n), (int64_t)blockIdx.x * kTT, n);
    float2 *qs = sm;                       // [kTT + K - 1]
    float2 *ps = sm + kTT + K - 1;         // [kJT][K]
    const float2 *qr = q + (int64_t)tile.ref * ld + u0;
    for (int i = threadIdx.x; i < kTT + K - 1; i += kThreads) qs[i] = qr[i];
    for (int i = threadIdx.x; i < kJT * K; i += kThreads) {
        const int a = i / K, k = i - a * K;
        ps[i] = (a < tile.count) ? taps[(int64_t)(tile.first + a) * k_stride + k]
                                 : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int tg = threadIdx.x >> 6, ts = threadIdx.x & 63;
    float ar[4][8], ai[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 8; ++i) ar[a][i] = ai[a][i] = 0.f;
    const float2 *pt = ps + (tg * 4) * K;
    for (int k = 0; k < K; ++k) {
        float2 pv[4], qv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) pv[a] = pt[a * K + k];
#pragma unroll
        for (int i = 0; i < 8; ++i) qv[i] = qs[ts + 64 * i + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                ar[a][i] = fmaf(pv[a].x, qv[i].x, ar[a][i]);
                ar[a][i] = fmaf(-pv[a].y, qv[i].y, ar[a][i]);
                ai[a][i] = fmaf(pv[a].x, qv[i].y, ai[a][i]);
                ai[a][i] = fmaf(pv[a].y, qv[i].x, ai[a][i]);
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int slot_in_tile = tg * 4 + a;
        const bool vt = slot_in_tile < tile.count;
        const int64_t slot = tile.first + (vt ? slot_in_tile : 0);
        const int32_t j = vt ? perm[slot] : 0;
        const int32_t o = vt ? off[slot] : 0;
        const float sc = vt ? scale[slot] : 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t u = u0 + ts + 64 * i;
            const uint32_t t = (uint32_t)((u + o) & (n - 1));
            emit_window_max(vt && j >= 0 && u < n, (uint32_t)j, t, ar[a][i] * sc, ai[a][i] * sc,
                            thr, W, cand, cap, count);
        }
    }
}

}  // namespace

int fir32_tile_templates() { return kJT; }

rfd_status fir32_launch(const rfd_plan *plan, const float2 *q, const int64_t *u_begin, rfd_candidate *cand,
                        int64_t cap, int64_t *count, cudaStream_t s) {
    const int64_t n = plan->grid.n;
    const size_t shm = (size_t)(kTT + plan->k_max - 1 + kJT * plan->k_max) * sizeof(float2);
    static size_t smem_set[64] = {};
    const int dev = plan->ctx->device < 64 ? plan->ctx->device : 63;
    if (shm > smem_set[dev]) {
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_fir32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        smem_set[dev] = shm;
    }
    const unsigned ntiles = (unsigned)plan->tiles.size();
    for (unsigned t0 = 0; t0 < ntiles; t0 += 65535) {
        dim3 grid((unsigned)(plan->out_len / kTT), std::min(65535u, ntiles - t0));
        k_fir32<<<grid, kThreads, shm, s>>>(
            (const RfdTile *)plan->d_tiles.p + t0, q, plan->ld, (const float2 *)plan->d_taps.p,
            plan->k_max, (const int32_t *)plan->d_perm.p, (const int32_t *)plan->d_off.p,
            (const float *)plan->d_scale.p, n, plan->threshold, (uint32_t)plan->window, cand, cap,
            (unsigned long long *)count, u_begin);
        RFD_LAUNCH_CHECK();
    }
    return RFD_OK;
}

}  // namespace rfd

namespace rfd {

namespace {

// P[slot][k] = rho_j[K_j - 1 - k] for k < K_j, 0 up to k_max; off = (s_j + K_j - 1) mod n;
// scale = 1 / sigma_eff,j.
__global__ void k_pack_fp32(const float2 *__restrict__ taps, int32_t k_stride,
                            const int32_t *__restrict__ perm, const int32_t *__restrict__ kslot,
                            const int32_t *__restrict__ lag, const double *__restrict__ sigma,
                            int64_t n, int32_t kmax, float2 *__restrict__ out,
                            int32_t *__restrict__ off, float *__restrict__ scale) {
    const int64_t slot = blockIdx.x;
    const int32_t j = perm[slot];
    const int32_t K = kslot[slot];
    for (int k = threadIdx.x; k < kmax; k += blockDim.x)
        out[slot * kmax + k] = (k < K) ? taps[(int64_t)j * k_stride + (K - 1 - k)] : make_float2(0.f, 0.f);
    if (threadIdx.x == 0) {
        off[slot] = (int32_t)((((int64_t)lag[j] + K - 1) % n + n) % n);
        // a window with no weight (e.g. K = 2 under a Tukey taper) has sigma_eff = 0: no triggers
        scale[slot] = sigma[j] > 0.0 ? (float)(1.0 / sigma[j]) : 0.f;
    }
}

}  // namespace

rfd_status pack_taps_fp32(rfd_plan *plan, const float2 *taps, int32_t k_stride, const int32_t *lag,
                          const double *sigma, cudaStream_t s) {
    if (plan->n_slots == 0) return RFD_OK;
    k_pack_fp32<<<(unsigned)plan->n_slots, 128, 0, s>>>(
        taps, k_stride, (const int32_t *)plan->d_perm.p, (const int32_t *)plan->d_kslot.p, lag, sigma,
        plan->grid.n, plan->k_max, (float2 *)plan->d_taps.p, (int32_t *)plan->d_off.p,
        (float *)plan->d_scale.p);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

}  // namespace rfd
