// Fused trigger epilogue: |z|^2 threshold and per-window maximum (Table II's peak find and
// trigger accumulation), shared by every filtering kernel.
#pragma once
#include "internal.cuh"

namespace rfd {

// One warp, one template: lane l holds the complex SNR z at true sample t_l.  Lanes whose
// |z|^2 exceeds `thr` are grouped by window w = t / W; for each group the lane with the
// largest |z|^2 (ties: smallest t) appends one candidate.  All 32 lanes must call this
// convergently with the same j.  Every float compare is on |z|^2 computed here once, so the
// candidate key and the stored z always agree.
__device__ __forceinline__ void emit_window_max(bool valid, uint32_t j, uint32_t t, float zr,
                                                float zi, float thr, uint32_t W,
                                                rfd_candidate *__restrict__ cand, int64_t cap,
                                                unsigned long long *__restrict__ count) {
    const float p = __fadd_rn(__fmul_rn(zr, zr), __fmul_rn(zi, zi));
    const bool pred = valid && (p > thr);
    unsigned pending = __ballot_sync(0xffffffffu, pred);
    if (!pending) return;
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t w = t / W;
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const uint32_t wl = __shfl_sync(0xffffffffu, w, leader);
        const unsigned same = __ballot_sync(0xffffffffu, pred && (w == wl)) & pending;
        const bool in = (same >> lane) & 1u;
        const uint32_t pb = in ? __float_as_uint(p) : 0u;   // p > 0: bit order = value order
        const uint32_t pmax = __reduce_max_sync(0xffffffffu, pb);
        const uint32_t tk = (in && pb == pmax) ? (0xffffffffu - t) : 0u;
        const uint32_t tkmax = __reduce_max_sync(0xffffffffu, tk);
        if (in && pb == pmax && tk == tkmax) {
            const unsigned long long idx = atomicAdd(count, 1ull);
            if ((int64_t)idx < cap) {
                rfd_candidate c;
                c.key = ((uint64_t)pmax << 32) | (uint64_t)tkmax;
                c.j = j;
                c.w = wl;
                c.zr = zr;
                c.zi = zi;
                cand[idx] = c;
            }
        }
        pending &= ~same;
    }
}

}  // namespace rfd
