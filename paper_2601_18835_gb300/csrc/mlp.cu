// Learned taps: one small MLP per reference maps a template to its 128 complex ratio-filter
// taps at the reference's fixed lag.  Inputs: (Mc, eta, chi_eff, Lambda~) standardised per
// network, and cos / sin of p_m = Dpsi(f_m) - Dpsi(f_a), Dpsi = Psi_j - Psi_r the ratio's phase
// (Eq. 2) in FP64 at eight frequencies log-spaced from 3 f_low to 0.45 fs around the anchor
// f_a (20 inputs, zero-padded to 64).  Training minimises the PSD-weighted chi^2 of Eq. 4
// between the taps' response and the exact taps' response, written in the tap domain
// through Parseval (Eqs. 5-6) and minimised over a constant phase of the target:
//   L = (rho^H M rho + a*^H M a* - 2 |a*^H M rho|) / (a*^H M a*),  M[b, a] = C_r[b - a].
// Layers: 20 -> 256 -> 256 -> 256 (GELU, tanh form) -> 256 = (Re, Im) of 128 taps.
//
// Every dense layer, forward and backward, is one tcgen05 GEMM (FP16 operands, FP32
// accumulation in tensor memory) C[128 x N] = A[128 x Kd] B[N x Kd]^T with both operands
// staged by cp.async into the K-major 128-byte-swizzle shared-memory layout and the bias /
// GELU / GELU' / transposed copies fused into the epilogue.  FP32 master weights, Adam
// (bias-corrected), dynamic loss scaling kept on the device (a step with a non-finite
// gradient is skipped and halves the scale; 1000 clean steps double it).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace rfd {
namespace {

using namespace tc;

constexpr int kH = 256;            // hidden width and output width
constexpr int kT = 128;            // taps
constexpr int kF = 64;             // inputs padded to one 64-element K chunk
constexpr int kIn = 20;            // inputs used: 4 physical features, 8 phasors (cos, sin)
constexpr int kPhasor = 8;
constexpr int kCw = 2 * kT - 1;    // C_r lags -(kT-1) .. kT-1
constexpr int64_t OFF_W1 = 0, OFF_B1 = kH * kIn, OFF_W2 = OFF_B1 + kH, OFF_B2 = OFF_W2 + kH * kH,
                  OFF_W3 = OFF_B2 + kH, OFF_B3 = OFF_W3 + kH * kH, OFF_W4 = OFF_B3 + kH, OFF_B4 = OFF_W4 + kH * kH,
                  kP = OFF_B4 + kH;
// FP16 copies per network: W1 padded [256][64], W2..W4 [out][in], and W2..W4 transposed [in][out]
constexpr int64_t HW1 = 0, HW2 = 16384, HW3 = HW2 + 65536, HW4 = HW3 + 65536, HT2 = HW4 + 65536, HT3 = HT2 + 65536,
                  HT4 = HT3 + 65536, kHP = HT4 + 65536;
constexpr int kNorm = 12;          // per network (double): mu[4], sd[4], out_scale, pad
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;
constexpr uint32_t kSpin = 1u << 24;

}  // namespace

struct MlpState {
    float loss_scale;
    int32_t good;      // clean steps since the last change of scale
    int32_t t;         // Adam steps taken
    int32_t inf;       // the last gradients had a non-finite value
    uint32_t err;      // a bounded wait gave up
    int32_t pad[3];
};

}  // namespace rfd

struct rfd_mlp {
    rfd_ctx *ctx = nullptr;
    rfd::Grid grid{};
    int32_t R = 0;
    std::vector<rfd::PNParams> refs;
    double fq[9] = {0};                // phasor frequencies, f_a = fq[4]
    std::vector<double> norm;          // [R][kNorm]
    std::vector<int32_t> lag;          // [R]
    rfd::DevBuf d_params, d_m, d_v, d_grads, d_wh, d_C, d_norm, d_lag, d_state, d_loss, d_refpn;
    rfd::DevBuf ws_train, ws_infer, ws_idx, ws_aux;
    int32_t batch = 0;                 // training batch per network the workspace is sized for
};

namespace rfd {
namespace {

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ float gelu_f(float u) {
    const float t = tanhf(kGeluC * (u + kGeluA * u * u * u));
    return 0.5f * u * (1.f + t);
}
__device__ __forceinline__ float gelu_grad_f(float u) {
    const float t = tanhf(kGeluC * (u + kGeluA * u * u * u));
    return 0.5f * (1.f + t) + 0.5f * u * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * u * u);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// rows x 64 halfs at g[r * ld + k0 ..] into a K-major 128-byte-swizzle tile at s (1024-aligned):
// 16-byte chunk c of row r lands at r * 128 + ((c ^ (r & 7)) * 16).
__device__ __forceinline__ void load_tile(uint32_t s, const __half *g, int64_t ld, int rows, int64_t k0, int tid) {
    for (int i = tid; i < rows * 8; i += 128) {
        const int r = i >> 3, c = i & 7;
        cp_async16(s + r * 128 + ((c ^ (r & 7)) << 4), g + (int64_t)r * ld + k0 + c * 8);
    }
}

__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpin; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------------ GEMM
enum GemmMode { kFwdHidden = 0, kFwdOut = 1, kBwdDH = 2, kDW = 3, kInferHidden = 4 };

struct GemmArgs {
    const __half *A; int64_t lda, a_gs;     // A [M][Kd] per activation group
    const __half *B; int64_t ldb, b_gs;     // B [N][Kd] per weight group
    int32_t N, Kd;                          // N: 64 or 256; Kd: multiple of 64
    const float *bias; int64_t bias_gs;
    float *oF; int64_t ldf, f_gs;           // FP32 output [M][ldf]
    __half *oH; int64_t ldh, h_gs;          // FP16 output [M][ldh]
    __half *oT; int64_t ldt, t_gs;          // FP16 transposed output [N][ldt]
    const float *Z; int64_t ldz, z_gs;      // pre-activations (kBwdDH)
    int32_t n_store;                        // kDW: columns stored
    const int32_t *tile_group;              // non-NULL: weight group of M-tile blockIdx.x (inference)
    uint32_t *err;
};

constexpr int kStageA = 128 * 128;          // bytes: 128 rows x 64 halfs
constexpr int kStageB = 256 * 128;
constexpr int kStage = kStageA + kStageB;
constexpr size_t kGemmSmem = 2 * kStage + 1024;

template <int MODE>
__global__ void __launch_bounds__(128, 1) k_mlp_gemm(GemmArgs a) {
    extern __shared__ uint8_t raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ag = blockIdx.z;
    const int64_t wg = a.tile_group ? a.tile_group[blockIdx.x] : blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * 128;
    const __half *A = a.A + ag * a.a_gs + m0 * a.lda;
    const __half *B = a.B + wg * a.b_gs;
    const uint32_t s0 = smem_u32(sm);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tbase), 256);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const int nk = a.Kd / 64;
    const uint32_t idesc = idesc_f16(128, (uint32_t)a.N, 0, 0);
    bool ok = true;

    load_tile(s0, A, a.lda, 128, 0, tid);
    load_tile(s0 + kStageA, B, a.ldb, a.N, 0, tid);
    cp_async_commit();
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc & 1;
        if (kc + 1 < nk) {
            if (kc >= 1 && ok) ok = wait_bounded(smem_u32(&bars[st ^ 1]), ((kc - 1) >> 1) & 1);
            const uint32_t sn = s0 + (st ^ 1) * kStage;
            load_tile(sn, A, a.lda, 128, (int64_t)(kc + 1) * 64, tid);
            load_tile(sn + kStageA, B, a.ldb, a.N, (int64_t)(kc + 1) * 64, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t sa = s0 + st * kStage, sb = sa + kStageA;
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16)
                mma_ss(tmem, desc_sw128(sa + k16 * 32), desc_sw128(sb + k16 * 32), idesc, (kc | k16) ? 1u : 0u);
            mma_commit(smem_u32(&bars[st]));
        }
    }
    {
        const int last = nk - 1;
        if (!wait_bounded(smem_u32(&bars[last & 1]), (last >> 1) & 1)) ok = false;
    }
    fence_after();
    if (!ok) {
        if (tid == 0) atomicOr(a.err, 1u);
    } else {
        const int64_t r = m0 + warp * 32 + lane;    // output row (within the activation group)
        for (int c0 = 0; c0 < a.N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tmem_ld_wait();
            if (MODE == kDW) {
                float *o = a.oF + ag * a.f_gs + r * a.ldf;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < a.n_store) o[c0 + j] = __uint_as_float(v[j]);
                continue;
            }
            float x[32];
            if (MODE == kFwdHidden || MODE == kFwdOut || MODE == kInferHidden) {
                const float *bias = a.bias + wg * a.bias_gs + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]) + bias[j];
            } else {   // kBwdDH
                const float *z = a.Z + ag * a.z_gs + r * a.ldz + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 zz = *(const float4 *)(z + j);
                    x[j] = __uint_as_float(v[j]) * gelu_grad_f(zz.x);
                    x[j + 1] = __uint_as_float(v[j + 1]) * gelu_grad_f(zz.y);
                    x[j + 2] = __uint_as_float(v[j + 2]) * gelu_grad_f(zz.z);
                    x[j + 3] = __uint_as_float(v[j + 3]) * gelu_grad_f(zz.w);
                }
            }
            if (MODE == kFwdHidden || MODE == kFwdOut) {
                float *o = a.oF + ag * a.f_gs + r * a.ldf + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 4) *(float4 *)(o + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
            }
            if (MODE == kFwdHidden || MODE == kInferHidden) {
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = gelu_f(x[j]);
            }
            if (MODE == kFwdHidden || MODE == kInferHidden || MODE == kBwdDH) {
                __half *o = a.oH + ag * a.h_gs + r * a.ldh + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 8) {
                    __align__(16) __half2 hh[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) hh[q] = __floats2half2_rn(x[j + 2 * q], x[j + 2 * q + 1]);
                    *(uint4 *)(o + j) = *(const uint4 *)hh;
                }
                if (MODE != kInferHidden && a.oT) {
                    __half *t = a.oT + ag * a.t_gs + (int64_t)c0 * a.ldt + r;
#pragma unroll
                    for (int j = 0; j < 32; ++j) t[(int64_t)j * a.ldt] = __float2half_rn(x[j]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------ features, gather
struct Phasors {
    double f[9];
};

__global__ void k_mlp_features(const rfd_params *__restrict__ p, const PNParams *__restrict__ tp,
                               const int32_t *__restrict__ net_of, const int32_t *__restrict__ row_of, int64_t n,
                               const double *__restrict__ norm, const PNParams *__restrict__ refpn, Phasors fq,
                               int32_t pn_flags, __half *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const rfd_params q = p[i];
    const int32_t g = net_of[i];
    const double M = q.m1 + q.m2, eta = q.m1 * q.m2 / (M * M);
    double x[4] = {M * pow(eta, 0.6), eta, (q.m1 * q.chi1 + q.m2 * q.chi2) / M, q.lambda_tilde};
    const double *nm = norm + (int64_t)g * kNorm;
    __half *o = out + (row_of ? (int64_t)row_of[i] : i) * kF;
#pragma unroll
    for (int f = 0; f < 4; ++f) o[f] = __float2half_rn((float)((x[f] - nm[f]) / nm[4 + f]));
    const PNParams tj = tp[i], tr = refpn[g];
    double d[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) d[m] = pn_phase(fq.f[m], tj, pn_flags) - pn_phase(fq.f[m], tr, pn_flags);
    int c = 0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        if (m == kPhasor / 2) continue;
        double sn, cs;
        sincos(d[m] - d[kPhasor / 2], &sn, &cs);
        o[4 + c] = __float2half_rn((float)cs);
        o[4 + kPhasor + c] = __float2half_rn((float)sn);
        ++c;
    }
}

// X[g][b] = feat[g][idx[g][b]], its transpose, and the target rows.
__global__ void k_mlp_gather(const __half *__restrict__ feat, const float2 *__restrict__ target,
                             const int32_t *__restrict__ idx, int32_t n_train, int32_t B, __half *__restrict__ X,
                             __half *__restrict__ Xt, float2 *__restrict__ Tb) {
    const int b = blockIdx.x, g = blockIdx.y, k = threadIdx.x;
    const int64_t src = (int64_t)g * n_train + idx[(int64_t)g * B + b];
    const int64_t row = (int64_t)g * B + b;
    if (k < kF) {
        const __half v = feat[src * kF + k];
        X[row * kF + k] = v;
        Xt[((int64_t)g * kF + k) * B + b] = v;
    }
    Tb[row * kT + k] = target[src * kT + k];
}

// ------------------------------------------------------------------ loss (Eq. 4 through Eqs. 5-6)
__device__ __forceinline__ float block_sum128(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return red[0] + red[1] + red[2] + red[3];
}

__global__ void __launch_bounds__(128) k_mlp_loss(const float *__restrict__ Y, const float2 *__restrict__ T,
                                                  const double2 *__restrict__ C, const double *__restrict__ norm,
                                                  const MlpState *__restrict__ st, int32_t B,
                                                  __half *__restrict__ dZ, __half *__restrict__ dZt,
                                                  float *__restrict__ lossv) {
    __shared__ float2 sC[kCw], sr[kT], stg[kT];
    __shared__ float red[4];
    const int b = blockIdx.x, g = blockIdx.y, k = threadIdx.x;
    const int64_t row = (int64_t)g * B + b;
    for (int i = k; i < kCw; i += 128) {
        const double2 c = C[(int64_t)g * kCw + i];
        sC[i] = make_float2((float)c.x, (float)c.y);
    }
    const float scale = (float)norm[(int64_t)g * kNorm + 8];
    const float2 rho = make_float2(scale * Y[row * kH + k], scale * Y[row * kH + kT + k]);
    const float2 t = T[row * kT + k];
    sr[k] = rho;
    stg[k] = t;
    __syncthreads();
    float mrr = 0.f, mri = 0.f, mtr = 0.f, mti = 0.f;
    for (int j = 0; j < kT; ++j) {       // (M x)[k] = sum_j C[k - j] x[j]
        const float2 c = sC[k - j + kT - 1], r = sr[j], u = stg[j];
        mrr += c.x * r.x - c.y * r.y;
        mri += c.x * r.y + c.y * r.x;
        mtr += c.x * u.x - c.y * u.y;
        mti += c.x * u.y + c.y * u.x;
    }
    const float s_r = block_sum128(rho.x * mrr + rho.y * mri, red);
    const float s_t = block_sum128(t.x * mtr + t.y * mti, red);
    // c = a*^H M rho = sum_k conj((M a*)[k]) rho[k]
    const float c_re = block_sum128(mtr * rho.x + mti * rho.y, red);
    const float c_im = block_sum128(mtr * rho.y - mti * rho.x, red);
    const float ca = sqrtf(c_re * c_re + c_im * c_im);
    const float pr = ca > 0.f ? c_re / ca : 1.f, pi = ca > 0.f ? c_im / ca : 0.f;
    const float f = 2.f * st->loss_scale * scale / (s_t * (float)B);
    const float gr = f * (mrr - (pr * mtr - pi * mti)), gi = f * (mri - (pr * mti + pi * mtr));
    dZ[row * kH + k] = __float2half_rn(gr);
    dZ[row * kH + kT + k] = __float2half_rn(gi);
    __half *dt = dZt + (int64_t)g * kH * B;
    dt[(int64_t)k * B + b] = __float2half_rn(gr);
    dt[(int64_t)(kT + k) * B + b] = __float2half_rn(gi);
    if (k == 0) lossv[row] = (s_r + s_t - 2.f * ca) / s_t;
}

// per-network mean of the per-sample losses (fixed order)
__global__ void k_mlp_loss_mean(const float *__restrict__ lossv, int32_t B, float *__restrict__ loss) {
    __shared__ float red[4];
    const int g = blockIdx.x;
    float v = 0.f;
    for (int b = threadIdx.x; b < B; b += 128) v += lossv[(int64_t)g * B + b];
    v = block_sum128(v, red);
    if (threadIdx.x == 0) loss[g] = v / (float)B;
}

// bias gradient: db[g][o] = sum_b dZt[g][o][b]
__global__ void k_mlp_colsum(const __half *__restrict__ dZt, int32_t B, float *__restrict__ grads, int64_t off) {
    const int g = blockIdx.y;
    const int o = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const __half *row = dZt + ((int64_t)g * kH + o) * B;
    float v = 0.f;
    for (int b = lane; b < B; b += 32) v += __half2float(row[b]);
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (lane == 0) grads[(int64_t)g * kP + off + o] = v;
}

// ------------------------------------------------------------------ optimiser
__device__ __forceinline__ void write_half(__half *wh, int64_t q, float p) {
    const __half h = __float2half_rn(p);
    if (q < OFF_B1) {
        wh[HW1 + (q / kIn) * kF + (q % kIn)] = h;
        return;
    }
    int64_t base, hw, ht;
    if (q >= OFF_W2 && q < OFF_B2) { base = OFF_W2; hw = HW2; ht = HT2; }
    else if (q >= OFF_W3 && q < OFF_B3) { base = OFF_W3; hw = HW3; ht = HT3; }
    else if (q >= OFF_W4 && q < OFF_B4) { base = OFF_W4; hw = HW4; ht = HT4; }
    else return;   // biases stay FP32
    const int64_t i = q - base, o = i >> 8, in = i & 255;
    wh[hw + i] = h;
    wh[ht + in * kH + o] = h;
}

__global__ void k_mlp_sync_half(const float *__restrict__ params, __half *__restrict__ wh, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    write_half(wh + (i / kP) * kHP, i % kP, params[i]);
}

__global__ void k_mlp_check(const float *__restrict__ grads, int64_t n, MlpState *st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t j = i; j < n; j += (int64_t)gridDim.x * blockDim.x) bad |= !isfinite(grads[j]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->inf, 1);
}

__global__ void k_mlp_adam(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grads, __half *__restrict__ wh, int64_t n, float lr,
                           float beta1, float beta2, float eps, const MlpState *__restrict__ st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || st->inf) return;
    const float t = (float)(st->t + 1);
    const float g = grads[i] / st->loss_scale;
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(beta1, t)), vh = vi / (1.f - powf(beta2, t));
    const float p = params[i] - lr * mh / (sqrtf(vh) + eps);
    params[i] = p;
    write_half(wh + (i / kP) * kHP, i % kP, p);
}

__global__ void k_mlp_unscale(const float *__restrict__ grads, const MlpState *__restrict__ st, int64_t n,
                              float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = grads[i] / st->loss_scale;
}

__global__ void k_mlp_scale(MlpState *st) {
    if (st->inf) {
        st->loss_scale = fmaxf(st->loss_scale * 0.5f, 1.f);
        st->good = 0;
        st->inf = 0;
    } else {
        st->t += 1;
        if (++st->good >= 1000) {
            st->loss_scale = fminf(st->loss_scale * 2.f, 16777216.f);
            st->good = 0;
        }
    }
}

// ------------------------------------------------------------------ inference output, matches
// sum_b conj(x2[b]) sum_a C[b - a] x1[a] over one template's taps (FP64), block of 128.
__device__ __forceinline__ double2 quad_form(const double2 *sC, const double2 *x1, const double2 *x2, double *red) {
    const int b = threadIdx.x;
    double ur = 0.0, ui = 0.0;
    for (int j = 0; j < kT; ++j) {
        const double2 c = sC[b - j + kT - 1], x = x1[j];
        ur += c.x * x.x - c.y * x.y;
        ui += c.x * x.y + c.y * x.x;
    }
    const double2 y = x2[b];
    double re = y.x * ur + y.y * ui, im = y.x * ui - y.y * ur;
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    __syncthreads();
    if ((b & 31) == 0) {
        red[(b >> 5) * 2] = re;
        red[(b >> 5) * 2 + 1] = im;
    }
    __syncthreads();
    return make_double2(red[0] + red[2] + red[4] + red[6], red[1] + red[3] + red[5] + red[7]);
}

// taps[j] = out_scale (y[k] + i y[128 + k]), lag[j] = s_r, sigma[j] = sqrt(rho^H M rho) of the
// stored (FP32) taps, for every valid row of the padded inference batch.
__global__ void __launch_bounds__(128) k_mlp_taps_out(const float *__restrict__ Y, const int32_t *__restrict__ row_tmpl,
                                                      const int32_t *__restrict__ row_net, const double *__restrict__ norm,
                                                      const double2 *__restrict__ C, const int32_t *__restrict__ lag_r,
                                                      int32_t k_stride, float2 *__restrict__ taps,
                                                      int32_t *__restrict__ lag, double *__restrict__ sigma) {
    __shared__ double2 sC[kCw], x[kT];
    __shared__ double red[8];
    const int64_t row = blockIdx.x;
    const int32_t j = row_tmpl[row];
    if (j < 0) return;
    const int g = row_net[row], k = threadIdx.x;
    for (int i = k; i < kCw; i += 128) sC[i] = C[(int64_t)g * kCw + i];
    const float scale = (float)norm[(int64_t)g * kNorm + 8];
    const float2 r = make_float2(scale * Y[row * kH + k], scale * Y[row * kH + kT + k]);
    x[k] = make_double2(r.x, r.y);
    float2 *o = taps + (int64_t)j * k_stride;
    o[k] = r;
    for (int i = kT + k; i < k_stride; i += 128) o[i] = make_float2(0.f, 0.f);
    if (k == 0) lag[j] = lag_r[g];
    __syncthreads();
    const double2 q = quad_form(sC, x, x, red);
    if (k == 0) sigma[j] = sqrt(fmax(q.x, 0.0));
}

// match between the responses of tap rows rho1[idx1[i]] and rho2[i] (same lag, same reference).
__global__ void __launch_bounds__(128) k_mlp_cross_match(const float2 *__restrict__ rho1, int64_t ld1,
                                                         const int32_t *__restrict__ idx1,
                                                         const float2 *__restrict__ rho2, int64_t ld2,
                                                         const int32_t *__restrict__ net, const double2 *__restrict__ C,
                                                         double *__restrict__ out) {
    __shared__ double2 sC[kCw], x1[kT], x2[kT];
    __shared__ double red[8];
    const int64_t i = blockIdx.x;
    const int k = threadIdx.x;
    const int g = net[i];
    for (int q = k; q < kCw; q += 128) sC[q] = C[(int64_t)g * kCw + q];
    const int64_t r1 = idx1 ? idx1[i] : i;
    const float2 a = rho1[r1 * ld1 + k], b = rho2[i * ld2 + k];
    x1[k] = make_double2(a.x, a.y);
    x2[k] = make_double2(b.x, b.y);
    __syncthreads();
    const double2 x12 = quad_form(sC, x1, x2, red);
    const double2 s1 = quad_form(sC, x1, x1, red);
    const double2 s2 = quad_form(sC, x2, x2, red);
    if (k == 0) out[i] = sqrt(x12.x * x12.x + x12.y * x12.y) / sqrt(s1.x * s2.x);
}

__global__ void k_scatter_taps(const float2 *__restrict__ src_taps, const int32_t *__restrict__ src_lag,
                               const double *__restrict__ src_sigma, const int32_t *__restrict__ dst_idx,
                               int32_t k_stride, float2 *__restrict__ taps, int32_t *__restrict__ lag,
                               double *__restrict__ sigma) {
    const int64_t i = blockIdx.x;
    const int64_t j = dst_idx[i];
    for (int k = threadIdx.x; k < k_stride; k += blockDim.x) taps[j * k_stride + k] = src_taps[i * k_stride + k];
    if (threadIdx.x == 0) {
        lag[j] = src_lag[i];
        sigma[j] = src_sigma[i];
    }
}

// ------------------------------------------------------------------ host side
template <int MODE>
rfd_status gemm(const GemmArgs &a, dim3 grid, cudaStream_t s) {
    static int attr_dev[64] = {0};
    int dev = 0;
    RFD_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr_dev[dev]) {
        RFD_TRY_CUDA(cudaFuncSetAttribute(k_mlp_gemm<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kGemmSmem));
        attr_dev[dev] = 1;
    }
    k_mlp_gemm<MODE><<<grid, 128, kGemmSmem, s>>>(a);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

// Training workspace for batch B per network (R networks), carved from one block.
struct TrainWs {
    __half *X, *Xt;                 // [R B][64], [R][64][B]
    float2 *T;                      // [R B][128]
    float *Z[3];                    // [R B][256]
    __half *Hh[3], *Ht[3];          // [R B][256], [R][256][B]
    float *Y;                       // [R B][256]
    __half *dZ[4], *dZt[4];         // index l = layer (0..3)
    float *lossv;                   // [R B]
};

size_t train_ws_bytes(int64_t R, int64_t B, TrainWs *w, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) / 256 * 256;
        return p;
    };
    const int64_t M = R * B;
    w->X = (__half *)take(M * kF * 2);
    w->Xt = (__half *)take(M * kF * 2);
    w->T = (float2 *)take(M * kT * 8);
    for (int l = 0; l < 3; ++l) {
        w->Z[l] = (float *)take(M * kH * 4);
        w->Hh[l] = (__half *)take(M * kH * 2);
        w->Ht[l] = (__half *)take(M * kH * 2);
    }
    w->Y = (float *)take(M * kH * 4);
    for (int l = 0; l < 4; ++l) {
        w->dZ[l] = (__half *)take(M * kH * 2);
        w->dZt[l] = (__half *)take(M * kH * 2);
    }
    w->lossv = (float *)take(M * 4);
    return off;
}

rfd_status mlp_forward_backward(rfd_mlp *P, const __half *feat, const float2 *target, int32_t n_train,
                                const int32_t *idx, int32_t B, cudaStream_t s) {
    const int64_t R = P->R;
    TrainWs w;
    const size_t bytes = train_ws_bytes(R, B, &w, nullptr);
    RFD_TRY(ensure(P->ws_train, bytes));
    train_ws_bytes(R, B, &w, (char *)P->ws_train.p);
    const float *prm = (const float *)P->d_params.p;
    const __half *wh = (const __half *)P->d_wh.p;
    float *grads = (float *)P->d_grads.p;
    uint32_t *err = &((MlpState *)P->d_state.p)->err;
    const int64_t hgs = (int64_t)B * kH;     // per-network stride of [B][256] activations
    const dim3 gm((unsigned)(B / 128), 1, (unsigned)R);

    k_mlp_gather<<<dim3((unsigned)B, (unsigned)R), 128, 0, s>>>(feat, target, idx, n_train, B, w.X, w.Xt, w.T);
    RFD_LAUNCH_CHECK();
    // forward: Z1 = X W1^T + b1 (K = 64 padded features), then two hidden layers, then the output
    const int64_t offW[4] = {HW1, HW2, HW3, HW4}, offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
    for (int l = 0; l < 4; ++l) {
        GemmArgs a{};
        a.A = l == 0 ? w.X : w.Hh[l - 1];
        a.lda = l == 0 ? kF : kH;
        a.a_gs = (int64_t)B * a.lda;
        a.B = wh + offW[l];
        a.ldb = l == 0 ? kF : kH;
        a.b_gs = kHP;
        a.N = kH;
        a.Kd = l == 0 ? kF : kH;
        a.bias = prm + offB[l];
        a.bias_gs = kP;
        a.err = err;
        if (l < 3) {
            a.oF = w.Z[l]; a.ldf = kH; a.f_gs = hgs;
            a.oH = w.Hh[l]; a.ldh = kH; a.h_gs = hgs;
            a.oT = w.Ht[l]; a.ldt = B; a.t_gs = hgs;
            RFD_TRY(gemm<kFwdHidden>(a, gm, s));
        } else {
            a.oF = w.Y; a.ldf = kH; a.f_gs = hgs;
            RFD_TRY(gemm<kFwdOut>(a, gm, s));
        }
    }
    k_mlp_loss<<<dim3((unsigned)B, (unsigned)R), 128, 0, s>>>(w.Y, w.T, (const double2 *)P->d_C.p,
                                                             (const double *)P->d_norm.p, (const MlpState *)P->d_state.p,
                                                             B, w.dZ[3], w.dZt[3], w.lossv);
    RFD_LAUNCH_CHECK();
    k_mlp_loss_mean<<<(unsigned)R, 128, 0, s>>>(w.lossv, B, (float *)P->d_loss.p);
    RFD_LAUNCH_CHECK();
    // backward
    const int64_t offWg[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
    const int64_t offT[4] = {0, HT2, HT3, HT4};
    for (int l = 3; l >= 0; --l) {
        {   // dW_l = dZ_l^T H_{l-1}  (M = 256 outputs in two tiles, N = inputs, K = batch)
            GemmArgs a{};
            a.A = w.dZt[l]; a.lda = B; a.a_gs = hgs;
            a.B = l == 0 ? w.Xt : w.Ht[l - 1];
            a.ldb = B;
            a.b_gs = l == 0 ? (int64_t)kF * B : hgs;
            a.N = l == 0 ? kF : kH;
            a.Kd = B;
            a.oF = grads + offWg[l]; a.ldf = l == 0 ? kIn : kH; a.f_gs = kP;
            a.n_store = l == 0 ? kIn : kH;
            a.err = err;
            RFD_TRY(gemm<kDW>(a, dim3(2, 1, (unsigned)R), s));
        }
        k_mlp_colsum<<<dim3(kH / 8, (unsigned)R), 256, 0, s>>>(w.dZt[l], B, grads, offB[l]);
        RFD_LAUNCH_CHECK();
        if (l > 0) {   // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
            GemmArgs a{};
            a.A = w.dZ[l]; a.lda = kH; a.a_gs = hgs;
            a.B = wh + offT[l]; a.ldb = kH; a.b_gs = kHP;
            a.N = kH;
            a.Kd = kH;
            a.Z = w.Z[l - 1]; a.ldz = kH; a.z_gs = hgs;
            a.oH = w.dZ[l - 1]; a.ldh = kH; a.h_gs = hgs;
            a.oT = w.dZt[l - 1]; a.ldt = B; a.t_gs = hgs;
            a.err = err;
            RFD_TRY(gemm<kBwdDH>(a, gm, s));
        }
    }
    return RFD_OK;
}

rfd_status check_train_args(rfd_mlp *P, const void *feat, const void *target, int32_t n_train, const int32_t *idx,
                            int32_t B) {
    RFD_REQUIRE(P && feat && target && idx, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(B >= 128 && B % 128 == 0 && B <= 8192, RFD_ERR_SHAPE, "batch=%d must be a multiple of 128 in [128, 8192]",
                B);
    RFD_REQUIRE(n_train >= 1, RFD_ERR_SHAPE, "n_train must be >= 1");
    return RFD_OK;
}

// Inference batch: templates grouped by network, each group padded to 128-row tiles.
struct InferPlan {
    std::vector<int32_t> row_tmpl, row_net, tile_net, row_of;
    int64_t rows = 0;
};

void plan_infer(const int32_t *net_of, int32_t n, int32_t R, InferPlan *ip) {
    std::vector<std::vector<int32_t>> by(R);
    for (int32_t j = 0; j < n; ++j) by[net_of[j]].push_back(j);
    ip->row_tmpl.clear();
    ip->row_net.clear();
    ip->tile_net.clear();
    ip->row_of.assign(n, -1);
    for (int32_t g = 0; g < R; ++g) {
        const int64_t cnt = (int64_t)by[g].size();
        const int64_t tiles = (cnt + 127) / 128;
        for (int64_t t = 0; t < tiles; ++t) {
            ip->tile_net.push_back(g);
            for (int r = 0; r < 128; ++r) {
                const int64_t i = t * 128 + r;
                const int32_t j = i < cnt ? by[g][i] : -1;
                if (j >= 0) ip->row_of[j] = (int32_t)ip->row_tmpl.size();
                ip->row_tmpl.push_back(j);
                ip->row_net.push_back(g);
            }
        }
    }
    ip->rows = (int64_t)ip->row_tmpl.size();
}

// Copies the templates' parameters and their FP64 phase constants to the device and writes
// the network inputs of row row_of[i] (or i) for template i.  Synchronises the stream (the
// staging buffers are reused by the next call).
rfd_status features_impl(rfd_mlp *P, const rfd_params *host, const int32_t *net_of_host, int64_t n,
                         const int32_t *row_of_dev, __half *out, cudaStream_t s) {
    std::vector<PNParams> pn;
    RFD_TRY(make_pn_vec(P->grid, host, (int32_t)n, &pn));
    const size_t bp = ((size_t)n * sizeof(rfd_params) + 255) / 256 * 256;
    const size_t bq = ((size_t)n * sizeof(PNParams) + 255) / 256 * 256;
    RFD_TRY(ensure(P->ws_aux, bp + bq + (size_t)n * 4));
    rfd_params *dp = (rfd_params *)P->ws_aux.p;
    PNParams *dq = (PNParams *)((char *)P->ws_aux.p + bp);
    int32_t *dn = (int32_t *)((char *)P->ws_aux.p + bp + bq);
    RFD_TRY_CUDA(cudaMemcpyAsync(dp, host, n * sizeof(rfd_params), cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(dq, pn.data(), n * sizeof(PNParams), cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(dn, net_of_host, n * 4, cudaMemcpyHostToDevice, s));
    Phasors fq;
    for (int m = 0; m < 9; ++m) fq.f[m] = P->fq[m];
    k_mlp_features<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dp, dq, dn, row_of_dev, n, (const double *)P->d_norm.p,
                                                               (const PNParams *)P->d_refpn.p, fq, P->grid.pn_flags,
                                                               out);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return RFD_OK;
}

rfd_status mlp_infer_impl(rfd_mlp *P, const rfd_params *params_host, const int32_t *net_of, int32_t n,
                          int32_t k_stride, float2 *taps, int32_t *lag, double *sigma, cudaStream_t s) {
    InferPlan ip;
    plan_infer(net_of, n, P->R, &ip);
    const int64_t rows = ip.rows, tiles = rows / 128;
    if (rows == 0) return RFD_OK;
    // workspace: X [rows][64] half, H0/H1 [rows][256] half, Y [rows][256] float, int32 tables
    const size_t bx = rows * kF * 2, bh = rows * kH * 2, by = rows * kH * 4, bi = rows * 4;
    const size_t bt = tiles * 4 + 256, bo = (size_t)n * 4;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    RFD_TRY(ensure(P->ws_infer, up(bx) + 2 * up(bh) + up(by) + 2 * up(bi) + up(bt) + up(bo)));
    char *base = (char *)P->ws_infer.p;
    __half *X = (__half *)base; base += up(bx);
    __half *H0 = (__half *)base; base += up(bh);
    __half *H1 = (__half *)base; base += up(bh);
    float *Y = (float *)base; base += up(by);
    int32_t *d_row_tmpl = (int32_t *)base; base += up(bi);
    int32_t *d_row_net = (int32_t *)base; base += up(bi);
    int32_t *d_tile_net = (int32_t *)base; base += up(bt);
    int32_t *d_row_of = (int32_t *)base;
    RFD_TRY_CUDA(cudaMemcpyAsync(d_row_tmpl, ip.row_tmpl.data(), bi, cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(d_row_net, ip.row_net.data(), bi, cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(d_tile_net, ip.tile_net.data(), tiles * 4, cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(d_row_of, ip.row_of.data(), bo, cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaMemsetAsync(X, 0, bx, s));
    RFD_TRY(features_impl(P, params_host, net_of, n, d_row_of, X, s));
    const float *prm = (const float *)P->d_params.p;
    const __half *wh = (const __half *)P->d_wh.p;
    uint32_t *err = &((MlpState *)P->d_state.p)->err;
    const int64_t offW[4] = {HW1, HW2, HW3, HW4}, offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
    __half *Hs[2] = {H0, H1};
    for (int l = 0; l < 4; ++l) {
        GemmArgs a{};
        a.A = l == 0 ? X : Hs[(l - 1) & 1];
        a.lda = l == 0 ? kF : kH;
        a.B = wh + offW[l];
        a.ldb = l == 0 ? kF : kH;
        a.b_gs = kHP;
        a.N = kH;
        a.Kd = l == 0 ? kF : kH;
        a.bias = prm + offB[l];
        a.bias_gs = kP;
        a.tile_group = d_tile_net;
        a.err = err;
        if (l < 3) {
            a.oH = Hs[l & 1];
            a.ldh = kH;
            RFD_TRY(gemm<kInferHidden>(a, dim3((unsigned)tiles), s));
        } else {
            a.oF = Y;
            a.ldf = kH;
            RFD_TRY(gemm<kFwdOut>(a, dim3((unsigned)tiles), s));
        }
    }
    k_mlp_taps_out<<<(unsigned)rows, 128, 0, s>>>(Y, d_row_tmpl, d_row_net, (const double *)P->d_norm.p,
                                                  (const double2 *)P->d_C.p, (const int32_t *)P->d_lag.p, k_stride,
                                                  taps, lag, sigma);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

rfd_status check_status(rfd_mlp *P, cudaStream_t s) {
    MlpState h;
    RFD_TRY_CUDA(cudaMemcpyAsync(&h, P->d_state.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    RFD_REQUIRE(!h.err, RFD_ERR_TIMEOUT, "an MLP kernel gave up waiting for its tensor-core work");
    return RFD_OK;
}

}  // namespace
}  // namespace rfd

using namespace rfd;

extern "C" {

int64_t rfd_mlp_param_count(void) { return kP; }

void rfd_mlp_destroy(rfd_mlp *P) {
    if (!P) return;
    DevBuf *bufs[] = {&P->d_params, &P->d_m, &P->d_v, &P->d_grads, &P->d_wh, &P->d_C, &P->d_norm, &P->d_lag,
                      &P->d_state, &P->d_loss, &P->d_refpn, &P->ws_train, &P->ws_infer, &P->ws_idx, &P->ws_aux};
    for (DevBuf *b : bufs) release(*b);
    delete P;
}

rfd_status rfd_mlp_create(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev, const rfd_params *refs_host,
                          int32_t n_ref, rfd_mlp **out) {
    RFD_REQUIRE(ctx && grid && psd_dev && refs_host && out, RFD_ERR_ARG, "NULL argument");
    *out = nullptr;
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_ref <= 4096, RFD_ERR_SHAPE, "n_ref=%d not in [1, 4096]", n_ref);
    RFD_REQUIRE(g.n >= 2 * kT, RFD_ERR_SHAPE, "n must be at least %d", 2 * kT);
    RFD_REQUIRE(0.45 * g.fs > 3.0 * g.f_low, RFD_ERR_ARG, "the phasor band 3 f_low .. 0.45 fs is empty");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    rfd_mlp *P = new rfd_mlp();
    P->ctx = ctx;
    P->grid = g;
    P->R = n_ref;
    rfd_status st = RFD_OK;
    do {
        if ((st = make_pn_vec(g, refs_host, n_ref, &P->refs)) != RFD_OK) break;
        const int64_t R = n_ref;
        if ((st = ensure(P->d_params, R * kP * 4)) || (st = ensure(P->d_m, R * kP * 4)) ||
            (st = ensure(P->d_v, R * kP * 4)) || (st = ensure(P->d_grads, R * kP * 4)) ||
            (st = ensure(P->d_wh, R * kHP * 2)) || (st = ensure(P->d_C, R * kCw * sizeof(double2))) ||
            (st = ensure(P->d_norm, R * kNorm * 8)) || (st = ensure(P->d_lag, R * 4)) ||
            (st = ensure(P->d_state, sizeof(MlpState))) || (st = ensure(P->d_loss, R * 4)) ||
            (st = ensure(P->d_refpn, R * sizeof(PNParams))))
            break;
        for (int m = 0; m < 9; ++m)
            P->fq[m] = 3.0 * g.f_low * std::pow(0.45 * g.fs / (3.0 * g.f_low), (double)m / 8.0);
        cudaError_t e;
        if ((e = cudaMemset(P->d_params.p, 0, R * kP * 4)) != cudaSuccess ||
            (e = cudaMemset(P->d_m.p, 0, R * kP * 4)) != cudaSuccess ||
            (e = cudaMemset(P->d_v.p, 0, R * kP * 4)) != cudaSuccess ||
            (e = cudaMemset(P->d_wh.p, 0, R * kHP * 2)) != cudaSuccess ||
            (e = cudaMemset(P->d_lag.p, 0, R * 4)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemset failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        MlpState s0{};
        s0.loss_scale = 65536.f;
        P->norm.assign(R * kNorm, 0.0);
        for (int64_t r = 0; r < R; ++r) {
            for (int f = 0; f < 4; ++f) P->norm[r * kNorm + 4 + f] = 1.0;
            P->norm[r * kNorm + 8] = 1.0;
        }
        P->lag.assign(R, 0);
        if ((e = cudaMemcpy(P->d_state.p, &s0, sizeof(s0), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(P->d_norm.p, P->norm.data(), R * kNorm * 8, cudaMemcpyHostToDevice)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        for (int64_t r = 0; r < R; ++r)
            if (P->refs[r].k_hi < g.k_lo) {
                set_error("reference %lld has an empty band (ISCO below f_low)", (long long)r);
                st = RFD_ERR_ARG;
            }
        if (st) break;
        // C_r rows through the library's FP64 path (one inverse FFT per reference)
        if ((st = ensure(ctx->ws[0], R * sizeof(PNParams)))) break;
        if ((e = cudaMemcpy(ctx->ws[0].p, P->refs.data(), R * sizeof(PNParams), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(P->d_refpn.p, P->refs.data(), R * sizeof(PNParams), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        if ((st = ref_autocorr_impl(ctx, g, psd_dev, (const PNParams *)ctx->ws[0].p, R, kT, (double2 *)P->d_C.p, 0)))
            break;
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("autocorrelation failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
        }
    } while (0);
    if (st != RFD_OK) {
        rfd_mlp_destroy(P);
        return st;
    }
    *out = P;
    return RFD_OK;
}

rfd_status rfd_mlp_set_weights(rfd_mlp *P, const float *host) {
    RFD_REQUIRE(P && host, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    const int64_t n = (int64_t)P->R * kP;
    for (int64_t i = 0; i < n; ++i)
        RFD_REQUIRE(std::isfinite(host[i]), RFD_ERR_ARG, "weight %lld is not finite", (long long)i);
    RFD_TRY_CUDA(cudaMemcpy(P->d_params.p, host, n * 4, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemset(P->d_m.p, 0, n * 4));
    RFD_TRY_CUDA(cudaMemset(P->d_v.p, 0, n * 4));
    MlpState s0{};
    s0.loss_scale = 65536.f;
    RFD_TRY_CUDA(cudaMemcpy(P->d_state.p, &s0, sizeof(s0), cudaMemcpyHostToDevice));
    k_mlp_sync_half<<<(unsigned)((n + 255) / 256), 256>>>((const float *)P->d_params.p, (__half *)P->d_wh.p, n);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    return RFD_OK;
}

rfd_status rfd_mlp_get_weights(const rfd_mlp *P, float *host) {
    RFD_REQUIRE(P && host, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    RFD_TRY_CUDA(cudaMemcpy(host, P->d_params.p, (size_t)P->R * kP * 4, cudaMemcpyDeviceToHost));
    return RFD_OK;
}

rfd_status rfd_mlp_set_norm(rfd_mlp *P, const double *mu, const double *sd, const double *out_scale,
                            const int32_t *lag) {
    RFD_REQUIRE(P && mu && sd && out_scale && lag, RFD_ERR_ARG, "NULL argument");
    const int64_t R = P->R;
    for (int64_t r = 0; r < R; ++r) {
        for (int f = 0; f < 4; ++f) {
            RFD_REQUIRE(std::isfinite(mu[r * 4 + f]) && std::isfinite(sd[r * 4 + f]) && sd[r * 4 + f] > 0,
                        RFD_ERR_ARG, "network %lld: feature %d needs a finite mean and a positive spread",
                        (long long)r, f);
            P->norm[r * kNorm + f] = mu[r * 4 + f];
            P->norm[r * kNorm + 4 + f] = sd[r * 4 + f];
        }
        RFD_REQUIRE(std::isfinite(out_scale[r]) && out_scale[r] > 0, RFD_ERR_ARG, "out_scale[%lld] must be > 0",
                    (long long)r);
        RFD_REQUIRE(lag[r] >= -(P->grid.n / 2) && lag[r] < P->grid.n / 2, RFD_ERR_ARG, "lag[%lld]=%d out of range",
                    (long long)r, lag[r]);
        P->norm[r * kNorm + 8] = out_scale[r];
        P->lag[r] = lag[r];
    }
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    RFD_TRY_CUDA(cudaMemcpy(P->d_norm.p, P->norm.data(), R * kNorm * 8, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_lag.p, P->lag.data(), R * 4, cudaMemcpyHostToDevice));
    return RFD_OK;
}

rfd_status rfd_mlp_get_autocorr(const rfd_mlp *P, double *host) {
    RFD_REQUIRE(P && host, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    RFD_TRY_CUDA(cudaMemcpy(host, P->d_C.p, (size_t)P->R * kCw * sizeof(double2), cudaMemcpyDeviceToHost));
    return RFD_OK;
}

rfd_status rfd_mlp_features(rfd_mlp *P, const rfd_params *params_host, const int32_t *net_of_host, int32_t n,
                            void *feat_dev, void *stream) {
    RFD_REQUIRE(P && params_host && net_of_host && feat_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n >= 0, RFD_ERR_SHAPE, "n < 0");
    if (n == 0) return RFD_OK;
    for (int32_t j = 0; j < n; ++j)
        RFD_REQUIRE(net_of_host[j] >= 0 && net_of_host[j] < P->R, RFD_ERR_ARG, "net_of[%d]=%d out of range", j,
                    net_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY_CUDA(cudaMemsetAsync(feat_dev, 0, (size_t)n * kF * 2, s));
    return features_impl(P, params_host, net_of_host, n, nullptr, (__half *)feat_dev, s);
}

rfd_status rfd_mlp_grads(rfd_mlp *P, const void *feat_dev, const void *target_dev, int32_t n_train,
                         const int32_t *idx_dev, int32_t batch, float *grads_dev, float *loss_dev, void *stream) {
    RFD_TRY(check_train_args(P, feat_dev, target_dev, n_train, idx_dev, batch));
    RFD_REQUIRE(grads_dev && loss_dev, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(mlp_forward_backward(P, (const __half *)feat_dev, (const float2 *)target_dev, n_train, idx_dev, batch, s));
    const int64_t n = (int64_t)P->R * kP;
    k_mlp_unscale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float *)P->d_grads.p,
                                                              (const MlpState *)P->d_state.p, n, grads_dev);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaMemcpyAsync(loss_dev, P->d_loss.p, (size_t)P->R * 4, cudaMemcpyDeviceToDevice, s));
    return check_status(P, s);
}

rfd_status rfd_mlp_train_step(rfd_mlp *P, const void *feat_dev, const void *target_dev, int32_t n_train,
                              const int32_t *idx_dev, int32_t batch, float lr, void *stream) {
    RFD_TRY(check_train_args(P, feat_dev, target_dev, n_train, idx_dev, batch));
    RFD_REQUIRE(std::isfinite(lr) && lr > 0.f, RFD_ERR_ARG, "lr must be > 0");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(mlp_forward_backward(P, (const __half *)feat_dev, (const float2 *)target_dev, n_train, idx_dev, batch, s));
    const int64_t n = (int64_t)P->R * kP;
    MlpState *st = (MlpState *)P->d_state.p;
    k_mlp_check<<<256, 256, 0, s>>>((const float *)P->d_grads.p, n, st);
    RFD_LAUNCH_CHECK();
    k_mlp_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float *)P->d_params.p, (float *)P->d_m.p,
                                                           (float *)P->d_v.p, (const float *)P->d_grads.p,
                                                           (__half *)P->d_wh.p, n, lr, 0.9f, 0.999f, 1e-8f, st);
    RFD_LAUNCH_CHECK();
    k_mlp_scale<<<1, 1, 0, s>>>(st);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

rfd_status rfd_mlp_state(rfd_mlp *P, float *loss_host, int32_t *step_host, float *loss_scale_host, void *stream) {
    RFD_REQUIRE(P, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(check_status(P, s));
    MlpState h;
    RFD_TRY_CUDA(cudaMemcpy(&h, P->d_state.p, sizeof(h), cudaMemcpyDeviceToHost));
    if (step_host) *step_host = h.t;
    if (loss_scale_host) *loss_scale_host = h.loss_scale;
    if (loss_host) RFD_TRY_CUDA(cudaMemcpy(loss_host, P->d_loss.p, (size_t)P->R * 4, cudaMemcpyDeviceToHost));
    return RFD_OK;
}

rfd_status rfd_mlp_infer(rfd_mlp *P, const rfd_params *params_host, const int32_t *net_of_host, int32_t n,
                         int32_t k_stride, void *taps_dev, int32_t *lag_dev, double *sigma_dev, void *stream) {
    RFD_REQUIRE(P && params_host && net_of_host && taps_dev && lag_dev && sigma_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n >= 0, RFD_ERR_SHAPE, "n < 0");
    RFD_REQUIRE(k_stride >= kT && k_stride <= 4096, RFD_ERR_SHAPE, "k_stride=%d not in [%d, 4096]", k_stride, kT);
    if (n == 0) return RFD_OK;
    for (int32_t j = 0; j < n; ++j)
        RFD_REQUIRE(net_of_host[j] >= 0 && net_of_host[j] < P->R, RFD_ERR_ARG, "net_of[%d]=%d out of range", j,
                    net_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(mlp_infer_impl(P, params_host, net_of_host, n, k_stride, (float2 *)taps_dev, lag_dev, sigma_dev, s));
    RFD_TRY(check_status(P, s));
    return RFD_OK;
}

rfd_status rfd_mlp_cross_match(rfd_mlp *P, const int32_t *net_of_host, int32_t n, const void *rho1_dev, int64_t ld1,
                               const void *rho2_dev, int64_t ld2, double *match_dev, void *stream) {
    RFD_REQUIRE(P && net_of_host && rho1_dev && rho2_dev && match_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n >= 0 && ld1 >= kT && ld2 >= kT, RFD_ERR_SHAPE, "need n >= 0 and row strides >= %d", kT);
    if (n == 0) return RFD_OK;
    for (int32_t j = 0; j < n; ++j)
        RFD_REQUIRE(net_of_host[j] >= 0 && net_of_host[j] < P->R, RFD_ERR_ARG, "net_of[%d]=%d out of range", j,
                    net_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(ensure(P->ws_idx, (size_t)n * 4));
    RFD_TRY_CUDA(cudaMemcpyAsync(P->ws_idx.p, net_of_host, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    k_mlp_cross_match<<<(unsigned)n, 128, 0, s>>>((const float2 *)rho1_dev, ld1, nullptr, (const float2 *)rho2_dev, ld2,
                                                  (const int32_t *)P->ws_idx.p, (const double2 *)P->d_C.p, match_dev);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return RFD_OK;
}

rfd_status rfd_learned_taps(rfd_mlp *P, const double *psd_dev, const rfd_params *tmpl_host,
                            const int32_t *ref_of_host, int32_t n_tmpl, int32_t spot_stride, double min_match,
                            int32_t k_stride, double tukey_alpha, void *taps_dev, int32_t *lag_dev, double *sigma_dev,
                            double *surrogate_match_dev, int32_t *source_dev, int64_t *stats_host, void *stream) {
    RFD_REQUIRE(P && psd_dev && tmpl_host && ref_of_host && taps_dev && lag_dev && sigma_dev && source_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(n_tmpl >= 0, RFD_ERR_SHAPE, "n_tmpl < 0");
    RFD_REQUIRE(spot_stride >= 1, RFD_ERR_ARG, "spot_stride must be >= 1");
    RFD_REQUIRE(std::isfinite(min_match) && min_match <= 1.0, RFD_ERR_ARG, "min_match must be <= 1");
    RFD_REQUIRE(k_stride >= kT && k_stride <= 4096 && k_stride <= P->grid.n, RFD_ERR_SHAPE,
                "k_stride=%d not in [%d, min(4096, n)]", k_stride, kT);
    if (n_tmpl == 0) return RFD_OK;
    for (int32_t j = 0; j < n_tmpl; ++j)
        RFD_REQUIRE(ref_of_host[j] >= 0 && ref_of_host[j] < P->R, RFD_ERR_ARG, "ref_of[%d]=%d out of range", j,
                    ref_of_host[j]);
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    rfd_ctx *ctx = P->ctx;
    const Grid &g = P->grid;
    // 1. surrogate taps for every template
    RFD_TRY(mlp_infer_impl(P, tmpl_host, ref_of_host, n_tmpl, k_stride, (float2 *)taps_dev, lag_dev, sigma_dev, s));
    // 2. spot sample: per reference, every spot_stride-th template in chirp-mass order, and the last
    std::vector<std::vector<int32_t>> by(P->R);
    std::vector<double> mc(n_tmpl);
    for (int32_t j = 0; j < n_tmpl; ++j) {
        const double M = tmpl_host[j].m1 + tmpl_host[j].m2;
        mc[j] = std::pow(tmpl_host[j].m1 * tmpl_host[j].m2, 0.6) / std::pow(M, 0.2);
        by[ref_of_host[j]].push_back(j);
    }
    std::vector<int32_t> spot, spot_ref, spot_lag, spot_k;
    std::vector<std::vector<int32_t>> spot_pos(P->R);    // positions (in Mc order) of the spot templates
    for (int32_t r = 0; r < P->R; ++r) {
        auto &v = by[r];
        std::stable_sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return mc[a] < mc[b]; });
        const int32_t cnt = (int32_t)v.size();
        for (int32_t p = 0; p < cnt; ++p)
            if (p % spot_stride == 0 || p == cnt - 1) {
                spot_pos[r].push_back(p);
                spot.push_back(v[p]);
                spot_ref.push_back(r);
                spot_lag.push_back(P->lag[r]);
                spot_k.push_back(kT);
            }
    }
    const int32_t ns = (int32_t)spot.size();
    // 3. exact taps of the spot sample at the reference's lag
    std::vector<rfd_params> spot_params(ns);
    for (int32_t i = 0; i < ns; ++i) spot_params[i] = tmpl_host[spot[i]];
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t bt = (size_t)std::max(ns, 1) * k_stride * sizeof(float2);
    DevBuf scratch;
    const size_t need = up(bt) + up((size_t)ns * 8) * 2 + up((size_t)ns * 4) * 3;
    RFD_TRY(ensure(scratch, need));
    char *base = (char *)scratch.p;
    float2 *ex_taps = (float2 *)base; base += up(bt);
    double *ex_sigma = (double *)base; base += up((size_t)ns * 8);
    double *smatch = (double *)base; base += up((size_t)ns * 8);
    int32_t *d_spot = (int32_t *)base; base += up((size_t)ns * 4);
    int32_t *d_spot_ref = (int32_t *)base; base += up((size_t)ns * 4);
    int32_t *d_lag_tmp = (int32_t *)base;
    rfd_status st = RFD_OK;
    do {
        std::vector<PNParams> tmpl_pn;
        if ((st = make_pn_vec(g, spot_params.data(), ns, &tmpl_pn))) break;
        if ((st = make_taps_impl(ctx, g, psd_dev, P->refs, tmpl_pn, spot_ref, spot_k, {}, spot_lag, 1.0, k_stride,
                                 tukey_alpha, ex_taps, nullptr, d_lag_tmp, ex_sigma, nullptr, s)))
            break;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(d_spot, spot.data(), ns * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_spot_ref, spot_ref.data(), ns * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("cudaMemcpyAsync failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        // 4. surrogate match against the exact taps
        k_mlp_cross_match<<<(unsigned)ns, 128, 0, s>>>((const float2 *)taps_dev, k_stride, d_spot, ex_taps, k_stride,
                                                       d_spot_ref, (const double2 *)P->d_C.p, smatch);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            set_error("k_mlp_cross_match launch failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        count_launch();
        std::vector<double> hm(ns);
        if ((e = cudaMemcpyAsync(hm.data(), smatch, ns * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("reading the spot matches failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        // 5. a template keeps its surrogate taps when the spot checks on both sides of it in
        //    chirp-mass order (or its own) reach min_match; the rest fall back to exact taps
        std::vector<int32_t> source(n_tmpl, 0);
        std::vector<double> smatch_all(n_tmpl, std::nan(""));
        int64_t spot_fail = 0;
        int32_t si = 0;
        for (int32_t r = 0; r < P->R; ++r) {
            const auto &v = by[r];
            const auto &pos = spot_pos[r];
            std::vector<double> m(pos.size());
            for (size_t q = 0; q < pos.size(); ++q, ++si) {
                m[q] = hm[si];
                smatch_all[v[pos[q]]] = hm[si];
                if (!(hm[si] >= min_match)) ++spot_fail;
            }
            for (size_t q = 0; q < pos.size(); ++q) {
                const bool ok_here = m[q] >= min_match;
                source[v[pos[q]]] = ok_here ? 2 : 1;
                if (q + 1 < pos.size()) {
                    const bool ok = ok_here && m[q + 1] >= min_match;
                    for (int32_t p = pos[q] + 1; p < pos[q + 1]; ++p) source[v[p]] = ok ? 0 : 1;
                }
            }
        }
        std::vector<int32_t> fb, fb_ref, fb_k;
        std::vector<rfd_params> fb_params;
        for (int32_t j = 0; j < n_tmpl; ++j)
            if (source[j] == 1) {
                fb.push_back(j);
                fb_ref.push_back(ref_of_host[j]);
                fb_k.push_back(kT);
                fb_params.push_back(tmpl_host[j]);
            }
        const int32_t nf = (int32_t)fb.size();
        // 6. exact extraction (own lag) for the fallback set, scattered into place
        if (nf > 0) {
            DevBuf fbuf;
            const size_t bft = (size_t)nf * k_stride * sizeof(float2);
            if ((st = ensure(fbuf, up(bft) + up((size_t)nf * 4) * 2 + up((size_t)nf * 8)))) break;
            char *fbase = (char *)fbuf.p;
            float2 *f_taps = (float2 *)fbase; fbase += up(bft);
            int32_t *f_lag = (int32_t *)fbase; fbase += up((size_t)nf * 4);
            int32_t *f_idx = (int32_t *)fbase; fbase += up((size_t)nf * 4);
            double *f_sigma = (double *)fbase;
            std::vector<PNParams> fb_pn;
            if ((st = make_pn_vec(g, fb_params.data(), nf, &fb_pn))) {
                release(fbuf);
                break;
            }
            st = make_taps_impl(ctx, g, psd_dev, P->refs, fb_pn, fb_ref, fb_k, {}, {}, 1.0, k_stride, tukey_alpha,
                                f_taps, nullptr, f_lag, f_sigma, nullptr, s);
            if (st == RFD_OK) {
                if ((e = cudaMemcpyAsync(f_idx, fb.data(), nf * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
                    (void)cudaGetLastError();
                    set_error("cudaMemcpyAsync failed: %s", cudaGetErrorString(e));
                    st = RFD_ERR_CUDA;
                } else {
                    k_scatter_taps<<<(unsigned)nf, 128, 0, s>>>(f_taps, f_lag, f_sigma, f_idx, k_stride,
                                                               (float2 *)taps_dev, lag_dev, sigma_dev);
                    if ((e = cudaGetLastError()) != cudaSuccess) {
                        set_error("k_scatter_taps launch failed: %s", cudaGetErrorString(e));
                        st = RFD_ERR_CUDA;
                    } else {
                        count_launch();
                        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
                            (void)cudaGetLastError();
                            set_error("fallback extraction failed: %s", cudaGetErrorString(e));
                            st = RFD_ERR_CUDA;
                        }
                    }
                }
            }
            release(fbuf);
            if (st) break;
        }
        if ((e = cudaMemcpyAsync(source_dev, source.data(), (size_t)n_tmpl * 4, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (surrogate_match_dev &&
             (e = cudaMemcpyAsync(surrogate_match_dev, smatch_all.data(), (size_t)n_tmpl * 8, cudaMemcpyHostToDevice,
                                  s)) != cudaSuccess) ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("writing the tap sources failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        if (stats_host) {
            int64_t n_mlp = 0;
            for (int32_t j = 0; j < n_tmpl; ++j) n_mlp += source[j] != 1;
            stats_host[0] = n_mlp;
            stats_host[1] = nf;
            stats_host[2] = ns;
            stats_host[3] = spot_fail;
        }
    } while (0);
    release(scratch);
    if (st) return st;
    return check_status(P, s);
}

}  // extern "C"

// ------------------------------------------------------------------ checkpoint
// File: 8-byte magic "RFDMLP" 0x00 0x01, uint64 (little endian) length of a JSON header, the
// header (ASCII), then the sections it lists, each at its offset from the end of the header
// (64-byte aligned): FP32 master weights, Adam first and second moments, the per-network
// normalisation (double [R][kNorm]: mu[4], sd[4], out_scale), the lags, the optimiser state
// (Adam step, dynamic loss scale and its clean-step count), the references' autocorrelations
// C_r (which depend on the grid, the PSD and the references' bands) and the references' phase
// constants, which together identify what the networks were trained for.
#include <cstdio>
#include <cstring>
#include <string>

namespace rfd {
namespace {

constexpr char kCkptMagic[8] = {'R', 'F', 'D', 'M', 'L', 'P', 0, 1};

struct CkptSection {
    const char *name;
    const char *dtype;
    int64_t rows, cols;
    size_t bytes;
};

// The sections of a checkpoint of P, in file order.
std::vector<CkptSection> ckpt_sections(const rfd_mlp *P) {
    const int64_t R = P->R;
    return {{"weights", "f32", R, kP, (size_t)(R * kP * 4)},
            {"adam_m", "f32", R, kP, (size_t)(R * kP * 4)},
            {"adam_v", "f32", R, kP, (size_t)(R * kP * 4)},
            {"norm", "f64", R, kNorm, (size_t)(R * kNorm * 8)},
            {"lag", "i32", R, 1, (size_t)(R * 4)},
            {"optimizer", "raw", 1, (int64_t)sizeof(MlpState), sizeof(MlpState)},
            {"autocorr", "c128", R, kCw, (size_t)(R * kCw * 16)},
            {"references", "raw", R, (int64_t)sizeof(PNParams), (size_t)(R * sizeof(PNParams))}};
}

size_t align64(size_t x) { return (x + 63) / 64 * 64; }

// Value of a number-valued key of the header ("key": number), or false when absent.
bool header_number(const std::string &h, const char *key, double *out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = h.find(k);
    if (at == std::string::npos) return false;
    char *end = nullptr;
    *out = std::strtod(h.c_str() + at + k.size(), &end);
    return end != h.c_str() + at + k.size();
}

}  // namespace
}  // namespace rfd

extern "C" {

rfd_status rfd_mlp_save(rfd_mlp *P, const char *path, void *stream) {
    using namespace rfd;
    RFD_REQUIRE(P && path, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY(check_status(P, s));
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    const std::vector<CkptSection> secs = ckpt_sections(P);
    std::vector<std::vector<char>> data(secs.size());
    for (size_t i = 0; i < secs.size(); ++i) data[i].resize(secs[i].bytes);
    const int64_t R = P->R;
    RFD_TRY_CUDA(cudaMemcpy(data[0].data(), P->d_params.p, secs[0].bytes, cudaMemcpyDeviceToHost));
    RFD_TRY_CUDA(cudaMemcpy(data[1].data(), P->d_m.p, secs[1].bytes, cudaMemcpyDeviceToHost));
    RFD_TRY_CUDA(cudaMemcpy(data[2].data(), P->d_v.p, secs[2].bytes, cudaMemcpyDeviceToHost));
    std::memcpy(data[3].data(), P->norm.data(), secs[3].bytes);
    std::memcpy(data[4].data(), P->lag.data(), secs[4].bytes);
    MlpState st{};
    RFD_TRY_CUDA(cudaMemcpy(&st, P->d_state.p, sizeof(st), cudaMemcpyDeviceToHost));
    std::memcpy(data[5].data(), &st, sizeof(st));
    RFD_TRY_CUDA(cudaMemcpy(data[6].data(), P->d_C.p, secs[6].bytes, cudaMemcpyDeviceToHost));
    std::memcpy(data[7].data(), P->refs.data(), secs[7].bytes);
    char buf[512];
    std::string h = "{\"format\": \"librfd learned-tap networks\", \"version\": 1";
    std::snprintf(buf, sizeof(buf),
                  ", \"n_ref\": %lld, \"param_count\": %lld, \"taps\": %d, \"inputs\": %d"
                  ", \"grid\": {\"fs\": %.17g, \"n\": %lld, \"f_low\": %.17g, \"pn_flags\": %d}"
                  ", \"adam_step\": %d, \"loss_scale\": %.9g, \"clean_steps\": %d, \"sections\": [",
                  (long long)R, (long long)kP, kT, kIn, P->grid.fs, (long long)P->grid.n, P->grid.f_low,
                  P->grid.pn_flags, st.t, (double)st.loss_scale, st.good);
    h += buf;
    size_t off = 0;
    for (size_t i = 0; i < secs.size(); ++i) {
        std::snprintf(buf, sizeof(buf), "%s{\"name\": \"%s\", \"dtype\": \"%s\", \"shape\": [%lld, %lld], "
                      "\"offset\": %zu, \"bytes\": %zu}", i ? ", " : "", secs[i].name, secs[i].dtype,
                      (long long)secs[i].rows, (long long)secs[i].cols, off, secs[i].bytes);
        h += buf;
        off = align64(off + secs[i].bytes);
    }
    h += "]}\n";
    FILE *f = std::fopen(path, "wb");
    RFD_REQUIRE(f, RFD_ERR_ARG, "mlp_save: cannot open %s for writing", path);
    const uint64_t hl = h.size();
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&hl, 8, 1, f) == 1 &&
              std::fwrite(h.data(), 1, h.size(), f) == h.size();
    const std::vector<char> zeros(64, 0);
    off = 0;
    for (size_t i = 0; ok && i < secs.size(); ++i) {
        ok = std::fwrite(data[i].data(), 1, secs[i].bytes, f) == secs[i].bytes;
        const size_t pad = align64(off + secs[i].bytes) - (off + secs[i].bytes);
        ok = ok && (pad == 0 || std::fwrite(zeros.data(), 1, pad, f) == pad);
        off = align64(off + secs[i].bytes);
    }
    ok = (std::fclose(f) == 0) && ok;
    RFD_REQUIRE(ok, RFD_ERR_ARG, "mlp_save: writing %s failed", path);
    return RFD_OK;
}

rfd_status rfd_mlp_load(rfd_mlp *P, const char *path, void *stream) {
    using namespace rfd;
    RFD_REQUIRE(P && path, RFD_ERR_ARG, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    RFD_REQUIRE(f, RFD_ERR_ARG, "mlp_load: cannot open %s", path);
    char magic[8];
    uint64_t hl = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(&hl, 8, 1, f) == 1 && hl > 0 && hl < (1u << 20);
    std::string h;
    if (ok) {
        h.resize(hl);
        ok = std::fread(&h[0], 1, hl, f) == hl;
    }
    const std::vector<CkptSection> secs = ckpt_sections(P);
    std::vector<std::vector<char>> data(secs.size());
    size_t off = 0;
    for (size_t i = 0; ok && i < secs.size(); ++i) {
        data[i].resize(secs[i].bytes);
        ok = std::fread(data[i].data(), 1, secs[i].bytes, f) == secs[i].bytes;
        const size_t pad = align64(off + secs[i].bytes) - (off + secs[i].bytes);
        char skip[64];
        ok = ok && (pad == 0 || std::fread(skip, 1, pad, f) == pad);
        off = align64(off + secs[i].bytes);
    }
    std::fclose(f);
    RFD_REQUIRE(ok, RFD_ERR_ARG, "mlp_load: %s is not a complete librfd network checkpoint", path);
    double v = 0;
    RFD_REQUIRE(header_number(h, "n_ref", &v) && (int64_t)v == P->R, RFD_ERR_SHAPE,
                "mlp_load: the checkpoint holds %g networks, this object %d", v, P->R);
    RFD_REQUIRE(header_number(h, "param_count", &v) && (int64_t)v == kP, RFD_ERR_SHAPE,
                "mlp_load: parameter count %g, expected %lld", v, (long long)kP);
    double fs = 0, n = 0, fl = 0, pf = 0;
    RFD_REQUIRE(header_number(h, "fs", &fs) && header_number(h, "n", &n) && header_number(h, "f_low", &fl) &&
                    header_number(h, "pn_flags", &pf) && fs == P->grid.fs && (int64_t)n == P->grid.n &&
                    fl == P->grid.f_low && (int32_t)pf == P->grid.pn_flags,
                RFD_ERR_ARG, "mlp_load: the checkpoint's grid differs from this object's");
    RFD_TRY_CUDA(cudaSetDevice(P->ctx->device));
    RFD_TRY_CUDA(cudaDeviceSynchronize());
    // the references' autocorrelations must be the same to the bit: same PSD, grid and references
    std::vector<char> C(secs[6].bytes);
    RFD_TRY_CUDA(cudaMemcpy(C.data(), P->d_C.p, C.size(), cudaMemcpyDeviceToHost));
    RFD_REQUIRE(std::memcmp(C.data(), data[6].data(), C.size()) == 0, RFD_ERR_ARG,
                "mlp_load: the checkpoint was trained with another PSD or band");
    RFD_REQUIRE(std::memcmp(P->refs.data(), data[7].data(), secs[7].bytes) == 0, RFD_ERR_ARG,
                "mlp_load: the checkpoint was trained for other references");
    const int64_t R = P->R;
    const float *w = (const float *)data[0].data();
    for (int64_t i = 0; i < R * kP; ++i)
        RFD_REQUIRE(std::isfinite(w[i]), RFD_ERR_ARG, "mlp_load: weight %lld is not finite", (long long)i);
    MlpState st{};
    std::memcpy(&st, data[5].data(), sizeof(st));
    st.inf = 0;
    st.err = 0;
    std::memcpy(P->norm.data(), data[3].data(), secs[3].bytes);
    std::memcpy(P->lag.data(), data[4].data(), secs[4].bytes);
    RFD_TRY_CUDA(cudaMemcpy(P->d_params.p, data[0].data(), secs[0].bytes, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_m.p, data[1].data(), secs[1].bytes, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_v.p, data[2].data(), secs[2].bytes, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_norm.p, P->norm.data(), secs[3].bytes, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_lag.p, P->lag.data(), secs[4].bytes, cudaMemcpyHostToDevice));
    RFD_TRY_CUDA(cudaMemcpy(P->d_state.p, &st, sizeof(st), cudaMemcpyHostToDevice));
    // the FP16 operand copies follow from the masters by the same rounding every step uses
    const int64_t nparam = R * kP;
    k_mlp_sync_half<<<(unsigned)((nparam + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        (const float *)P->d_params.p, (__half *)P->d_wh.p, nparam);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return RFD_OK;
}

}  // extern "C"
