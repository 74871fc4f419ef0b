// Internal declarations of librfd (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <map>
#include <vector>

#include "rfd.h"

namespace rfd {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTSun = 4.925490947641267e-6;   // G Msun / c^3, seconds

void set_error(const char *fmt, ...);

#define RFD_TRY_CUDA(expr)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (void)cudaGetLastError(); /* a failed call leaves no error for the next check */ \
            ::rfd::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                      \
            return RFD_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)

#define RFD_REQUIRE(cond, code, ...)                                                         \
    do {                                                                                     \
        if (!(cond)) {                                                                       \
            ::rfd::set_error(__VA_ARGS__);                                                   \
            return code;                                                                     \
        }                                                                                    \
    } while (0)

#define RFD_TRY(expr)                                                                        \
    do {                                                                                     \
        rfd_status s_ = (expr);                                                              \
        if (s_ != RFD_OK) return s_;                                                         \
    } while (0)

// Every kernel launch site is followed by RFD_LAUNCH_CHECK(), which also counts the launch
// (rfd_kernel_launches() reports the running total).
void count_launch();
#define RFD_LAUNCH_CHECK()                                                                   \
    do {                                                                                     \
        ::rfd::count_launch();                                                               \
        RFD_TRY_CUDA(cudaGetLastError());                                                    \
    } while (0)

// ------------------------------------------------------------------ grid
struct Grid {
    double fs, f_low, df;
    int64_t n, nf;    // samples, one-sided bins n/2+1
    int64_t k_lo;     // first in-band bin
    int32_t pn_flags;
    int32_t log2n;
};
rfd_status check_grid(const rfd_grid *g, Grid *out);

// Per-template constants of the TaylorF2 phase, evaluated on the host in FP64.
struct PNParams {
    double mt;        // total mass in seconds
    double eta;       // symmetric mass ratio
    double beta;      // spin-orbit coefficient (0 unless RFD_PN_SO)
    double lam;       // tidal deformability (0 unless RFD_PN_TIDAL)
    int64_t k_hi;     // last non-zero bin: min(n/2 - 1, floor(f_ISCO / df))
    int64_t pad;
};
rfd_status make_pn(const Grid &g, const rfd_params *p, PNParams *out);

// FP64 TaylorF2 phase Psi(f) (t_c = phi_c = 0).
// Output window of a filtering call: its first position *u_begin (device memory, so that a
// captured graph can be replayed for another window), taken modulo n and rounded down to a
// multiple of 512; 0 without a window.  Positions inside it wrap around the circular segment.
__device__ __forceinline__ int64_t window_base(const int64_t *u_begin, int64_t n) {
    if (!u_begin) return 0;
    int64_t b = *u_begin % n;
    if (b < 0) b += n;
    return b & ~(int64_t)511;
}
__device__ __forceinline__ int64_t wrap_pos(int64_t base, int64_t off, int64_t n) {
    const int64_t u = base + off;    // base < n, off < n
    return u >= n ? u - n : u;
}

__device__ __forceinline__ double pn_phase(double f, const PNParams &p, int flags) {
    const double v = cbrt(kPi * p.mt * f);
    const double v2 = v * v, v3 = v2 * v, v5 = v3 * v2;
    double br = 1.0 + (3715.0 / 756.0 + 55.0 * p.eta / 9.0) * v2 + (4.0 * p.beta - 16.0 * kPi) * v3;
    if (flags & RFD_PN_TIDAL) br -= 19.5 * p.lam * (v5 * v5);
    return -0.25 * kPi + 3.0 / (128.0 * p.eta * v5) * br;
}

// ------------------------------------------------------------------ workspaces
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
// Grow-only device buffer.  Growing synchronises the device before freeing the old block.
rfd_status ensure(DevBuf &b, size_t bytes);
// While a captured graph is alive (graphs_pin .. graphs_unpin), ensure() and release() keep
// replaced blocks allocated, so the graph's pointers stay valid.
void graphs_pin();
void graphs_unpin();
void release(DevBuf &b);

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// ------------------------------------------------------------------ FFT (fft.cu)
// Unnormalised complex FFT of `batch` rows of length n (power of two) by Stockham passes.
// in: rows at stride in_stride; out: rows at stride out_stride; tmp: batch * n elements.
// in, out, tmp must not overlap.  inverse: exp(+2 pi i k m / n), forward: exp(-...).
template <typename T>
rfd_status fft_c2c(rfd_ctx *ctx, int64_t n, int64_t batch, const typename Cplx<T>::type *in,
                   int64_t in_stride, typename Cplx<T>::type *out, int64_t out_stride,
                   typename Cplx<T>::type *tmp, bool inverse, cudaStream_t s);
// Stage twiddles of a length-2^logL Stockham transform (the passes in order: a radix-2, -4 or
// -8 pass first when logL is not a multiple of 4, then radix 16; pass p with radix R after
// ns = product of the earlier radices holds exp(+2 pi i r k / (ns R)) at
// base_p + (r - 1) ns + k), FP32, cached in the context.
rfd_status fft_stage_twiddles32(rfd_ctx *ctx, int logL, const float2 **out, cudaStream_t s);
// FINDCHIRP (Eq. 1) for J templates h (complex64 [J][nf]) in two fused passes (fft.cu): the
// spectrum G[k] conj(h[k]) formed inside the first FFT pass from GW[k] = (Re G, Im G, Wt, 0),
// G = 4 df d / S on the data band and Wt = 4 df / S (length n/2), z = q / sigma with the trigger
// epilogue inside the last.  tmp: J n complex64; part: J x 2048 doubles; sig2: J doubles.
rfd_status findchirp_fused(rfd_ctx *ctx, int64_t n, int64_t J, const float4 *GW, const float2 *h,
                           int64_t nf, int32_t j0, float thr, int32_t W, float2 *tmp, double *part,
                           double *sig2, rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s);

// ------------------------------------------------------------------ taps (taps.cu)
// lag_in empty: the lag is searched (Sec. V placement); otherwise it is taken from lag_in.
// K empty: K chosen from `buckets`.  fit_eps > 0: the taps are the chi^2 fit of Sec. V.A with
// ridge fit_eps C_r[0] (at the same lag), and `match` is its closed form.
rfd_status make_taps_impl(rfd_ctx *ctx, const Grid &g, const double *psd, const std::vector<PNParams> &refs,
                          const std::vector<PNParams> &tmpl, const std::vector<int32_t> &ref_of,
                          const std::vector<int32_t> &K, const std::vector<int32_t> &buckets,
                          const std::vector<int32_t> &lag_in, double energy_frac, int32_t k_stride, double alpha,
                          float2 *taps, int32_t *k_out, int32_t *lag, double *sigma, double *match, cudaStream_t s,
                          double fit_eps = 0.0);
rfd_status make_taps_fit_dynamic(rfd_ctx *ctx, const Grid &g, const double *psd, const std::vector<PNParams> &refs,
                                 const std::vector<PNParams> &tmpl, const std::vector<int32_t> &ref_of,
                                 const std::vector<int32_t> &buckets, double target, double eps, int32_t k_stride,
                                 double alpha, float2 *taps, int32_t *k_out, int32_t *lag, double *sigma,
                                 double *match, cudaStream_t s);
rfd_status ref_autocorr_impl(rfd_ctx *ctx, const Grid &g, const double *psd, const PNParams *refs_dev, int64_t R,
                             int32_t kmax, double2 *C, cudaStream_t s);
rfd_status make_pn_vec(const Grid &g, const rfd_params *p, int32_t n, std::vector<PNParams> *out);

// ------------------------------------------------------------------ triggers (triggers.cu)
struct TrigReadback {
    int64_t count;    // candidates produced (bit 62: a filtering kernel timed out)
    int64_t total;    // triggers
    int32_t bad;      // candidates naming a template out of range
    int32_t pad;
};
rfd_status find_triggers_enqueue(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand,
                                 const int64_t *cand_count, int64_t cap, rfd_trigger *trig,
                                 int64_t trig_cap, TrigReadback *host, cudaStream_t s);
rfd_status find_triggers_check(const TrigReadback &h, int32_t n_tmpl, int64_t cap, int64_t trig_cap,
                               int64_t *n_trig_host);
rfd_status find_triggers_impl(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand,
                              const int64_t *cand_count, int64_t cap, rfd_trigger *trig,
                              int64_t trig_cap, int64_t *n_trig_host, cudaStream_t s);

}  // namespace rfd

// ------------------------------------------------------------------ opaque handles
struct rfd_ctx {
    int device = 0;
    int num_sms = 0;
    std::map<int64_t, void *> tw32, tw64;   // twiddle tables exp(+2 pi i m / n), m < n
    std::map<int64_t, void *> stw32, stw64; // per-pass (stage) twiddles of short transforms, by log2 length
    rfd::DevBuf ws[16];                      // scratch slots, see the users for their roles
};

// Tile of the ratio-filter contraction: templates [first, first + count) of the plan's
// permuted template order, all assigned to reference `ref`, padded to k_tile taps.
struct RfdTile {
    int32_t ref;
    int32_t first;
    int32_t count;
    int32_t k_tile;
};

// Tile of the tensor-core contraction (see rf_tc.cu): up to nt templates (64, or 32 when the
// tile's K exceeds 256) of one reference; nk16 16-tap MMA steps, kpad = 16 nk16 taps, nch
// 64-tap chunks; its pre-swizzled B-operand image is taps_bytes bytes at taps_off.
struct TcTile {
    int32_t ref, first, count, k_tile;
    int32_t nt, nch, nk16, kpad;
    int64_t taps_off;
    int32_t taps_bytes, pad;
};

// Tile of the block-FFT ratio filter (rf_fft.cu): up to 64 templates of one reference.
struct FftTile {
    int32_t ref, first, count, pad;
};

struct rfd_plan {
    rfd_ctx *ctx = nullptr;
    rfd::Grid grid{};
    int32_t n_ref = 0, n_tmpl = 0, precision = 0, window = 1, halo = 0;
    float threshold = 0.f;
    int64_t ld = 0;                  // q_ref row length
    int64_t out_len = 0;             // outputs per filtering call (n, or a window of it)
    int32_t k_max = 0;
    int32_t tile_j = 0;              // templates per tile
    std::vector<int32_t> ref_of, k_of;
    std::vector<int32_t> perm;       // permuted template order (tile-major)
    std::vector<RfdTile> tiles;
    // device state
    rfd::DevBuf d_tiles;             // RfdTile [n_tiles]
    rfd::DevBuf d_perm;              // int32 [n_slots]: template index of each slot (-1 pad)
    rfd::DevBuf d_taps;              // packed taps (layout depends on precision)
    rfd::DevBuf d_off;               // int32 [n_slots]: (s_j + K_j - 1) mod n
    rfd::DevBuf d_scale;             // float [n_slots]: 1 / (sigma_eff 2^e_j)
    rfd::DevBuf d_kslot;             // int32 [n_slots]: K_j
    int64_t n_slots = 0;
    bool taps_set = false;
    // tensor-core path
    std::vector<TcTile> tc_tiles;
    // long-tap kernel (rf_tc_long.cu): tiles of 64 templates, items of 256 outputs
    std::vector<TcTile> tl_tiles;
    rfd::DevBuf d_tl_tiles, d_tl_ranges, d_tl_taps;
    int32_t tl_grid = 0;
    uint32_t tl_ystride = 0, tl_qwin = 0;
    rfd::DevBuf d_ranges;            // int64 [tc_grid + 1] item ranges per CTA
    uint32_t tc_taps_cap = 0, tc_win = 0;
    int32_t tc_grid = 0;
    double executed_flops = 0.0;     // tensor (or FMA) flops one ratio_filter_batch executes
    int32_t debug_flags = 0;         // RFD_DEBUG_* (testing only)
    // block-FFT path (rf_fft.cu): templates with fft_k < K <= 1024
    std::vector<FftTile> fft_tiles;
    std::vector<int32_t> fft_refs;   // references with block-FFT templates
    rfd::DevBuf d_fft_tiles, d_fft_ranges, d_fft_refs, d_fft_P, d_fft_X;
    const float2 *fft_stw = nullptr; // stage twiddles of length 2048 (context-owned)
    int32_t fft_grid = 0, fft_L = 0, fft_nb = 0, fft_nbg = 0;
    int64_t fft_slot0 = 0, fft_nslots = 0;
    double fft_flops = 0.0;          // nominal FP32 flops of the block-FFT path per call
};
