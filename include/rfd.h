/*
 * rfd.h -- C ABI of the GB300 ratio-filter dechirping library (librfd.so).
 *
 * Method: A. H. Nitz, K. Kacanja, K. Soni, "Beyond FINDCHIRP: ... Ratio-Filter
 * Dechirping" (arXiv 2601.18835).  The data are matched-filtered once per reference
 * template (Eq. 1: point-wise d conj(h_ref) / S, then an inverse FFT), giving a complex
 * series q_ref.  Each target template's SNR series comes from a short complex FIR applied
 * to q_ref (Eq. 3); the FIR is the windowed, truncated inverse transform of conj(h/h_ref)
 * (Eq. 2, Sec. V).  The SNR series is reduced to |z|^2 threshold crossings and
 * per-window maxima (Table II: peak find, trigger accumulation).
 *
 * Conventions for every call:
 *   - Plain C99 types only.  Pointers named *_dev are device pointers, *_host host
 *     pointers.  All data buffers are allocated and owned by the caller; the library owns
 *     only contexts, plans and their workspaces, released by the matching *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Every call
 *     is stream-ordered and asynchronous unless its comment says it synchronises.
 *   - Errors are return codes; nothing throws.  Arguments are checked before any launch
 *     (RFD_ERR_ARG / RFD_ERR_SHAPE).  rfd_last_error() gives a message for the calling
 *     thread's last failing call.
 *   - Complex arrays are interleaved (re, im) float32 ("complex64") unless stated.
 *   - Frequency grid: f_k = k df, df = fs / n, k = 0 .. n/2 (one-sided, n/2+1 bins).
 *     n is a power of two, 2^10 <= n <= 2^22.  A template is non-zero for
 *     ceil(f_low/df) <= k <= min(n/2 - 1, floor(f_ISCO/df)).
 *   - Time index m = 0 .. n-1; every convolution is circular over the segment.
 */
#ifndef RFD_H
#define RFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RFD_VERSION 5

typedef enum {
    RFD_OK = 0,
    RFD_ERR_ARG = -1,          /* null pointer, bad enum, non-finite parameter */
    RFD_ERR_SHAPE = -2,        /* sizes inconsistent or out of the supported range */
    RFD_ERR_UNSUPPORTED = -3,  /* a valid request the library does not implement */
    RFD_ERR_CUDA = -4,         /* a CUDA runtime call failed (message has the CUDA error) */
    RFD_ERR_NOMEM = -5,        /* workspace allocation failed */
    RFD_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
    RFD_ERR_OVERFLOW = -7      /* an output list was too small; the required size is returned */
} rfd_status;

/* Post-Newtonian phase terms beyond 0/1/1.5PN. */
enum { RFD_PN_SO = 1,          /* aligned-spin 1.5PN spin-orbit term (beta) */
       RFD_PN_TIDAL = 2 };     /* 5PN tidal term -(39/2) Lambda v^10 */

/* Arithmetic of the ratio-filter contraction (and the layout of the q_ref buffer). */
enum { RFD_PREC_FP32 = 0,      /* complex64 q_ref, FP32 CUDA-core FIR */
       RFD_PREC_FP16X3 = 1,    /* fp16 hi+lo planes, 3-product tensor-core contraction */
       RFD_PREC_BF16X3 = 2 };  /* bf16 hi+lo planes, 3-product tensor-core contraction */

typedef struct rfd_ctx rfd_ctx;    /* opaque: device, FFT tables, workspaces */
typedef struct rfd_plan rfd_plan;  /* opaque: one bank's filtering schedule and packed taps */

/* Sampling grid of one data segment. */
typedef struct {
    double fs;          /* sample rate, Hz */
    int64_t n;          /* samples per segment (power of two) */
    double f_low;       /* lower frequency cutoff, Hz */
    int32_t pn_flags;   /* RFD_PN_* bits applied to every template and reference */
    int32_t reserved;   /* must be 0 */
} rfd_grid;

/* Intrinsic parameters of one TaylorF2 template (masses in solar masses). */
typedef struct {
    double m1, m2, chi1, chi2, lambda_tilde;
} rfd_params;

/* One candidate from the fused epilogue: the maximum over a run of samples that share a
 * (template, window) pair.  key = (float bits of |z|^2) << 32 | (0xFFFFFFFF - t), so the
 * larger key is the larger |z|^2 and, on equal |z|^2, the smaller t.  24 bytes. */
typedef struct {
    uint64_t key;
    uint32_t j;         /* template index */
    uint32_t w;         /* window index floor(t / window) */
    float zr, zi;       /* complex SNR at that sample */
} rfd_candidate;

/* One trigger: the per-window maximum of |z|^2 above threshold.  20 bytes. */
typedef struct {
    int32_t j;          /* template index */
    int32_t t;          /* sample index of the maximum, 0 .. n-1 */
    float snr2;         /* |z|^2 at t */
    float zr, zi;       /* complex SNR at t */
} rfd_trigger;

/* ------------------------------------------------------------------ housekeeping */
int32_t rfd_version(void);
const char *rfd_status_string(rfd_status s);
/* Message of the calling thread's last failing call ("" if none).  Owned by the library,
 * valid until the thread's next failing call. */
const char *rfd_last_error(void);

/* Number of kernels this library has launched in the process so far (all contexts). */
int64_t rfd_kernel_launches(void);

/* Create a context on CUDA device `device` (made current for the calling thread).
 * The context is not thread-safe: use one per host thread. */
rfd_status rfd_ctx_create(int32_t device, rfd_ctx **out);
void rfd_ctx_destroy(rfd_ctx *ctx);
/* Frees the context's scratch workspaces (they are re-created on demand).  Synchronises the
 * device. */
void rfd_ctx_trim(rfd_ctx *ctx);

/* Elements per reference row of a q_ref buffer: n + halo rounded up to a multiple of 64.
 * A q_ref buffer holds n_ref * 8 * rfd_qref_ld(n, halo) bytes in every precision. */
int64_t rfd_qref_ld(int64_t n, int32_t halo);

/* ------------------------------------------------------------------ templates
 * TaylorF2 templates (the h(f) of Eq. 1) evaluated with FP64 phase:
 *   h(f_k) = f_k^(-7/6) exp(-i Psi(f_k)),
 *   Psi = -pi/4 + 3/(128 eta v^5) [1 + (3715/756 + 55 eta/9) v^2 + (4 beta - 16 pi) v^3
 *                                  - (39/2) Lambda v^10],  v = (pi M f)^(1/3),
 * zero outside the template's band.  h_dev: complex64 [n_tmpl][n/2+1], caller-allocated. */
rfd_status rfd_gen_templates(rfd_ctx *ctx, const rfd_grid *grid, const rfd_params *params_host,
                             int32_t n_tmpl, void *h_dev, void *stream);

/* ------------------------------------------------------------------ make_taps
 * Ratio-filter taps for each template against its reference (Eq. 2, Eq. 3, Sec. V;
 * normalisation Eqs. 5-6).  All arithmetic before the final cast is FP64 on the device:
 *   G[k]   = exp(+i (Psi_j - Psi_r)) in the reference band up to the template's cutoff,
 *            0 above the template's cutoff, and a linear magnitude / shortest-arc phase
 *            fill from G[k_hi] round the out-of-band arc to G[k_lo];
 *   g      = (1/n) IDFT_n(G)                              (hand-written FP64 Stockham FFT);
 *   K_j    = k_host[j], or, when k_host is NULL, the smallest entry of buckets_host whose
 *            best circular window of that many samples holds energy_frac of sum |g|^2 (the
 *            largest bucket when none does) -- the tap count from the ratio's bandwidth;
 *   s_j    = argmax over s in [-n/2, n/2) of E[s] = sum_k w[k]^2 |g[(s+k) mod n]|^2,
 *            w = symmetric Tukey(K_j, tukey_alpha); values within 1e-9 relative of the
 *            maximum tie, and ties go to the s closest to -K_j/2, then to the smaller s (found
 *            exactly, evaluating E only where the unweighted window energy can reach it);
 *   rho[k] = w[k] g[(s_j + k) mod n], k < K_j;
 *   sigma_eff^2 = sum_{a,b} rho[a] conj(rho[b]) C_r[b - a],
 *            C_r[l] = 4 df sum_{k in band_r} |h_r,k|^2 / S_k exp(+2 pi i k l / n);
 *   match  = |<h_j, h_eff>| / (|h_j| |h_eff|), h_eff = h_r conj(A), A = DFT of the placed taps.
 * Inputs: psd_dev float64 [n/2+1]; refs_host [n_ref]; tmpl_host [n_tmpl];
 *   ref_of_tmpl_host int32 [n_tmpl] in [0, n_ref); k_host int32 [n_tmpl] with
 *   1 <= K <= k_stride, or NULL with buckets_host int32 [n_buckets] increasing, each
 *   <= k_stride, and energy_frac in (0, 1].
 * Outputs (device, caller-allocated): taps_dev complex64 [n_tmpl][k_stride] (entries past K
 *   are zeroed), k_dev int32 [n_tmpl] (K_j; may be NULL when k_host is given),
 *   lag_dev int32 [n_tmpl] (s_j), sigma_dev float64 [n_tmpl], match_dev float64 [n_tmpl] or
 *   NULL to skip the match (it costs one more FFT per template).
 * Synchronises the stream before returning (its FP64 workspace is sized per batch). */
rfd_status rfd_make_taps(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                         const rfd_params *refs_host, int32_t n_ref,
                         const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host,
                         int32_t n_tmpl, const int32_t *k_host, const int32_t *buckets_host,
                         int32_t n_buckets, double energy_frac, int32_t k_stride,
                         double tukey_alpha, void *taps_dev, int32_t *k_dev, int32_t *lag_dev,
                         double *sigma_dev, double *match_dev, void *stream);

/* Chi^2-fitted taps (Sec. V.A, Eq. 4): instead of windowing, the taps minimise
 *   sum_k w_k |G_k - A_k|^2 + lam |rho|^2,  A_k = sum_n rho_n exp(-2 pi i k (s_j + n) / n),
 * G = conj(h_j / h_ref) (Eq. 2 conjugated), w_k = 4 df |h_ref,k|^2 / S_k on the reference band
 * (the data reach the ratio filter band-passed by the reference), lam = ridge C_r[0]; i.e.
 *   sum_m (C_r[n - m] + lam delta_nm) rho_m = b_n,  b_n = sum_k w_k G_k exp(+2 pi i k (s_j + n)/N),
 * solved per template by the Levinson recursion in FP64.  The lag s_j is placed as in
 * rfd_make_taps (window-energy rule with the Tukey window of K taps).  match_dev (required)
 * receives the fitted taps' match to the template, |rho^H b| / (sigma_eff sigma_j).
 * K: k_host int32 [n_tmpl] per template, or k_host = NULL and buckets_host [n_buckets]: each
 * template gets the smallest bucket whose fitted match reaches match_target (the largest bucket
 * otherwise), written to k_dev (may be NULL with k_host).  ridge in (0, 1); k_stride <= 512.
 * Outputs as for rfd_make_taps.  Synchronises the stream before returning. */
rfd_status rfd_make_taps_fit(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                             const rfd_params *refs_host, int32_t n_ref, const rfd_params *tmpl_host,
                             const int32_t *ref_of_tmpl_host, int32_t n_tmpl, const int32_t *k_host,
                             const int32_t *buckets_host, int32_t n_buckets, double match_target,
                             double ridge, int32_t k_stride, double tukey_alpha, void *taps_dev,
                             int32_t *k_dev, int32_t *lag_dev, double *sigma_dev, double *match_dev,
                             void *stream);

/* Taps at a given lag: as rfd_make_taps with fixed K, except that the placement s_j is
 * lag_host[j] (in [-n/2, n/2)) instead of the window-energy maximiser, so
 * rho_j[k] = w[k] g_j[(s_j + k) mod n].  These are the targets the learned-tap networks are
 * trained on (each network's taps sit at one lag per reference).  sigma_dev / match_dev as
 * for rfd_make_taps (match_dev may be NULL).  Synchronises the stream before returning. */
rfd_status rfd_make_taps_at_lag(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                                const rfd_params *refs_host, int32_t n_ref,
                                const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host,
                                int32_t n_tmpl, const int32_t *k_host, const int32_t *lag_host,
                                int32_t k_stride, double tukey_alpha, void *taps_dev,
                                double *sigma_dev, double *match_dev, void *stream);

/* ------------------------------------------------------------------ tap banks on disk
 * Tap extraction (Sec. V) is the set-up's dominant cost, and its outputs depend only on its
 * inputs, so a bank's taps can be stored once and read back by later runs.
 *
 * rfd_taps_key writes to key_out (32 bytes) the SHA-256 digest (FIPS 180-4) of this
 * serialisation of rfd_make_taps' inputs, native little-endian (other hosts get
 * RFD_ERR_UNSUPPORTED), no padding between fields:
 *   the 12 bytes "librfd-taps" and its NUL; int32 RFD_VERSION; int32 mode (0: k_host given,
 *   1: bucket list); grid fs (double), n (int64), f_low (double), pn_flags (int32); int32
 *   n_ref, n_tmpl, k_stride; double tukey_alpha; double energy_frac (0 in mode 0); int32
 *   n_buckets (0 in mode 0); refs_host [n_ref] and tmpl_host [n_tmpl] as rfd_params (five
 *   doubles each); ref_of_tmpl_host int32 [n_tmpl]; k_host int32 [n_tmpl] (mode 0) or
 *   buckets_host int32 [n_buckets] (mode 1); psd_host double [n/2+1].
 * Host only; arguments as for rfd_make_taps except that the PSD is a host array. */
rfd_status rfd_taps_key(const rfd_grid *grid, const double *psd_host, const rfd_params *refs_host,
                        int32_t n_ref, const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host,
                        int32_t n_tmpl, const int32_t *k_host, const int32_t *buckets_host,
                        int32_t n_buckets, double energy_frac, int32_t k_stride, double tukey_alpha,
                        uint8_t *key_out);
/* rfd_make_taps through a cache directory.  The bank's key (rfd_taps_key, with the PSD read
 * back from psd_dev) names the file <cache_dir>/<key as 64 hex digits>.rfdtaps.  When that
 * file holds this key, n_tmpl and k_stride (and a match section, when match_dev is given), its
 * taps, K, lags, sigma_eff and match are copied to the outputs and *hit_host = 1.  Otherwise
 * rfd_make_taps runs with the same arguments, its outputs are written to that file (under a
 * temporary name, then renamed, so a reader never sees a partial file; cache_dir is created
 * if missing, one level) and *hit_host = 0.  A file that is truncated, holds another key or
 * fails the checks on its contents (1 <= K <= k_stride, lag in [-n/2, n/2), finite
 * sigma_eff >= 0) is recomputed and replaced.  The file: the 8-byte magic "RFDTAPS" 0x01, a
 * little-endian uint64 header length, a JSON header (key, n_tmpl, k_stride, has_match, and
 * per section its name, dtype, shape, offset and bytes), then the sections, 64-byte aligned
 * from the end of the header: taps complex64 [n_tmpl][k_stride], K int32 [n_tmpl], lag int32
 * [n_tmpl], sigma_eff float64 [n_tmpl] and, when present, match float64 [n_tmpl].
 * Outputs as for rfd_make_taps (k_dev and match_dev may be NULL).  When the taps were
 * extracted but the file cannot be written, the outputs are valid and RFD_ERR_ARG reports the
 * write.  Synchronises the stream. */
rfd_status rfd_make_taps_cached(const char *cache_dir, rfd_ctx *ctx, const rfd_grid *grid,
                                const double *psd_dev, const rfd_params *refs_host, int32_t n_ref,
                                const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host,
                                int32_t n_tmpl, const int32_t *k_host, const int32_t *buckets_host,
                                int32_t n_buckets, double energy_frac, int32_t k_stride,
                                double tukey_alpha, void *taps_dev, int32_t *k_dev, int32_t *lag_dev,
                                double *sigma_dev, double *match_dev, int32_t *hit_host,
                                void *stream);

/* ------------------------------------------------------------------ filter_reference
 * The reference SNR series of Eq. 3, (s|h)_ref, one per reference (Eq. 1 discretised):
 *   c_r[k] = 4 df d[k] conj(h_r[k]) / S[k] for k <= n/2 (h_r is zero outside its band),
 *            0 for k > n/2;
 *   q_r[m] = sum_k c_r[k] exp(+2 pi i k m / n)   (hand-written FP32 Stockham inverse FFT),
 * stored with a wrap halo q_r[n + i] = q_r[i], i < halo, so every FIR window
 * [u, u + K) with u < n is contiguous (halo >= K_max - 1; the tensor-core path reads K
 * rounded up to 16).
 * Inputs: dtilde_dev complex64 [n/2+1]; psd_dev float64 [n/2+1]; href_dev complex64
 * [n_ref][n/2+1], the reference templates as written by rfd_gen_templates (set-up work: the
 * references do not change from segment to segment).
 * Output qref_dev, row length ld = rfd_qref_ld(n, halo):
 *   RFD_PREC_FP32:   complex64 q[r * ld + m];
 *   RFD_PREC_FP16X3 / BF16X3: four 2-byte planes per reference, plane p of reference r at
 *     element offset (4 r + p) ld, p = 0 re_hi, 1 im_hi, 2 re_lo, 3 im_lo, with
 *     hi = round(x 2^e_r), lo = round(x 2^e_r - hi).
 * qscale_dev int32 [n_ref] receives e_r (0 for FP32); e_r puts the rms of the scaled series
 *   near 2^8, lowered where needed so that the largest component of the scaled series is at
 *   most 2^14 (a very loud sample cannot overflow the FP16 hi part).  Deterministic: the
 *   floating-point reductions run in a fixed order (the largest component is an integer
 *   maximum over float bits, exact in any order). */
rfd_status rfd_filter_reference(rfd_ctx *ctx, const rfd_grid *grid, const void *dtilde_dev,
                                const double *psd_dev, const void *href_dev, int32_t n_ref,
                                int32_t halo, int32_t precision, void *qref_dev,
                                int32_t *qscale_dev, void *stream);

/* ------------------------------------------------------------------ plans
 * A plan fixes one bank's schedule: templates grouped by reference into tiles of the
 * contraction Z[J_r x T] = P[J_r x K] Q[K x T] (Eq. 3 for all templates that share a
 * reference), the arithmetic, the trigger window and the threshold.
 * ref_of_tmpl_host int32 [n_tmpl]; k_host int32 [n_tmpl] (taps per template, as given to
 * rfd_make_taps); window >= 1 samples; threshold on |z|^2 (strict >); halo as for
 * rfd_filter_reference (>= max K - 1).  Copies everything it needs. */
rfd_status rfd_plan_create(rfd_ctx *ctx, const rfd_grid *grid, int32_t n_ref, int32_t n_tmpl,
                           const int32_t *ref_of_tmpl_host, const int32_t *k_host,
                           int32_t precision, int32_t window, float threshold, int32_t halo,
                           rfd_plan **out);
void rfd_plan_destroy(rfd_plan *plan);

/* Tile choices of the tensor-core path (what the autotuner varies). */
typedef struct {
    int32_t tile_nt[3];   /* templates per tile (multiple of 16) for K rounded to 16 in (0,128],
                             (128,256], (256,512]: at most 128, 64, 32 (the taps image of a tile,
                             3 x templates x K x hi/lo, stays within 192 KB of shared memory) */
    int32_t mix_k;        /* 1: a tile may hold templates whose K differ (padded to the largest);
                             0: tiles also split where the number of 16-tap steps changes */
    int32_t grid_ctas;    /* persistent CTAs of the tensor-core kernel, 0 = one per SM */
    int32_t long_k;       /* templates with K > long_k go to the long-tap kernel (64 templates
                             on the MMA's M side, 256 output positions on its N side, taps
                             streamed, so every MMA is full width for any K <= 512): 0 = every
                             template, 512 = none (tile_nt[1], tile_nt[2] then apply) */
    int32_t fft_k;        /* templates with fft_k < K <= 1024 go to the block-FFT kernel instead
                             (overlap-save blocks of 2048 samples, FP32 transforms in shared
                             memory, the paper's own realisation of the FIR): 0 = every template
                             with K <= 1024, 4096 = none */
    int32_t out_len;      /* outputs per filtering call: 0 = the whole segment (n); otherwise a
                             multiple of 512 (n a multiple of 512 too): rfd_ratio_filter_window
                             then filters out_len positions from a start held in device memory
                             (streaming, Sec. VII.A) */
    int32_t fft_rem;      /* per reference, the templates bound for the long-tap kernel fill
                             tiles of 64; when they leave a last tile of at most fft_rem
                             templates (a tile whose empty rows the MMAs still compute), those
                             templates (the ones with the largest K) go to the block-FFT kernel
                             instead (needs K <= 1024): 0 = never, at most 63 */
    int32_t debug_flags;  /* testing only, 0 otherwise.  RFD_DEBUG_STALL_TAPS: the tensor-core
                             kernels never copy the taps and give up their waits after a few
                             thousand polls, so that rfd_find_triggers reports RFD_ERR_TIMEOUT
                             (the test of the bounded-wait abort path) */
} rfd_plan_options;
#define RFD_DEBUG_STALL_TAPS 1
/* Fills the defaults: tile_nt = {128, 64, 32}, mix_k = 1, grid_ctas = 0, long_k = 64,
 * fft_k = 4096, out_len = 0, fft_rem = 0, debug_flags = 0. */
void rfd_plan_options_default(rfd_plan_options *options);
/* rfd_plan_create with explicit tile choices (NULL = defaults). */
rfd_status rfd_plan_create_ex(rfd_ctx *ctx, const rfd_grid *grid, int32_t n_ref, int32_t n_tmpl,
                              const int32_t *ref_of_tmpl_host, const int32_t *k_host,
                              int32_t precision, int32_t window, float threshold, int32_t halo,
                              const rfd_plan_options *options, rfd_plan **out);

/* Packs the taps from rfd_make_taps into the plan's own layout (reversed, scaled, split
 * into hi/lo parts for the tensor-core path) and stores 1/sigma_eff and the lags.
 * taps_dev complex64 [n_tmpl][k_stride]; lag_dev int32 [n_tmpl]; sigma_dev float64 [n_tmpl].
 * Must be called before rfd_ratio_filter_batch; stream-ordered. */
rfd_status rfd_plan_set_taps(rfd_plan *plan, const void *taps_dev, int32_t k_stride,
                             const int32_t *lag_dev, const double *sigma_dev, void *stream);

/* ------------------------------------------------------------------ ratio_filter_batch
 * Eq. 3 for every template of the plan, with the trigger reduction fused in:
 *   qhat_j[m] = sum_{k<K_j} rho_j[k] q_r[(m - s_j - k) mod n],  z_j = qhat_j / sigma_eff,j,
 * computed as Y[j, u] = sum_k rho_j[K_j-1-k] q_r[u + k] at true time m = (u + s_j + K_j - 1)
 * mod n; |z|^2 is compared with the threshold in registers and, for each run of samples
 * sharing (j, window), the maximum key is appended to cand_dev.  No SNR series is written.
 * qref_dev / qscale_dev as written by rfd_filter_reference in the plan's precision.
 * cand_dev rfd_candidate [cand_capacity]; cand_count_dev int64 (device) is reset to 0 by this
 * call, then counts every candidate produced, including those past the capacity (which are
 * dropped; rfd_find_triggers reports RFD_ERR_OVERFLOW and the needed capacity).
 * RFD_PREC_FP32 runs an FP32 CUDA-core FIR.  RFD_PREC_FP16X3 / BF16X3 run the tcgen05 kernel:
 * taps and q are split into hi + lo parts and the complex product is formed from three
 * real-block-form products hi*hi + hi*lo + lo*hi accumulated in FP32 (K <= 512; the plan's halo
 * must cover K rounded up to 16).  Its waits are bounded: a wait that gives up sets bit 62 of
 * *cand_count_dev, which rfd_find_triggers reports as RFD_ERR_TIMEOUT. */
rfd_status rfd_ratio_filter_batch(rfd_plan *plan, const void *qref_dev,
                                  const int32_t *qscale_dev, rfd_candidate *cand_dev,
                                  int64_t cand_capacity, int64_t *cand_count_dev, void *stream);

/* The same over a window of the plan's out_len output positions u = u_0 .. u_0 + out_len - 1
 * (mod n), u_0 = *u_begin_dev (int64 in device memory, read by the kernels, so that a captured
 * graph can be replayed for the next window; taken modulo n and rounded down to a multiple of
 * 512).  This is the streaming form of Sec. VII.A: the next block of SNR needs only the most
 * recent reference series plus a K-sample halo.  The triggers of windows that tile the segment,
 * merged per (j, window) by the maximum key, are those of rfd_ratio_filter_batch on a plan
 * without a window (bit for bit on the tensor-core and FP32 kernels; the block-FFT kernel cuts
 * its blocks at the window start, so there the SNRs agree to rounding). */
rfd_status rfd_ratio_filter_window(rfd_plan *plan, const void *qref_dev, const int32_t *qscale_dev,
                                   const int64_t *u_begin_dev, rfd_candidate *cand_dev,
                                   int64_t cand_capacity, int64_t *cand_count_dev, void *stream);

/* Tensor-core (or FMA) flops one rfd_ratio_filter_batch call of this plan executes. */
double rfd_plan_executed_flops(const rfd_plan *plan);
/* Which kernel filters each template of the plan: kernel_host int32 [n_tmpl] receives
 * RFD_KERNEL_FP32 (CUDA-core direct FIR), RFD_KERNEL_TC_TIME_ON_M / _TC_TEMPLATES_ON_M (the
 * two tensor-core contractions) or RFD_KERNEL_BLOCK_FFT (overlap-save blocks).  Host only. */
#define RFD_KERNEL_FP32 0
#define RFD_KERNEL_TC_TIME_ON_M 1
#define RFD_KERNEL_TC_TEMPLATES_ON_M 2
#define RFD_KERNEL_BLOCK_FFT 3
rfd_status rfd_plan_template_kernels(const rfd_plan *plan, int32_t *kernel_host);

/* ------------------------------------------------------------------ find_triggers
 * Merges candidates into triggers: per (j, w) the maximum key (the largest |z|^2, ties to the
 * smallest t), emitted sorted by (j, w).  Integer-only, deterministic.
 * cand_dev / cand_count_dev / cand_capacity as filled by a filtering call; n_tmpl templates;
 * trig_dev rfd_trigger [trig_capacity].  *n_trig_host receives the number of triggers.
 * Synchronises the stream (it reads the counts back).  Returns RFD_ERR_OVERFLOW when the
 * candidate list overflowed (then *n_trig_host = the candidate capacity needed) or when
 * trig_capacity is too small (then *n_trig_host = the trigger capacity needed). */
rfd_status rfd_find_triggers(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand_dev,
                             const int64_t *cand_count_dev, int64_t cand_capacity,
                             rfd_trigger *trig_dev, int64_t trig_capacity,
                             int64_t *n_trig_host, void *stream);

/* ------------------------------------------------------------------ whole segment as one graph
 * One data segment through filter_reference, ratio_filter_batch and the trigger merge,
 * captured once into a CUDA graph and replayed per segment (the per-segment loop of Table II
 * with one launch).  All buffers (as described for the three calls) are bound at creation;
 * to search the next segment, write its spectrum into dtilde_dev and run again.
 * rfd_search_create runs the step once outside the capture (sizing every workspace), then
 * captures it on `stream`, which must be a created stream (not the legacy default stream),
 * and synchronises.  rfd_search_run launches the graph on `stream`, waits for it, and returns
 * the trigger count in *n_trig_host with the status rules of rfd_find_triggers.  The plan and
 * the buffers must outlive the search; runs of one search must not overlap.  The graph also
 * holds the context's scratch buffers: while any search exists, a later call that needs a
 * larger scratch buffer gets a new one and the old block stays allocated (freed when the last
 * search is destroyed), so other calls on the same context may run between replays, in the
 * same stream order (not concurrently on another stream). */
typedef struct rfd_search rfd_search;
rfd_status rfd_search_create(rfd_plan *plan, const void *dtilde_dev, const double *psd_dev,
                             const void *href_dev, void *qref_dev, int32_t *qscale_dev,
                             rfd_candidate *cand_dev, int64_t cand_capacity,
                             int64_t *cand_count_dev, rfd_trigger *trig_dev,
                             int64_t trig_capacity, void *stream, rfd_search **out);
rfd_status rfd_search_run(rfd_search *search, void *stream, int64_t *n_trig_host);
/* Streaming (Sec. VII.A) with a plan whose out_len is a window: the next run filters the
 * window starting at u_begin (a multiple of 512 in [0, n); the value is copied to device
 * memory the graph reads, then the graph is launched as by rfd_search_run).  A plan without a
 * window ignores it. */
rfd_status rfd_search_run_at(rfd_search *search, int64_t u_begin, void *stream, int64_t *n_trig_host);
/* One segment end to end from host memory: copies the data spectrum dtilde_host (complex64
 * [n/2+1], host memory; pinned memory makes the copy asynchronous with respect to other host
 * work) into the search's bound dtilde_dev on `stream`, replays the graph as rfd_search_run,
 * then copies the triggers (rfd_trigger, sorted by (j, w)) into trig_host [trig_host_capacity].
 * Returns the trigger count in *n_trig_host with the status rules of rfd_find_triggers, and
 * RFD_ERR_OVERFLOW (with the count) when trig_host_capacity is too small; nothing is copied
 * to trig_host then.  Synchronises the stream twice (the count decides the read-back size). */
rfd_status rfd_search_run_host(rfd_search *search, const void *dtilde_host, rfd_trigger *trig_host,
                               int64_t trig_host_capacity, void *stream, int64_t *n_trig_host);
/* Kernels one run launches (they are counted in rfd_kernel_launches as they are replayed). */
int64_t rfd_search_kernels_per_run(const rfd_search *search);
/* Device time (ms) of the ratio-filter kernel in the last completed run (CUDA events recorded
 * inside the graph around it), or -1. */
double rfd_search_filter_ms(const rfd_search *search);
/* Device time (ms) of the whole last completed run, first to last node of the graph, or -1. */
double rfd_search_step_ms(const rfd_search *search);
void rfd_search_destroy(rfd_search *search);

/* ------------------------------------------------------------------ find_triggers, no allocation
 * The same merge as rfd_find_triggers, for callers that cannot allocate device memory while
 * they run: code that must not call cudaMalloc / cudaFree once set up (both can synchronise
 * the whole device and stall other streams, which low-latency search loops cannot afford),
 * callers whose device memory is owned by another allocator or memory pool, and callers that
 * hold no librfd context.  The paper has no counterpart; this is a deployment variant.
 *
 * It allocates nothing.  Its scratch is one fixed array of static device memory (4.0 MiB,
 * sized for RFD_NOALLOC_MAX_TEMPLATES templates and RFD_NOALLOC_MAX_CANDIDATES candidates)
 * that every GPU loading librfd holds until the process exits.  It runs on
 * the calling thread's current device.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress).  Under CUDA's lazy module loading that lookup is
 * also what loads librfd's device code on that device and backs the array, which can
 * synchronise the device: make the first call on each device during set-up; later calls only
 * reuse the cached address.
 * n_tmpl > RFD_NOALLOC_MAX_TEMPLATES or cand_capacity > RFD_NOALLOC_MAX_CANDIDATES is
 * rejected with RFD_ERR_SHAPE before anything runs.  Every call on a device shares the one
 * array: each call clears the counters it needs, but calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the caller.
 * Arguments, outputs, synchronisation and RFD_ERR_OVERFLOW as for rfd_find_triggers. */
#define RFD_NOALLOC_MAX_TEMPLATES 32768
#define RFD_NOALLOC_MAX_CANDIDATES 131072
rfd_status rfd_find_triggers_noalloc(int32_t n_tmpl, const rfd_candidate *cand_dev,
                                     const int64_t *cand_count_dev, int64_t cand_capacity,
                                     rfd_trigger *trig_dev, int64_t trig_capacity,
                                     int64_t *n_trig_host, void *stream);

/* ------------------------------------------------------------------ FINDCHIRP baseline
 * The standard frequency-domain matched filter of Eq. 1 for every template (Sec. II-III):
 * per template, c = 4 df d conj(h_j) / S, an n-point FP32 Stockham inverse FFT,
 * z = q / sigma(h_j), and the same threshold / window reduction into candidates as
 * rfd_ratio_filter_batch.  h_dev complex64 [n_tmpl][n/2+1] holds the templates (written by
 * rfd_gen_templates once per bank).  The comparison path for the ratio filter.  Two kernels
 * per batch of templates: the product 4 df d conj(h_j) / S is formed inside the first pass
 * of the two-pass inverse FFT (the zero upper half of the spectrum is never read) and the
 * threshold / window maximum runs inside the last pass (the series is never stored);
 * n in [2^12, 2^22]. */
rfd_status rfd_findchirp(rfd_ctx *ctx, const rfd_grid *grid, const void *dtilde_dev,
                         const double *psd_dev, const void *h_dev, int32_t n_tmpl,
                         int32_t window, float threshold, rfd_candidate *cand_dev,
                         int64_t cand_capacity, int64_t *cand_count_dev, void *stream);

/* Inverse FFT (unnormalised, exp(+2 pi i k m / n)) of `batch` complex64 rows of length n
 * with the library's Stockham kernels: in_dev and out_dev may not overlap. */
rfd_status rfd_ifft_c2c(rfd_ctx *ctx, int64_t n, int32_t batch, const void *in_dev,
                        void *out_dev, void *stream);

/* The same transform in either direction and precision: fp64 = 0 for complex64 rows, 1 for
 * complex128 rows; inverse = 1 for exp(+2 pi i k m / n), 0 for exp(-2 pi i k m / n); no
 * normalisation.  n a power of two in [4, 2^24]; for 2^12 <= n <= 2^22 the rows go through the
 * two-pass (four-step) form, otherwise one pass per radix.  in_dev and out_dev hold batch * n
 * elements on the device and may not overlap.  RFD_ERR_SHAPE / RFD_ERR_ARG on bad sizes or
 * pointers, before any launch. */
rfd_status rfd_fft_c2c(rfd_ctx *ctx, int64_t n, int32_t batch, int32_t fp64, int32_t inverse,
                       const void *in_dev, void *out_dev, void *stream);

/* ------------------------------------------------------------------ sub-band chi^2
 * The time-frequency chi^2 signal-consistency test through the ratio filter (Sec. VI): the
 * reference's band is split into p sub-bands of equal reference SNR (w_k = 4 df |h_ref,k|^2 / S_k;
 * edge e_b is one past the first bin at which the running FP64 sum of w from k_lo reaches
 * b W / p); the data are matched-filtered per sub-band once per reference; a template's
 * sub-band SNRs at a trigger are its ratio FIR (Eq. 3) of the reference's sub-band series,
 *   z_b = (1/sigma_eff) sum_k rho[k] q_r,b[(t - s - k) mod n],  z = sum_b z_b,
 * and chi^2 = sum_b |z_b - u_b z|^2 / u_b with u_b the effective template's share of power in
 * band b (2 (p - 1) degrees of freedom in Gaussian noise).  Evaluated at the triggers only. */
typedef struct rfd_subband rfd_subband;
/* p in [2, 64]; computes the band edges (synchronous).  rfd_subband_edges copies them out as
 * int32 [n_ref][p + 1]. */
rfd_status rfd_subband_create(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                              const rfd_params *refs_host, int32_t n_ref, int32_t p,
                              rfd_subband **out);
void rfd_subband_destroy(rfd_subband *sb);
rfd_status rfd_subband_edges(const rfd_subband *sb, int32_t *edges_host);
/* q_r,b of every reference and band: qband_dev complex64 [n_ref][p][ld], ld = rfd_qref_ld(n,
 * halo), wrap halo as for rfd_filter_reference; href_dev as for rfd_filter_reference. */
rfd_status rfd_subband_filter_reference(rfd_subband *sb, const void *dtilde_dev, const double *psd_dev,
                                        const void *href_dev, int32_t halo, void *qband_dev,
                                        void *stream);
/* u_dev float [n_tmpl][p]: each template's band shares (forward FFT of its placed taps).
 * taps_dev complex64 [n_tmpl][k_stride], k_dev / lag_dev int32 [n_tmpl] (device), ref_of_host
 * int32 [n_tmpl].  Per bank, set-up.  Synchronises the stream. */
rfd_status rfd_subband_shares(rfd_subband *sb, const double *psd_dev, const void *taps_dev,
                              int32_t k_stride, const int32_t *k_dev, const int32_t *lag_dev,
                              const int32_t *ref_of_host, int32_t n_tmpl, float *u_dev, void *stream);
/* chi^2 of each trigger (rfd_trigger [n_trig], device) into chi2_dev float [n_trig]; zb_dev
 * complex64 [n_trig][p] (may be NULL) receives the sub-band SNRs.  sigma_dev float64 [n_tmpl].
 * Synchronises the stream. */
rfd_status rfd_subband_chi2(rfd_subband *sb, const void *qband_dev, int32_t halo, const void *taps_dev,
                            int32_t k_stride, const int32_t *k_dev, const int32_t *lag_dev,
                            const double *sigma_dev, const float *u_dev, const int32_t *ref_of_host,
                            int32_t n_tmpl, const rfd_trigger *trig_dev, int64_t n_trig,
                            float *chi2_dev, void *zb_dev, void *stream);

/* ------------------------------------------------------------------ learned taps
 * A surrogate for make_taps: one network per reference maps a template to 128 complex taps
 * at the network's fixed lag.  Inputs (20): the features
 *   x = (Mc, eta, chi_eff, Lambda~),  Mc = M eta^(3/5), chi_eff = (m1 chi1 + m2 chi2) / M,
 * standardised per network, xh = (x - mu) / sd, then cos p_m and sin p_m of the ratio's phase
 * (Eq. 2) p_m = Dpsi(f_m) - Dpsi(f_4), Dpsi = Psi_j - Psi_r in FP64, at the eight frequencies
 * f_m (m = 0..8, m != 4) log-spaced from 3 f_low to 0.45 fs.  Layers
 *   h1 = gelu(W1 in + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3), y = W4 h3 + b4
 * (widths 20 -> 256 -> 256 -> 256 -> 256; gelu(u) = u/2 (1 + tanh(sqrt(2/pi)(u + 0.044715 u^3))))
 * give rho[k] = out_scale (y[k] + i y[128 + k]).
 * Training minimises the PSD-weighted chi^2 of Eq. 4 (Sec. V.A) between the response of rho
 * and that of the exact taps a* at the same lag, written in the tap domain through Parseval
 * (Eqs. 5-6) and minimised over a constant phase of a* (which only rotates z):
 *   L = (rho^H M rho + a*^H M a* - 2 |a*^H M rho|) / (a*^H M a*),  M[b, a] = C_r[b - a],
 * averaged over the batch.  FP16 operands on the tensor cores, FP32 master weights, Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8), dynamic loss scaling on the device.
 * Weights (host float32), per network in this order: W1 [256][20], b1 [256], W2 [256][256],
 * b2, W3 [256][256], b3, W4 [256][256], b4: rfd_mlp_param_count() floats per network. */
#define RFD_MLP_TAPS 128
#define RFD_MLP_INPUTS 20
#define RFD_MLP_FEATURES_LD 64     /* halfs per row of an input buffer (20 used, zero padded) */
typedef struct rfd_mlp rfd_mlp;
int64_t rfd_mlp_param_count(void);
/* One network per reference; computes the references' autocorrelations C_r[l], |l| < 128
 * (Eq. 6 on the sample grid, FP64).  Weights start at zero: call rfd_mlp_set_weights. */
rfd_status rfd_mlp_create(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                          const rfd_params *refs_host, int32_t n_ref, rfd_mlp **out);
void rfd_mlp_destroy(rfd_mlp *mlp);
/* Sets the FP32 master weights of every network (host [n_ref][param_count]) and resets the
 * optimiser (step 0, loss scale 2^16).  Synchronous.  get_weights copies them back. */
rfd_status rfd_mlp_set_weights(rfd_mlp *mlp, const float *weights_host);
rfd_status rfd_mlp_get_weights(const rfd_mlp *mlp, float *weights_host);
/* Per network: feature mean and spread (host double [n_ref][4] each, spread > 0), output
 * scale (double [n_ref], > 0) and lag s_r (int32 [n_ref], in [-n/2, n/2)).  Synchronous. */
rfd_status rfd_mlp_set_norm(rfd_mlp *mlp, const double *mu_host, const double *sd_host,
                            const double *out_scale_host, const int32_t *lag_host);
/* C_r rows as complex128 [n_ref][255], lag l at index l + 127.  Synchronous. */
rfd_status rfd_mlp_get_autocorr(const rfd_mlp *mlp, double *autocorr_host);
/* FP16 network inputs of n templates (row j uses network net_of_host[j]) into feat_dev
 * half [n][64].  Synchronises the stream. */
rfd_status rfd_mlp_features(rfd_mlp *mlp, const rfd_params *params_host,
                            const int32_t *net_of_host, int32_t n, void *feat_dev, void *stream);
/* One optimiser step of every network on a batch: network g uses the rows
 * idx_dev[g][b] (int32 [n_ref][batch], each < n_train) of feat_dev (half
 * [n_ref][n_train][64]) and target_dev (complex64 [n_ref][n_train][128], the exact taps).
 * batch: multiple of 128 in [128, 8192].  Stream-ordered, no host synchronisation; a step
 * whose gradients are not finite is skipped on the device. */
rfd_status rfd_mlp_train_step(rfd_mlp *mlp, const void *feat_dev, const void *target_dev,
                              int32_t n_train, const int32_t *idx_dev, int32_t batch, float lr,
                              void *stream);
/* Forward and backward only: unscaled gradients into grads_dev (float [n_ref][param_count],
 * the weight layout) and the batch-mean loss per network into loss_dev (float [n_ref]).
 * Synchronises the stream. */
rfd_status rfd_mlp_grads(rfd_mlp *mlp, const void *feat_dev, const void *target_dev,
                         int32_t n_train, const int32_t *idx_dev, int32_t batch,
                         float *grads_dev, float *loss_dev, void *stream);
/* After the last step: batch-mean loss per network (host float [n_ref], may be NULL), steps
 * taken and the current loss scale.  Synchronises the stream; RFD_ERR_TIMEOUT if a kernel
 * gave up a bounded wait. */
rfd_status rfd_mlp_state(rfd_mlp *mlp, float *loss_host, int32_t *step_host,
                         float *loss_scale_host, void *stream);
/* Checkpoint of the networks' training state (the paper has no training code to resume;
 * this makes training restartable): rfd_mlp_save writes, after the stream's work, the FP32
 * master weights, Adam's moments, the normalisation, the lags, the optimiser state (Adam step,
 * dynamic loss scale and its clean-step count), the references' autocorrelations and their
 * phase constants to `path`: an 8-byte magic, a little-endian uint64 header length, a JSON
 * header naming each section (dtype, shape, offset, bytes), then the raw sections, 64-byte
 * aligned.  rfd_mlp_load reads such a file into a network object created for the same grid,
 * PSD and references (checked: the grid, the counts, the autocorrelations and the references'
 * constants bit for bit, else RFD_ERR_ARG / RFD_ERR_SHAPE) and rebuilds the FP16 operand copies from the masters, so that
 * training continues exactly as it would have without the save.  Both synchronise. */
rfd_status rfd_mlp_save(rfd_mlp *mlp, const char *path, void *stream);
rfd_status rfd_mlp_load(rfd_mlp *mlp, const char *path, void *stream);
/* Surrogate taps of n templates: taps_dev complex64 [n][k_stride] (k_stride >= 128, taps
 * 128.. zero), lag_dev int32 [n] (the network's lag), sigma_dev float64 [n] (sigma_eff of
 * the stored taps, Eqs. 5-6).  The outputs are what rfd_plan_set_taps takes.  Synchronises
 * the stream. */
rfd_status rfd_mlp_infer(rfd_mlp *mlp, const rfd_params *params_host,
                         const int32_t *net_of_host, int32_t n, int32_t k_stride,
                         void *taps_dev, int32_t *lag_dev, double *sigma_dev, void *stream);
/* Match between the responses of tap rows rho1[i] and rho2[i] (complex64, row strides ld1,
 * ld2 >= 128, first 128 taps, same lag) under reference net_of_host[i]'s C_r:
 * |rho2^H M rho1| / sqrt(rho1^H M rho1 rho2^H M rho2) into match_dev float64 [n].
 * Synchronises the stream. */
rfd_status rfd_mlp_cross_match(rfd_mlp *mlp, const int32_t *net_of_host, int32_t n,
                               const void *rho1_dev, int64_t ld1, const void *rho2_dev,
                               int64_t ld2, double *match_dev, void *stream);
/* Taps for a bank with the surrogate and exact extraction as the fallback.  Every template
 * gets surrogate taps; per reference, templates are ordered by chirp mass and every
 * spot_stride-th one (and the last) is spot-checked: its exact taps at the network's lag
 * (rfd_make_taps_at_lag) are compared with its surrogate taps by the match above.  A
 * template keeps its surrogate taps when the spot checks on both sides of it in that order
 * (or its own, for a spot-checked one) reach min_match (0.999 is the intended bar); the rest
 * get exact taps from rfd_make_taps (their own lag, K = 128).
 * Outputs: taps_dev complex64 [n_tmpl][k_stride], lag_dev, sigma_dev as for rfd_make_taps;
 * surrogate_match_dev float64 [n_tmpl] (may be NULL): the measured match of spot-checked
 * templates, NaN elsewhere; source_dev int32 [n_tmpl]: 0 surrogate, 1 exact fallback,
 * 2 surrogate and spot-checked; stats_host int64 [4] (may be NULL): templates on surrogate
 * taps, on exact taps, spot-checked, spot checks below min_match.  Synchronous. */
rfd_status rfd_learned_taps(rfd_mlp *mlp, const double *psd_dev, const rfd_params *tmpl_host,
                            const int32_t *ref_of_tmpl_host, int32_t n_tmpl, int32_t spot_stride,
                            double min_match, int32_t k_stride, double tukey_alpha,
                            void *taps_dev, int32_t *lag_dev, double *sigma_dev,
                            double *surrogate_match_dev, int32_t *source_dev,
                            int64_t *stats_host, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RFD_H */
