// C ABI entry points of librfd: argument checks, host-side planning, dispatch to kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <numeric>

#include "internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace {
// A profiler-visible range (NVTX) over one C-ABI call, so that Nsight tools show the library's
// calls by name; with no tool attached a push or pop costs a pointer test.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace rfd {

// implemented in the kernel files
rfd_status gen_templates_impl(rfd_ctx *, const Grid &, const std::vector<PNParams> &, float2 *,
                              cudaStream_t);
rfd_status filter_reference_impl(rfd_ctx *, const Grid &, const float2 *, const double *, const float2 *,
                                 int64_t, int32_t, int32_t, void *, int32_t *, cudaStream_t);
rfd_status findchirp_impl(rfd_ctx *, const Grid &, const float2 *, const double *, const float2 *, int64_t,
                          int32_t, float, rfd_candidate *, int64_t, int64_t *, cudaStream_t);
int fir32_tile_templates();
rfd_status fir32_launch(const rfd_plan *, const float2 *, const int64_t *, rfd_candidate *, int64_t, int64_t *,
                        cudaStream_t);
rfd_status pack_taps_fp32(rfd_plan *, const float2 *, int32_t, const int32_t *, const double *,
                          cudaStream_t);
rfd_status tc_pack(rfd_plan *, const float2 *, int32_t, const int32_t *, const double *, cudaStream_t);
rfd_status tl_pack(rfd_plan *, const float2 *, int32_t, const int32_t *, const double *, cudaStream_t);
rfd_status tl_launch(const rfd_plan *, const void *, const int32_t *, const int64_t *, rfd_candidate *, int64_t,
                     int64_t *,
                     cudaStream_t);
uint32_t tl_ystride(int32_t kpad_max);
uint32_t tl_qwin(int32_t kpad_max);
int tl_rows_per_item();
int tl_tile_templates();
rfd_status tc_launch(const rfd_plan *, const void *, const int32_t *, const int64_t *, rfd_candidate *, int64_t,
                     int64_t *,
                     cudaStream_t);
int tc_rows_per_item();
int fft_fir_block_len();
int fft_fir_tile_templates();
int fft_fir_blocks_per_cta();
rfd_status fft_pack(rfd_plan *, const float2 *, int32_t, const int32_t *, const double *, cudaStream_t);
rfd_status fft_launch(const rfd_plan *, const void *, const int32_t *, const int64_t *, rfd_candidate *, int64_t,
                      int64_t *,
                      cudaStream_t);

// Tensor-core tiles: per reference, templates in increasing K, cut so that a tile holds at
// most 128 templates (64 once its K exceeds 128, 32 once it exceeds 256: the taps image,
// 3 NT rows x K taps x hi/lo, stays within 192 KB of shared memory); NT is the tile's count
// rounded up to 16.  Item ranges per CTA balance the MMA work.
static int32_t tc_nt_cap(const rfd_plan_options &o, int32_t kpad) {
    return kpad <= 128 ? o.tile_nt[0] : (kpad <= 256 ? o.tile_nt[1] : o.tile_nt[2]);
}

// Cost-balanced contiguous item ranges (one per CTA) over tiles of n_it items each, an item of
// tile t costing cost[t].
static std::vector<int64_t> balanced_ranges(const std::vector<double> &cost, int64_t n_it, int64_t G) {
    const int64_t ntiles = (int64_t)cost.size();
    const int64_t total_items = ntiles * n_it;
    std::vector<double> prefix(ntiles + 1, 0.0);
    for (int64_t t = 0; t < ntiles; ++t) prefix[t + 1] = prefix[t] + cost[t] * n_it;
    std::vector<int64_t> ranges(G + 1, 0);
    ranges[G] = total_items;
    int64_t t = 0;
    for (int64_t g = 1; g < G; ++g) {
        const double target = prefix[ntiles] * (double)g / (double)G;
        while (t + 1 < ntiles && prefix[t + 1] <= target) ++t;
        int64_t within = (int64_t)((target - prefix[t]) / cost[t]);
        within = std::min<int64_t>(std::max<int64_t>(within, 0), n_it);
        ranges[g] = std::max(ranges[g - 1], t * n_it + within);
    }
    return ranges;
}

// Long-tap tiles: per reference, up to 64 templates with K > long_k (mix_k as for the other
// kernel); appended to the plan's slot order.
static rfd_status plan_tl_tiles(rfd_plan *p, const std::vector<int32_t> &order, int num_sms,
                                const rfd_plan_options &opt) {
    const int64_t n_tb = p->out_len / tl_rows_per_item();
    const int32_t nt = tl_tile_templates();
    int64_t taps_off = 0;
    int32_t kpad_max = 0;
    size_t i = 0;
    while (i < order.size()) {
        const int32_t r = p->ref_of[order[i]];
        TcTile t{};
        t.ref = r;
        t.first = (int32_t)p->perm.size();
        while (i < order.size() && p->ref_of[order[i]] == r && t.count < nt) {
            const int32_t kt = std::max(t.k_tile, p->k_of[order[i]]);
            if (!opt.mix_k && t.count > 0 && (kt + 15) / 16 != (t.k_tile + 15) / 16) break;
            t.k_tile = kt;
            ++t.count;
            p->perm.push_back(order[i]);
            ++i;
        }
        t.nk16 = (t.k_tile + 15) / 16;
        t.kpad = 16 * t.nk16;
        t.nt = nt;
        t.nch = (t.kpad + 63) / 64;
        t.taps_bytes = t.nch * 2 * 3 * nt * 128;
        t.taps_off = taps_off;
        taps_off += t.taps_bytes;
        kpad_max = std::max(kpad_max, t.kpad);
        p->tl_tiles.push_back(t);
        p->executed_flops += (double)n_tb * t.nk16 * 6.0 * 2.0 * 128.0 * (double)tl_rows_per_item() * 16.0;
    }
    const int64_t ntiles = (int64_t)p->tl_tiles.size();
    if (ntiles == 0) return RFD_OK;
    RFD_REQUIRE(p->ld >= p->grid.n + kpad_max, RFD_ERR_SHAPE,
                "tensor-core path reads %d taps past each block: halo=%d too small (need >= %d)", kpad_max,
                p->halo, kpad_max - 1);
    p->tl_ystride = tl_ystride(kpad_max);
    p->tl_qwin = tl_qwin(kpad_max);
    // cost of one item in SM cycles, measured on the kernel (uniform K, every SM busy): the MMAs
    // take 768 cycles per 16-tap step plus ~370 of hand-offs, and no item takes less than about
    // 3850 (the epilogue drains 128 x 256 accumulators per item whatever K is): 3864 cycles at
    // K = 16, 4012 at 64, 4989 at 96, 6508 at 128.  Items of short-K tiles priced by their MMAs
    // alone made the CTAs that hold them finish last.
    std::vector<double> cost(ntiles);
    for (int64_t t = 0; t < ntiles; ++t) {
        const double nk = (double)p->tl_tiles[t].nk16;
        cost[t] = std::max(768.0 * nk + 370.0, 3850.0 + 40.0 * nk);
    }
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(opt.grid_ctas > 0 ? opt.grid_ctas : num_sms,
                                                           ntiles * n_tb));
    const std::vector<int64_t> ranges = balanced_ranges(cost, n_tb, G);
    p->tl_grid = (int32_t)G;
    RFD_TRY(ensure(p->d_tl_ranges, (G + 1) * sizeof(int64_t)));
    RFD_TRY_CUDA(cudaMemcpy(p->d_tl_ranges.p, ranges.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    RFD_TRY(ensure(p->d_tl_taps, (size_t)taps_off));
    RFD_TRY(ensure(p->d_tl_tiles, ntiles * sizeof(TcTile)));
    RFD_TRY_CUDA(
        cudaMemcpy(p->d_tl_tiles.p, p->tl_tiles.data(), ntiles * sizeof(TcTile), cudaMemcpyHostToDevice));
    return RFD_OK;
}

// Block-FFT tiles: per reference, up to 64 templates (order: by reference, then K), appended
// to the plan's slot order.  Blocks of L = 2048 - K_max + 1 outputs, four per CTA item; item
// ranges per persistent CTA balance the templates transformed.
static rfd_status plan_fft_tiles(rfd_plan *p, const std::vector<int32_t> &order, int num_sms,
                                 const rfd_plan_options &opt) {
    if (order.empty()) return RFD_OK;
    const int32_t M = fft_fir_block_len(), nt = fft_fir_tile_templates(), gpc = fft_fir_blocks_per_cta();
    int32_t kmax = 0;
    for (int32_t j : order) kmax = std::max(kmax, p->k_of[j]);
    p->fft_L = M - kmax + 1;
    p->fft_nb = (int32_t)((p->out_len + p->fft_L - 1) / p->fft_L);
    p->fft_nbg = (p->fft_nb + gpc - 1) / gpc;
    p->fft_slot0 = (int64_t)p->perm.size();
    size_t i = 0;
    while (i < order.size()) {
        const int32_t r = p->ref_of[order[i]];
        FftTile t{};
        t.ref = r;
        t.first = (int32_t)p->perm.size();
        while (i < order.size() && p->ref_of[order[i]] == r && t.count < nt) {
            p->perm.push_back(order[i]);
            ++t.count;
            ++i;
        }
        if (p->fft_refs.empty() || p->fft_refs.back() != r) p->fft_refs.push_back(r);
        p->fft_tiles.push_back(t);
    }
    p->fft_nslots = (int64_t)p->perm.size() - p->fft_slot0;
    const double log2m = std::log2((double)M);
    p->fft_flops = (double)p->fft_nslots * p->fft_nb * M * (6.0 + 5.0 * log2m) +
                   (double)p->fft_refs.size() * p->fft_nb * M * 5.0 * log2m;
    const int64_t ntiles = (int64_t)p->fft_tiles.size();
    // cost of one item in template-block groups: a per-CTA span fit on C3 and C5 gave 1.77 us
    // per template-block group and 1.9-2.7 us per item (the block spectra loads, the ring's
    // first copy), so an item costs about one group besides its templates
    std::vector<double> cost(ntiles);
    for (int64_t t = 0; t < ntiles; ++t) cost[t] = (double)p->fft_tiles[t].count + 1.0;
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(opt.grid_ctas > 0 ? opt.grid_ctas : num_sms,
                                                           ntiles * p->fft_nbg));
    const std::vector<int64_t> ranges = balanced_ranges(cost, p->fft_nbg, G);
    p->fft_grid = (int32_t)G;
    RFD_TRY(fft_stage_twiddles32(p->ctx, 11, &p->fft_stw, 0));
    RFD_TRY_CUDA(cudaStreamSynchronize(0));
    RFD_TRY(ensure(p->d_fft_ranges, (G + 1) * sizeof(int64_t)));
    RFD_TRY_CUDA(cudaMemcpy(p->d_fft_ranges.p, ranges.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    RFD_TRY(ensure(p->d_fft_tiles, ntiles * sizeof(FftTile)));
    RFD_TRY_CUDA(
        cudaMemcpy(p->d_fft_tiles.p, p->fft_tiles.data(), ntiles * sizeof(FftTile), cudaMemcpyHostToDevice));
    RFD_TRY(ensure(p->d_fft_refs, p->fft_refs.size() * sizeof(int32_t)));
    RFD_TRY_CUDA(cudaMemcpy(p->d_fft_refs.p, p->fft_refs.data(), p->fft_refs.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    RFD_TRY(ensure(p->d_fft_P, (size_t)p->fft_nslots * M * sizeof(float2)));
    RFD_TRY(ensure(p->d_fft_X, (size_t)p->n_ref * p->fft_nb * M * sizeof(float2)));
    return RFD_OK;
}

static rfd_status plan_tc_tiles(rfd_plan *p, const std::vector<int32_t> &all, int num_sms,
                                const rfd_plan_options &opt) {
    const int64_t n_tt = p->out_len / tc_rows_per_item();
    int64_t taps_off = 0;
    int32_t kpad_max = 0;
    uint32_t cap = 0;
    const int32_t long_k = opt.long_k;
    std::vector<int32_t> order, order_long;
    for (int32_t j : all) (p->k_of[j] > long_k ? order_long : order).push_back(j);
    size_t i = 0;
    while (i < order.size()) {
        const int32_t r = p->ref_of[order[i]];
        TcTile t{};
        t.ref = r;
        t.first = (int32_t)p->perm.size();
        while (i < order.size() && p->ref_of[order[i]] == r) {
            const int32_t kt = std::max(t.k_tile, p->k_of[order[i]]);
            if (t.count + 1 > tc_nt_cap(opt, 16 * ((kt + 15) / 16))) break;
            // without mixing, a tile ends where the 16-tap step count changes
            if (!opt.mix_k && t.count > 0 && (kt + 15) / 16 != (t.k_tile + 15) / 16) break;
            t.k_tile = kt;
            ++t.count;
            p->perm.push_back(order[i]);
            ++i;
        }
        t.nk16 = (t.k_tile + 15) / 16;
        t.kpad = 16 * t.nk16;
        t.nt = 16 * ((t.count + 15) / 16);
        t.nch = (t.kpad + 63) / 64;
        t.taps_bytes = 2 * t.nch * 3 * t.nt * 128;
        t.taps_off = taps_off;
        taps_off += t.taps_bytes;
        kpad_max = std::max(kpad_max, t.kpad);
        cap = std::max(cap, (uint32_t)t.taps_bytes);
        p->tc_tiles.push_back(t);
        p->executed_flops += (double)n_tt * t.nk16 * 6.0 * 2.0 * 128.0 * (2.0 * t.nt) * 16.0;
    }
    p->tc_taps_cap = (cap + 1023u) / 1024u * 1024u;
    p->tc_win = (uint32_t)(128 + kpad_max + 8);
    RFD_REQUIRE(p->ld >= p->grid.n + kpad_max, RFD_ERR_SHAPE,
                "tensor-core path reads %d taps past each block: halo=%d too small (need >= %d)", kpad_max,
                p->halo, kpad_max - 1);
    RFD_TRY(plan_tl_tiles(p, order_long, num_sms, opt));
    p->n_slots = (int64_t)p->perm.size();
    const int64_t ntiles = (int64_t)p->tc_tiles.size();
    if (ntiles == 0) return RFD_OK;
    // cost-balanced contiguous item ranges, one per CTA (MMAs cost the same for any N <= 256)
    std::vector<double> cost(ntiles);
    for (int64_t t = 0; t < ntiles; ++t) cost[t] = (double)p->tc_tiles[t].nk16 * 6.0 + 2.0;
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(opt.grid_ctas > 0 ? opt.grid_ctas : num_sms,
                                                           ntiles * n_tt));
    const std::vector<int64_t> ranges = balanced_ranges(cost, n_tt, G);
    p->tc_grid = (int32_t)G;
    RFD_TRY(ensure(p->d_ranges, (G + 1) * sizeof(int64_t)));
    RFD_TRY_CUDA(cudaMemcpy(p->d_ranges.p, ranges.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    RFD_TRY(ensure(p->d_taps, (size_t)std::max<int64_t>(taps_off, 1024)));
    RFD_TRY(ensure(p->d_tiles, ntiles * sizeof(TcTile)));
    RFD_TRY_CUDA(cudaMemcpy(p->d_tiles.p, p->tc_tiles.data(), ntiles * sizeof(TcTile), cudaMemcpyHostToDevice));
    return RFD_OK;
}

namespace {
thread_local char g_err[1024] = {0};
std::atomic<int64_t> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// A captured graph (rfd_search) holds raw pointers into workspaces and plan buffers.  While
// any graph is alive, a block that is replaced or released is kept (retired) instead of
// freed, and the retired blocks are freed when the last graph goes away.
static std::mutex g_retire_mu;
static int g_live_graphs = 0;
static std::vector<void *> g_retired;

void graphs_pin() {
    std::lock_guard<std::mutex> lk(g_retire_mu);
    ++g_live_graphs;
}

void graphs_unpin() {
    std::lock_guard<std::mutex> lk(g_retire_mu);
    if (--g_live_graphs > 0) return;
    g_live_graphs = 0;
    if (g_retired.empty()) return;
    cudaDeviceSynchronize();
    for (void *p : g_retired) cudaFree(p);
    g_retired.clear();
}

static void free_or_retire(void *p) {
    std::lock_guard<std::mutex> lk(g_retire_mu);
    if (g_live_graphs > 0)
        g_retired.push_back(p);
    else
        cudaFree(p);
}

rfd_status ensure(DevBuf &b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return RFD_OK;
    if (b.p) {
        // earlier stream work may still use the old block
        RFD_TRY_CUDA(cudaDeviceSynchronize());
        free_or_retire(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    const size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        b.p = nullptr;
        set_error("workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return RFD_ERR_NOMEM;
    }
    b.bytes = want;
    return RFD_OK;
}

void release(DevBuf &b) {
    if (b.p) free_or_retire(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

rfd_status check_grid(const rfd_grid *g, Grid *out) {
    RFD_REQUIRE(g != nullptr, RFD_ERR_ARG, "grid is NULL");
    RFD_REQUIRE(std::isfinite(g->fs) && g->fs > 0, RFD_ERR_ARG, "grid.fs must be finite and > 0");
    RFD_REQUIRE(g->n >= 1024 && g->n <= (int64_t(1) << 22) && (g->n & (g->n - 1)) == 0, RFD_ERR_SHAPE,
                "grid.n=%lld must be a power of two in [2^10, 2^22]", (long long)g->n);
    RFD_REQUIRE(std::isfinite(g->f_low) && g->f_low > 0 && g->f_low < 0.5 * g->fs, RFD_ERR_ARG,
                "grid.f_low must lie in (0, fs/2)");
    RFD_REQUIRE(g->reserved == 0, RFD_ERR_ARG, "grid.reserved must be 0");
    RFD_REQUIRE((g->pn_flags & ~(RFD_PN_SO | RFD_PN_TIDAL)) == 0, RFD_ERR_ARG, "unknown pn_flags bits");
    out->fs = g->fs;
    out->n = g->n;
    out->nf = g->n / 2 + 1;
    out->f_low = g->f_low;
    out->df = g->fs / (double)g->n;
    out->k_lo = (int64_t)std::ceil(g->f_low / out->df - 1e-12);
    out->pn_flags = g->pn_flags;
    int l = 0;
    while ((int64_t(1) << l) < g->n) ++l;
    out->log2n = l;
    RFD_REQUIRE(out->k_lo >= 1 && out->k_lo <= g->n / 2 - 1, RFD_ERR_ARG, "empty data band");
    return RFD_OK;
}

rfd_status make_pn(const Grid &g, const rfd_params *p, PNParams *out) {
    RFD_REQUIRE(std::isfinite(p->m1) && std::isfinite(p->m2) && p->m1 > 0 && p->m2 > 0, RFD_ERR_ARG,
                "masses must be finite and > 0");
    RFD_REQUIRE(std::isfinite(p->chi1) && std::isfinite(p->chi2) && std::isfinite(p->lambda_tilde),
                RFD_ERR_ARG, "spins and lambda must be finite");
    const double mtot = p->m1 + p->m2;
    out->mt = mtot * kTSun;
    out->eta = p->m1 * p->m2 / (mtot * mtot);
    out->beta = 0.0;
    if (g.pn_flags & RFD_PN_SO) {
        const double q1 = p->m1 / mtot, q2 = p->m2 / mtot;
        out->beta = ((113.0 * (q1 * q1) + 75.0 * out->eta) * p->chi1 +
                     (113.0 * (q2 * q2) + 75.0 * out->eta) * p->chi2) / 12.0;
    }
    out->lam = (g.pn_flags & RFD_PN_TIDAL) ? p->lambda_tilde : 0.0;
    const double fisco = 1.0 / (std::pow(6.0, 1.5) * kPi * out->mt);
    out->k_hi = std::min<int64_t>(g.n / 2 - 1, (int64_t)std::floor(fisco / g.df));
    out->pad = 0;
    return RFD_OK;
}

rfd_status make_pn_vec(const Grid &g, const rfd_params *p, int32_t count,
                              std::vector<PNParams> *out) {
    out->resize(count);
    for (int32_t i = 0; i < count; ++i) RFD_TRY(make_pn(g, &p[i], &(*out)[i]));
    return RFD_OK;
}

}  // namespace rfd

using namespace rfd;

extern "C" {

int32_t rfd_version(void) { return RFD_VERSION; }

const char *rfd_status_string(rfd_status s) {
    switch (s) {
        case RFD_OK: return "ok";
        case RFD_ERR_ARG: return "invalid argument";
        case RFD_ERR_SHAPE: return "invalid shape";
        case RFD_ERR_UNSUPPORTED: return "unsupported";
        case RFD_ERR_CUDA: return "CUDA error";
        case RFD_ERR_NOMEM: return "out of device memory";
        case RFD_ERR_TIMEOUT: return "device wait timed out";
        case RFD_ERR_OVERFLOW: return "output capacity exceeded";
    }
    return "unknown status";
}

const char *rfd_last_error(void) { return g_err; }

int64_t rfd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t rfd_qref_ld(int64_t n, int32_t halo) { return ((n + (int64_t)halo + 63) / 64) * 64; }

rfd_status rfd_ctx_create(int32_t device, rfd_ctx **out) {
    RFD_REQUIRE(out != nullptr, RFD_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    RFD_TRY_CUDA(cudaGetDeviceCount(&ndev));
    RFD_REQUIRE(device >= 0 && device < ndev, RFD_ERR_ARG, "device %d not present (%d devices)", device, ndev);
    RFD_TRY_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    RFD_TRY_CUDA(cudaGetDeviceProperties(&prop, device));
    RFD_REQUIRE(prop.major == 10 && prop.minor == 3, RFD_ERR_UNSUPPORTED,
                "librfd is built for sm_103a (GB300); device %d is sm_%d%d", device, prop.major, prop.minor);
    rfd_ctx *c = new rfd_ctx();
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    *out = c;
    return RFD_OK;
}

void rfd_ctx_destroy(rfd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->tw32) cudaFree(kv.second);
    for (auto &kv : ctx->tw64) cudaFree(kv.second);
    for (auto &kv : ctx->stw32) cudaFree(kv.second);
    for (auto &kv : ctx->stw64) cudaFree(kv.second);
    for (auto &b : ctx->ws) release(b);
    delete ctx;
}

void rfd_ctx_trim(rfd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &b : ctx->ws) release(b);
}

rfd_status rfd_gen_templates(rfd_ctx *ctx, const rfd_grid *grid, const rfd_params *params_host,
                             int32_t n_tmpl, void *h_dev, void *stream) {
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_tmpl >= 0, RFD_ERR_SHAPE, "n_tmpl < 0");
    if (n_tmpl == 0) return RFD_OK;
    RFD_REQUIRE(params_host && h_dev, RFD_ERR_ARG, "NULL params or output");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<PNParams> pn;
    RFD_TRY(make_pn_vec(g, params_host, n_tmpl, &pn));
    return gen_templates_impl(ctx, g, pn, (float2 *)h_dev, (cudaStream_t)stream);
}

rfd_status rfd_make_taps(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                         const rfd_params *refs_host, int32_t n_ref, const rfd_params *tmpl_host,
                         const int32_t *ref_of_tmpl_host, int32_t n_tmpl, const int32_t *k_host,
                         const int32_t *buckets_host, int32_t n_buckets, double energy_frac, int32_t k_stride,
                         double tukey_alpha, void *taps_dev, int32_t *k_dev, int32_t *lag_dev, double *sigma_dev,
                         double *match_dev, void *stream) {
    NvtxRange nvtx_range("rfd_make_taps");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_tmpl >= 0, RFD_ERR_SHAPE, "need n_ref >= 1 and n_tmpl >= 0");
    if (n_tmpl == 0) return RFD_OK;
    RFD_REQUIRE(psd_dev && refs_host && tmpl_host && ref_of_tmpl_host && taps_dev && lag_dev && sigma_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(k_host || (buckets_host && n_buckets >= 1), RFD_ERR_ARG,
                "give either k_host or a non-empty bucket list");
    RFD_REQUIRE(k_stride >= 1 && k_stride <= 4096 && k_stride <= g.n, RFD_ERR_SHAPE,
                "k_stride=%d out of [1, min(4096, n)]", k_stride);
    RFD_REQUIRE(std::isfinite(tukey_alpha) && tukey_alpha >= 0.0, RFD_ERR_ARG, "tukey_alpha must be >= 0");
    std::vector<int32_t> ref_of(ref_of_tmpl_host, ref_of_tmpl_host + n_tmpl), K, buckets;
    for (int32_t j = 0; j < n_tmpl; ++j)
        RFD_REQUIRE(ref_of[j] >= 0 && ref_of[j] < n_ref, RFD_ERR_ARG, "ref_of_tmpl[%d]=%d out of range", j, ref_of[j]);
    if (k_host) {
        K.assign(k_host, k_host + n_tmpl);
        for (int32_t j = 0; j < n_tmpl; ++j)
            RFD_REQUIRE(K[j] >= 1 && K[j] <= k_stride, RFD_ERR_SHAPE, "K[%d]=%d not in [1, k_stride]", j, K[j]);
    } else {
        RFD_REQUIRE(std::isfinite(energy_frac) && energy_frac > 0.0 && energy_frac <= 1.0, RFD_ERR_ARG,
                    "energy_frac must be in (0, 1]");
        buckets.assign(buckets_host, buckets_host + n_buckets);
        for (int32_t i = 0; i < n_buckets; ++i) {
            RFD_REQUIRE(buckets[i] >= 1 && buckets[i] <= k_stride, RFD_ERR_SHAPE, "bucket %d=%d not in [1, k_stride]",
                        i, buckets[i]);
            RFD_REQUIRE(i == 0 || buckets[i] > buckets[i - 1], RFD_ERR_ARG, "buckets must increase");
        }
    }
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<PNParams> refs, tmpl;
    RFD_TRY(make_pn_vec(g, refs_host, n_ref, &refs));
    RFD_TRY(make_pn_vec(g, tmpl_host, n_tmpl, &tmpl));
    for (int32_t r = 0; r < n_ref; ++r)
        RFD_REQUIRE(refs[r].k_hi >= g.k_lo, RFD_ERR_ARG, "reference %d has an empty band (ISCO below f_low)", r);
    return make_taps_impl(ctx, g, psd_dev, refs, tmpl, ref_of, K, buckets, {}, energy_frac, k_stride, tukey_alpha,
                          (float2 *)taps_dev, k_dev, lag_dev, sigma_dev, match_dev, (cudaStream_t)stream);
}

rfd_status rfd_make_taps_fit(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev, const rfd_params *refs_host,
                             int32_t n_ref, const rfd_params *tmpl_host, const int32_t *ref_of_tmpl_host,
                             int32_t n_tmpl, const int32_t *k_host, const int32_t *buckets_host, int32_t n_buckets,
                             double match_target, double ridge, int32_t k_stride, double tukey_alpha, void *taps_dev,
                             int32_t *k_dev, int32_t *lag_dev, double *sigma_dev, double *match_dev, void *stream) {
    NvtxRange nvtx_range("rfd_make_taps_fit");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_tmpl >= 0, RFD_ERR_SHAPE, "need n_ref >= 1 and n_tmpl >= 0");
    if (n_tmpl == 0) return RFD_OK;
    RFD_REQUIRE(psd_dev && refs_host && tmpl_host && ref_of_tmpl_host && taps_dev && lag_dev && sigma_dev && match_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(k_host || (buckets_host && n_buckets >= 1), RFD_ERR_ARG, "give either k_host or a non-empty bucket list");
    RFD_REQUIRE(std::isfinite(ridge) && ridge > 0.0 && ridge < 1.0, RFD_ERR_ARG, "ridge must be in (0, 1)");
    RFD_REQUIRE(k_stride >= 1 && k_stride <= 512 && k_stride <= g.n, RFD_ERR_SHAPE,
                "k_stride=%d out of [1, min(512, n)] for the fitted taps", k_stride);
    RFD_REQUIRE(std::isfinite(tukey_alpha) && tukey_alpha >= 0.0, RFD_ERR_ARG, "tukey_alpha must be >= 0");
    std::vector<int32_t> ref_of(ref_of_tmpl_host, ref_of_tmpl_host + n_tmpl), K, buckets;
    for (int32_t j = 0; j < n_tmpl; ++j)
        RFD_REQUIRE(ref_of[j] >= 0 && ref_of[j] < n_ref, RFD_ERR_ARG, "ref_of_tmpl[%d]=%d out of range", j, ref_of[j]);
    if (k_host) {
        K.assign(k_host, k_host + n_tmpl);
        for (int32_t j = 0; j < n_tmpl; ++j)
            RFD_REQUIRE(K[j] >= 1 && K[j] <= k_stride, RFD_ERR_SHAPE, "K[%d]=%d not in [1, k_stride]", j, K[j]);
    } else {
        RFD_REQUIRE(std::isfinite(match_target) && match_target <= 1.0, RFD_ERR_ARG, "match_target must be <= 1");
        buckets.assign(buckets_host, buckets_host + n_buckets);
        for (int32_t i = 0; i < n_buckets; ++i)
            RFD_REQUIRE(buckets[i] >= 1 && buckets[i] <= k_stride, RFD_ERR_SHAPE, "bucket %d=%d not in [1, k_stride]",
                        i, buckets[i]);
    }
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<PNParams> refs, tmpl;
    RFD_TRY(make_pn_vec(g, refs_host, n_ref, &refs));
    RFD_TRY(make_pn_vec(g, tmpl_host, n_tmpl, &tmpl));
    for (int32_t r = 0; r < n_ref; ++r)
        RFD_REQUIRE(refs[r].k_hi >= g.k_lo, RFD_ERR_ARG, "reference %d has an empty band (ISCO below f_low)", r);
    cudaStream_t s = (cudaStream_t)stream;
    if (k_host) {
        RFD_TRY(make_taps_impl(ctx, g, psd_dev, refs, tmpl, ref_of, K, {}, {}, 1.0, k_stride, tukey_alpha,
                               (float2 *)taps_dev, k_dev, lag_dev, sigma_dev, match_dev, s, ridge));
        return RFD_OK;
    }
    return make_taps_fit_dynamic(ctx, g, psd_dev, refs, tmpl, ref_of, buckets, match_target, ridge, k_stride,
                                 tukey_alpha, (float2 *)taps_dev, k_dev, lag_dev, sigma_dev, match_dev, s);
}

rfd_status rfd_make_taps_at_lag(rfd_ctx *ctx, const rfd_grid *grid, const double *psd_dev,
                                const rfd_params *refs_host, int32_t n_ref, const rfd_params *tmpl_host,
                                const int32_t *ref_of_tmpl_host, int32_t n_tmpl, const int32_t *k_host,
                                const int32_t *lag_host, int32_t k_stride, double tukey_alpha, void *taps_dev,
                                double *sigma_dev, double *match_dev, void *stream) {
    NvtxRange nvtx_range("rfd_make_taps_at_lag");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_tmpl >= 0, RFD_ERR_SHAPE, "need n_ref >= 1 and n_tmpl >= 0");
    if (n_tmpl == 0) return RFD_OK;
    RFD_REQUIRE(psd_dev && refs_host && tmpl_host && ref_of_tmpl_host && k_host && lag_host && taps_dev && sigma_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(k_stride >= 1 && k_stride <= 4096 && k_stride <= g.n, RFD_ERR_SHAPE,
                "k_stride=%d out of [1, min(4096, n)]", k_stride);
    RFD_REQUIRE(std::isfinite(tukey_alpha) && tukey_alpha >= 0.0, RFD_ERR_ARG, "tukey_alpha must be >= 0");
    std::vector<int32_t> ref_of(ref_of_tmpl_host, ref_of_tmpl_host + n_tmpl), K(k_host, k_host + n_tmpl),
        lag(lag_host, lag_host + n_tmpl);
    for (int32_t j = 0; j < n_tmpl; ++j) {
        RFD_REQUIRE(ref_of[j] >= 0 && ref_of[j] < n_ref, RFD_ERR_ARG, "ref_of_tmpl[%d]=%d out of range", j, ref_of[j]);
        RFD_REQUIRE(K[j] >= 1 && K[j] <= k_stride, RFD_ERR_SHAPE, "K[%d]=%d not in [1, k_stride]", j, K[j]);
        RFD_REQUIRE(lag[j] >= -(g.n / 2) && lag[j] < g.n / 2, RFD_ERR_ARG, "lag[%d]=%d not in [-n/2, n/2)", j, lag[j]);
    }
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<PNParams> refs, tmpl;
    RFD_TRY(make_pn_vec(g, refs_host, n_ref, &refs));
    RFD_TRY(make_pn_vec(g, tmpl_host, n_tmpl, &tmpl));
    for (int32_t r = 0; r < n_ref; ++r)
        RFD_REQUIRE(refs[r].k_hi >= g.k_lo, RFD_ERR_ARG, "reference %d has an empty band (ISCO below f_low)", r);
    // the placed lag is written back; it equals lag_host
    RFD_TRY(ensure(ctx->ws[12], (size_t)n_tmpl * sizeof(int32_t)));
    int32_t *lag_dev = (int32_t *)ctx->ws[12].p;
    return make_taps_impl(ctx, g, psd_dev, refs, tmpl, ref_of, K, {}, lag, 1.0, k_stride, tukey_alpha,
                          (float2 *)taps_dev, nullptr, lag_dev, sigma_dev, match_dev, (cudaStream_t)stream);
}

rfd_status rfd_filter_reference(rfd_ctx *ctx, const rfd_grid *grid, const void *dtilde_dev,
                                const double *psd_dev, const void *href_dev, int32_t n_ref, int32_t halo,
                                int32_t precision, void *qref_dev, int32_t *qscale_dev, void *stream) {
    NvtxRange nvtx_range("rfd_filter_reference");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 0, RFD_ERR_SHAPE, "n_ref < 0");
    if (n_ref == 0) return RFD_OK;
    RFD_REQUIRE(dtilde_dev && psd_dev && href_dev && qref_dev && qscale_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(halo >= 0 && halo < g.n, RFD_ERR_SHAPE, "halo=%d must be in [0, n)", halo);
    RFD_REQUIRE(precision >= RFD_PREC_FP32 && precision <= RFD_PREC_BF16X3, RFD_ERR_ARG, "bad precision %d",
                precision);
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    return filter_reference_impl(ctx, g, (const float2 *)dtilde_dev, psd_dev, (const float2 *)href_dev, n_ref, halo,
                                 precision, qref_dev, qscale_dev, (cudaStream_t)stream);
}

rfd_status rfd_plan_create(rfd_ctx *ctx, const rfd_grid *grid, int32_t n_ref, int32_t n_tmpl,
                           const int32_t *ref_of_tmpl_host, const int32_t *k_host, int32_t precision,
                           int32_t window, float threshold, int32_t halo, rfd_plan **out) {
    return rfd_plan_create_ex(ctx, grid, n_ref, n_tmpl, ref_of_tmpl_host, k_host, precision, window, threshold,
                              halo, nullptr, out);
}

void rfd_plan_options_default(rfd_plan_options *o) {
    if (!o) return;
    *o = rfd_plan_options{};
    o->tile_nt[0] = 128;
    o->tile_nt[1] = 64;
    o->tile_nt[2] = 32;
    o->mix_k = 1;
    o->grid_ctas = 0;
    o->long_k = 64;
    o->fft_k = 4096;
    o->fft_rem = 0;
    o->debug_flags = 0;
}

rfd_status rfd_plan_create_ex(rfd_ctx *ctx, const rfd_grid *grid, int32_t n_ref, int32_t n_tmpl,
                              const int32_t *ref_of_tmpl_host, const int32_t *k_host, int32_t precision,
                              int32_t window, float threshold, int32_t halo, const rfd_plan_options *options,
                              rfd_plan **out) {
    NvtxRange nvtx_range("rfd_plan_create_ex");
    rfd_plan_options opt;
    rfd_plan_options_default(&opt);
    if (options) opt = *options;
    {
        static const int32_t cap[3] = {128, 64, 32};
        for (int c = 0; c < 3; ++c)
            RFD_REQUIRE(opt.tile_nt[c] >= 16 && opt.tile_nt[c] <= cap[c] && opt.tile_nt[c] % 16 == 0, RFD_ERR_ARG,
                        "tile_nt[%d]=%d must be a multiple of 16 in [16, %d]", c, opt.tile_nt[c], cap[c]);
        RFD_REQUIRE(opt.grid_ctas >= 0, RFD_ERR_ARG, "grid_ctas must be >= 0");
        RFD_REQUIRE(opt.long_k >= 0 && opt.long_k <= 512, RFD_ERR_ARG, "long_k must be in [0, 512]");
        RFD_REQUIRE(opt.fft_k >= 0 && opt.fft_k <= 4096, RFD_ERR_ARG, "fft_k must be in [0, 4096]");
        RFD_REQUIRE(opt.out_len >= 0 && opt.out_len % 512 == 0, RFD_ERR_ARG,
                    "out_len=%d must be 0 or a positive multiple of 512", opt.out_len);
        RFD_REQUIRE(opt.fft_rem >= 0 && opt.fft_rem < 64, RFD_ERR_ARG, "fft_rem must be in [0, 63]");
        RFD_REQUIRE((opt.debug_flags & ~RFD_DEBUG_STALL_TAPS) == 0, RFD_ERR_ARG, "unknown debug_flags bits");
    }
    RFD_REQUIRE(ctx && out, RFD_ERR_ARG, "NULL ctx or out");
    *out = nullptr;
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_ref >= 1 && n_tmpl >= 1, RFD_ERR_SHAPE, "need n_ref >= 1 and n_tmpl >= 1");
    RFD_REQUIRE(ref_of_tmpl_host && k_host, RFD_ERR_ARG, "NULL ref_of or k");
    RFD_REQUIRE(window >= 1, RFD_ERR_ARG, "window must be >= 1");
    RFD_REQUIRE(std::isfinite(threshold) && threshold >= 0.f, RFD_ERR_ARG, "threshold must be finite, >= 0");
    RFD_REQUIRE(precision >= RFD_PREC_FP32 && precision <= RFD_PREC_BF16X3, RFD_ERR_ARG, "bad precision");
    int32_t kmax = 0;
    for (int32_t j = 0; j < n_tmpl; ++j) {
        RFD_REQUIRE(ref_of_tmpl_host[j] >= 0 && ref_of_tmpl_host[j] < n_ref, RFD_ERR_ARG,
                    "ref_of_tmpl[%d] out of range", j);
        RFD_REQUIRE(k_host[j] >= 1 && k_host[j] <= 4096, RFD_ERR_SHAPE, "K[%d]=%d out of [1, 4096]", j, k_host[j]);
        RFD_REQUIRE(precision == RFD_PREC_FP32 || k_host[j] <= 512, RFD_ERR_UNSUPPORTED,
                    "K[%d]=%d: the tensor-core path supports K <= 512", j, k_host[j]);
        kmax = std::max(kmax, k_host[j]);
    }
    RFD_REQUIRE(halo >= kmax - 1 && halo < g.n, RFD_ERR_SHAPE, "halo=%d must be >= max K - 1 = %d and < n",
                halo, kmax - 1);
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    rfd_plan *p = new rfd_plan();
    p->ctx = ctx;
    p->grid = g;
    p->n_ref = n_ref;
    p->n_tmpl = n_tmpl;
    p->precision = precision;
    p->window = window;
    p->threshold = threshold;
    p->halo = halo;
    p->ld = rfd_qref_ld(g.n, halo);
    RFD_REQUIRE(opt.out_len <= g.n && (opt.out_len == 0 || g.n % 512 == 0), RFD_ERR_SHAPE,
                "out_len=%d must be <= n=%lld, and n a multiple of 512 for a window", opt.out_len, (long long)g.n);
    p->out_len = opt.out_len > 0 ? opt.out_len : g.n;
    p->k_max = kmax;
    p->ref_of.assign(ref_of_tmpl_host, ref_of_tmpl_host + n_tmpl);
    p->k_of.assign(k_host, k_host + n_tmpl);
    // tiles: per reference, templates ordered by K (stable)
    std::vector<int32_t> order(n_tmpl);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (p->ref_of[a] != p->ref_of[b]) return p->ref_of[a] < p->ref_of[b];
        return p->k_of[a] < p->k_of[b];
    });
    // templates with fft_k < K <= 1024 go to the block-FFT path
    std::vector<int32_t> order_fft, order_rest;
    for (int32_t j : order) (p->k_of[j] > opt.fft_k && p->k_of[j] <= 1024 ? order_fft : order_rest).push_back(j);
    if (precision != RFD_PREC_FP32 && opt.fft_rem > 0) {
        // per reference, the long-tap kernel's last partial tile (its largest-K templates) goes
        // to the block-FFT kernel when it holds at most fft_rem templates
        const int32_t nt = tl_tile_templates();
        std::vector<int32_t> keep;
        size_t i = 0;
        while (i < order_rest.size()) {
            const int32_t r = p->ref_of[order_rest[i]];
            size_t e = i;
            while (e < order_rest.size() && p->ref_of[order_rest[e]] == r) ++e;
            std::vector<int32_t> lng;
            for (size_t q = i; q < e; ++q) {
                const int32_t j = order_rest[q];
                if (p->k_of[j] > opt.long_k) lng.push_back(j); else keep.push_back(j);
            }
            const int32_t rem = (int32_t)(lng.size() % (size_t)nt);
            const bool move = rem > 0 && rem <= opt.fft_rem && p->k_of[lng.back()] <= 1024;
            for (size_t q = 0; q < lng.size(); ++q)
                (move && q >= lng.size() - (size_t)rem ? order_fft : keep).push_back(lng[q]);
            i = e;
        }
        order_rest.swap(keep);
        std::stable_sort(order_rest.begin(), order_rest.end(), [&](int32_t a, int32_t b) {
            if (p->ref_of[a] != p->ref_of[b]) return p->ref_of[a] < p->ref_of[b];
            return p->k_of[a] < p->k_of[b];
        });
        std::stable_sort(order_fft.begin(), order_fft.end(), [&](int32_t a, int32_t b) {
            if (p->ref_of[a] != p->ref_of[b]) return p->ref_of[a] < p->ref_of[b];
            return p->k_of[a] < p->k_of[b];
        });
    }
    p->debug_flags = opt.debug_flags;
    order.swap(order_rest);
    if (precision != RFD_PREC_FP32) {
        rfd_status st = plan_tc_tiles(p, order, ctx->num_sms, opt);
        if (st == RFD_OK) st = plan_fft_tiles(p, order_fft, ctx->num_sms, opt);
        if (st == RFD_OK) p->n_slots = (int64_t)p->perm.size();
        if (st == RFD_OK) {
            do {
                if ((st = ensure(p->d_perm, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
                if ((st = ensure(p->d_kslot, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
                if ((st = ensure(p->d_off, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
                if ((st = ensure(p->d_scale, p->n_slots * sizeof(float))) != RFD_OK) break;
                std::vector<int32_t> kslot(p->n_slots);
                for (int64_t s2 = 0; s2 < p->n_slots; ++s2) kslot[s2] = p->k_of[p->perm[s2]];
                cudaError_t e1 = cudaMemcpy(p->d_perm.p, p->perm.data(), p->n_slots * sizeof(int32_t),
                                            cudaMemcpyHostToDevice);
                cudaError_t e2 = cudaMemcpy(p->d_kslot.p, kslot.data(), p->n_slots * sizeof(int32_t),
                                            cudaMemcpyHostToDevice);
                if (e1 != cudaSuccess || e2 != cudaSuccess) {
                    set_error("plan upload failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
                    st = RFD_ERR_CUDA;
                }
            } while (0);
        }
        if (st != RFD_OK) {
            rfd_plan_destroy(p);
            return st;
        }
        *out = p;
        return RFD_OK;
    }
    p->tile_j = fir32_tile_templates();
    int32_t slot = 0;
    for (size_t i = 0; i < order.size();) {
        const int32_t r = p->ref_of[order[i]];
        size_t e = i;
        while (e < order.size() && p->ref_of[order[e]] == r && (int32_t)(e - i) < p->tile_j) ++e;
        RfdTile t;
        t.ref = r;
        t.first = slot;
        t.count = (int32_t)(e - i);
        t.k_tile = 0;
        for (size_t q = i; q < e; ++q) {
            t.k_tile = std::max(t.k_tile, p->k_of[order[q]]);
            p->perm.push_back(order[q]);
        }
        slot += t.count;
        p->tiles.push_back(t);
        p->executed_flops += 8.0 * t.k_tile * (double)p->tile_j * (double)p->out_len;
        i = e;
    }
    rfd_status st = plan_fft_tiles(p, order_fft, ctx->num_sms, opt);
    p->n_slots = (int64_t)p->perm.size();
    do {
        if (st != RFD_OK) break;
        if ((st = ensure(p->d_tiles, p->tiles.size() * sizeof(RfdTile))) != RFD_OK) break;
        if ((st = ensure(p->d_perm, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
        if ((st = ensure(p->d_kslot, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
        if ((st = ensure(p->d_off, p->n_slots * sizeof(int32_t))) != RFD_OK) break;
        if ((st = ensure(p->d_scale, p->n_slots * sizeof(float))) != RFD_OK) break;
        if ((st = ensure(p->d_taps, (size_t)p->n_slots * p->k_max * sizeof(float2))) != RFD_OK) break;
        std::vector<int32_t> kslot(p->n_slots);
        for (int64_t s = 0; s < p->n_slots; ++s) kslot[s] = p->k_of[p->perm[s]];
        cudaError_t e1 = cudaMemcpy(p->d_tiles.p, p->tiles.data(), p->tiles.size() * sizeof(RfdTile),
                                    cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(p->d_perm.p, p->perm.data(), p->n_slots * sizeof(int32_t),
                                    cudaMemcpyHostToDevice);
        cudaError_t e3 = cudaMemcpy(p->d_kslot.p, kslot.data(), p->n_slots * sizeof(int32_t),
                                    cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            set_error("plan upload failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
            st = RFD_ERR_CUDA;
        }
    } while (0);
    if (st != RFD_OK) {
        rfd_plan_destroy(p);
        return st;
    }
    *out = p;
    return RFD_OK;
}

void rfd_plan_destroy(rfd_plan *plan) {
    if (!plan) return;
    cudaSetDevice(plan->ctx->device);
    cudaDeviceSynchronize();
    release(plan->d_tiles);
    release(plan->d_perm);
    release(plan->d_taps);
    release(plan->d_off);
    release(plan->d_scale);
    release(plan->d_kslot);
    release(plan->d_ranges);
    release(plan->d_tl_tiles);
    release(plan->d_tl_ranges);
    release(plan->d_tl_taps);
    release(plan->d_fft_tiles);
    release(plan->d_fft_ranges);
    release(plan->d_fft_refs);
    release(plan->d_fft_P);
    release(plan->d_fft_X);
    delete plan;
}

rfd_status rfd_plan_set_taps(rfd_plan *plan, const void *taps_dev, int32_t k_stride, const int32_t *lag_dev,
                             const double *sigma_dev, void *stream) {
    NvtxRange nvtx_range("rfd_plan_set_taps");
    RFD_REQUIRE(plan, RFD_ERR_ARG, "plan is NULL");
    RFD_REQUIRE(taps_dev && lag_dev && sigma_dev, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(k_stride >= plan->k_max, RFD_ERR_SHAPE, "k_stride=%d < max K=%d", k_stride, plan->k_max);
    RFD_TRY_CUDA(cudaSetDevice(plan->ctx->device));
    if (plan->precision == RFD_PREC_FP32)
        RFD_TRY(pack_taps_fp32(plan, (const float2 *)taps_dev, k_stride, lag_dev, sigma_dev, (cudaStream_t)stream));
    else {
        RFD_TRY(tc_pack(plan, (const float2 *)taps_dev, k_stride, lag_dev, sigma_dev, (cudaStream_t)stream));
        RFD_TRY(tl_pack(plan, (const float2 *)taps_dev, k_stride, lag_dev, sigma_dev, (cudaStream_t)stream));
    }
    RFD_TRY(fft_pack(plan, (const float2 *)taps_dev, k_stride, lag_dev, sigma_dev, (cudaStream_t)stream));
    plan->taps_set = true;
    return RFD_OK;
}

}  // extern "C"

namespace rfd {
// Every filtering kernel of a plan, in order, on one stream (the call and the search graph
// both go through here).
rfd_status ratio_filter_enqueue(const rfd_plan *plan, const void *q, const int32_t *qscale, const int64_t *u_begin,
                                rfd_candidate *cand, int64_t cap, int64_t *count, cudaStream_t s) {
    if (plan->precision == RFD_PREC_FP32) {
        RFD_TRY(fir32_launch(plan, (const float2 *)q, u_begin, cand, cap, count, s));
    } else {
        RFD_TRY(tc_launch(plan, q, qscale, u_begin, cand, cap, count, s));
        RFD_TRY(tl_launch(plan, q, qscale, u_begin, cand, cap, count, s));
    }
    return fft_launch(plan, q, qscale, u_begin, cand, cap, count, s);
}
}  // namespace rfd

extern "C" {

rfd_status rfd_ratio_filter_batch(rfd_plan *plan, const void *qref_dev, const int32_t *qscale_dev,
                                  rfd_candidate *cand_dev, int64_t cand_capacity, int64_t *cand_count_dev,
                                  void *stream) {
    NvtxRange nvtx_range("rfd_ratio_filter_batch");
    RFD_REQUIRE(plan, RFD_ERR_ARG, "plan is NULL");
    RFD_REQUIRE(plan->taps_set, RFD_ERR_ARG, "rfd_plan_set_taps has not been called");
    RFD_REQUIRE(qref_dev && cand_count_dev && (cand_dev || cand_capacity == 0), RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(cand_capacity >= 0, RFD_ERR_SHAPE, "negative capacity");
    RFD_REQUIRE(plan->precision == RFD_PREC_FP32 || qscale_dev, RFD_ERR_ARG, "qscale_dev is NULL");
    RFD_TRY_CUDA(cudaSetDevice(plan->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY_CUDA(cudaMemsetAsync(cand_count_dev, 0, sizeof(int64_t), s));
    return ratio_filter_enqueue(plan, qref_dev, qscale_dev, nullptr, cand_dev, cand_capacity, cand_count_dev, s);
}

rfd_status rfd_ratio_filter_window(rfd_plan *plan, const void *qref_dev, const int32_t *qscale_dev,
                                   const int64_t *u_begin_dev, rfd_candidate *cand_dev, int64_t cand_capacity,
                                   int64_t *cand_count_dev, void *stream) {
    NvtxRange nvtx_range("rfd_ratio_filter_window");
    RFD_REQUIRE(plan, RFD_ERR_ARG, "plan is NULL");
    RFD_REQUIRE(plan->taps_set, RFD_ERR_ARG, "rfd_plan_set_taps has not been called");
    RFD_REQUIRE(qref_dev && u_begin_dev && cand_count_dev && (cand_dev || cand_capacity == 0), RFD_ERR_ARG,
                "NULL argument");
    RFD_REQUIRE(cand_capacity >= 0, RFD_ERR_SHAPE, "negative capacity");
    RFD_REQUIRE(plan->precision == RFD_PREC_FP32 || qscale_dev, RFD_ERR_ARG, "qscale_dev is NULL");
    RFD_TRY_CUDA(cudaSetDevice(plan->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY_CUDA(cudaMemsetAsync(cand_count_dev, 0, sizeof(int64_t), s));
    return ratio_filter_enqueue(plan, qref_dev, qscale_dev, u_begin_dev, cand_dev, cand_capacity, cand_count_dev, s);
}

double rfd_plan_executed_flops(const rfd_plan *plan) { return plan ? plan->executed_flops : 0.0; }

rfd_status rfd_plan_template_kernels(const rfd_plan *plan, int32_t *kernel_host) {
    RFD_REQUIRE(plan && kernel_host, RFD_ERR_ARG, "NULL argument");
    for (int32_t j = 0; j < plan->n_tmpl; ++j) kernel_host[j] = -1;
    auto mark = [&](int32_t first, int32_t count, int32_t kind) {
        for (int32_t a = 0; a < count; ++a) kernel_host[plan->perm[first + a]] = kind;
    };
    for (const RfdTile &t : plan->tiles) mark(t.first, t.count, RFD_KERNEL_FP32);
    for (const TcTile &t : plan->tc_tiles) mark(t.first, t.count, RFD_KERNEL_TC_TIME_ON_M);
    for (const TcTile &t : plan->tl_tiles) mark(t.first, t.count, RFD_KERNEL_TC_TEMPLATES_ON_M);
    for (const FftTile &t : plan->fft_tiles) mark(t.first, t.count, RFD_KERNEL_BLOCK_FFT);
    for (int32_t j = 0; j < plan->n_tmpl; ++j)
        RFD_REQUIRE(kernel_host[j] >= 0, RFD_ERR_ARG, "template %d is in no tile (internal error)", j);
    return RFD_OK;
}

rfd_status rfd_find_triggers(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand_dev,
                             const int64_t *cand_count_dev, int64_t cand_capacity, rfd_trigger *trig_dev,
                             int64_t trig_capacity, int64_t *n_trig_host, void *stream) {
    NvtxRange nvtx_range("rfd_find_triggers");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    RFD_REQUIRE(n_tmpl >= 1, RFD_ERR_SHAPE, "n_tmpl must be >= 1");
    RFD_REQUIRE(cand_count_dev && n_trig_host && (cand_dev || cand_capacity == 0) &&
                    (trig_dev || trig_capacity == 0),
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(cand_capacity >= 0 && trig_capacity >= 0, RFD_ERR_SHAPE, "negative capacity");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    return find_triggers_impl(ctx, n_tmpl, cand_dev, cand_count_dev, cand_capacity, trig_dev, trig_capacity,
                              n_trig_host, (cudaStream_t)stream);
}

rfd_status rfd_findchirp(rfd_ctx *ctx, const rfd_grid *grid, const void *dtilde_dev, const double *psd_dev,
                         const void *h_dev, int32_t n_tmpl, int32_t window, float threshold,
                         rfd_candidate *cand_dev, int64_t cand_capacity, int64_t *cand_count_dev, void *stream) {
    NvtxRange nvtx_range("rfd_findchirp");
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    Grid g;
    RFD_TRY(check_grid(grid, &g));
    RFD_REQUIRE(n_tmpl >= 1, RFD_ERR_SHAPE, "n_tmpl must be >= 1");
    RFD_REQUIRE(dtilde_dev && psd_dev && h_dev && cand_count_dev && (cand_dev || cand_capacity == 0), RFD_ERR_ARG,
                "NULL argument");
    RFD_REQUIRE(window >= 1 && std::isfinite(threshold) && threshold >= 0.f, RFD_ERR_ARG, "bad window/threshold");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    return findchirp_impl(ctx, g, (const float2 *)dtilde_dev, psd_dev, (const float2 *)h_dev, n_tmpl, window,
                          threshold, cand_dev, cand_capacity, cand_count_dev, (cudaStream_t)stream);
}

rfd_status rfd_ifft_c2c(rfd_ctx *ctx, int64_t n, int32_t batch, const void *in_dev, void *out_dev, void *stream) {
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    RFD_REQUIRE(n >= 4 && n <= (int64_t(1) << 24) && (n & (n - 1)) == 0, RFD_ERR_SHAPE, "n must be a power of two");
    RFD_REQUIRE(batch >= 0, RFD_ERR_SHAPE, "batch < 0");
    if (batch == 0) return RFD_OK;
    RFD_REQUIRE(in_dev && out_dev && in_dev != out_dev, RFD_ERR_ARG, "NULL or aliased buffers");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    RFD_TRY(ensure(ctx->ws[14], (size_t)batch * n * sizeof(float2)));
    return fft_c2c<float>(ctx, n, batch, (const float2 *)in_dev, n, (float2 *)out_dev, n, (float2 *)ctx->ws[14].p,
                          true, (cudaStream_t)stream);
}

rfd_status rfd_fft_c2c(rfd_ctx *ctx, int64_t n, int32_t batch, int32_t fp64, int32_t inverse, const void *in_dev,
                       void *out_dev, void *stream) {
    RFD_REQUIRE(ctx, RFD_ERR_ARG, "ctx is NULL");
    RFD_REQUIRE(n >= 4 && n <= (int64_t(1) << 24) && (n & (n - 1)) == 0, RFD_ERR_SHAPE, "n must be a power of two");
    RFD_REQUIRE(batch >= 0, RFD_ERR_SHAPE, "batch < 0");
    RFD_REQUIRE(fp64 == 0 || fp64 == 1, RFD_ERR_ARG, "fp64 must be 0 or 1");
    RFD_REQUIRE(inverse == 0 || inverse == 1, RFD_ERR_ARG, "inverse must be 0 or 1");
    if (batch == 0) return RFD_OK;
    RFD_REQUIRE(in_dev && out_dev && in_dev != out_dev, RFD_ERR_ARG, "NULL or aliased buffers");
    RFD_TRY_CUDA(cudaSetDevice(ctx->device));
    if (fp64) {
        RFD_TRY(ensure(ctx->ws[14], (size_t)batch * n * sizeof(double2)));
        return fft_c2c<double>(ctx, n, batch, (const double2 *)in_dev, n, (double2 *)out_dev, n,
                               (double2 *)ctx->ws[14].p, inverse != 0, (cudaStream_t)stream);
    }
    RFD_TRY(ensure(ctx->ws[14], (size_t)batch * n * sizeof(float2)));
    return fft_c2c<float>(ctx, n, batch, (const float2 *)in_dev, n, (float2 *)out_dev, n, (float2 *)ctx->ws[14].p,
                          inverse != 0, (cudaStream_t)stream);
}

}  // extern "C"
