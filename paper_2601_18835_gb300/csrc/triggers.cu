// find_triggers: candidates -> one trigger per (template, window), sorted by (j, w).
// Table II's "trigger accumulation".  Integer keys only, so the result does not depend on
// the order in which candidates were appended.
//
//   1. count candidates per template;  2. exclusive scan -> bucket offsets;
//   3. scatter into per-template buckets;
//   4. per template, pick each window's winner (largest key = largest |z|^2, ties to the
//      smallest t) and its rank among the template's winners in window order: a warp per
//      template when it has at most 32 candidates (every lane compares its candidate with the
//      others), else a block per template that takes the windows in ranges of kRange through
//      shared-memory tables (key maximum, then the smallest bucket index holding it, then an
//      occupancy scan for the ranks), O(c) per range;
//   5. exclusive scan of the winner counts -> trigger offsets;  6. each winner writes itself
//      at its template's offset plus its rank.
// A winner keeps its rank in the bucket entry's j field (the bucket already names the
// template); a losing entry gets bit 31 of its window index set.
#include <algorithm>

#include "internal.cuh"

namespace rfd {

namespace {

// A filtering kernel whose bounded wait gave up sets bit 62 of the candidate count.
constexpr int64_t kTimeoutBit = (int64_t)1 << 62;
constexpr int64_t kCountMask = kTimeoutBit - 1;

__global__ void k_count(const rfd_candidate *__restrict__ c, const int64_t *__restrict__ count,
                        int64_t cap, int32_t n_tmpl, int32_t *__restrict__ cnt,
                        int32_t *__restrict__ bad) {
    const int64_t nc = min(*count & kCountMask, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = c[i].j;
        if (j < (uint32_t)n_tmpl) atomicAdd(&cnt[j], 1);
        else atomicAdd(bad, 1);
    }
}

// Exclusive scan of int32 counts into int64 offsets with one block; out[n] = total.
__global__ void k_scan(const int32_t *__restrict__ in, int32_t n, int64_t *__restrict__ out) {
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int32_t per = (n + nt - 1) / nt;
    const int32_t b = min(n, tid * per), e = min(n, b + per);
    int64_t s = 0;
    for (int32_t i = b; i < e; ++i) s += in[i];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {       // inclusive Hillis-Steele
        const int64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t run = tid ? part[tid - 1] : 0;
    for (int32_t i = b; i < e; ++i) {
        out[i] = run;
        run += in[i];
    }
    if (tid == nt - 1) out[n] = part[nt - 1];
}

__global__ void k_scatter(const rfd_candidate *__restrict__ c, const int64_t *__restrict__ count,
                          int64_t cap, int32_t n_tmpl, const int64_t *__restrict__ off,
                          int32_t *__restrict__ cur, rfd_candidate *__restrict__ bucket) {
    const int64_t nc = min(*count & kCountMask, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const rfd_candidate v = c[i];
        if (v.j >= (uint32_t)n_tmpl) continue;
        const int32_t p = atomicAdd(&cur[v.j], 1);
        bucket[off[v.j] + p] = v;
    }
}

constexpr uint32_t kLoser = 0x80000000u;
constexpr int kRange = 2048;              // windows per shared-memory pass of the block merge
constexpr int kMergeThreads = 256;

// Step 4 for templates with at most 32 candidates (one warp each); larger ones are listed in
// big[] for k_merge_big.
__global__ void k_merge_small(rfd_candidate *__restrict__ bucket, const int64_t *__restrict__ off, int32_t n_tmpl,
                              int32_t *__restrict__ ntrig, int32_t *__restrict__ big, int32_t *__restrict__ nbig) {
    const int32_t j = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_tmpl) return;
    const int64_t b = off[j];
    const int64_t c = off[j + 1] - b;
    if (c > 32) {
        if (lane == 0) big[atomicAdd(nbig, 1)] = j;
        return;
    }
    const bool have = lane < c;
    uint32_t w = 0xffffffffu;
    unsigned long long key = 0ull;
    if (have) {
        w = bucket[b + lane].w;
        key = bucket[b + lane].key;
    }
    bool beaten = false;
    for (int k = 0; k < (int)c; ++k) {
        const uint32_t wk = __shfl_sync(0xffffffffu, w, k);
        const unsigned long long kk = __shfl_sync(0xffffffffu, key, k);
        beaten |= wk == w && (kk > key || (kk == key && k < lane));
    }
    const bool win = have && !beaten;
    const unsigned winners = __ballot_sync(0xffffffffu, win);
    uint32_t rank = 0;
    for (int k = 0; k < (int)c; ++k) {
        const uint32_t wk = __shfl_sync(0xffffffffu, w, k);
        rank += ((winners >> k) & 1u) && wk < w;
    }
    if (have) {
        if (win)
            bucket[b + lane].j = rank;
        else
            bucket[b + lane].w = w | kLoser;
    }
    if (lane == 0) ntrig[j] = __popc(winners);
}

// Step 4 for the listed templates with more than 32 candidates: one block per template (a
// block loops over the list), windows [wmin, wmax] in ranges of kRange.
__global__ void __launch_bounds__(kMergeThreads) k_merge_big(rfd_candidate *__restrict__ bucket,
                                                             const int64_t *__restrict__ off,
                                                             int32_t *__restrict__ ntrig,
                                                             const int32_t *__restrict__ big,
                                                             const int32_t *__restrict__ nbig) {
    __shared__ unsigned long long s_key[kRange];
    __shared__ uint32_t s_idx[kRange];
    __shared__ uint32_t s_part[kMergeThreads];
    __shared__ uint32_t s_wmin, s_wmax;
    constexpr int kPer = kRange / kMergeThreads;
    const int tid = threadIdx.x;
    const int32_t nb = *nbig;
    for (int32_t bi = blockIdx.x; bi < nb; bi += gridDim.x) {
        const int32_t j = big[bi];
        const int64_t b = off[j];
        const int64_t c = off[j + 1] - b;
        if (tid == 0) {
            s_wmin = 0xffffffffu;
            s_wmax = 0u;
        }
        __syncthreads();
        uint32_t lmin = 0xffffffffu, lmax = 0u;
        for (int64_t i = tid; i < c; i += kMergeThreads) {
            const uint32_t w = bucket[b + i].w;
            lmin = min(lmin, w);
            lmax = max(lmax, w);
        }
        atomicMin(&s_wmin, lmin);
        atomicMax(&s_wmax, lmax);
        __syncthreads();
        const uint32_t wmin = s_wmin, wmax = s_wmax;
        uint32_t running = 0;
        for (uint64_t w0 = wmin; w0 <= wmax; w0 += kRange) {
            for (int x = tid; x < kRange; x += kMergeThreads) {
                s_key[x] = 0ull;
                s_idx[x] = 0xffffffffu;
            }
            __syncthreads();
            for (int64_t i = tid; i < c; i += kMergeThreads) {
                const uint64_t d = (uint64_t)bucket[b + i].w - w0;
                if (d < (uint64_t)kRange) atomicMax(&s_key[d], (unsigned long long)bucket[b + i].key);
            }
            __syncthreads();
            for (int64_t i = tid; i < c; i += kMergeThreads) {
                const uint64_t d = (uint64_t)bucket[b + i].w - w0;
                if (d < (uint64_t)kRange && bucket[b + i].key == s_key[d]) atomicMin(&s_idx[d], (uint32_t)i);
            }
            __syncthreads();
            // ranks: exclusive scan of the occupied windows of this range
            uint32_t local = 0;
#pragma unroll
            for (int q = 0; q < kPer; ++q) local += s_idx[tid * kPer + q] != 0xffffffffu;
            s_part[tid] = local;
            __syncthreads();
            for (int o = 1; o < kMergeThreads; o <<= 1) {
                const uint32_t v = tid >= o ? s_part[tid - o] : 0u;
                __syncthreads();
                s_part[tid] += v;
                __syncthreads();
            }
            const uint32_t total = s_part[kMergeThreads - 1];
            // rewrite s_key[x] as the rank of window w0 + x among this range's winners
            uint32_t r = s_part[tid] - local;
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int x = tid * kPer + q;
                s_key[x] = r;
                r += s_idx[x] != 0xffffffffu;
            }
            __syncthreads();
            for (int64_t i = tid; i < c; i += kMergeThreads) {
                const uint32_t w = bucket[b + i].w;
                const uint64_t d = (uint64_t)w - w0;
                if (d >= (uint64_t)kRange) continue;
                if (s_idx[d] == (uint32_t)i)
                    bucket[b + i].j = running + (uint32_t)s_key[d];
                else
                    bucket[b + i].w = w | kLoser;
            }
            running += total;
            __syncthreads();
        }
        if (tid == 0) ntrig[j] = (int32_t)running;
        __syncthreads();
    }
}

// Step 6: a warp per template writes its winners at toff[j] + rank.
__global__ void k_write(const rfd_candidate *__restrict__ bucket, const int64_t *__restrict__ off,
                        const int64_t *__restrict__ toff, int32_t n_tmpl, int64_t trig_cap,
                        rfd_trigger *__restrict__ trig) {
    const int32_t j = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_tmpl) return;
    const int64_t b = off[j], e = off[j + 1], o = toff[j];
    for (int64_t i = b + lane; i < e; i += 32) {
        const rfd_candidate c = bucket[i];
        if (c.w & kLoser) continue;
        const int64_t at = o + (int64_t)c.j;
        if (at < trig_cap) {
            rfd_trigger t;
            t.j = j;
            t.t = (int32_t)(0xffffffffu - (uint32_t)(c.key & 0xffffffffull));
            t.snr2 = __uint_as_float((uint32_t)(c.key >> 32));
            t.zr = c.zr;
            t.zi = c.zi;
            trig[at] = t;
        }
    }
}

// Steps 1-6 on caller-given scratch.  i32: cnt[J] cur[J] ntrig[J] big[J] bad nbig, zeroed
// here; off, toff: int64 [J + 1]; bucket: cap candidates.
rfd_status merge_enqueue(int32_t n_tmpl, const rfd_candidate *cand, const int64_t *cand_count, int64_t cap,
                         rfd_trigger *trig, int64_t trig_cap, int32_t *i32, int64_t *off, int64_t *toff,
                         rfd_candidate *bucket, int merge_blocks, cudaStream_t s) {
    const size_t J = (size_t)n_tmpl;
    int32_t *cnt = i32, *cur = cnt + J, *ntrig = cur + J, *big = ntrig + J, *bad = big + J, *nbig = bad + 1;
    RFD_TRY_CUDA(cudaMemsetAsync(i32, 0, (4 * J + 2) * sizeof(int32_t), s));
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, (cap + 255) / 256));
    const unsigned gw = (unsigned)((J * 32 + 255) / 256);
    k_count<<<gb, 256, 0, s>>>(cand, cand_count, cap, n_tmpl, cnt, bad);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(cnt, n_tmpl, off);
    RFD_LAUNCH_CHECK();
    k_scatter<<<gb, 256, 0, s>>>(cand, cand_count, cap, n_tmpl, off, cur, bucket);
    RFD_LAUNCH_CHECK();
    k_merge_small<<<gw, 256, 0, s>>>(bucket, off, n_tmpl, ntrig, big, nbig);
    RFD_LAUNCH_CHECK();
    k_merge_big<<<(unsigned)std::max(1, merge_blocks), kMergeThreads, 0, s>>>(bucket, off, ntrig, big, nbig);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(ntrig, n_tmpl, toff);
    RFD_LAUNCH_CHECK();
    k_write<<<gw, 256, 0, s>>>(bucket, off, toff, n_tmpl, trig_cap, trig);
    RFD_LAUNCH_CHECK();
    return RFD_OK;
}

}  // namespace

// Scratch: ctx->ws[12] holds the int32 / int64 arrays, ctx->ws[13] the bucketed candidates.
// Enqueues the merge and the read-back of (candidate count, trigger total, bad count) into
// `host` (pinned memory when the stream is being captured into a graph).
rfd_status find_triggers_enqueue(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand,
                                 const int64_t *cand_count, int64_t cap, rfd_trigger *trig,
                                 int64_t trig_cap, TrigReadback *host, cudaStream_t s) {
    const size_t J = (size_t)n_tmpl;
    const size_t i32_bytes = ((4 * J + 2) * sizeof(int32_t) + 15) / 16 * 16;
    const size_t bytes = i32_bytes + 2 * (J + 1) * sizeof(int64_t);
    RFD_TRY(ensure(ctx->ws[12], bytes));
    RFD_TRY(ensure(ctx->ws[13], (size_t)std::max<int64_t>(cap, 1) * sizeof(rfd_candidate)));
    char *base = (char *)ctx->ws[12].p;
    int32_t *i32 = (int32_t *)base;
    int64_t *off = (int64_t *)(base + i32_bytes), *toff = off + (J + 1);
    RFD_TRY(merge_enqueue(n_tmpl, cand, cand_count, cap, trig, trig_cap, i32, off, toff,
                          (rfd_candidate *)ctx->ws[13].p, 2 * ctx->num_sms, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->count, cand_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->total, toff + J, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->bad, i32 + 4 * J, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    return RFD_OK;
}

// Interprets a completed read-back.
rfd_status find_triggers_check(const TrigReadback &h, int32_t n_tmpl, int64_t cap, int64_t trig_cap,
                               int64_t *n_trig_host) {
    RFD_REQUIRE((h.count & kTimeoutBit) == 0, RFD_ERR_TIMEOUT,
                "find_triggers: the filtering kernel gave up waiting on the device (timeout)");
    RFD_REQUIRE(h.bad == 0, RFD_ERR_ARG, "find_triggers: %d candidates name a template >= n_tmpl=%d", h.bad, n_tmpl);
    if (h.count > cap) {
        *n_trig_host = h.count;
        ::rfd::set_error("find_triggers: %lld candidates produced, capacity %lld", (long long)h.count,
                         (long long)cap);
        return RFD_ERR_OVERFLOW;
    }
    *n_trig_host = h.total;
    if (h.total > trig_cap) {
        ::rfd::set_error("find_triggers: %lld triggers, capacity %lld", (long long)h.total, (long long)trig_cap);
        return RFD_ERR_OVERFLOW;
    }
    return RFD_OK;
}

rfd_status find_triggers_impl(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand,
                              const int64_t *cand_count, int64_t cap, rfd_trigger *trig,
                              int64_t trig_cap, int64_t *n_trig_host, cudaStream_t s) {
    TrigReadback h{};
    RFD_TRY(find_triggers_enqueue(ctx, n_tmpl, cand, cand_count, cap, trig, trig_cap, &h, s));
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return find_triggers_check(h, n_tmpl, cap, trig_cap, n_trig_host);
}

}  // namespace rfd

// ------------------------------------------------------------------ no-allocation variant
// rfd_find_triggers_noalloc runs the same merge kernels with its scratch in a fixed,
// file-scope device array instead of context workspaces, so it never allocates.  The array
// lives in every GPU that loads this library until the process exits.  Host code cannot use
// the array's name as a device address, so the address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

namespace rfd {
namespace {

constexpr size_t kNaI32Bytes = ((4 * (size_t)RFD_NOALLOC_MAX_TEMPLATES + 2) * sizeof(int32_t) + 255) / 256 * 256;
constexpr size_t kNaI64Bytes = (2 * ((size_t)RFD_NOALLOC_MAX_TEMPLATES + 1) * sizeof(int64_t) + 255) / 256 * 256;
constexpr size_t kNaScratchBytes = kNaI32Bytes + kNaI64Bytes +
                                   (size_t)RFD_NOALLOC_MAX_CANDIDATES * sizeof(rfd_candidate);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kNaMaxDevices] = {};

}  // namespace
}  // namespace rfd

extern "C" rfd_status rfd_find_triggers_noalloc(int32_t n_tmpl, const rfd_candidate *cand_dev,
                                                const int64_t *cand_count_dev, int64_t cand_capacity,
                                                rfd_trigger *trig_dev, int64_t trig_capacity,
                                                int64_t *n_trig_host, void *stream) {
    using namespace rfd;
    RFD_REQUIRE(n_tmpl >= 1 && n_tmpl <= RFD_NOALLOC_MAX_TEMPLATES, RFD_ERR_SHAPE,
                "find_triggers_noalloc: n_tmpl=%d outside [1, %d] (the static scratch maximum)", n_tmpl,
                RFD_NOALLOC_MAX_TEMPLATES);
    RFD_REQUIRE(cand_capacity >= 0 && cand_capacity <= RFD_NOALLOC_MAX_CANDIDATES, RFD_ERR_SHAPE,
                "find_triggers_noalloc: cand_capacity=%lld outside [0, %d] (the static scratch maximum)",
                (long long)cand_capacity, RFD_NOALLOC_MAX_CANDIDATES);
    RFD_REQUIRE(trig_capacity >= 0, RFD_ERR_SHAPE, "negative trigger capacity");
    RFD_REQUIRE(cand_count_dev && n_trig_host && (cand_dev || cand_capacity == 0) && (trig_dev || trig_capacity == 0),
                RFD_ERR_ARG, "NULL argument");
    int dev = 0;
    RFD_TRY_CUDA(cudaGetDevice(&dev));
    RFD_REQUIRE(dev >= 0 && dev < kNaMaxDevices, RFD_ERR_UNSUPPORTED, "device index %d too large", dev);
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            RFD_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t J = (size_t)n_tmpl;
    char *b = (char *)base;
    int32_t *i32 = (int32_t *)b;
    int64_t *off = (int64_t *)(b + kNaI32Bytes), *toff = off + (J + 1);
    rfd_candidate *bucket = (rfd_candidate *)(b + kNaI32Bytes + kNaI64Bytes);
    int32_t *bad = i32 + 4 * J;
    // the array keeps the previous call's contents: merge_enqueue clears the counters it
    // accumulates into; every other word it reads was written earlier in the same call
    int nsm = 0;
    RFD_TRY_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RFD_TRY(merge_enqueue(n_tmpl, cand_dev, cand_count_dev, cand_capacity, trig_dev, trig_capacity, i32, off, toff,
                          bucket, 2 * nsm, s));
    int64_t host[2] = {0, 0};
    int32_t hbad = 0;
    RFD_TRY_CUDA(cudaMemcpyAsync(&host[0], cand_count_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host[1], toff + J, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    RFD_REQUIRE((host[0] & kTimeoutBit) == 0, RFD_ERR_TIMEOUT,
                "find_triggers_noalloc: the filtering kernel gave up waiting on the device (timeout)");
    RFD_REQUIRE(hbad == 0, RFD_ERR_ARG, "find_triggers_noalloc: %d candidates name a template >= n_tmpl=%d", hbad,
                n_tmpl);
    if (host[0] > cand_capacity) {
        *n_trig_host = host[0];
        set_error("find_triggers_noalloc: %lld candidates produced, capacity %lld", (long long)host[0],
                  (long long)cand_capacity);
        return RFD_ERR_OVERFLOW;
    }
    *n_trig_host = host[1];
    if (host[1] > trig_capacity) {
        set_error("find_triggers_noalloc: %lld triggers, capacity %lld", (long long)host[1],
                  (long long)trig_capacity);
        return RFD_ERR_OVERFLOW;
    }
    return RFD_OK;
}
