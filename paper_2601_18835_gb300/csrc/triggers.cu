// find_triggers: candidates -> one trigger per (template, window), sorted by (j, w).
// Table II's "trigger accumulation".  Integer keys only, so the result does not depend on
// the order in which candidates were appended.
//
//   1. count candidates per template;  2. exclusive scan -> bucket offsets;
//   3. scatter into per-template buckets;  4. per template, sort its bucket by (w, key desc)
//      and count distinct windows;  5. exclusive scan -> trigger offsets;  6. write.
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

__device__ __forceinline__ bool before(const rfd_candidate &a, const rfd_candidate &b) {
    return a.w < b.w || (a.w == b.w && a.key > b.key);
}

__global__ void k_merge(rfd_candidate *__restrict__ bucket, const int64_t *__restrict__ off,
                        int32_t n_tmpl, int32_t *__restrict__ ntrig) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_tmpl) return;
    const int64_t b = off[j], e = off[j + 1];
    for (int64_t i = b + 1; i < e; ++i) {    // insertion sort: buckets are short
        const rfd_candidate v = bucket[i];
        int64_t k = i - 1;
        while (k >= b && before(v, bucket[k])) {
            bucket[k + 1] = bucket[k];
            --k;
        }
        bucket[k + 1] = v;
    }
    int32_t nt = 0;
    for (int64_t i = b; i < e; ++i)
        if (i == b || bucket[i].w != bucket[i - 1].w) ++nt;
    ntrig[j] = nt;
}

__global__ void k_write(const rfd_candidate *__restrict__ bucket, const int64_t *__restrict__ off,
                        const int64_t *__restrict__ toff, int32_t n_tmpl, int64_t trig_cap,
                        rfd_trigger *__restrict__ trig) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_tmpl) return;
    const int64_t b = off[j], e = off[j + 1];
    int64_t o = toff[j];
    for (int64_t i = b; i < e; ++i) {
        if (i != b && bucket[i].w == bucket[i - 1].w) continue;
        if (o < trig_cap) {
            const rfd_candidate c = bucket[i];
            rfd_trigger t;
            t.j = j;
            t.t = (int32_t)(0xffffffffu - (uint32_t)(c.key & 0xffffffffull));
            t.snr2 = __uint_as_float((uint32_t)(c.key >> 32));
            t.zr = c.zr;
            t.zi = c.zi;
            trig[o] = t;
        }
        ++o;
    }
}

}  // namespace

// Scratch: ctx->ws[12] holds the int32 / int64 arrays, ctx->ws[13] the bucketed candidates.
// Enqueues the six kernels and the read-back of (candidate count, trigger total, bad count)
// into `host` (pinned memory when the stream is being captured into a graph).
rfd_status find_triggers_enqueue(rfd_ctx *ctx, int32_t n_tmpl, const rfd_candidate *cand,
                                 const int64_t *cand_count, int64_t cap, rfd_trigger *trig,
                                 int64_t trig_cap, TrigReadback *host, cudaStream_t s) {
    const size_t J = (size_t)n_tmpl;
    // layout: cnt[J] cur[J] ntrig[J] bad[1] (int32, padded) | off[J+1] toff[J+1] (int64)
    const size_t i32_bytes = ((3 * J + 1) * sizeof(int32_t) + 15) / 16 * 16;
    const size_t bytes = i32_bytes + 2 * (J + 1) * sizeof(int64_t);
    RFD_TRY(ensure(ctx->ws[12], bytes));
    RFD_TRY(ensure(ctx->ws[13], (size_t)std::max<int64_t>(cap, 1) * sizeof(rfd_candidate)));
    char *base = (char *)ctx->ws[12].p;
    int32_t *cnt = (int32_t *)base, *cur = cnt + J, *ntrig = cur + J, *bad = ntrig + J;
    int64_t *off = (int64_t *)(base + i32_bytes), *toff = off + (J + 1);
    rfd_candidate *bucket = (rfd_candidate *)ctx->ws[13].p;
    RFD_TRY_CUDA(cudaMemsetAsync(base, 0, i32_bytes, s));
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, (cap + 255) / 256));
    const unsigned gj = (unsigned)((J + 255) / 256);
    k_count<<<gb, 256, 0, s>>>(cand, cand_count, cap, n_tmpl, cnt, bad);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(cnt, n_tmpl, off);
    RFD_LAUNCH_CHECK();
    k_scatter<<<gb, 256, 0, s>>>(cand, cand_count, cap, n_tmpl, off, cur, bucket);
    RFD_LAUNCH_CHECK();
    k_merge<<<gj, 256, 0, s>>>(bucket, off, n_tmpl, ntrig);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(ntrig, n_tmpl, toff);
    RFD_LAUNCH_CHECK();
    k_write<<<gj, 256, 0, s>>>(bucket, off, toff, n_tmpl, trig_cap, trig);
    RFD_LAUNCH_CHECK();
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->count, cand_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->total, toff + J, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RFD_TRY_CUDA(cudaMemcpyAsync(&host->bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
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
// rfd_find_triggers_noalloc runs the same six kernels with its scratch in a fixed,
// file-scope device array instead of context workspaces, so it never allocates.  The array
// lives in every GPU that loads this library until the process exits.  Host code cannot use
// the array's name as a device address, so the address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

namespace rfd {
namespace {

constexpr size_t kNaI32Bytes = ((3 * (size_t)RFD_NOALLOC_MAX_TEMPLATES + 1) * sizeof(int32_t) + 255) / 256 * 256;
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
    int32_t *cnt = (int32_t *)b, *cur = cnt + J, *ntrig = cur + J, *bad = ntrig + J;
    int64_t *off = (int64_t *)(b + kNaI32Bytes), *toff = off + (J + 1);
    rfd_candidate *bucket = (rfd_candidate *)(b + kNaI32Bytes + kNaI64Bytes);
    // the array keeps the previous call's contents: clear the counters this call accumulates into
    const size_t i32_bytes = (3 * J + 1) * sizeof(int32_t);
    RFD_TRY_CUDA(cudaMemsetAsync(cnt, 0, i32_bytes, s));
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, (cand_capacity + 255) / 256));
    const unsigned gj = (unsigned)((J + 255) / 256);
    k_count<<<gb, 256, 0, s>>>(cand_dev, cand_count_dev, cand_capacity, n_tmpl, cnt, bad);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(cnt, n_tmpl, off);
    RFD_LAUNCH_CHECK();
    k_scatter<<<gb, 256, 0, s>>>(cand_dev, cand_count_dev, cand_capacity, n_tmpl, off, cur, bucket);
    RFD_LAUNCH_CHECK();
    k_merge<<<gj, 256, 0, s>>>(bucket, off, n_tmpl, ntrig);
    RFD_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(ntrig, n_tmpl, toff);
    RFD_LAUNCH_CHECK();
    k_write<<<gj, 256, 0, s>>>(bucket, off, toff, n_tmpl, trig_capacity, trig_dev);
    RFD_LAUNCH_CHECK();
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
