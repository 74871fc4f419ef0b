// One data segment through the whole per-segment path as a single CUDA graph:
// filter_reference (Eq. 1 per reference, Stockham IFFT, split + halo), ratio_filter_batch
// (Eq. 3 for every template with the fused Table II reduction) and the trigger merge, with
// the read-back of the counts into pinned host memory.  Buffers are bound at creation; each
// run replays the graph, waits for it and checks the counts.
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
rfd_status filter_reference_impl(rfd_ctx *, const Grid &, const float2 *, const double *, const float2 *,
                                 int64_t, int32_t, int32_t, void *, int32_t *, cudaStream_t);
rfd_status ratio_filter_enqueue(const rfd_plan *, const void *, const int32_t *, const int64_t *, rfd_candidate *,
                                int64_t, int64_t *, cudaStream_t);
void add_launches(int64_t n);
int64_t launch_count();
}  // namespace rfd

struct rfd_search {
    rfd_plan *plan = nullptr;
    const float2 *d = nullptr;
    const double *psd = nullptr;
    const float2 *href = nullptr;
    void *qref = nullptr;
    int32_t *qscale = nullptr;
    rfd_candidate *cand = nullptr;
    int64_t cap = 0;
    int64_t *count = nullptr;
    rfd_trigger *trig = nullptr;
    int64_t trig_cap = 0;
    rfd::TrigReadback *host = nullptr;     // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels_per_run = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the ratio-filter kernel, inside the graph
    cudaEvent_t evs = nullptr, eve = nullptr;   // first and last node of the graph
    bool pinned = false;                        // holds a graphs_pin()
    int64_t *d_ubase = nullptr;                 // window start read by the filtering kernels
    int64_t *h_ubase = nullptr;                 // pinned staging for it
};

namespace rfd {
namespace {

// Inside a stream capture an event must be recorded as "external" to become an event-record
// node of the graph (a plain record only marks a capture dependency).
cudaError_t record(cudaEvent_t ev, cudaStream_t s, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

rfd_status enqueue_step(rfd_search *S, cudaStream_t s, bool capturing) {
    rfd_plan *p = S->plan;
    RFD_TRY_CUDA(record(S->evs, s, capturing));
    RFD_TRY(filter_reference_impl(p->ctx, p->grid, S->d, S->psd, S->href, p->n_ref, p->halo, p->precision, S->qref,
                                  S->qscale, s));
    RFD_TRY_CUDA(cudaMemsetAsync(S->count, 0, sizeof(int64_t), s));
    RFD_TRY_CUDA(record(S->ev0, s, capturing));
    RFD_TRY(ratio_filter_enqueue(p, S->qref, S->qscale, S->d_ubase, S->cand, S->cap, S->count, s));
    RFD_TRY_CUDA(record(S->ev1, s, capturing));
    RFD_TRY(find_triggers_enqueue(p->ctx, p->n_tmpl, S->cand, S->count, S->cap, S->trig, S->trig_cap, S->host, s));
    RFD_TRY_CUDA(record(S->eve, s, capturing));
    return RFD_OK;
}

}  // namespace
}  // namespace rfd

using namespace rfd;

extern "C" {

void rfd_search_destroy(rfd_search *S) {
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->pinned) graphs_unpin();
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->host) cudaFreeHost(S->host);
    if (S->h_ubase) cudaFreeHost(S->h_ubase);
    if (S->d_ubase) cudaFree(S->d_ubase);
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev1) cudaEventDestroy(S->ev1);
    if (S->evs) cudaEventDestroy(S->evs);
    if (S->eve) cudaEventDestroy(S->eve);
    delete S;
}

rfd_status rfd_search_create(rfd_plan *plan, const void *dtilde_dev, const double *psd_dev, const void *href_dev,
                             void *qref_dev, int32_t *qscale_dev, rfd_candidate *cand_dev, int64_t cand_capacity,
                             int64_t *cand_count_dev, rfd_trigger *trig_dev, int64_t trig_capacity, void *stream,
                             rfd_search **out) {
    NvtxRange nvtx_range("rfd_search_create");
    RFD_REQUIRE(plan && out, RFD_ERR_ARG, "NULL plan or out");
    *out = nullptr;
    RFD_REQUIRE(plan->taps_set, RFD_ERR_ARG, "rfd_plan_set_taps has not been called");
    RFD_REQUIRE(dtilde_dev && psd_dev && href_dev && qref_dev && qscale_dev && cand_dev && cand_count_dev && trig_dev,
                RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(cand_capacity >= 1 && trig_capacity >= 1, RFD_ERR_SHAPE, "capacities must be >= 1");
    RFD_REQUIRE(stream != nullptr, RFD_ERR_ARG, "graph capture needs a created stream (not the legacy stream)");
    RFD_TRY_CUDA(cudaSetDevice(plan->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    rfd_search *S = new rfd_search();
    S->plan = plan;
    S->d = (const float2 *)dtilde_dev;
    S->psd = psd_dev;
    S->href = (const float2 *)href_dev;
    S->qref = qref_dev;
    S->qscale = qscale_dev;
    S->cand = cand_dev;
    S->cap = cand_capacity;
    S->count = cand_count_dev;
    S->trig = trig_dev;
    S->trig_cap = trig_capacity;
    rfd_status st = RFD_OK;
    do {
        cudaError_t e = cudaMallocHost((void **)&S->host, sizeof(TrigReadback));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_ubase, sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_ubase, sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMemset(S->d_ubase, 0, sizeof(int64_t));
        if (e != cudaSuccess) {
            set_error("search allocation failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_NOMEM;
            break;
        }
        if ((e = cudaEventCreate(&S->ev0)) != cudaSuccess || (e = cudaEventCreate(&S->ev1)) != cudaSuccess ||
            (e = cudaEventCreate(&S->evs)) != cudaSuccess || (e = cudaEventCreate(&S->eve)) != cudaSuccess) {
            set_error("cudaEventCreate failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        // warm-up pass: sizes every workspace and sets kernel attributes outside the capture
        const int64_t l0 = launch_count();
        if ((st = enqueue_step(S, s, false)) != RFD_OK) break;
        S->kernels_per_run = launch_count() - l0;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
            set_error("warm-up failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            set_error("cudaStreamBeginCapture failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        const int64_t l1 = launch_count();
        const rfd_status st_cap = enqueue_step(S, s, true);
        add_launches(-(launch_count() - l1));      // captured, not launched
        e = cudaStreamEndCapture(s, &S->graph);
        if (st_cap != RFD_OK) {
            st = st_cap;
            break;
        }
        if (e != cudaSuccess) {
            set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        if ((e = cudaGraphInstantiate(&S->exec, S->graph, 0)) != cudaSuccess) {
            set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
            st = RFD_ERR_CUDA;
            break;
        }
        graphs_pin();
        S->pinned = true;
    } while (0);
    if (st != RFD_OK) {
        rfd_search_destroy(S);
        return st;
    }
    *out = S;
    return RFD_OK;
}

rfd_status rfd_search_run_at(rfd_search *S, int64_t u_begin, void *stream, int64_t *n_trig_host) {
    NvtxRange nvtx_range("rfd_search_run_at");
    RFD_REQUIRE(S && n_trig_host, RFD_ERR_ARG, "NULL argument");
    RFD_REQUIRE(u_begin >= 0 && u_begin < S->plan->grid.n && u_begin % 512 == 0, RFD_ERR_ARG,
                "u_begin=%lld must be a multiple of 512 in [0, n)", (long long)u_begin);
    RFD_TRY_CUDA(cudaSetDevice(S->plan->ctx->device));
    *S->h_ubase = u_begin;
    RFD_TRY_CUDA(cudaMemcpyAsync(S->d_ubase, S->h_ubase, sizeof(int64_t), cudaMemcpyHostToDevice,
                                 (cudaStream_t)stream));
    return rfd_search_run(S, stream, n_trig_host);
}

rfd_status rfd_search_run(rfd_search *S, void *stream, int64_t *n_trig_host) {
    NvtxRange nvtx_range("rfd_search_run");
    RFD_REQUIRE(S && n_trig_host, RFD_ERR_ARG, "NULL argument");
    RFD_TRY_CUDA(cudaSetDevice(S->plan->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RFD_TRY_CUDA(cudaGraphLaunch(S->exec, s));
    add_launches(S->kernels_per_run);
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    return find_triggers_check(*S->host, S->plan->n_tmpl, S->cap, S->trig_cap, n_trig_host);
}

rfd_status rfd_search_run_host(rfd_search *S, const void *dtilde_host, rfd_trigger *trig_host,
                               int64_t trig_host_capacity, void *stream, int64_t *n_trig_host) {
    NvtxRange nvtx_range("rfd_search_run_host");
    RFD_REQUIRE(S && dtilde_host && n_trig_host && (trig_host || trig_host_capacity == 0), RFD_ERR_ARG,
                "NULL argument");
    RFD_REQUIRE(trig_host_capacity >= 0, RFD_ERR_SHAPE, "negative trigger capacity");
    RFD_TRY_CUDA(cudaSetDevice(S->plan->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t in_bytes = (size_t)S->plan->grid.nf * sizeof(float2);
    RFD_TRY_CUDA(cudaMemcpyAsync((void *)S->d, dtilde_host, in_bytes, cudaMemcpyHostToDevice, s));
    RFD_TRY_CUDA(cudaGraphLaunch(S->exec, s));
    add_launches(S->kernels_per_run);
    RFD_TRY_CUDA(cudaStreamSynchronize(s));
    int64_t n = 0;
    RFD_TRY(find_triggers_check(*S->host, S->plan->n_tmpl, S->cap, S->trig_cap, &n));
    *n_trig_host = n;
    RFD_REQUIRE(n <= trig_host_capacity, RFD_ERR_OVERFLOW, "search_run_host: %lld triggers, host capacity %lld",
                (long long)n, (long long)trig_host_capacity);
    if (n > 0) {
        RFD_TRY_CUDA(cudaMemcpyAsync(trig_host, S->trig, (size_t)n * sizeof(rfd_trigger), cudaMemcpyDeviceToHost, s));
        RFD_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return RFD_OK;
}

int64_t rfd_search_kernels_per_run(const rfd_search *S) { return S ? S->kernels_per_run : 0; }

static double elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        (void)cudaGetLastError();   // leave no error behind for a later launch check
        return -1.0;
    }
    return (double)ms;
}

double rfd_search_step_ms(const rfd_search *S) { return S ? elapsed(S->evs, S->eve) : -1.0; }

double rfd_search_filter_ms(const rfd_search *S) { return S ? elapsed(S->ev0, S->ev1) : -1.0; }

}  // extern "C"
