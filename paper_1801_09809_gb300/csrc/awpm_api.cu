// Host side of libawpm: the C ABI declared in include/awpm.h.
//
// A context owns a device workspace sized for the largest problem seen, the
// staging buffers for host-resident inputs and a cache of instantiated CUDA
// graphs.  One solve is one graph launch: validation and initialisation, a
// conditional WHILE node whose body is one pass of Steps A-D (the control
// kernel at the end of the body decides on the device whether another pass
// runs, Algorithm 2), and the final weight reduction.  The host waits once,
// at the end, to read the statistics.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "awpm.h"
#include "awpm_internal.h"

using namespace awpm;

namespace {

thread_local char g_last_error[512] = "";

void note_cuda(cudaError_t e, const char *what, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at awpm_api.cu:%d: %s",
             cudaGetErrorName(e), what, line, cudaGetErrorString(e));
}

#define CUDA_TRY(x)                                                        \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) {                                           \
            note_cuda(e_, #x, __LINE__);                                   \
            return e_ == cudaErrorMemoryAllocation ? AWPM_ERR_OOM          \
                                                   : AWPM_ERR_CUDA;        \
        }                                                                  \
    } while (0)

#define AWPM_TRY(x)            \
    do {                       \
        int rc_ = (x);         \
        if (rc_ != AWPM_OK)    \
            return rc_;        \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct GraphKey {
    int32_t n = -1, nnz = -1, max_passes = 0, lookup = 0, count = 0;
    const void *colptr = nullptr, *rowidx = nullptr, *w = nullptr, *mate_in = nullptr,
               *n_off = nullptr;
    bool operator==(const GraphKey &o) const
    {
        return n == o.n && nnz == o.nnz && max_passes == o.max_passes && lookup == o.lookup &&
               count == o.count && colptr == o.colptr && rowidx == o.rowidx && w == o.w &&
               mate_in == o.mate_in && n_off == o.n_off;
    }
};

}  // namespace

struct awpm_ctx {
    std::mutex mu;
    awpm_options opt{};
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t held = 0;
    // workspace
    DevBuf mc, mr, wm, rr, wmr, colsig, best, dsel, tile_col, starts, ctl, wpart, htab;
    int search_u = 1;
    int search_bps[2][2] = {{1, 1}, {1, 1}};  // [batch][hash]: resident blocks per SM
    // staging of host-resident arrays
    DevBuf s_colptr, s_rowidx, s_w, s_mate, s_gain, s_row;
    // batched solves
    DevBuf b_noff, b_colmat, b_tilemat, b_i32, b_u64, b_f64;
    void *h_batch = nullptr;  // pinned per-matrix results
    size_t h_batch_bytes = 0;
    Ctl *h_ctl = nullptr;       // pinned
    int32_t *h_active = nullptr;  // pinned ring of the timed loop
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    std::vector<cudaEvent_t> tev;     // timing pairs of the timed loop
    std::vector<cudaEvent_t> flagev;  // ring of the timed loop
    // cached solve graph
    bool g_valid = false;
    GraphKey g_key;
    cudaGraphExec_t g_exec = nullptr;
};

namespace {

constexpr int kLookahead = 2;
constexpr int kRing = 4;

int release(awpm_ctx *c, DevBuf &b)
{
    if (b.p) {
        cudaFree(b.p);
        c->held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    return AWPM_OK;
}

void drop_graph(awpm_ctx *c)
{
    if (c->g_exec)
        cudaGraphExecDestroy(c->g_exec);
    c->g_exec = nullptr;
    c->g_valid = false;
}

int ensure(awpm_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (b.bytes >= bytes)
        return AWPM_OK;
    drop_graph(c);
    release(c, b);
    size_t want = bytes + bytes / 8;  // headroom against small growth steps
    if (c->opt.mem_budget_bytes && c->held + want > c->opt.mem_budget_bytes) {
        want = bytes;
        if (c->held + want > c->opt.mem_budget_bytes)
            return AWPM_ERR_BUDGET;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        note_cuda(e, "cudaMalloc", __LINE__);
        cudaGetLastError();
        return AWPM_ERR_OOM;
    }
    b.p = p;
    b.bytes = want;
    c->held += want;
    return AWPM_OK;
}

// 1 = device memory of the context's GPU, 0 = host memory, -1 = another GPU.
int where(const awpm_ctx *c, const void *p)
{
    if (!p)
        return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        if (a.type == cudaMemoryTypeDevice && a.device != c->device)
            return -1;
        return 1;
    }
    return 0;
}

int code_of(unsigned err)
{
    if (err & kErrInvalid)
        return AWPM_ERR_INVALID_ARG;
    if (err & kErrUnsorted)
        return AWPM_ERR_UNSORTED_OR_DUP;
    if (err & kErrNonfinite)
        return AWPM_ERR_NONFINITE;
    if (err & kErrNotPerfect)
        return AWPM_ERR_NOT_PERFECT;
    if (err)
        return AWPM_ERR_TIMEOUT;
    return AWPM_OK;
}

int check_launch()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda(e, "kernel launch", __LINE__);
        return AWPM_ERR_CUDA;
    }
    return AWPM_OK;
}

int build_graph(awpm_ctx *c, const Work &wk, int max_passes, int lookup)
{
    cudaStream_t s = c->stream;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t g_init = nullptr, g_final = nullptr, top = nullptr;
    int rc = AWPM_OK;
    cudaError_t e;

    e = cudaStreamBeginCapture(s, mode);
    if (e != cudaSuccess) {
        note_cuda(e, "cudaStreamBeginCapture", __LINE__);
        return AWPM_ERR_CUDA;
    }
    launch_init(wk, max_passes, c->num_sms, s);
    launch_weight_sum(wk, false, s);
    launch_batch_weight_sum(wk, false, s);
    e = cudaStreamEndCapture(s, &g_init);
    if (e != cudaSuccess) {
        note_cuda(e, "capture of the initialisation", __LINE__);
        return AWPM_ERR_CUDA;
    }
    e = cudaStreamBeginCapture(s, mode);
    if (e == cudaSuccess) {
        launch_weight_sum(wk, true, s);
        launch_batch_weight_sum(wk, true, s);
        e = cudaStreamEndCapture(s, &g_final);
    }
    if (e != cudaSuccess) {
        note_cuda(e, "capture of the final reduction", __LINE__);
        cudaGraphDestroy(g_init);
        return AWPM_ERR_CUDA;
    }

    cudaGraphNode_t n_init, n_cond, n_final;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cudaGraph_t body = nullptr;
    if ((e = cudaGraphCreate(&top, 0)) != cudaSuccess ||
        (e = cudaGraphAddChildGraphNode(&n_init, top, nullptr, 0, g_init)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault)) !=
            cudaSuccess) {
        note_cuda(e, "graph assembly", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_cond, top, &n_init, nullptr, 1, &cp)) != cudaSuccess) {
        note_cuda(e, "conditional node", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, mode)) != cudaSuccess) {
        note_cuda(e, "capture of the pass body", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    launch_reset_best(wk, s);
    launch_search(wk, c->num_sms, s);
    launch_select_and_flip(wk, c->num_sms, s);
    launch_control(wk, true, h, s);
    if ((e = cudaStreamEndCapture(s, &body)) != cudaSuccess) {
        note_cuda(e, "capture of the pass body", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_final, top, &n_cond, 1, g_final)) != cudaSuccess ||
        (e = cudaGraphInstantiate(&c->g_exec, top, 0)) != cudaSuccess) {
        note_cuda(e, "graph instantiation", __LINE__);
        c->g_exec = nullptr;
        rc = AWPM_ERR_CUDA;
        goto done;
    }
done:
    if (top)
        cudaGraphDestroy(top);
    if (g_init)
        cudaGraphDestroy(g_init);
    if (g_final)
        cudaGraphDestroy(g_final);
    cudaGetLastError();
    return rc;
}

int ensure_timing_events(awpm_ctx *c, size_t pairs)
{
    while (c->tev.size() < 2 * pairs) {
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreate(&ev));
        c->tev.push_back(ev);
    }
    return AWPM_OK;
}

// Host-driven pass loop (AWPM_FLAG_TIME_SEARCH): CUDA events around every
// search launch; the host stays kLookahead passes ahead of the device and
// stops enqueueing once a finished pass reports that the loop ended.  Passes
// enqueued after the end are no-ops (every kernel checks ctl->active).
int run_timed(awpm_ctx *c, const Work &wk, int max_passes, int lookup, double *ms_search,
              int *passes_enqueued)
{
    cudaStream_t s = c->stream;
    launch_init(wk, max_passes, c->num_sms, s);
    launch_weight_sum(wk, false, s);
    launch_batch_weight_sum(wk, false, s);
    AWPM_TRY(check_launch());
    int t = 0;
    for (; t < max_passes; ++t) {
        if (t >= kLookahead) {
            int slot = (t - kLookahead) % kRing;
            CUDA_TRY(cudaEventSynchronize(c->flagev[slot]));
            if (!c->h_active[slot])
                break;
        }
        AWPM_TRY(ensure_timing_events(c, (size_t)t + 1));
        launch_reset_best(wk, s);
        CUDA_TRY(cudaEventRecord(c->tev[2 * t], s));
        launch_search(wk, c->num_sms, s);
        CUDA_TRY(cudaEventRecord(c->tev[2 * t + 1], s));
        launch_select_and_flip(wk, c->num_sms, s);
        launch_control(wk, false, cudaGraphConditionalHandle(), s);
        AWPM_TRY(check_launch());
        CUDA_TRY(cudaMemcpyAsync(&c->h_active[t % kRing], &wk.ctl->active, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(c->flagev[t % kRing], s));
    }
    launch_weight_sum(wk, true, s);
    launch_batch_weight_sum(wk, true, s);
    AWPM_TRY(check_launch());
    *passes_enqueued = t;
    *ms_search = 0.0;
    return AWPM_OK;
}

int setup_ctx(awpm_ctx *c, const awpm_options *opt)
{
    if (opt)
        c->opt = *opt;
    else
        awpm_default_options(&c->opt);
    if (c->opt.max_iters < 0 || c->opt.lookup < 0 || c->opt.lookup > 2)
        return AWPM_ERR_INVALID_ARG;
    int dev = c->opt.device;
    if (dev < 0)
        CUDA_TRY(cudaGetDevice(&dev));
    c->device = dev;
    CUDA_TRY(cudaSetDevice(dev));
    CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    c->search_u = default_search_u();
    for (int b = 0; b < 2; ++b) {
        c->search_bps[b][0] = search_blocks_per_sm(AWPM_LOOKUP_BSEARCH, c->search_u, b == 1);
        c->search_bps[b][1] = search_blocks_per_sm(AWPM_LOOKUP_HASH, 1, b == 1);
    }
    if (c->opt.stream) {
        c->stream = (cudaStream_t)c->opt.stream;
        c->own_stream = false;
    } else {
        CUDA_TRY(cudaStreamCreate(&c->stream));
        c->own_stream = true;
    }
    CUDA_TRY(cudaMallocHost((void **)&c->h_ctl, sizeof(Ctl)));
    CUDA_TRY(cudaMallocHost((void **)&c->h_active, sizeof(int32_t) * kRing));
    CUDA_TRY(cudaEventCreate(&c->ev_a));
    CUDA_TRY(cudaEventCreate(&c->ev_b));
    for (int i = 0; i < kRing; ++i) {
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->flagev.push_back(ev);
    }
    return AWPM_OK;
}

void teardown_ctx(awpm_ctx *c)
{
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    drop_graph(c);
    DevBuf *bufs[] = {&c->mc, &c->mr, &c->wm, &c->rr, &c->wmr, &c->colsig, &c->best, &c->dsel,
                      &c->tile_col, &c->starts, &c->htab, &c->b_noff, &c->b_colmat,
                      &c->b_tilemat, &c->b_i32, &c->b_u64, &c->b_f64,
                      &c->ctl, &c->wpart, &c->s_colptr, &c->s_rowidx, &c->s_w, &c->s_mate,
                      &c->s_gain, &c->s_row};
    for (DevBuf *b : bufs)
        release(c, *b);
    if (c->h_ctl)
        cudaFreeHost(c->h_ctl);
    if (c->h_batch)
        cudaFreeHost(c->h_batch);
    if (c->h_active)
        cudaFreeHost(c->h_active);
    for (cudaEvent_t ev : c->tev)
        cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->flagev)
        cudaEventDestroy(ev);
    if (c->ev_a)
        cudaEventDestroy(c->ev_a);
    if (c->ev_b)
        cudaEventDestroy(c->ev_b);
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
    cudaGetLastError();
}

template <typename T>
int stage_in(awpm_ctx *c, DevBuf &buf, const T *src, size_t count, int loc, const T **out)
{
    if (loc == 1) {
        *out = src;
        return AWPM_OK;
    }
    AWPM_TRY(ensure(c, buf, sizeof(T) * count));
    if (count)
        CUDA_TRY(cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
    *out = (const T *)buf.p;
    return AWPM_OK;
}

// The whole call: argument checks, staging, the solve (or the single
// search), results and statistics.
int run(awpm_ctx *c, int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *weight,
        const int32_t *mate_in, int32_t *mate_out, awpm_stats *st, bool search_only,
        double *gain_out, int32_t *row_out, int32_t count = 0, const int32_t *n_off = nullptr,
        awpm_stats *per_matrix = nullptr)
{
    if (!c || n < 0 || (n > 0 && (!colptr || !mate_in)) || (!search_only && n > 0 && !mate_out) ||
        (search_only && n > 0 && (!gain_out || !row_out)))
        return AWPM_ERR_INVALID_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    awpm_stats S;
    std::memset(&S, 0, sizeof(S));
    if (n == 0) {
        S.iterations = search_only ? 0 : 1;
        S.converged = 1;
        S.lookup_used = AWPM_LOOKUP_BSEARCH;
        if (st)
            *st = S;
        return AWPM_OK;
    }
    const int l_colptr = where(c, colptr), l_rowidx = where(c, rowidx), l_w = where(c, weight),
              l_mate = where(c, mate_in);
    const int l_out = search_only ? 0 : where(c, mate_out);
    const int l_gain = search_only ? where(c, gain_out) : 0;
    const int l_row = search_only ? where(c, row_out) : 0;
    if (l_colptr < 0 || l_rowidx < 0 || l_w < 0 || l_mate < 0 || l_out < 0 || l_gain < 0 ||
        l_row < 0)
        return AWPM_ERR_INVALID_ARG;

    int32_t nnz = 0;
    if (l_colptr == 1) {
        CUDA_TRY(cudaMemcpyAsync(c->h_ctl, colptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        std::memcpy(&nnz, c->h_ctl, sizeof(int32_t));
    } else {
        nnz = colptr[n];
    }
    if (nnz < 0 || (nnz > 0 && (!rowidx || !weight)))
        return AWPM_ERR_INVALID_ARG;
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    const int32_t max_passes = c->opt.max_iters > 0 ? c->opt.max_iters : AWPM_PASS_CAP;
    const int lookup = c->opt.lookup == AWPM_LOOKUP_HASH ? AWPM_LOOKUP_HASH : AWPM_LOOKUP_BSEARCH;

    AWPM_TRY(ensure(c, c->mc, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mr, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->wm, sizeof(double) * n));
    AWPM_TRY(ensure(c, c->rr, sizeof(RowRec) * n));
    AWPM_TRY(ensure(c, c->wmr, sizeof(double) * n));
    AWPM_TRY(ensure(c, c->colsig, sizeof(unsigned long long) * n));
    AWPM_TRY(ensure(c, c->best, sizeof(Rec) * n));
    AWPM_TRY(ensure(c, c->dsel, sizeof(Sel) * n));
    AWPM_TRY(ensure(c, c->tile_col, sizeof(int32_t) * ((size_t)ntiles + 1)));
    AWPM_TRY(ensure(c, c->starts, sizeof(uint32_t) * (((size_t)nnz + 31) / 32 + 1)));
    AWPM_TRY(ensure(c, c->ctl, sizeof(Ctl)));
    AWPM_TRY(ensure(c, c->wpart, sizeof(double) * kWsumBlocks));
    if (lookup == AWPM_LOOKUP_HASH)
        AWPM_TRY(ensure(c, c->htab, sizeof(unsigned long long) * 2 * (size_t)nnz));

    CUDA_TRY(cudaEventRecord(c->ev_a, c->stream));
    Work wk;
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = ntiles;
    wk.lookup = lookup;
    wk.htab = lookup == AWPM_LOOKUP_HASH ? (unsigned long long *)c->htab.p : nullptr;
    wk.search_u = lookup == AWPM_LOOKUP_HASH ? 1 : c->search_u;
    wk.search_bps = c->search_bps[count > 0 ? 1 : 0][lookup == AWPM_LOOKUP_HASH ? 1 : 0];
    AWPM_TRY(stage_in(c, c->s_colptr, colptr, (size_t)n + 1, l_colptr, &wk.colptr));
    AWPM_TRY(stage_in(c, c->s_rowidx, rowidx, (size_t)nnz, l_rowidx, &wk.rowidx));
    AWPM_TRY(stage_in(c, c->s_w, weight, (size_t)nnz, l_w, &wk.w));
    AWPM_TRY(stage_in(c, c->s_mate, mate_in, (size_t)n, l_mate, &wk.mate_in));
    if (count > 0) {
        const int l_off = where(c, n_off);
        if (l_off < 0)
            return AWPM_ERR_INVALID_ARG;
        BatchWork &bw = wk.bw;
        bw.count = count;
        AWPM_TRY(stage_in(c, c->b_noff, n_off, (size_t)count + 1, l_off, &bw.n_off));
        AWPM_TRY(ensure(c, c->b_colmat, sizeof(int32_t) * n));
        AWPM_TRY(ensure(c, c->b_tilemat, sizeof(int32_t) * ((size_t)ntiles + 1)));
        AWPM_TRY(ensure(c, c->b_i32, sizeof(int32_t) * (5 * (size_t)count + 1)));
        AWPM_TRY(ensure(c, c->b_u64, sizeof(unsigned long long) * 2 * (size_t)count));
        AWPM_TRY(ensure(c, c->b_f64, sizeof(double) * 2 * (size_t)count));
        bw.colmat = (int32_t *)c->b_colmat.p;
        bw.tilemat = (int32_t *)c->b_tilemat.p;
        int32_t *i32 = (int32_t *)c->b_i32.p;
        bw.mdone = i32;
        bw.miter = i32 + count;
        bw.mconv = i32 + 2 * (size_t)count;
        bw.mnnz = i32 + 3 * (size_t)count;
        bw.active = i32 + 5 * (size_t)count;
        unsigned long long *u64 = (unsigned long long *)c->b_u64.p;
        bw.mflips = u64;
        bw.mcycles = u64 + count;
        double *f64 = (double *)c->b_f64.p;
        bw.mw_in = f64;
        bw.mw_out = f64 + count;
    }
    wk.mc = (int32_t *)c->mc.p;
    wk.mr = (int32_t *)c->mr.p;
    wk.wm = (double *)c->wm.p;
    wk.rr = (RowRec *)c->rr.p;
    wk.wmr = (double *)c->wmr.p;
    wk.colsig = (unsigned long long *)c->colsig.p;
    wk.best = (Rec *)c->best.p;
    wk.dsel = (Sel *)c->dsel.p;
    wk.tile_col = (int32_t *)c->tile_col.p;
    wk.starts = (uint32_t *)c->starts.p;
    wk.ctl = (Ctl *)c->ctl.p;
    wk.wpart = (double *)c->wpart.p;

    int passes_enqueued = 0;
    double ms_search = 0.0;
    const bool timed = (c->opt.flags & AWPM_FLAG_TIME_SEARCH) != 0;
    if (search_only) {
        launch_init(wk, 1, c->num_sms, c->stream);
        launch_search(wk, c->num_sms, c->stream);
        double *g = gain_out;
        int32_t *r = row_out;
        if (l_gain != 1) {
            AWPM_TRY(ensure(c, c->s_gain, sizeof(double) * n));
            g = (double *)c->s_gain.p;
        }
        if (l_row != 1) {
            AWPM_TRY(ensure(c, c->s_row, sizeof(int32_t) * n));
            r = (int32_t *)c->s_row.p;
        }
        launch_export_stepc(wk, g, r, c->stream);
        AWPM_TRY(check_launch());
        if (l_gain != 1)
            CUDA_TRY(cudaMemcpyAsync(gain_out, g, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                     c->stream));
        if (l_row != 1)
            CUDA_TRY(cudaMemcpyAsync(row_out, r, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                     c->stream));
    } else if (timed) {
        AWPM_TRY(run_timed(c, wk, max_passes, lookup, &ms_search, &passes_enqueued));
    } else {
        GraphKey key;
        key.n = n;
        key.nnz = nnz;
        key.max_passes = max_passes;
        key.lookup = lookup;
        key.colptr = wk.colptr;
        key.rowidx = wk.rowidx;
        key.w = wk.w;
        key.mate_in = wk.mate_in;
        key.count = count;
        key.n_off = wk.bw.n_off;
        if (!c->g_valid || !(c->g_key == key)) {
            drop_graph(c);
            AWPM_TRY(build_graph(c, wk, max_passes, lookup));
            c->g_key = key;
            c->g_valid = true;
        }
        CUDA_TRY(cudaGraphLaunch(c->g_exec, c->stream));
    }
    if (!search_only) {
        CUDA_TRY(cudaMemcpyAsync(mate_out, wk.mc, sizeof(int32_t) * n,
                                 l_out == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(c->h_ctl, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    // per-matrix results: miter, mconv, mnnz (3 x i32), mcycles (u64), mw_in, mw_out (f64)
    const size_t pm_bytes = (size_t)count * (3 * sizeof(int32_t) + 3 * 8);
    if (count > 0 && per_matrix) {
        if (c->h_batch_bytes < pm_bytes) {
            if (c->h_batch)
                cudaFreeHost(c->h_batch);
            c->h_batch = nullptr;
            c->h_batch_bytes = 0;
            CUDA_TRY(cudaMallocHost(&c->h_batch, pm_bytes));
            c->h_batch_bytes = pm_bytes;
        }
        char *hb = (char *)c->h_batch;
        CUDA_TRY(cudaMemcpyAsync(hb, wk.bw.miter, sizeof(int32_t) * 3 * (size_t)count,
                                 cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(hb + 12 * (size_t)count, wk.bw.mcycles, 8 * (size_t)count,
                                 cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(hb + 20 * (size_t)count, wk.bw.mw_in, 16 * (size_t)count,
                                 cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaEventRecord(c->ev_b, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));

    const Ctl &h = *c->h_ctl;
    int rc = code_of(h.err);
    if (rc != AWPM_OK)
        return rc;
    if (timed && !search_only) {
        for (int t = 0; t < h.iterations && t < passes_enqueued; ++t) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, c->tev[2 * t], c->tev[2 * t + 1]));
            ms_search += ms;
        }
    }
    float ms_total = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms_total, c->ev_a, c->ev_b));
    S.iterations = h.iterations;
    S.converged = h.converged;
    S.cycles_applied = (int64_t)h.cycles;
    S.edge_checks = (int64_t)(nnz - n) * (int64_t)(search_only ? 1 : h.iterations);
    S.candidates = (int64_t)h.candidates;
    S.closing_found = (int64_t)h.found;
    S.positive = (int64_t)h.positive;
    S.weight_in = h.weight_in;
    S.weight_out = search_only ? h.weight_in : h.weight_out;
    S.ms_total = ms_total;
    S.ms_search = ms_search;
    S.lookup_used = lookup;
    if (count > 0 && per_matrix) {
        const char *hb = (const char *)c->h_batch;
        const int32_t *miter = (const int32_t *)hb;
        const int32_t *mconv = miter + count;
        const int32_t *mnnz = miter + 2 * (size_t)count;
        const unsigned long long *mcyc = (const unsigned long long *)(hb + 12 * (size_t)count);
        const double *mwi = (const double *)(hb + 20 * (size_t)count);
        const double *mwo = mwi + count;
        std::vector<int32_t> off((size_t)count + 1);
        if (where(c, n_off) == 1)
            CUDA_TRY(cudaMemcpy(off.data(), n_off, sizeof(int32_t) * off.size(),
                                cudaMemcpyDeviceToHost));
        else
            std::memcpy(off.data(), n_off, sizeof(int32_t) * off.size());
        int all_conv = 1;
        for (int32_t b = 0; b < count; ++b) {
            awpm_stats &m = per_matrix[b];
            std::memset(&m, 0, sizeof(m));
            m.iterations = miter[b];
            m.converged = mconv[b];
            all_conv &= mconv[b];
            m.cycles_applied = (int64_t)mcyc[b];
            m.edge_checks = (int64_t)(mnnz[b] - (off[b + 1] - off[b])) * miter[b];
            m.weight_in = mwi[b];
            m.weight_out = mwo[b];
            m.ms_total = ms_total;
            m.lookup_used = lookup;
        }
        S.converged = all_conv;
    }
    if (count > 0) {
        // edge checks of a batch: each matrix counts only its own passes
        S.edge_checks = 0;
        if (per_matrix)
            for (int32_t b = 0; b < count; ++b)
                S.edge_checks += per_matrix[b].edge_checks;
    }
    if (st)
        *st = S;
    return AWPM_OK;
}

std::mutex g_default_mu;
std::map<int, awpm_ctx *> g_default;

}  // namespace

extern "C" {

const char *awpm_strerror(int code)
{
    switch (code) {
    case AWPM_OK: return "ok";
    case AWPM_ERR_INVALID_ARG: return "invalid argument";
    case AWPM_ERR_NOT_PERFECT: return "mate_in is not a perfect matching of stored entries";
    case AWPM_ERR_UNSORTED_OR_DUP: return "rows not strictly increasing within a column";
    case AWPM_ERR_NONFINITE: return "non-finite weight";
    case AWPM_ERR_OOM: return "out of memory";
    case AWPM_ERR_BUDGET: return "device memory budget exceeded";
    case AWPM_ERR_CUDA: return "CUDA error";
    case AWPM_ERR_TIMEOUT: return "bounded device wait gave up";
    case AWPM_ERR_NOT_FOUND: return "unknown ticket";
    default: return "unknown error";
    }
}

const char *awpm_last_error(void)
{
    return g_last_error;
}

void awpm_default_options(awpm_options *opt)
{
    if (!opt)
        return;
    std::memset(opt, 0, sizeof(*opt));
    opt->device = -1;
    opt->max_iters = 0;
    opt->lookup = AWPM_LOOKUP_AUTO;
    opt->flags = 0;
    opt->stream = nullptr;
    opt->mem_budget_bytes = 0;
}

int awpm_create(awpm_ctx **out, const awpm_options *opt)
{
    if (!out)
        return AWPM_ERR_INVALID_ARG;
    *out = nullptr;
    awpm_ctx *c = new (std::nothrow) awpm_ctx();
    if (!c)
        return AWPM_ERR_OOM;
    int rc = setup_ctx(c, opt);
    if (rc != AWPM_OK) {
        teardown_ctx(c);
        delete c;
        return rc;
    }
    *out = c;
    return AWPM_OK;
}

int awpm_destroy(awpm_ctx *ctx)
{
    if (!ctx)
        return AWPM_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        teardown_ctx(ctx);
    }
    delete ctx;
    return AWPM_OK;
}

int awpm_improve_ctx(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                     const double *weight, const int32_t *mate_in, int32_t *mate_out,
                     awpm_stats *stats)
{
    if (!ctx)
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run(ctx, n, colptr, rowidx, weight, mate_in, mate_out, stats, false, nullptr, nullptr);
}

int awpm_improve(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *weight,
                 const int32_t *mate_in, int32_t *mate_out, awpm_stats *stats)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        note_cuda(e, "cudaGetDevice", __LINE__);
        return AWPM_ERR_CUDA;
    }
    awpm_ctx *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_default_mu);
        auto it = g_default.find(dev);
        if (it == g_default.end()) {
            awpm_options o;
            awpm_default_options(&o);
            o.device = dev;
            int rc = awpm_create(&c, &o);
            if (rc != AWPM_OK)
                return rc;
            g_default[dev] = c;
        } else {
            c = it->second;
        }
    }
    return awpm_improve_ctx(c, n, colptr, rowidx, weight, mate_in, mate_out, stats);
}

int awpm_improve_batch(awpm_ctx *ctx, int32_t count, const int32_t *n_off, const int32_t *colptr,
                       const int32_t *rowidx, const double *weight, const int32_t *mate_in,
                       int32_t *mate_out, awpm_stats *per_matrix, awpm_stats *total)
{
    if (!ctx || count < 0 || (count > 0 && !n_off))
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (count == 0) {
        if (total) {
            std::memset(total, 0, sizeof(*total));
            total->converged = 1;
        }
        return AWPM_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        note_cuda(e, "cudaSetDevice", __LINE__);
        return AWPM_ERR_CUDA;
    }
    int32_t n = 0;
    if (where(ctx, n_off) == 1) {
        e = cudaMemcpy(&n, n_off + count, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            note_cuda(e, "cudaMemcpy", __LINE__);
            return AWPM_ERR_CUDA;
        }
    } else {
        n = n_off[count];
    }
    if (n <= 0)
        return AWPM_ERR_INVALID_ARG;
    std::vector<awpm_stats> tmp;
    awpm_stats *pm = per_matrix;
    if (!pm) {
        tmp.resize((size_t)count);
        pm = tmp.data();
    }
    return run(ctx, n, colptr, rowidx, weight, mate_in, mate_out, total, false, nullptr, nullptr,
               count, n_off, pm);
}

int awpm_search(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const double *weight, const int32_t *mate, double *stepc_gain, int32_t *stepc_row,
                awpm_stats *stats)
{
    if (!ctx)
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run(ctx, n, colptr, rowidx, weight, mate, nullptr, stats, true, stepc_gain, stepc_row);
}

}  // extern "C"
