// Host side of libawpm: contexts and the synchronous C ABI of include/awpm.h.
//
// A context owns a device workspace sized for the largest problem seen, the
// staging buffers for host-resident inputs, a device-resident problem
// descriptor (Work) and one instantiated CUDA graph per launch shape.  One
// solve is: write the descriptor, launch the graph (validation and
// initialisation; a conditional WHILE node whose body is one pass of Steps
// A-D, the control kernel at the end of the body deciding on the device
// whether another pass runs, Algorithm 2; the final weight reduction), copy
// the results back.  The host waits once, at the end.  Because every kernel
// reads the problem from the descriptor and runs a GPU-sized grid, the same
// graph serves every problem of the context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "awpm.h"
#include "awpm_ctx.h"
#include "awpm_internal.h"

using namespace awpm;

namespace awpm {

thread_local char g_last_error[512] = "";

void note_cuda_error(cudaError_t e, const char *what, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at line %d: %s", cudaGetErrorName(e),
             what, line, cudaGetErrorString(e));
}

}  // namespace awpm

namespace {

#define CUDA_TRY(x)                                                        \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) {                                           \
            note_cuda_error(e_, #x, __LINE__);                             \
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

// Largest nnz: positions up to nnz + 31 (a tile's last lane) stay in int32.
constexpr int32_t kMaxNnz = 0x7fffffff - 63;
// Largest nnz served by the hash lookup (slot 2 * position in int32).
constexpr int32_t kMaxHashNnz = (1 << 30) - 1;
constexpr int kLookahead = 2;
constexpr int kRing = 4;

void release(awpm_ctx *c, DevBuf &b)
{
    if (b.p) {
        cudaFree(b.p);
        c->held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
}

int ensure(awpm_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (b.bytes >= bytes)
        return AWPM_OK;
    release(c, b);
    size_t want = bytes + bytes / 8;  // headroom against small growth steps
    if (c->opt.mem_budget_bytes && c->held + want > c->opt.mem_budget_bytes) {
        want = bytes;
        if (c->held + want > c->opt.mem_budget_bytes)
            return AWPM_ERR_BUDGET;
    }
    if (c->fail_after >= 0) {  // injected failure (awpm_inject_alloc_failure)
        if (c->fail_after == 0) {
            c->fail_after = -1;
            return AWPM_ERR_OOM;
        }
        --c->fail_after;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        note_cuda_error(e, "cudaMalloc", __LINE__);
        cudaGetLastError();
        return AWPM_ERR_OOM;
    }
    b.p = p;
    b.bytes = want;
    c->held += want;
    if (c->held > c->peak)
        c->peak = c->held;
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

// Bloom filters of the long columns with the binary-search lookup (default
// on; the environment variable AWPM_BLOOM=0 switches them off, a tuning knob:
// results are the same either way).
bool bloom_enabled()
{
    static const bool on = [] {
        const char *v = getenv("AWPM_BLOOM");
        return !(v && v[0] == '0' && v[1] == 0);
    }();
    return on;
}

int code_of(unsigned err)
{
    return awpm_code_of_bits(err);
}

int check_sink(const Sink &k)
{
    if (k.err != cudaSuccess) {
        note_cuda_error(k.err, "kernel launch", __LINE__);
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    return AWPM_OK;
}

// Index of a lookup in the per-lookup tables: binary search, hash, row marking.
int lookup_slot(int lookup)
{
    return lookup == AWPM_LOOKUP_HASH ? 1 : lookup == AWPM_LOOKUP_ROWMARK ? 2 : 0;
}

Shape shape_of(const awpm_ctx *c, bool batch, int lookup, bool wide, int32_t ntiles)
{
    Shape sh;
    sh.num_sms = c->num_sms;
    sh.batch = batch;
    sh.lookup = lookup;
    sh.wide = wide;
    sh.search_bps = c->search_bps[batch ? 1 : 0][lookup_slot(lookup)][wide ? 1 : 0];
    sh.search_waves = search_waves(sh.num_sms, sh.search_bps, ntiles);
    sh.select = c->opt.select == AWPM_SELECT_GREEDY ? AWPM_SELECT_GREEDY : AWPM_SELECT_STEP_D;
    return sh;
}

int ilog2(int64_t x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        ++l;
    }
    return l;
}

// The solve graph of one launch shape: initialisation, WHILE{pass}, final
// sum, assembled node by node (no stream capture).
int build_graph(awpm_ctx *c, const Shape &sh, cudaGraphExec_t *out)
{
    const Work *d = (const Work *)c->d_work.p;
    cudaGraph_t top = nullptr, g_init = nullptr, g_final = nullptr;
    cudaGraphNode_t n_init, n_cond, n_final;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    int rc = AWPM_OK;
    cudaError_t e;
    Sink si, sf, sb;
    if ((e = cudaGraphCreate(&g_init, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&g_final, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&top, 0)) != cudaSuccess) {
        note_cuda_error(e, "cudaGraphCreate", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    si.graph = g_init;
    launch_init(d, sh, si);
    launch_weight_sum(d, sh, false, si);
    sf.graph = g_final;
    launch_weight_sum(d, sh, true, sf);
    if (si.err != cudaSuccess || sf.err != cudaSuccess) {
        note_cuda_error(si.err != cudaSuccess ? si.err : sf.err, "kernel nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_init, top, nullptr, 0, g_init)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault)) !=
            cudaSuccess) {
        note_cuda_error(e, "graph assembly", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_cond, top, &n_init, nullptr, 1, &cp)) != cudaSuccess) {
        note_cuda_error(e, "conditional node", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    sb.graph = cp.conditional.phGraph_out[0];
    launch_search(d, sh, sb);
    if (sh.select == AWPM_SELECT_GREEDY) {
        // the selection's rounds: a WHILE node nested in the pass body
        cudaGraphConditionalHandle h2;
        cudaGraphNodeParams cp2 = {cudaGraphNodeTypeConditional};
        cudaGraphNode_t n_inner;
        if ((e = cudaGraphConditionalHandleCreate(&h2, sb.graph, 0, 0)) != cudaSuccess) {
            note_cuda_error(e, "inner conditional handle", __LINE__);
            rc = AWPM_ERR_CUDA;
            goto done;
        }
        launch_greedy_select_begin(d, sh, true, h2, sb);
        cp2.conditional.handle = h2;
        cp2.conditional.type = cudaGraphCondTypeWhile;
        cp2.conditional.size = 1;
        if (sb.err != cudaSuccess ||
            (e = cudaGraphAddNode(&n_inner, sb.graph, &sb.last, nullptr, 1, &cp2)) !=
                cudaSuccess) {
            note_cuda_error(sb.err != cudaSuccess ? sb.err : e, "inner conditional node",
                            __LINE__);
            rc = AWPM_ERR_CUDA;
            goto done;
        }
        Sink sr;
        sr.graph = cp2.conditional.phGraph_out[0];
        launch_greedy_select_round(d, sh, true, h2, sr);
        if (sr.err != cudaSuccess) {
            note_cuda_error(sr.err, "selection round nodes", __LINE__);
            rc = AWPM_ERR_CUDA;
            goto done;
        }
        sb.last = n_inner;
        launch_greedy_select_end_and_flip(d, sh, sb);
    } else if (!sh.batch) {
        // the flip's last block ends the pass (no control kernel)
        launch_select_flip_control_graph(d, sh, h, sb);
    } else {
        launch_select_and_flip(d, sh, sb);
    }
    if (sh.batch || sh.select == AWPM_SELECT_GREEDY)
        launch_control(d, sh, true, h, sb);
    if (sb.err != cudaSuccess) {
        note_cuda_error(sb.err, "pass body nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_final, top, &n_cond, 1, g_final)) != cudaSuccess ||
        (e = cudaGraphInstantiate(out, top, 0)) != cudaSuccess) {
        note_cuda_error(e, "graph instantiation", __LINE__);
        *out = nullptr;
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

// Graph of the greedy maximal matching: state reset and input checks, a
// conditional WHILE node over the rounds, the matched-weight sum.
int build_greedy_graph(awpm_ctx *c, const Shape &sh, cudaGraphExec_t *out)
{
    const Work *d = (const Work *)c->d_work.p;
    cudaGraph_t top = nullptr, g_init = nullptr, g_final = nullptr;
    cudaGraphNode_t n_init, n_cond, n_final;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    int rc = AWPM_OK;
    cudaError_t e;
    Sink si, sf, sb;
    if ((e = cudaGraphCreate(&g_init, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&g_final, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&top, 0)) != cudaSuccess) {
        note_cuda_error(e, "cudaGraphCreate", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    si.graph = g_init;
    launch_greedy_init(d, sh, si);
    sf.graph = g_final;
    launch_weight_sum(d, sh, true, sf);
    if (si.err != cudaSuccess || sf.err != cudaSuccess) {
        note_cuda_error(si.err != cudaSuccess ? si.err : sf.err, "kernel nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_init, top, nullptr, 0, g_init)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault)) !=
            cudaSuccess) {
        note_cuda_error(e, "graph assembly", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_cond, top, &n_init, nullptr, 1, &cp)) != cudaSuccess) {
        note_cuda_error(e, "conditional node", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    sb.graph = cp.conditional.phGraph_out[0];
    launch_greedy_round(d, sh, true, h, sb);
    if (sb.err != cudaSuccess) {
        note_cuda_error(sb.err, "round body nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_final, top, &n_cond, 1, g_final)) != cudaSuccess ||
        (e = cudaGraphInstantiate(out, top, 0)) != cudaSuccess) {
        note_cuda_error(e, "graph instantiation", __LINE__);
        *out = nullptr;
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

// Graph of the maximum cardinality matching: load and checks; a WHILE node
// over the phases whose body starts a phase, runs a WHILE node over the
// levels, augments and decides whether to continue; the result stored.
int build_mcm_graph(awpm_ctx *c, const Shape &sh, cudaGraphExec_t *out)
{
    const Work *d = (const Work *)c->d_work.p;
    cudaGraph_t top = nullptr, g_init = nullptr, g_final = nullptr;
    cudaGraphNode_t n_init, n_cond, n_final, n_inner;
    cudaGraphConditionalHandle h1, h2;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cudaGraphNodeParams cp2 = {cudaGraphNodeTypeConditional};
    int rc = AWPM_OK;
    cudaError_t e;
    Sink si, sf, sb, sl;
    if ((e = cudaGraphCreate(&g_init, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&g_final, 0)) != cudaSuccess ||
        (e = cudaGraphCreate(&top, 0)) != cudaSuccess) {
        note_cuda_error(e, "cudaGraphCreate", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    si.graph = g_init;
    launch_mcm_load(d, sh, si);
    sf.graph = g_final;
    launch_mcm_store(d, sh, sf);
    if (si.err != cudaSuccess || sf.err != cudaSuccess) {
        note_cuda_error(si.err != cudaSuccess ? si.err : sf.err, "kernel nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_init, top, nullptr, 0, g_init)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h1, top, 1, cudaGraphCondAssignDefault)) !=
            cudaSuccess) {
        note_cuda_error(e, "graph assembly", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    cp.conditional.handle = h1;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_cond, top, &n_init, nullptr, 1, &cp)) != cudaSuccess) {
        note_cuda_error(e, "phase node", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    sb.graph = cp.conditional.phGraph_out[0];
    if ((e = cudaGraphConditionalHandleCreate(&h2, sb.graph, 0, 0)) != cudaSuccess) {
        note_cuda_error(e, "level handle", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    launch_mcm_phase(d, sh, sb);
    launch_mcm_cond_level(d, sh, h2, sb);
    cp2.conditional.handle = h2;
    cp2.conditional.type = cudaGraphCondTypeWhile;
    cp2.conditional.size = 1;
    if (sb.err != cudaSuccess ||
        (e = cudaGraphAddNode(&n_inner, sb.graph, &sb.last, nullptr, 1, &cp2)) != cudaSuccess) {
        note_cuda_error(sb.err != cudaSuccess ? sb.err : e, "level node", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    sl.graph = cp2.conditional.phGraph_out[0];
    launch_mcm_level_graph(d, sh, h2, sl);
    sb.last = n_inner;
    launch_mcm_augment(d, sh, sb);
    launch_mcm_cond_phase(d, sh, h1, sb);
    if (sb.err != cudaSuccess || sl.err != cudaSuccess) {
        note_cuda_error(sb.err != cudaSuccess ? sb.err : sl.err, "phase body nodes", __LINE__);
        rc = AWPM_ERR_CUDA;
        goto done;
    }
    if ((e = cudaGraphAddChildGraphNode(&n_final, top, &n_cond, 1, g_final)) != cudaSuccess ||
        (e = cudaGraphInstantiate(out, top, 0)) != cudaSuccess) {
        note_cuda_error(e, "graph instantiation", __LINE__);
        *out = nullptr;
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
int run_timed(awpm_ctx *c, const Shape &sh, int max_passes, int *passes_enqueued)
{
    cudaStream_t s = c->stream;
    const Work *d = (const Work *)c->d_work.p;
    Ctl *ctl = (Ctl *)c->ctl.p;
    Sink k;
    k.stream = s;
    launch_init(d, sh, k);
    launch_weight_sum(d, sh, false, k);
    AWPM_TRY(check_sink(k));
    int t = 0;
    for (; t < max_passes; ++t) {
        if (t >= kLookahead) {
            const int slot = (t - kLookahead) % kRing;
            CUDA_TRY(cudaEventSynchronize(c->flagev[slot]));
            if (!c->h_active[slot])
                break;
        }
        NvtxRange pass_range("pass");
        AWPM_TRY(ensure_timing_events(c, (size_t)t + 1));
        CUDA_TRY(cudaEventRecord(c->tev[2 * t], s));
        launch_search(d, sh, k);
        CUDA_TRY(cudaEventRecord(c->tev[2 * t + 1], s));
        if (sh.select == AWPM_SELECT_GREEDY) {
            // the selection's rounds, driven from the host by the count of
            // undecided winners
            launch_greedy_select_begin(d, sh, false, cudaGraphConditionalHandle(), k);
            for (;;) {
                AWPM_TRY(check_sink(k));
                CUDA_TRY(cudaMemcpyAsync(&c->h_ctl->live, &ctl->live, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
                CUDA_TRY(cudaStreamSynchronize(s));
                const int32_t live = c->h_ctl->live;
                CUDA_TRY(cudaMemsetAsync(&ctl->live, 0, sizeof(int32_t), s));
                if (live <= 0)
                    break;
                launch_greedy_select_round(d, sh, false, cudaGraphConditionalHandle(), k);
            }
            launch_greedy_select_end_and_flip(d, sh, k);
        } else {
            launch_select_and_flip(d, sh, k);
        }
        launch_control(d, sh, false, cudaGraphConditionalHandle(), k);
        AWPM_TRY(check_sink(k));
        CUDA_TRY(cudaMemcpyAsync(&c->h_active[t % kRing], &ctl->active, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(c->flagev[t % kRing], s));
    }
    launch_weight_sum(d, sh, true, k);
    AWPM_TRY(check_sink(k));
    *passes_enqueued = t;
    return AWPM_OK;
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

std::mutex g_default_mu;
std::map<int, awpm_ctx *> g_default;

}  // namespace

namespace awpm {

size_t ctx_bytes_needed(int32_t n, int32_t nnz, bool host_inputs, int lookup, int select)
{
    const size_t N = (size_t)n, Z = (size_t)nnz, T = Z / kTile + 1;
    size_t b = N * (4 + 4 + 8 + sizeof(RowRange) + 8 + 8 + sizeof(Rec) + sizeof(Sel) + 4) + N / 8 +
               4 * T +
               4 * (Z / 32 + 1) + sizeof(Ctl) + 8 * kWsumBlocks;
    if (lookup != AWPM_LOOKUP_BSEARCH)  // hash tables (AUTO may pick them)
        b += 16 * Z;
    if (lookup != AWPM_LOOKUP_HASH && lookup != AWPM_LOOKUP_ROWMARK)  // Bloom filters
        b += Z + 4;
    if (lookup == AWPM_LOOKUP_ROWMARK)  // marks, transpose, radix-sort buffers
        b += 12 * N + 4 + 16 * Z + 4 * (size_t)kRsBins * (Z / kRsTile + 1) + 4 * kRsBins;
    if (host_inputs)
        b += 4 * (N + 1) + 12 * Z + 8 * N;
    if (select == AWPM_SELECT_GREEDY)  // selection records and three bitmaps
        b += sizeof(Sel) * N + 3 * 4 * (N / 32 + 1);
    return b + b / 8;
}

size_t ctx_bytes_held(const awpm_ctx *c)
{
    return c->held;
}

void ctx_trim(awpm_ctx *c)
{
    DevBuf *bufs[] = {&c->mc,      &c->mr,       &c->wm,       &c->rr,       &c->rsig,
                      &c->colsig,  &c->best,     &c->dsel,     &c->tile_col, &c->starts,
                      &c->wpart,   &c->htab,     &c->b_noff,   &c->b_colmat, &c->b_tilemat,
                      &c->b_tlist, &c->b_i32,    &c->b_u64,    &c->b_f64,    &c->s_colptr,
                      &c->s_rowidx, &c->s_w,     &c->s_mate,   &c->s_out,    &c->s_gain,
                      &c->s_row,   &c->winbits,  &c->wkey,     &c->bloom,    &c->gckey,
                      &c->gcpos,   &c->grkey,    &c->grcol,    &c->gmate,    &c->gtdead,
                      &c->psel,    &c->pslive,   &c->pstaken,  &c->psused,   &c->wt_cmax,
                      &c->wt_rmax, &c->wt_stage, &c->mroot,    &c->mrpar,    &c->mfront,
                      &c->mnext,   &c->mroff,    &c->mtend,    &c->mtouch,
                      &c->mstage,  &c->mcolof,   &c->mtiles,   &c->rowsig,   &c->trowptr,
                      &c->rs_k0,   &c->rs_k1,    &c->rs_v0,    &c->rs_v1,    &c->rs_hist,
                      &c->rs_sums};
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    for (DevBuf *b : bufs)
        release(c, *b);
    c->rec_clean = 0;
    cudaGetLastError();
}

int setup_ctx(awpm_ctx *c, const awpm_options *opt)
{
    if (opt)
        c->opt = *opt;
    else
        awpm_default_options(&c->opt);
    if (c->opt.max_iters < 0 || c->opt.lookup < 0 || c->opt.lookup > 3 || c->opt.slots < 0 ||
        c->opt.select < 0 || c->opt.select > 1)
        return AWPM_ERR_INVALID_ARG;
    int dev = c->opt.device;
    if (dev < 0)
        CUDA_TRY(cudaGetDevice(&dev));
    c->device = dev;
    CUDA_TRY(cudaSetDevice(dev));
    CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    c->search_wide = default_search_wide();
    for (int b = 0; b < 2; ++b)
        for (int p = 0; p < 2; ++p) {
            c->search_bps[b][0][p] = search_blocks_per_sm(AWPM_LOOKUP_BSEARCH, b == 1, p == 1);
            c->search_bps[b][1][p] = search_blocks_per_sm(AWPM_LOOKUP_HASH, b == 1, p == 1);
            c->search_bps[b][2][p] = search_blocks_per_sm(AWPM_LOOKUP_ROWMARK, b == 1, p == 1);
        }
    if (c->opt.stream) {
        c->stream = (cudaStream_t)c->opt.stream;
        c->own_stream = false;
    } else {
        CUDA_TRY(cudaStreamCreate(&c->stream));
        c->own_stream = true;
    }
    AWPM_TRY(ensure(c, c->d_work, sizeof(Work)));
    CUDA_TRY(cudaMallocHost((void **)&c->h_work, sizeof(Work)));
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
    for (int b = 0; b < 2; ++b)
        for (int h = 0; h < 3; ++h)
            for (int p = 0; p < 2; ++p)
                for (int v = 0; v < 2; ++v)
                    for (int q = 0; q < 2; ++q)
                        if (c->g_exec[b][h][p][v][q]) {
                            cudaGraphExecDestroy(c->g_exec[b][h][p][v][q]);
                            c->g_exec[b][h][p][v][q] = nullptr;
                        }
    for (int v = 0; v < 2; ++v) {
        if (c->g_greedy[v]) {
            cudaGraphExecDestroy(c->g_greedy[v]);
            c->g_greedy[v] = nullptr;
        }
        if (c->g_mcm[v]) {
            cudaGraphExecDestroy(c->g_mcm[v]);
            c->g_mcm[v] = nullptr;
        }
    }
    DevBuf *bufs[] = {&c->mc,      &c->mr,       &c->wm,       &c->rr,       &c->rsig,
                      &c->colsig,  &c->best,     &c->dsel,     &c->tile_col, &c->starts,
                      &c->ctl,     &c->wpart,    &c->htab,     &c->b_noff,   &c->b_colmat,
                      &c->b_tilemat, &c->b_tlist, &c->b_i32,  &c->b_u64,    &c->b_f64,    &c->s_colptr,
                      &c->s_rowidx, &c->s_w,     &c->s_mate,   &c->s_out,    &c->s_gain,
                      &c->s_row,   &c->d_work,   &c->winbits,  &c->wkey,     &c->bloom,    &c->gckey,
                      &c->gcpos,   &c->grkey,    &c->grcol,    &c->gmate,
                      &c->gtdead,  &c->psel,     &c->pslive,   &c->pstaken,  &c->psused,
                      &c->wt_cmax, &c->wt_rmax,  &c->wt_stage,
                      &c->mroot,   &c->mrpar,    &c->mfront,   &c->mnext,    &c->mroff,
                      &c->mtend,   &c->mtouch,   &c->mstage,   &c->mcolof,
                      &c->mtiles,  &c->rowsig,   &c->trowptr,  &c->rs_k0,    &c->rs_k1,
                      &c->rs_v0,   &c->rs_v1,    &c->rs_hist,  &c->rs_sums};
    for (DevBuf *b : bufs)
        release(c, *b);
    if (c->h_work)
        cudaFreeHost(c->h_work);
    if (c->h_ctl)
        cudaFreeHost(c->h_ctl);
    if (c->h_active)
        cudaFreeHost(c->h_active);
    if (c->h_batch)
        cudaFreeHost(c->h_batch);
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

int ctx_enqueue(awpm_ctx *c, const Request &r)
{
    NvtxRange nvtx_range("enqueue");
    Pending &pd = c->pend;
    pd = Pending();
    const int32_t n = r.n;
    if (n < 0 || (n > 0 && (!r.colptr || !r.mate_in)) ||
        (!r.search_only && n > 0 && !r.mate_out) ||
        (r.search_only && n > 0 && (!r.gain_out || !r.row_out)) || r.count < 0 ||
        (r.count > 0 && !r.n_off))
        return AWPM_ERR_INVALID_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    pd.lookup = (c->opt.lookup == AWPM_LOOKUP_HASH || c->opt.lookup == AWPM_LOOKUP_ROWMARK)
                    ? c->opt.lookup
                    : AWPM_LOOKUP_BSEARCH;
    pd.search_only = r.search_only;
    if (n == 0) {
        pd.active = true;
        pd.trivial = true;
        return AWPM_OK;
    }
    const int l_colptr = where(c, r.colptr), l_rowidx = where(c, r.rowidx),
              l_w = where(c, r.weight), l_mate = where(c, r.mate_in);
    const int l_out = r.search_only ? 0 : where(c, r.mate_out);
    const int l_gain = r.search_only ? where(c, r.gain_out) : 0;
    const int l_row = r.search_only ? where(c, r.row_out) : 0;
    const int l_off = r.count > 0 ? where(c, r.n_off) : 0;
    if (l_colptr < 0 || l_rowidx < 0 || l_w < 0 || l_mate < 0 || l_out < 0 || l_gain < 0 ||
        l_row < 0 || l_off < 0)
        return AWPM_ERR_INVALID_ARG;

    int32_t nnz = r.nnz;
    if (nnz < 0) {
        if (l_colptr == 1) {
            CUDA_TRY(cudaMemcpyAsync(c->h_ctl, r.colptr + n, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            std::memcpy(&nnz, c->h_ctl, sizeof(int32_t));
        } else {
            nnz = r.colptr[n];
        }
    }
    // tile arithmetic is int32: positions up to nnz + 31 must fit
    if (nnz < 0 || nnz > kMaxNnz || (nnz > 0 && (!r.rowidx || !r.weight)))
        return AWPM_ERR_INVALID_ARG;
    const bool timed = (c->opt.flags & AWPM_FLAG_TIME_SEARCH) != 0;
    // launch configuration: given, or the autotuner's (AWPM_LOOKUP_AUTO)
    int lookup = pd.lookup;
    bool wide = c->search_wide;
    if (c->opt.lookup == AWPM_LOOKUP_AUTO && !r.search_only && !timed) {
        const uint64_t key = ((uint64_t)(r.count > 0) << 62) | ((uint64_t)ilog2(n) << 32) |
                             (uint64_t)ilog2(nnz > 0 ? nnz : 1);
        TuneEntry &te = c->tune[key];
        const int cfg = te.chosen >= 0 ? te.chosen : te.trials;
        lookup = kTune[cfg].lookup;
        wide = kTune[cfg].wide;
        if (te.chosen < 0) {
            pd.tune_cfg = cfg;
            pd.tune_key = key;
        }
    }
    // hash slots are addressed as 2 * position in int32
    if (lookup == AWPM_LOOKUP_HASH && nnz > kMaxHashNnz)
        lookup = AWPM_LOOKUP_BSEARCH;
    pd.lookup = lookup;
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    const int32_t max_passes = c->opt.max_iters > 0 ? c->opt.max_iters : AWPM_PASS_CAP;
    const int32_t count = r.count;

    AWPM_TRY(ensure(c, c->mc, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mr, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->wm, sizeof(double) * n));
    AWPM_TRY(ensure(c, c->rr, sizeof(RowRange) * n));
    AWPM_TRY(ensure(c, c->rsig, sizeof(unsigned long long) * n));
    AWPM_TRY(ensure(c, c->colsig, sizeof(unsigned long long) * n));
    const void *best_was = c->best.p, *dsel_was = c->dsel.p;
    AWPM_TRY(ensure(c, c->best, sizeof(Rec) * n));
    AWPM_TRY(ensure(c, c->dsel, sizeof(Sel) * n));
    if (c->best.p != best_was || c->dsel.p != dsel_was)
        c->rec_clean = 0;
    AWPM_TRY(ensure(c, c->winbits, sizeof(uint32_t) * ((size_t)n / 32 + 1)));
    AWPM_TRY(ensure(c, c->wkey, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->tile_col, sizeof(int32_t) * ((size_t)ntiles + 1)));
    AWPM_TRY(ensure(c, c->starts, sizeof(uint32_t) * (((size_t)nnz + 31) / 32 + 1)));
    AWPM_TRY(ensure(c, c->ctl, sizeof(Ctl)));
    AWPM_TRY(ensure(c, c->wpart, sizeof(double) * kWsumBlocks));
    const int32_t rs_tiles = (int32_t)(((int64_t)nnz + kRsTile - 1) / kRsTile);
    int32_t rs_passes = 1;
    while (rs_passes < 4 && ((int64_t)(n - 1) >> (8 * rs_passes)) > 0)
        ++rs_passes;
    if (lookup == AWPM_LOOKUP_HASH) {
        AWPM_TRY(ensure(c, c->htab, sizeof(unsigned long long) * 2 * (size_t)nnz));
    } else if (lookup == AWPM_LOOKUP_ROWMARK) {
        const size_t m = (size_t)kRsBins * (size_t)rs_tiles;
        AWPM_TRY(ensure(c, c->rowsig, sizeof(unsigned long long) * n));
        AWPM_TRY(ensure(c, c->trowptr, sizeof(int32_t) * ((size_t)n + 1)));
        AWPM_TRY(ensure(c, c->rs_k0, sizeof(int32_t) * ((size_t)nnz + 1)));
        AWPM_TRY(ensure(c, c->rs_k1, sizeof(int32_t) * ((size_t)nnz + 1)));
        AWPM_TRY(ensure(c, c->rs_v0, sizeof(int32_t) * ((size_t)nnz + 1)));
        AWPM_TRY(ensure(c, c->rs_v1, sizeof(int32_t) * ((size_t)nnz + 1)));
        AWPM_TRY(ensure(c, c->rs_hist, sizeof(int32_t) * (m + 1)));
        AWPM_TRY(ensure(c, c->rs_sums, sizeof(int32_t) * (m / kScanChunk + 2)));
    } else {
        AWPM_TRY(ensure(c, c->bloom, sizeof(uint32_t) * ((size_t)nnz / 4 + 1)));
    }
    const bool ps = c->opt.select == AWPM_SELECT_GREEDY && !r.search_only;
    if (ps) {
        AWPM_TRY(ensure(c, c->psel, sizeof(Sel) * n));
        AWPM_TRY(ensure(c, c->pslive, sizeof(uint32_t) * ((size_t)n / 32 + 1)));
        AWPM_TRY(ensure(c, c->pstaken, sizeof(uint32_t) * ((size_t)n / 32 + 1)));
        AWPM_TRY(ensure(c, c->psused, sizeof(uint32_t) * ((size_t)n / 32 + 1)));
    }

    // the solve graph of this launch shape, built once (before the timed span)
    const Shape sh = shape_of(c, count > 0, lookup, wide, ntiles);
    cudaGraphExec_t gexec = nullptr;
    if (!r.search_only && !timed) {
        cudaGraphExec_t &g = c->g_exec[count > 0 ? 1 : 0][lookup_slot(lookup)]
                                      [wide ? 1 : 0][sh.search_waves - 1][sh.select];
        if (!g)
            AWPM_TRY(build_graph(c, sh, &g));
        gexec = g;
    }
    CUDA_TRY(cudaEventRecord(c->ev_a, c->stream));
    Work &wk = *c->h_work;
    std::memset(&wk, 0, sizeof(Work));
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = ntiles;
    wk.max_passes = max_passes;
    wk.lookup = lookup;
    AWPM_TRY(stage_in(c, c->s_colptr, r.colptr, (size_t)n + 1, l_colptr, &wk.colptr));
    AWPM_TRY(stage_in(c, c->s_rowidx, r.rowidx, (size_t)nnz, l_rowidx, &wk.rowidx));
    AWPM_TRY(stage_in(c, c->s_w, r.weight, (size_t)nnz, l_w, &wk.w));
    AWPM_TRY(stage_in(c, c->s_mate, r.mate_in, (size_t)n, l_mate, &wk.mate_in));
    wk.mc = (int32_t *)c->mc.p;
    wk.mr = (int32_t *)c->mr.p;
    wk.wm = (double *)c->wm.p;
    wk.rsig = (unsigned long long *)c->rsig.p;
    wk.rrange = (RowRange *)c->rr.p;
    wk.colsig = (unsigned long long *)c->colsig.p;
    wk.htab = lookup == AWPM_LOOKUP_HASH ? (unsigned long long *)c->htab.p : nullptr;
    wk.bloom = lookup == AWPM_LOOKUP_BSEARCH && bloom_enabled() ? (uint32_t *)c->bloom.p : nullptr;
    if (lookup == AWPM_LOOKUP_ROWMARK) {
        wk.rowsig = (unsigned long long *)c->rowsig.p;
        wk.trowptr = (int32_t *)c->trowptr.p;
        wk.rs_key[0] = (int32_t *)c->rs_k0.p;
        wk.rs_key[1] = (int32_t *)c->rs_k1.p;
        wk.rs_val[0] = (int32_t *)c->rs_v0.p;
        wk.rs_val[1] = (int32_t *)c->rs_v1.p;
        wk.rs_hist = (int32_t *)c->rs_hist.p;
        wk.rs_sums = (int32_t *)c->rs_sums.p;
        wk.rs_tiles = rs_tiles;
        wk.rs_passes = rs_passes;
        wk.tpos = wk.rs_val[(rs_passes - 1) & 1];
    }
    if (ps) {
        wk.psel = (Sel *)c->psel.p;
        wk.pslive = (uint32_t *)c->pslive.p;
        wk.pstaken = (uint32_t *)c->pstaken.p;
        wk.psused = (uint32_t *)c->psused.p;
    }
    wk.best = (Rec *)c->best.p;
    wk.dsel = (Sel *)c->dsel.p;
    {
        // solves with Step D's selection (single or batched) leave the
        // records empty: every pass's flip clears the records of its winners
        const bool keeps_clean = !r.search_only && !ps;
        wk.rec_clean = keeps_clean && (int64_t)n <= c->rec_clean ? 1 : 0;
        pd.rec_clean_after = keeps_clean ? std::max<int64_t>(n, c->rec_clean) : 0;
        c->rec_clean = 0;
    }
    wk.winbits = (uint32_t *)c->winbits.p;
    wk.wkey = (int32_t *)c->wkey.p;
    wk.tile_col = (int32_t *)c->tile_col.p;
    wk.starts = (uint32_t *)c->starts.p;
    wk.ctl = (Ctl *)c->ctl.p;
    wk.wpart = (double *)c->wpart.p;
    if (count > 0) {
        BatchWork &bw = wk.bw;
        bw.count = count;
        AWPM_TRY(stage_in(c, c->b_noff, r.n_off, (size_t)count + 1, l_off, &bw.n_off));
        AWPM_TRY(ensure(c, c->b_colmat, sizeof(int32_t) * n));
        AWPM_TRY(ensure(c, c->b_tilemat, sizeof(int32_t) * ((size_t)ntiles + 1)));
        AWPM_TRY(ensure(c, c->b_i32, sizeof(int32_t) * (5 * (size_t)count + 2)));
        AWPM_TRY(ensure(c, c->b_tlist, sizeof(int32_t) * ((size_t)ntiles + 1)));
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
        bw.tlist_n = i32 + 5 * (size_t)count + 1;
        bw.tlist = (int32_t *)c->b_tlist.p;
        unsigned long long *u64 = (unsigned long long *)c->b_u64.p;
        bw.mflips = u64;
        bw.mcycles = u64 + count;
        double *f64 = (double *)c->b_f64.p;
        bw.mw_in = f64;
        bw.mw_out = f64 + count;
        pd.n_off.resize((size_t)count + 1);
        if (l_off == 1)
            CUDA_TRY(cudaMemcpyAsync(pd.n_off.data(), r.n_off, sizeof(int32_t) * (count + 1),
                                     cudaMemcpyDeviceToHost, c->stream));
        else
            std::memcpy(pd.n_off.data(), r.n_off, sizeof(int32_t) * (count + 1));
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_work.p, c->h_work, sizeof(Work), cudaMemcpyHostToDevice,
                             c->stream));
    const Work *d = (const Work *)c->d_work.p;

    if (r.search_only) {
        Sink k;
        k.stream = c->stream;
        launch_init(d, sh, k);
        launch_search(d, sh, k);
        double *g = r.gain_out;
        int32_t *row = r.row_out;
        if (l_gain != 1) {
            AWPM_TRY(ensure(c, c->s_gain, sizeof(double) * n));
            g = (double *)c->s_gain.p;
        }
        if (l_row != 1) {
            AWPM_TRY(ensure(c, c->s_row, sizeof(int32_t) * n));
            row = (int32_t *)c->s_row.p;
        }
        launch_export_stepc(d, sh, g, row, k);
        AWPM_TRY(check_sink(k));
        if (l_gain != 1)
            CUDA_TRY(cudaMemcpyAsync(r.gain_out, g, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                     c->stream));
        if (l_row != 1)
            CUDA_TRY(cudaMemcpyAsync(r.row_out, row, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                     c->stream));
    } else if (timed) {
        AWPM_TRY(run_timed(c, sh, max_passes, &pd.passes_enqueued));
    } else {
        CUDA_TRY(cudaGraphLaunch(gexec, c->stream));
    }
    if (!r.search_only)
        CUDA_TRY(cudaMemcpyAsync(r.mate_out, wk.mc, sizeof(int32_t) * n,
                                 l_out == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->h_ctl, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    if (count > 0) {
        // per-matrix results: miter, mconv, mnnz (i32), mcycles (u64), mw_in, mw_out (f64)
        const size_t pm_bytes = (size_t)count * (3 * sizeof(int32_t) + 3 * 8);
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
    pd.active = true;
    pd.timed = timed && !r.search_only;
    pd.n = n;
    pd.nnz = nnz;
    pd.count = count;
    return AWPM_OK;
}

int ctx_finish(awpm_ctx *c, awpm_stats *st, awpm_stats *per_matrix)
{
    NvtxRange nvtx_range("finish");
    Pending &pd = c->pend;
    if (!pd.active)
        return AWPM_ERR_INVALID_ARG;
    pd.active = false;
    awpm_stats S;
    std::memset(&S, 0, sizeof(S));
    S.lookup_used = pd.lookup;
    if (pd.trivial) {
        S.iterations = pd.search_only ? 0 : 1;
        S.converged = 1;
        if (st)
            *st = S;
        return AWPM_OK;
    }
    CUDA_TRY(cudaEventSynchronize(c->ev_b));
    const Ctl &h = *c->h_ctl;
    const int rc = code_of(h.err);
    if (rc != AWPM_OK)
        return rc;
    c->rec_clean = pd.rec_clean_after;
    double ms_search = 0.0;
    if (pd.timed) {
        for (int t = 0; t < h.iterations && t < pd.passes_enqueued; ++t) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, c->tev[2 * t], c->tev[2 * t + 1]));
            ms_search += ms;
        }
    }
    float ms_total = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms_total, c->ev_a, c->ev_b));
    if (pd.tune_cfg >= 0) {
        TuneEntry &te = c->tune[pd.tune_key];
        if (te.chosen < 0 && pd.tune_cfg == te.trials) {
            te.ms[te.trials++] = ms_total;
            if (te.trials == kTuneConfigs) {
                int best = 0;
                for (int k = 1; k < kTuneConfigs; ++k)
                    if (te.ms[k] < te.ms[best])
                        best = k;
                te.chosen = best;
            }
        }
        pd.tune_cfg = -1;
    }
    S.iterations = h.iterations;
    S.converged = h.converged;
    S.cycles_applied = (int64_t)h.cycles;
    S.edge_checks = (int64_t)(pd.nnz - pd.n) * (int64_t)(pd.search_only ? 1 : h.iterations);
    S.candidates = (int64_t)h.candidates;
    S.closing_found = (int64_t)h.found;
    S.positive = (int64_t)h.positive;
    S.weight_in = h.weight_in;
    S.weight_out = pd.search_only ? h.weight_in : h.weight_out;
    S.ms_total = ms_total;
    S.ms_search = ms_search;
    if (pd.count > 0) {
        const int32_t count = pd.count;
        const char *hb = (const char *)c->h_batch;
        const int32_t *miter = (const int32_t *)hb;
        const int32_t *mconv = miter + count;
        const int32_t *mnnz = miter + 2 * (size_t)count;
        const unsigned long long *mcyc = (const unsigned long long *)(hb + 12 * (size_t)count);
        const double *mwi = (const double *)(hb + 20 * (size_t)count);
        const double *mwo = mwi + count;
        int all_conv = 1;
        S.edge_checks = 0;
        for (int32_t b = 0; b < count; ++b) {
            const int64_t ec = (int64_t)(mnnz[b] - (pd.n_off[b + 1] - pd.n_off[b])) * miter[b];
            S.edge_checks += ec;
            all_conv &= mconv[b];
            if (!per_matrix)
                continue;
            awpm_stats &m = per_matrix[b];
            std::memset(&m, 0, sizeof(m));
            m.iterations = miter[b];
            m.converged = mconv[b];
            m.cycles_applied = (int64_t)mcyc[b];
            m.edge_checks = ec;
            m.weight_in = mwi[b];
            m.weight_out = mwo[b];
            m.ms_total = ms_total;
            m.lookup_used = pd.lookup;
        }
        S.converged = all_conv;
    }
    if (st)
        *st = S;
    return AWPM_OK;
}

}  // namespace awpm

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
    case AWPM_ERR_TIMEOUT: return "a bounded device-side retry or loop gave up";
    case AWPM_ERR_NOT_FOUND: return "unknown ticket";
    case AWPM_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of awpm_search_noalloc";
    case AWPM_ERR_INTERNAL: return "internal consistency check failed (library bug)";
    case AWPM_ERR_CANCELLED: return "request cancelled before it started";
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
    opt->slots = 0;
    opt->select = AWPM_SELECT_STEP_D;
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

void awpm_server_shutdown(awpm_ctx *ctx);

int awpm_destroy(awpm_ctx *ctx)
{
    if (!ctx)
        return AWPM_OK;
    awpm_server_shutdown(ctx);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        teardown_ctx(ctx);
    }
    delete ctx;
    return AWPM_OK;
}

int awpm_inject_alloc_failure(awpm_ctx *ctx, int32_t after)
{
    if (!ctx || after < -1)
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->fail_after = after;
    return AWPM_OK;
}

void awpm_server_memory(awpm_ctx *ctx, size_t *held, size_t *peak);

int awpm_bytes_needed(awpm_ctx *ctx, int32_t n, int32_t nnz, int32_t host_inputs, size_t *bytes)
{
    if (!ctx || !bytes || n < 0 || nnz < 0)
        return AWPM_ERR_INVALID_ARG;
    *bytes = ctx_bytes_needed(n, nnz, host_inputs != 0, ctx->opt.lookup, ctx->opt.select);
    return AWPM_OK;
}

int awpm_memory_held(awpm_ctx *ctx, size_t *held, size_t *peak)
{
    if (!ctx || !held || !peak)
        return AWPM_ERR_INVALID_ARG;
    size_t h, p;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        h = ctx->held;
        p = ctx->peak;
    }
    size_t sh = 0, sp = 0;
    awpm_server_memory(ctx, &sh, &sp);
    *held = h + sh;
    *peak = p > sp ? p : sp;
    return AWPM_OK;
}

static int solve_sync(awpm_ctx *c, const Request &r, awpm_stats *st, awpm_stats *per_matrix)
{
    std::lock_guard<std::mutex> lk(c->mu);
    int rc = ctx_enqueue(c, r);
    if (rc != AWPM_OK) {
        if (c->stream)
            cudaStreamSynchronize(c->stream);
        cudaGetLastError();
        c->pend.active = false;
        return rc;
    }
    return ctx_finish(c, st, per_matrix);
}

int awpm_improve_ctx(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                     const double *weight, const int32_t *mate_in, int32_t *mate_out,
                     awpm_stats *stats)
{
    NvtxRange nvtx_range("awpm_improve");
    if (!ctx)
        return AWPM_ERR_INVALID_ARG;
    Request r;
    r.n = n;
    r.colptr = colptr;
    r.rowidx = rowidx;
    r.weight = weight;
    r.mate_in = mate_in;
    r.mate_out = mate_out;
    if (!mate_in && n > 0) {
        // no matching given: start from the greedy maximal matching
        if (!mate_out)
            return AWPM_ERR_INVALID_ARG;
        int32_t *gm = nullptr;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            CUDA_TRY(cudaSetDevice(ctx->device));
            AWPM_TRY(ensure(ctx, ctx->gmate, sizeof(int32_t) * (size_t)n));
            gm = (int32_t *)ctx->gmate.p;
        }
        awpm_greedy_stats gs;
        AWPM_TRY(awpm_greedy(ctx, n, colptr, rowidx, weight, gm, &gs));
        int32_t card = gs.cardinality;
        if (card != n) {
            // greedy is not perfect: complete it with augmenting paths
            awpm_mcm_stats ms;
            AWPM_TRY(awpm_mcm(ctx, n, colptr, rowidx, weight, gm, &ms));
            card = ms.cardinality;
        }
        if (card != n) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            const int l_out = where(ctx, mate_out);
            if (l_out < 0)
                return AWPM_ERR_INVALID_ARG;
            CUDA_TRY(cudaMemcpyAsync(mate_out, gm, sizeof(int32_t) * (size_t)n,
                                     l_out == 1 ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyDeviceToHost,
                                     ctx->stream));
            CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            return AWPM_ERR_NOT_PERFECT;
        }
        r.mate_in = gm;
    }
    return solve_sync(ctx, r, stats, nullptr);
}

int awpm_improve(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *weight,
                 const int32_t *mate_in, int32_t *mate_out, awpm_stats *stats)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        note_cuda_error(e, "cudaGetDevice", __LINE__);
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
    NvtxRange nvtx_range("awpm_improve_batch");
    if (!ctx || count < 0 || (count > 0 && !n_off))
        return AWPM_ERR_INVALID_ARG;
    if (count == 0) {
        if (total) {
            std::memset(total, 0, sizeof(*total));
            total->converged = 1;
        }
        return AWPM_OK;
    }
    int32_t n = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e == cudaSuccess && where(ctx, n_off) == 1)
            e = cudaMemcpy(&n, n_off + count, sizeof(int32_t), cudaMemcpyDeviceToHost);
        else if (e == cudaSuccess)
            n = n_off[count];
        if (e != cudaSuccess) {
            note_cuda_error(e, "reading the batch offsets", __LINE__);
            return AWPM_ERR_CUDA;
        }
    }
    if (n <= 0)
        return AWPM_ERR_INVALID_ARG;
    Request r;
    r.n = n;
    r.colptr = colptr;
    r.rowidx = rowidx;
    r.weight = weight;
    r.mate_in = mate_in;
    r.mate_out = mate_out;
    r.count = count;
    r.n_off = n_off;
    return solve_sync(ctx, r, total, per_matrix);
}

int awpm_greedy(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const double *weight, int32_t *mate_out, awpm_greedy_stats *stats)
{
    NvtxRange nvtx_range("awpm_greedy");
    if (!ctx || n < 0 || (n > 0 && (!colptr || !mate_out)))
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    awpm_ctx *c = ctx;
    awpm_greedy_stats S;
    std::memset(&S, 0, sizeof(S));
    if (n == 0) {
        S.rounds = 1;  // one round, which matches nothing
        if (stats)
            *stats = S;
        return AWPM_OK;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    const int l_colptr = where(c, colptr), l_rowidx = where(c, rowidx), l_w = where(c, weight),
              l_out = where(c, mate_out);
    if (l_colptr < 0 || l_rowidx < 0 || l_w < 0 || l_out < 0)
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
    if (nnz < 0 || nnz > kMaxNnz || (nnz > 0 && (!rowidx || !weight)))
        return AWPM_ERR_INVALID_ARG;
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    AWPM_TRY(ensure(c, c->mc, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mr, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->wm, sizeof(double) * n));
    AWPM_TRY(ensure(c, c->gckey, sizeof(long long) * n));
    AWPM_TRY(ensure(c, c->gcpos, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->grkey, sizeof(long long) * n));
    AWPM_TRY(ensure(c, c->grcol, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->gtdead, (size_t)ntiles + 1));
    AWPM_TRY(ensure(c, c->tile_col, sizeof(int32_t) * ((size_t)ntiles + 1)));
    AWPM_TRY(ensure(c, c->starts, sizeof(uint32_t) * (((size_t)nnz + 31) / 32 + 1)));
    AWPM_TRY(ensure(c, c->ctl, sizeof(Ctl)));
    AWPM_TRY(ensure(c, c->wpart, sizeof(double) * kWsumBlocks));
    const Shape sh = shape_of(c, false, AWPM_LOOKUP_BSEARCH, true, ntiles);
    // AWPM_FLAG_TIME_SEARCH: a host loop over the rounds (every kernel a
    // separate stream launch, visible to profilers) instead of the graph
    const bool host_loop = (c->opt.flags & AWPM_FLAG_TIME_SEARCH) != 0;
    cudaGraphExec_t g = nullptr;
    if (!host_loop) {
        cudaGraphExec_t &gg = c->g_greedy[sh.search_waves - 1];
        if (!gg)
            AWPM_TRY(build_greedy_graph(c, sh, &gg));
        g = gg;
    }
    CUDA_TRY(cudaEventRecord(c->ev_a, c->stream));
    Work &wk = *c->h_work;
    std::memset(&wk, 0, sizeof(Work));
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = ntiles;
    // at most n rounds match something, then one matches nothing
    wk.max_passes = n < 0x7fffffff ? n + 1 : n;
    wk.lookup = AWPM_LOOKUP_BSEARCH;
    AWPM_TRY(stage_in(c, c->s_colptr, colptr, (size_t)n + 1, l_colptr, &wk.colptr));
    AWPM_TRY(stage_in(c, c->s_rowidx, rowidx, (size_t)nnz, l_rowidx, &wk.rowidx));
    AWPM_TRY(stage_in(c, c->s_w, weight, (size_t)nnz, l_w, &wk.w));
    wk.mc = (int32_t *)c->mc.p;
    wk.mr = (int32_t *)c->mr.p;
    wk.wm = (double *)c->wm.p;
    wk.tile_col = (int32_t *)c->tile_col.p;
    wk.starts = (uint32_t *)c->starts.p;
    wk.ctl = (Ctl *)c->ctl.p;
    wk.wpart = (double *)c->wpart.p;
    wk.gckey = (long long *)c->gckey.p;
    wk.gcpos = (int32_t *)c->gcpos.p;
    wk.grkey = (long long *)c->grkey.p;
    wk.grcol = (int32_t *)c->grcol.p;
    wk.gtdead = (uint8_t *)c->gtdead.p;
    CUDA_TRY(cudaMemcpyAsync(c->d_work.p, c->h_work, sizeof(Work), cudaMemcpyHostToDevice,
                             c->stream));
    if (host_loop) {
        const Work *d = (const Work *)c->d_work.p;
        Sink k;
        k.stream = c->stream;
        launch_greedy_init(d, sh, k);
        for (int32_t round = 0; round < wk.max_passes; ++round) {
            launch_greedy_round(d, sh, false, cudaGraphConditionalHandle(), k);
            AWPM_TRY(check_sink(k));
            CUDA_TRY(cudaMemcpyAsync(c->h_ctl, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                     c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            if (!c->h_ctl->active)
                break;
        }
        launch_weight_sum(d, sh, true, k);
        AWPM_TRY(check_sink(k));
    } else {
        CUDA_TRY(cudaGraphLaunch(g, c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(mate_out, wk.mc, sizeof(int32_t) * n,
                             l_out == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->h_ctl, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaEventRecord(c->ev_b, c->stream));
    CUDA_TRY(cudaEventSynchronize(c->ev_b));
    const Ctl &h = *c->h_ctl;
    const int rc = code_of(h.err);
    if (rc != AWPM_OK)
        return rc;
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_a, c->ev_b));
    S.rounds = h.iterations;
    S.cardinality = (int32_t)h.cycles;
    S.weight = h.weight_out;
    S.ms_total = ms;
    if (stats)
        *stats = S;
    return AWPM_OK;
}

int awpm_mcm(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
             const double *weight, int32_t *mate, awpm_mcm_stats *stats)
{
    NvtxRange nvtx_range("awpm_mcm");
    if (!ctx || n < 0 || (n > 0 && (!colptr || !mate)))
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    awpm_ctx *c = ctx;
    awpm_mcm_stats S;
    std::memset(&S, 0, sizeof(S));
    if (n == 0) {
        S.phases = 1;
        if (stats)
            *stats = S;
        return AWPM_OK;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    const int l_colptr = where(c, colptr), l_rowidx = where(c, rowidx), l_w = where(c, weight),
              l_m = where(c, mate);
    if (l_colptr < 0 || l_rowidx < 0 || l_w < 0 || l_m < 0)
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
    if (nnz < 0 || nnz > kMaxNnz || (nnz > 0 && (!rowidx || !weight)))
        return AWPM_ERR_INVALID_ARG;
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    const size_t words = (size_t)n / 32 + 1;
    AWPM_TRY(ensure(c, c->mc, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mr, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mroot, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mrpar, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mroff, sizeof(Off) * n));
    AWPM_TRY(ensure(c, c->mtend, sizeof(Off) * n));
    AWPM_TRY(ensure(c, c->mtouch, sizeof(int32_t) * n));
    AWPM_TRY(ensure(c, c->mfront, sizeof(uint32_t) * words));
    AWPM_TRY(ensure(c, c->mcolof, sizeof(int32_t) * ((size_t)nnz + 1)));
    AWPM_TRY(ensure(c, c->mnext, sizeof(uint32_t) * words));
    // the level's tile list: at most min(nnz, nnz/32 + 2n) entries
    const size_t tiles_cap = std::min((size_t)nnz, (size_t)ntiles + 2 * (size_t)n);
    AWPM_TRY(ensure(c, c->mtiles, sizeof(int32_t) * (tiles_cap + 1)));
    AWPM_TRY(ensure(c, c->tile_col, sizeof(int32_t) * ((size_t)ntiles + 1)));
    AWPM_TRY(ensure(c, c->starts, sizeof(uint32_t) * (((size_t)nnz + 31) / 32 + 1)));
    AWPM_TRY(ensure(c, c->ctl, sizeof(Ctl)));
    int32_t *dmate = mate;
    if (l_m != 1) {
        AWPM_TRY(ensure(c, c->mstage, sizeof(int32_t) * n));
        dmate = (int32_t *)c->mstage.p;
        CUDA_TRY(cudaMemcpyAsync(dmate, mate, sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                                 c->stream));
    }
    const Shape sh = shape_of(c, false, AWPM_LOOKUP_BSEARCH, true, ntiles);
    CUDA_TRY(cudaEventRecord(c->ev_a, c->stream));
    Work &wk = *c->h_work;
    std::memset(&wk, 0, sizeof(Work));
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = ntiles;
    AWPM_TRY(stage_in(c, c->s_colptr, colptr, (size_t)n + 1, l_colptr, &wk.colptr));
    AWPM_TRY(stage_in(c, c->s_rowidx, rowidx, (size_t)nnz, l_rowidx, &wk.rowidx));
    AWPM_TRY(stage_in(c, c->s_w, weight, (size_t)nnz, l_w, &wk.w));
    wk.mc = (int32_t *)c->mc.p;
    wk.mr = (int32_t *)c->mr.p;
    wk.tile_col = (int32_t *)c->tile_col.p;
    wk.starts = (uint32_t *)c->starts.p;
    wk.ctl = (Ctl *)c->ctl.p;
    wk.mroot = (int32_t *)c->mroot.p;
    wk.mrpar = (int32_t *)c->mrpar.p;
    wk.mfront = (uint32_t *)c->mfront.p;
    wk.mnext = (uint32_t *)c->mnext.p;
    wk.mroff = (Off *)c->mroff.p;
    wk.mtend = (Off *)c->mtend.p;
    wk.mtouch = (int32_t *)c->mtouch.p;
    wk.mmate = dmate;
    wk.mcolof = (int32_t *)c->mcolof.p;
    wk.mtiles = (int32_t *)c->mtiles.p;
    wk.mtiles_cap = (int64_t)tiles_cap + 1;
    CUDA_TRY(cudaMemcpyAsync(c->d_work.p, c->h_work, sizeof(Work), cudaMemcpyHostToDevice,
                             c->stream));
    const Work *d = (const Work *)c->d_work.p;
    Ctl *dctl = (Ctl *)c->ctl.p;
    if (!(c->opt.flags & AWPM_FLAG_TIME_SEARCH)) {
        // the whole search in one graph launch (loops on the device)
        cudaGraphExec_t &g = c->g_mcm[sh.search_waves - 1];
        if (!g)
            AWPM_TRY(build_mcm_graph(c, sh, &g));
        CUDA_TRY(cudaGraphLaunch(g, c->stream));
        if (l_m != 1)
            CUDA_TRY(cudaMemcpyAsync(mate, dmate, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                     c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->h_ctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaEventRecord(c->ev_b, c->stream));
        CUDA_TRY(cudaEventSynchronize(c->ev_b));
        const int rc = code_of(c->h_ctl->err);
        if (rc != AWPM_OK)
            return rc;
        float gms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&gms, c->ev_a, c->ev_b));
        S.phases = c->h_ctl->iterations;
        S.cardinality = (int32_t)c->h_ctl->cycles;
        S.levels = (int64_t)c->h_ctl->levels;
        S.ms_total = gms;
        if (stats)
            *stats = S;
        return AWPM_OK;
    }
    // AWPM_FLAG_TIME_SEARCH: levels and phases driven from the host
    Sink k;
    k.stream = c->stream;
    launch_mcm_load(d, sh, k);
    AWPM_TRY(check_sink(k));
    // read one counter of the control block, then zero it on the device
    auto take = [&](void *field, size_t bytes, void *host) -> int {
        CUDA_TRY(cudaMemcpyAsync(host, field, bytes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(&c->h_ctl->err, &dctl->err, sizeof(unsigned),
                                 cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        CUDA_TRY(cudaMemsetAsync(field, 0, bytes, c->stream));
        return code_of(c->h_ctl->err);
    };
    unsigned long long have = 0;
    AWPM_TRY(take(&dctl->cycles, sizeof(unsigned long long), &have));
    unsigned long long total = have;
    for (int32_t phase = 0; phase <= n; ++phase) {
        S.phases += 1;
        launch_mcm_phase(d, sh, k);
        AWPM_TRY(check_sink(k));
        for (int32_t level = 0; level <= n; ++level) {
            int32_t live = 0;
            AWPM_TRY(take(&dctl->live, sizeof(int32_t), &live));
            if (live <= 0)
                break;
            S.levels += 1;
            launch_mcm_level(d, sh, k);
            AWPM_TRY(check_sink(k));
        }
        launch_mcm_augment(d, sh, k);
        AWPM_TRY(check_sink(k));
        unsigned long long aug = 0;
        AWPM_TRY(take(&dctl->pass_flips, sizeof(unsigned long long), &aug));
        total += aug;
        if (aug == 0)
            break;
    }
    launch_mcm_store(d, sh, k);
    AWPM_TRY(check_sink(k));
    if (l_m != 1)
        CUDA_TRY(cudaMemcpyAsync(mate, dmate, sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                 c->stream));
    CUDA_TRY(cudaEventRecord(c->ev_b, c->stream));
    CUDA_TRY(cudaEventSynchronize(c->ev_b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_a, c->ev_b));
    S.cardinality = (int32_t)total;
    S.ms_total = ms;
    if (stats)
        *stats = S;
    return AWPM_OK;
}

int awpm_weights(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                 const double *values, int32_t mode, double *weight_out)
{
    NvtxRange nvtx_range("awpm_weights");
    if (!ctx || n < 0 || (n > 0 && !colptr) ||
        (mode != AWPM_WEIGHTS_SUM && mode != AWPM_WEIGHTS_PRODUCT))
        return AWPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    awpm_ctx *c = ctx;
    if (n == 0)
        return AWPM_OK;
    CUDA_TRY(cudaSetDevice(c->device));
    const int l_colptr = where(c, colptr), l_rowidx = where(c, rowidx), l_a = where(c, values),
              l_out = where(c, weight_out);
    if (l_colptr < 0 || l_rowidx < 0 || l_a < 0 || l_out < 0)
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
    if (nnz < 0 || nnz > kMaxNnz || (nnz > 0 && (!rowidx || !values || !weight_out)))
        return AWPM_ERR_INVALID_ARG;
    const int32_t ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    AWPM_TRY(ensure(c, c->wt_cmax, sizeof(double) * n));
    AWPM_TRY(ensure(c, c->wt_rmax, sizeof(unsigned long long) * n));
    AWPM_TRY(ensure(c, c->ctl, sizeof(Ctl)));
    double *dout = weight_out;
    if (l_out != 1) {
        AWPM_TRY(ensure(c, c->wt_stage, sizeof(double) * (size_t)nnz));
        dout = (double *)c->wt_stage.p;
    }
    const Shape sh = shape_of(c, false, AWPM_LOOKUP_BSEARCH, true, ntiles);
    Work &wk = *c->h_work;
    std::memset(&wk, 0, sizeof(Work));
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = ntiles;
    AWPM_TRY(stage_in(c, c->s_colptr, colptr, (size_t)n + 1, l_colptr, &wk.colptr));
    AWPM_TRY(stage_in(c, c->s_rowidx, rowidx, (size_t)nnz, l_rowidx, &wk.rowidx));
    AWPM_TRY(stage_in(c, c->s_w, values, (size_t)nnz, l_a, &wk.wt_a));
    wk.wt_out = dout;
    wk.wt_cmax = (double *)c->wt_cmax.p;
    wk.wt_rmax = (unsigned long long *)c->wt_rmax.p;
    wk.wt_mode = mode;
    wk.ctl = (Ctl *)c->ctl.p;
    CUDA_TRY(cudaMemcpyAsync(c->d_work.p, c->h_work, sizeof(Work), cudaMemcpyHostToDevice,
                             c->stream));
    Sink k;
    k.stream = c->stream;
    launch_weights((const Work *)c->d_work.p, sh, k);
    AWPM_TRY(check_sink(k));
    if (l_out != 1 && nnz > 0)
        CUDA_TRY(cudaMemcpyAsync(weight_out, dout, sizeof(double) * (size_t)nnz,
                                 cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->h_ctl, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    // a column without entries is no error here (no matching is asked for)
    return code_of(c->h_ctl->err & ~kErrNotPerfect);
}

int awpm_search(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const double *weight, const int32_t *mate, double *stepc_gain, int32_t *stepc_row,
                awpm_stats *stats)
{
    NvtxRange nvtx_range("awpm_search");
    if (!ctx)
        return AWPM_ERR_INVALID_ARG;
    Request r;
    r.n = n;
    r.colptr = colptr;
    r.rowidx = rowidx;
    r.weight = weight;
    r.mate_in = mate;
    r.search_only = true;
    r.gain_out = stepc_gain;
    r.row_out = stepc_row;
    return solve_sync(ctx, r, stats, nullptr);
}

}  // extern "C"
