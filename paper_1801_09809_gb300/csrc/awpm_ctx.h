// Host-side context of libawpm, shared by the synchronous entry points
// (awpm_api.cu) and the request server (awpm_serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "awpm.h"
#include "awpm_internal.h"

namespace awpm {

// NVTX range of a host-side step (an entry point, the enqueue of a solve,
// the wait for it, a pass of the host-driven loop): profilers show where the
// host time goes; without a profiler attached a push/pop costs a few
// nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// One problem handed to a context (single, batched or search only).
struct Request {
    int32_t n = 0;
    int32_t nnz = -1;  // -1: read colptr[n]
    const int32_t *colptr = nullptr;
    const int32_t *rowidx = nullptr;
    const double *weight = nullptr;
    const int32_t *mate_in = nullptr;
    int32_t *mate_out = nullptr;
    int32_t count = 0;  // > 0: batched union with offsets n_off
    const int32_t *n_off = nullptr;
    bool search_only = false;
    double *gain_out = nullptr;
    int32_t *row_out = nullptr;
};

// Launch configurations the autotuner tries (AWPM_LOOKUP_AUTO): closing-edge
// lookup and whether the search kernel takes four tiles per warp round.
struct TuneConfig {
    int lookup;
    bool wide;
};
constexpr int kTuneConfigs = 3;
constexpr TuneConfig kTune[kTuneConfigs] = {
    {AWPM_LOOKUP_BSEARCH, true}, {AWPM_LOOKUP_BSEARCH, false}, {AWPM_LOOKUP_HASH, true}};

// Per problem class (batched or not, log2 of n and of nnz): the time of each
// configuration's trial solve and the configuration chosen once all ran.
struct TuneEntry {
    int trials = 0;
    float ms[kTuneConfigs] = {};
    int chosen = -1;
};

// What finish() needs to turn the device results into statistics.
struct Pending {
    bool active = false;
    int32_t n = 0, nnz = 0, count = 0, lookup = 0;
    bool search_only = false, timed = false, trivial = false;
    int64_t rec_clean_after = 0;  // the context's rec_clean once the solve ends without error
    int passes_enqueued = 0;
    std::vector<int32_t> n_off;  // host copy of the batch offsets
    int tune_cfg = -1;           // autotuner trial of this solve, or -1
    uint64_t tune_key = 0;
};

int setup_ctx(struct ::awpm_ctx *c, const awpm_options *opt);
void teardown_ctx(struct ::awpm_ctx *c);
// Enqueue a whole solve on the context's stream without waiting for it;
// the context's done event is recorded after the last copy.
int ctx_enqueue(struct ::awpm_ctx *c, const Request &r);
// Wait for the enqueued solve (a no-op if it already finished) and fill the
// statistics (per_matrix: count entries for a batch, may be null).
int ctx_finish(struct ::awpm_ctx *c, awpm_stats *st, awpm_stats *per_matrix);
// Device bytes a context needs to solve a problem of this size.
size_t ctx_bytes_needed(int32_t n, int32_t nnz, bool host_inputs, int lookup, int select);
size_t ctx_bytes_held(const struct ::awpm_ctx *c);
// Free the per-solve workspace of an idle context (its descriptor and graphs
// stay; the next solve allocates again).
void ctx_trim(struct ::awpm_ctx *c);
void note_cuda_error(cudaError_t e, const char *what, int line);

}  // namespace awpm

struct awpm_ctx {
    std::mutex mu;
    awpm_options opt{};
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t held = 0;
    size_t peak = 0;        // most device bytes held at once
    int32_t fail_after = -1;  // test hook: allocations left before one fails (-1: off)
    // The Step-C and Step-D records (best, dsel) of columns [0, rec_clean) are
    // known to be empty: a solve with Step D's selection that ends without
    // error clears every record it wrote (each pass's flip empties its
    // winners' records), so the next solve's reset can skip them.  Zero
    // while a solve is in flight, after an error, and when the buffers are
    // reallocated or released.
    int64_t rec_clean = 0;
    int search_bps[2][3][2] = {};  // [batch][lookup slot][wide]
    bool search_wide = true;      // default when the lookup is given explicitly
    // per-solve device workspace
    awpm::DevBuf mc, mr, wm, rr, rsig, colsig, best, dsel, tile_col, starts, ctl, wpart, htab;
    awpm::DevBuf winbits, wkey, bloom;
    awpm::DevBuf gckey, gcpos, grkey, grcol, gtdead;  // greedy matching records
    awpm::DevBuf gmate;                       // greedy start of awpm_improve_ctx
    awpm::DevBuf psel, pslive, pstaken, psused;  // greedy (Pettie-Sanders) selection
    awpm::DevBuf wt_cmax, wt_rmax, wt_stage;     // weights from matrix values
    awpm::DevBuf mroot, mrpar, mfront, mnext, mroff, mtend, mtouch, mstage,
        mcolof, mtiles;  // maximum matching
    awpm::DevBuf rowsig, trowptr, rs_k0, rs_k1, rs_v0, rs_v1, rs_hist, rs_sums;  // row marking
    awpm::DevBuf b_noff, b_colmat, b_tilemat, b_tlist, b_i32, b_u64, b_f64;
    // staging of host-resident arrays
    awpm::DevBuf s_colptr, s_rowidx, s_w, s_mate, s_out, s_gain, s_row;
    awpm::DevBuf d_work;             // device copy of the Work descriptor
    awpm::Work *h_work = nullptr;    // pinned
    awpm::Ctl *h_ctl = nullptr;      // pinned
    int32_t *h_active = nullptr;     // pinned ring of the timed loop
    void *h_batch = nullptr;         // pinned per-matrix results
    size_t h_batch_bytes = 0;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    std::vector<cudaEvent_t> tev;     // timing pairs of the timed loop
    std::vector<cudaEvent_t> flagev;  // ring of the timed loop
    // one instantiated graph per [batch][lookup slot][wide][search waves - 1][select]
    cudaGraphExec_t g_exec[2][3][2][2][2] = {};
    cudaGraphExec_t g_greedy[2] = {};  // greedy matching, [search waves - 1] of the shape
    cudaGraphExec_t g_mcm[2] = {};     // maximum matching, [search waves - 1] of the shape
    std::map<uint64_t, awpm::TuneEntry> tune;  // autotuner state per problem class
    awpm::Pending pend;
    // the request server of this context (awpm_submit), created on first use
    struct awpm_server_impl *server = nullptr;
};
