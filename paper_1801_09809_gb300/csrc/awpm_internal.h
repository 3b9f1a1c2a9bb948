// Internal declarations shared by the kernels and the host side of libawpm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "awpm.h"

namespace awpm {

// Nonzeros handled by one warp per tile of the edge-parallel kernels; tiles
// start at multiples of kTile, so tile t owns word t of the column-start
// bitmap.
constexpr int kTile = 32;

// Error bits raised on the device; the host maps them to the public code
// (priority INVALID > UNSORTED > NONFINITE > NOTPERF > INTERNAL > TIMEOUT).
constexpr unsigned kErrInvalid = 1u;
constexpr unsigned kErrUnsorted = 2u;
constexpr unsigned kErrNonfinite = 4u;
constexpr unsigned kErrNotPerfect = 8u;
constexpr unsigned kErrInternal = 16u;  // a consistency check of the library's own state failed
constexpr unsigned kErrTimeout = 32u;   // a bounded retry loop or level loop gave up
constexpr unsigned kErrBounds = 64u;    // AWPM_DEBUG_BOUNDS builds: an index check failed

// Public code of a set of device error bits (host side).
inline int awpm_code_of_bits(unsigned err)
{
    if (err & kErrInvalid)
        return AWPM_ERR_INVALID_ARG;
    if (err & kErrUnsorted)
        return AWPM_ERR_UNSORTED_OR_DUP;
    if (err & kErrNonfinite)
        return AWPM_ERR_NONFINITE;
    if (err & kErrNotPerfect)
        return AWPM_ERR_NOT_PERFECT;
    if (err & (kErrInternal | kErrBounds))
        return AWPM_ERR_INTERNAL;
    if (err & kErrTimeout)
        return AWPM_ERR_TIMEOUT;
    if (err)
        return AWPM_ERR_INTERNAL;
    return AWPM_OK;
}

// Step-C record of a root column j (Algorithm 5): best positive gain, the
// position p of (i, j) in column j and the position q of the closing entry
// (m_j, m_i) in column m_i.  g == 0 means "no cycle".
struct alignas(16) Rec {
    double g;
    int32_t p;
    int32_t q;
};

// Per-row view of the column matched to row i (m_i), in two arrays:
//   rsig[i]   a 64-bit signature of column m_i's rows (the bits sig_mask(r)
//             set for every stored row r): a clear bit proves that the
//             closing entry (m_j, m_i) is absent without touching the column;
//             every candidate gathers these 8 bytes;
//   rrange[i] where column m_i's rows sit in the CSC arrays and the matched
//             weight w(i, m_i): read only for the candidates that pass.
// Both are rewritten whenever row i changes mate.
struct alignas(16) RowRange {
    int32_t s;
    int32_t e;
    double w;
};

// Maximum matching: the best offer a row received at this level (order key
// of the edge weight, then the lowest column), or a tree's end (order key of
// its last edge, then the lowest row); one 128-bit compare-and-swap updates
// both fields together.
struct alignas(16) Off {
    long long key;
    int32_t who;
    int32_t pad;
};

// Step-D selection at a key column k (Algorithm 6): best gain and its root j.
struct alignas(16) Sel {
    double g;
    int32_t j;
    int32_t pad;
};

// Device-resident control block of one solve.
struct Ctl {
    unsigned int err;            // kErr* bits
    int32_t active;              // 1 while the pass loop continues
    int32_t iterations;          // passes run
    int32_t converged;           // last pass flipped nothing
    int32_t max_passes;          // cap on passes
    int32_t live;                // greedy selection: winners still undecided
    int32_t nonempty;            // maximum matching: no column is empty
    int32_t phase_levels;        // maximum matching: levels of the running phase
    int32_t level_tiles;         // maximum matching: tiles listed for the next level
    int32_t level_listed;        // maximum matching: tiles listed for this level
    uint32_t flip_done;          // blocks done with the pass's flip (graph form)
    uint32_t pad_fd;
    uint32_t level_done;         // maximum matching: blocks done with the level's last step
    int32_t touched;             // maximum matching: rows listed in mtouch this level
    unsigned long long levels;   // maximum matching: search levels run
    unsigned long long pass_flips;   // cycles flipped in the running pass
    unsigned long long cycles;       // cycles flipped in total
    unsigned long long candidates;   // Step A requests (i > m_j)
    unsigned long long found;        // closing edge present
    unsigned long long positive;     // closing edge present and g > 0
    double weight_in;
    double weight_out;
};

// Batched solve of many independent matrices as one block-diagonal union
// (count > 0).  Matrix b owns columns and rows [n_off[b], n_off[b+1]).
struct BatchWork {
    int32_t count;
    int32_t pad;
    const int32_t *n_off;   // count + 1 offsets
    int32_t *colmat;        // matrix of each column
    int32_t *tilemat;       // matrix of each tile's first nonzero | kTileSingle
    int32_t *mdone;         // matrix finished (converged or pass cap)
    int32_t *miter;         // passes run per matrix
    int32_t *mconv;         // converged per matrix
    int32_t *mnnz;          // nonzeros per matrix
    unsigned long long *mflips;   // cycles flipped in the running pass
    unsigned long long *mcycles;  // cycles flipped in total
    double *mw_in;
    double *mw_out;
    int32_t *active;        // matrices still running after a pass
    int32_t *tlist;         // tiles the next pass searches (running matrices,
                            // and every tile spanning two matrices)
    int32_t *tlist_n;       // their number
};

// Tile whose nonzeros all belong to one matrix.
constexpr int32_t kTileSingle = (int32_t)0x80000000;

// Descriptor of one solve.  It lives in device memory and every kernel reads
// it from there, so launch configurations do not depend on the problem and
// one instantiated CUDA graph serves every problem of a context: a new
// problem only rewrites the descriptor before the graph launch.
struct Work {
    int32_t n;
    int32_t nnz;
    int32_t ntiles;
    int32_t max_passes;
    int32_t lookup;     // AWPM_LOOKUP_BSEARCH, _HASH or _ROWMARK
    int32_t rec_clean;  // the Step-C and Step-D records of columns [0, n) are all empty
    const int32_t *colptr;
    const int32_t *rowidx;
    const double *w;
    const int32_t *mate_in;
    int32_t *mc;        // row matched to column j
    int32_t *mr;        // column matched to row i
    double *wm;         // w(mc[j], j)
    unsigned long long *rsig;  // per row i: signature of the rows of column mr[i]
    RowRange *rrange;          // per row i: that column's range and w(i, mr[i])
    unsigned long long *colsig;  // per column: signature of its rows
    unsigned long long *htab;    // per-column hash tables (2 slots per nonzero), or null
    uint32_t *bloom;    // blocked Bloom filters of the long columns (a word per 4 nonzeros), or null
    Rec *best;          // Step-C records
    Sel *dsel;          // Step-D selections
    uint32_t *winbits;  // bit j: column j holds a Step-C winner this pass
    int32_t *wkey;      // key column of winner j (set by Step D), -1 if dropped
    int32_t *tile_col;  // column holding the first nonzero of each tile
    uint32_t *starts;   // bit p set when a column starts at nonzero p
    Ctl *ctl;
    double *wpart;      // partial sums of the weight reduction
    BatchWork bw;       // batched solve (bw.count > 0), else zero
    // greedy maximal matching: per column the best free entry (order key,
    // then position), per row the best free entry (order key, then column)
    long long *gckey;
    int32_t *gcpos;
    long long *grkey;
    int32_t *grcol;
    uint8_t *gtdead;    // per tile: every column of the tile is matched
    // greedy (Pettie-Sanders) selection: per column the first remaining
    // winner touching it; bitmaps of undecided and kept winners and of the
    // columns of kept cycles
    Sel *psel;
    uint32_t *pslive;
    uint32_t *pstaken;
    uint32_t *psused;
    // weights from matrix values: values, output, column maxima, row maxima
    // (bit patterns of positive doubles), mode (0 scaled magnitude, 1 its log)
    const double *wt_a;
    double *wt_out;
    double *wt_cmax;
    unsigned long long *wt_rmax;
    int32_t wt_mode;
    int32_t wt_pad;
    // maximum cardinality matching: tree of a column, column that reached a
    // row, frontier bitmaps, per row the best offer (key, column), per tree
    // its end (key of the last edge, row); mate in/out
    int32_t *mroot;
    int32_t *mrpar;
    uint32_t *mfront;
    uint32_t *mnext;
    Off *mroff;         // per row: the level's best offer (key, column)
    Off *mtend;         // per tree (root column): its end (key of the last edge, row)
    int32_t *mtouch;    // rows offered something at this level (each once)
    int32_t *mmate;
    int32_t *mcolof;    // column of every entry
    int32_t *mtiles;    // tiles holding a frontier column, this level
    int64_t mtiles_cap; // capacity of mtiles
    // row marking: per row the mark of its columns (a signature), the
    // transpose (row pointers; CSC positions row by row, ascending), the
    // radix sort that builds it (keys and values in two buffers each, digit
    // counts per block tile, then their offsets; sums per scan chunk)
    unsigned long long *rowsig;
    int32_t *trowptr;
    int32_t *tpos;
    int32_t *rs_key[2];
    int32_t *rs_val[2];
    int32_t *rs_hist;
    int32_t *rs_sums;
    int32_t rs_tiles;   // block tiles of kRsTile entries
    int32_t rs_passes;  // 8-bit digits of the largest row index (at least 1)
};

// Radix sort of the transpose: 256 threads, 8 entries each per block tile,
// 8-bit digits; scans run over chunks of 2048 counts.
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsBins = 256;
constexpr int kScanChunk = kRsThreads * 8;

// Launch shape of a context: fixed grids sized by the GPU, not the problem.
struct Shape {
    int num_sms;
    int search_bps;     // resident blocks per SM of the chosen search kernel
    int lookup;         // AWPM_LOOKUP_BSEARCH, _HASH or _ROWMARK
    bool batch;
    bool wide;          // search kernel takes four tiles per warp round (else one)
    int search_waves;   // size class: 2 when there are at least 64 tiles per resident
                        // search warp, else 1 (keys the cached graphs; Step D's grid)
    int select;         // AWPM_SELECT_STEP_D or AWPM_SELECT_GREEDY
};

constexpr int kWsumBlocks = 1024;
constexpr int kWsumThreads = 256;

// Where launches go: a stream (launched at once, asynchronously) or a graph
// (appended as kernel nodes, each depending on the previous one).  Graphs are
// built node by node rather than by stream capture, so building one never
// interacts with work other threads submit meanwhile.
struct Sink {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
    void launch(const void *func, unsigned grid, unsigned block, void **args);
};

// Launch sequences; `d` is the device copy of the Work.
void launch_init(const Work *d, const Shape &sh, Sink &k);
void launch_weight_sum(const Work *d, const Shape &sh, bool out, Sink &k);
void launch_search(const Work *d, const Shape &sh, Sink &k);
void launch_select_and_flip(const Work *d, const Shape &sh, Sink &k);
// Graph form for single problems with Step D: the selection and the flip,
// whose last block also ends the pass (no separate control kernel).
void launch_select_flip_control_graph(const Work *d, const Shape &sh,
                                      cudaGraphConditionalHandle h, Sink &k);
// Greedy selection: the kernels before the rounds (keys, undecided set,
// condition of the rounds' loop), one round (the loop condition is set at
// its end), and the kernels after (records for the flip).  With graph ==
// false the conditions are not set; the host reads Ctl::live instead.
void launch_greedy_select_begin(const Work *d, const Shape &sh, bool graph,
                                cudaGraphConditionalHandle h, Sink &k);
void launch_greedy_select_round(const Work *d, const Shape &sh, bool graph,
                                cudaGraphConditionalHandle h, Sink &k);
void launch_greedy_select_end_and_flip(const Work *d, const Shape &sh, Sink &k);
// Weights from matrix values (equilibration, Options A / B).
void launch_weights(const Work *d, const Shape &sh, Sink &k);
// Maximum cardinality matching: load and check the starting matching; start
// a phase (Ctl::live = free columns); one level of the searches (Ctl::live =
// next frontier); augment (Ctl::pass_flips = paths augmented); write back.
void launch_mcm_load(const Work *d, const Shape &sh, Sink &k);
void launch_mcm_phase(const Work *d, const Shape &sh, Sink &k);
void launch_mcm_level(const Work *d, const Shape &sh, Sink &k);
// Graph form of a level: its steps, the last one also setting the level
// loop's condition (no separate condition kernel).
void launch_mcm_level_graph(const Work *d, const Shape &sh, cudaGraphConditionalHandle h,
                            Sink &k);
void launch_mcm_augment(const Work *d, const Shape &sh, Sink &k);
void launch_mcm_store(const Work *d, const Shape &sh, Sink &k);
// Graph forms: the condition of the level loop (undecided frontier left),
// and the end of a phase (count it, continue while it augmented).
void launch_mcm_cond_level(const Work *d, const Shape &sh, cudaGraphConditionalHandle h, Sink &k);
void launch_mcm_cond_phase(const Work *d, const Shape &sh, cudaGraphConditionalHandle h, Sink &k);
void launch_control(const Work *d, const Shape &sh, bool graph, cudaGraphConditionalHandle h,
                    Sink &k);
void launch_export_stepc(const Work *d, const Shape &sh, double *gain, int32_t *row, Sink &k);
// Greedy maximal matching: state reset and input checks; one round (the
// control kernel ends the loop after a round that matched nothing).
void launch_greedy_init(const Work *d, const Shape &sh, Sink &k);
void launch_greedy_round(const Work *d, const Shape &sh, bool graph, cudaGraphConditionalHandle h,
                         Sink &k);
// Resident blocks per SM of the search kernel for a lookup strategy.
int search_blocks_per_sm(int lookup, bool batch, bool wide);
// Waves of the search grid for a problem of ntiles tiles: 2 once every warp
// of a single wave would take at least 64 tiles (more blocks than resident
// slots shorten the tail of uneven warps), else 1.
int search_waves(int num_sms, int search_bps, int32_t ntiles);
// Whether the search kernel takes four tiles per warp round (default on; the
// environment variable AWPM_SEARCH_WIDE=0/1 overrides it, a tuning knob).
bool default_search_wide();
// Whether single-problem searches use the pipelined kernel (default on; the
// environment variable AWPM_SEARCH_PIPE=0/1 overrides it, a tuning knob).
bool search_pipe();

}  // namespace awpm
