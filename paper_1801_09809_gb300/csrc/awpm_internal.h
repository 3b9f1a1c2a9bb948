// Internal declarations shared by the kernels and the host API of libawpm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace awpm {

// Nonzeros handled by one warp per tile of the edge-parallel kernels.
constexpr int kTile = 32;

// Error bits raised by the device-side validation; the host maps the lowest
// set bit to the public code (priority INVALID > UNSORTED > NONFINITE > NOTPERF).
constexpr unsigned kErrInvalid = 1u;
constexpr unsigned kErrUnsorted = 2u;
constexpr unsigned kErrNonfinite = 4u;
constexpr unsigned kErrNotPerfect = 8u;
constexpr unsigned kErrInternal = 16u;  // a bounded retry loop gave up

// Step-C record of a root column j (Algorithm 5): best positive gain, the
// position p of (i, j) in column j and the position q of the closing entry
// (m_j, m_i) in column m_i.  g == 0 means "no cycle".
struct alignas(16) Rec {
    double g;
    int32_t p;
    int32_t q;
};

// Per-row view of the column matched to row i (m_i): where its rows sit in
// the CSC arrays and a 64-bit signature of those rows (bit sig_bit(r) set for
// every stored row r).  A clear bit proves that the closing entry (m_j, m_i)
// is absent without touching the column; the record is rewritten whenever
// row i changes mate.
struct alignas(16) RowRec {
    int32_t s;
    int32_t e;
    unsigned long long sig;
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
    int32_t pad0;
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
    int32_t count = 0;
    const int32_t *n_off = nullptr;  // count + 1 offsets
    int32_t *colmat = nullptr;       // matrix of each column
    int32_t *tilemat = nullptr;      // matrix of each tile's first nonzero | kTileSingle
    int32_t *mdone = nullptr;        // matrix finished (converged or pass cap)
    int32_t *miter = nullptr;        // passes run per matrix
    int32_t *mconv = nullptr;        // converged per matrix
    int32_t *mnnz = nullptr;         // nonzeros per matrix
    unsigned long long *mflips = nullptr;   // cycles flipped in the running pass
    unsigned long long *mcycles = nullptr;  // cycles flipped in total
    double *mw_in = nullptr;
    double *mw_out = nullptr;
    int32_t *active = nullptr;       // matrices still running after a pass
};

// Tile whose nonzeros all belong to one matrix.
constexpr int32_t kTileSingle = (int32_t)0x80000000;

// Device pointers of one solve.
struct Work {
    int32_t n;
    int32_t nnz;
    int32_t ntiles;
    int32_t lookup;      // AWPM_LOOKUP_BSEARCH or AWPM_LOOKUP_HASH
    int32_t search_u;    // tiles in flight per warp in the search kernel (1, 2, 4)
    int32_t search_bps;  // resident blocks per SM of that search kernel
    const int32_t *colptr;
    const int32_t *rowidx;
    const double *w;
    const int32_t *mate_in;
    int32_t *mc;        // row matched to column j
    int32_t *mr;        // column matched to row i
    double *wm;         // w(mc[j], j)
    RowRec *rr;         // per row i: rows of column mr[i] (range + signature)
    double *wmr;        // per row i: wm[mr[i]] = w(i, mr[i])
    unsigned long long *colsig;  // per column: signature of its rows
    unsigned long long *htab;    // per-column hash tables (2 slots per nonzero), or null
    Rec *best;          // Step-C records
    Sel *dsel;          // Step-D selections
    int32_t *tile_col;  // column holding the first nonzero of each tile
    uint32_t *starts;   // bit p set when a column starts at nonzero p
    Ctl *ctl;
    double *wpart;      // partial sums of the weight reduction
    BatchWork bw;       // batched solve (bw.count > 0), else unused
};

constexpr int kWsumBlocks = 256;
constexpr int kWsumThreads = 256;

// Launchers (all asynchronous on `s`).  `num_sms` sizes persistent grids.
void launch_init(const Work &wk, int max_passes, int num_sms, cudaStream_t s);
void launch_weight_sum(const Work &wk, bool out, cudaStream_t s);
void launch_search(const Work &wk, int num_sms, cudaStream_t s);
void launch_select_and_flip(const Work &wk, int num_sms, cudaStream_t s);
void launch_control(const Work &wk, bool graph, cudaGraphConditionalHandle h, cudaStream_t s);
// Per-matrix weight sums of a batched solve.
void launch_batch_weight_sum(const Work &wk, bool out, cudaStream_t s);
void launch_export_stepc(const Work &wk, double *gain, int32_t *row, cudaStream_t s);
void launch_reset_best(const Work &wk, cudaStream_t s);
// Resident blocks per SM of the search kernel for a lookup strategy and u
// tiles in flight per warp (for a one-wave grid).
int search_blocks_per_sm(int lookup, int u, bool batch);
// Default tiles in flight per warp; the environment variable AWPM_SEARCH_U
// (1, 2 or 4) overrides it, as a tuning knob.
int default_search_u();

}  // namespace awpm
