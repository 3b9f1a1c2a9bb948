/*
 * awpm.h -- C ABI of the GB300 library for the weight-increasing alternating
 * 4-cycle phase of heavy-weight perfect matching (Azad, Buluc, Li, Wang and
 * Langguth, "A distributed-memory algorithm for computing a heavy-weight
 * perfect matching on bipartite graphs", arXiv 1801.09809).
 *
 * Given a perfect matching M of a weighted bipartite graph (rows and columns of
 * a sparse n x n matrix), the phase repeatedly finds vertex-disjoint
 * alternating 4-cycles of positive gain and flips M along them, until a pass
 * finds none (Section 5.3, Algorithms 2-6).  The gain of the cycle through
 * column j, row i, and their mates m_j (a row) and m_i (a column) is
 *     g(i, j, m_j, m_i) = w(i,j) + w(m_j,m_i) - w(i,m_i) - w(m_j,j)   (Section 3)
 * evaluated left to right in IEEE double precision.
 *
 * Data conventions (all entry points):
 *   - n: number of rows = number of columns, 0 <= n < 2^31.
 *   - colptr[n+1] int32, rowidx[nnz] int32, weight[nnz] double: the matrix in
 *     compressed sparse column form, nnz = colptr[n] <= 2^31 - 64, colptr[0] = 0,
 *     colptr non-decreasing, rows strictly increasing inside each column,
 *     every weight finite.  The library never modifies them.
 *   - mate_in[n] int32: the matching, mate_in[j] = row matched to column j.
 *     It must be a permutation of 0..n-1 and every (mate_in[j], j) must be a
 *     stored entry.  mate_out[n] int32 receives the result in the same
 *     convention; it may alias mate_in.
 *   - Each array pointer may be host memory (pageable or pinned) or device
 *     memory of the context's GPU; the library tells them apart with
 *     cudaPointerGetAttributes.  Host arrays are copied in (and mate_out out);
 *     device arrays are read (or written) in place and are borrowed only
 *     until the call returns.  The caller owns every array; the library never
 *     frees caller memory.
 *   - Every step of the computation (input validation included) runs in CUDA
 *     kernels on the GPU.  There is no CPU fallback: without a usable GPU the
 *     calls return AWPM_ERR_CUDA.
 *
 * Error behaviour: every entry point returns an int, AWPM_OK (0) on success or
 * one of the AWPM_ERR_* codes; outputs are unspecified after an error.  When
 * an input breaks several rules, the first class in this order is reported:
 * INVALID_ARG, UNSORTED_OR_DUP, NONFINITE, NOT_PERFECT.  Reaching max_iters is
 * not an error (stats.converged = 0).
 *
 * Thread safety: a context serialises its own calls with a mutex; distinct
 * contexts may be used from different threads.
 */
#ifndef AWPM_H
#define AWPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AWPM_OK 0
#define AWPM_ERR_INVALID_ARG 1     /* bad n / pointer / colptr / row index / option   */
#define AWPM_ERR_NOT_PERFECT 2     /* mate_in not a perfect matching of stored entries */
#define AWPM_ERR_UNSORTED_OR_DUP 3 /* rows not strictly increasing within a column    */
#define AWPM_ERR_NONFINITE 4       /* a weight is NaN or infinite                     */
#define AWPM_ERR_OOM 5             /* device or pinned host allocation failed         */
#define AWPM_ERR_BUDGET 6          /* the context's device-memory budget is exceeded  */
#define AWPM_ERR_CUDA 7            /* a CUDA call failed (message: awpm_last_error)   */
#define AWPM_ERR_TIMEOUT 8         /* a bounded device-side retry or loop gave up     */
#define AWPM_ERR_NOT_FOUND 9       /* unknown ticket                                  */
#define AWPM_ERR_TOO_LARGE 10      /* problem exceeds awpm_search_noalloc's scratch   */
#define AWPM_ERR_INTERNAL 11       /* a device-side consistency check of the library's
                                      own state failed (a full hash table, a broken
                                      transpose or search tree): a library bug, not an
                                      input error; the context stays usable           */
#define AWPM_ERR_CANCELLED 12      /* the request was cancelled before it started     */

/* Closing-edge lookup strategy of the cycle search (Step B). */
#define AWPM_LOOKUP_AUTO 0    /* the library picks (per matrix)                         */
#define AWPM_LOOKUP_BSEARCH 1 /* binary search in the sorted rows of column m_i         */
#define AWPM_LOOKUP_HASH 2    /* per-column open-addressing table built once per solve
                                 (nnz < 2^30; larger problems use the binary search,
                                 as awpm_stats.lookup_used reports)                    */
#define AWPM_LOOKUP_ROWMARK 3 /* row marking (Section 4): the neighbourhood of row m_j
                                 is marked once per solve (a 64-bit signature of its
                                 columns) and confirmed in the transpose of the
                                 pattern (built once per solve by a radix sort), so
                                 every candidate of root j reads row m_j's data;
                                 never picked by AWPM_LOOKUP_AUTO; the batched and
                                 single paths only (awpm_search_noalloc: binary
                                 search)                                              */

/* awpm_options.select: how a pass turns its Step-C winners into the disjoint
 * cycles it flips.
 *   AWPM_SELECT_STEP_D (default): Step D of Algorithm 6 -- drop a winner whose
 *     second matched edge is the root edge of another winner, keep per
 *     remaining key column the largest gain (equal gains: lowest root).
 *   AWPM_SELECT_GREEDY: the selection the paper attributes to Pettie and
 *     Sanders (Section 4): the winners in order of gain, descending (equal
 *     gains: lower root column first), each kept when it shares no vertex
 *     with a cycle kept before.  On the GPU it is computed in rounds: every
 *     column names the first remaining winner that touches it, and a winner
 *     named by both of its columns is kept; the winners touching a kept
 *     cycle are dropped.  Searches (awpm_search, awpm_search_noalloc) stop
 *     before either selection. */
#define AWPM_SELECT_STEP_D 0
#define AWPM_SELECT_GREEDY 1

/* awpm_options.flags */
#define AWPM_FLAG_TIME_SEARCH 1u /* time every cycle-search launch with CUDA events
                                    (host-driven pass loop instead of one CUDA graph) */

/* Passes run when max_iters = 0 ("until a pass finds nothing") are capped here. */
#define AWPM_PASS_CAP 65536

typedef struct awpm_ctx awpm_ctx;

typedef struct {
    int32_t device;            /* CUDA device ordinal; -1 = the current device       */
    int32_t max_iters;         /* at most this many passes; 0 = until none is found  */
    int32_t lookup;            /* AWPM_LOOKUP_*                                      */
    uint32_t flags;            /* AWPM_FLAG_*                                        */
    void *stream;              /* cudaStream_t to run on; NULL = a stream the context
                                  creates and owns                                   */
    size_t mem_budget_bytes;   /* device bytes the context may hold; 0 = unlimited;
                                  for the request server: all its slots together     */
    int32_t slots;             /* request server: concurrent solves (0 = 4)          */
    int32_t select;            /* AWPM_SELECT_*: how a pass picks disjoint cycles    */
} awpm_options;

/* One request of the request server (awpm_submit). */
typedef struct {
    int32_t n;                 /* matrix order                                       */
    int32_t nnz;               /* colptr[n]; -1 = read it (a device colptr then costs
                                  a synchronisation at admission)                    */
    const int32_t *colptr;     /* the awpm_improve arguments, host or device memory, */
    const int32_t *rowidx;     /*   borrowed until awpm_poll reports the request done */
    const double *weight;
    const int32_t *mate_in;
    int32_t *mate_out;
} awpm_problem;

typedef struct {
    int32_t iterations;      /* passes of Steps A-D run, the last empty one included  */
    int32_t converged;       /* 1 if the last pass found no weight-increasing cycle   */
    int64_t cycles_applied;  /* 4-cycles flipped in total                              */
    int64_t edge_checks;     /* (nnz - n) * iterations: non-matching entries examined  */
    int64_t candidates;      /* entries (i, j) with i > m_j examined (Step A requests) */
    int64_t closing_found;   /* candidates whose closing edge {m_j, m_i} exists        */
    int64_t positive;        /* of those, gain > 0 (Step B requests)                   */
    double weight_in;        /* sum of matched weights before / after                  */
    double weight_out;       /*   (device reduction; order differs from a serial sum) */
    double ms_total;         /* wall time of the call on the stream (CUDA events)      */
    double ms_search;        /* summed cycle-search kernel time, only with
                                AWPM_FLAG_TIME_SEARCH (else 0)                         */
    int32_t lookup_used;     /* AWPM_LOOKUP_BSEARCH, _HASH or _ROWMARK                 */
    int32_t reserved;
} awpm_stats;

/* Message of an error code (static string). */
const char *awpm_strerror(int code);

/* Text of the last CUDA error seen by this thread (static per thread). */
const char *awpm_last_error(void);

/* Fill *opt with defaults: device -1, max_iters 0, lookup AUTO, no flags,
 * NULL stream, no budget, 4 server slots. */
void awpm_default_options(awpm_options *opt);

/*
 * Create a context on opt->device (opt may be NULL: defaults).  The context
 * owns its device workspace (grown on demand, kept between calls, bounded by
 * mem_budget_bytes), its CUDA graphs and, unless opt->stream is given, its
 * stream.  Errors: INVALID_ARG (out == NULL, bad option), CUDA.
 */
int awpm_create(awpm_ctx **out, const awpm_options *opt);

/* Free everything the context owns.  NULL is accepted. */
int awpm_destroy(awpm_ctx *ctx);

/*
 * The whole phase (Algorithm 2): validate the inputs, initialise mates and
 * matched weights, then run passes of
 *   Step A+B (Algorithms 3-4): every stored (i, j) with i > m_j looks up the
 *            closing edge {m_j, m_i} and computes the gain;
 *   Step C   (Algorithm 5): per root column j keep the maximum positive gain,
 *            equal gains to the lowest row i;
 *   Step D   (Algorithm 6): drop a winner whose second matched edge {i, m_i}
 *            is the root edge of another Step-C winner; per matched edge
 *            {i, m_i} keep the maximum gain, equal gains to the lowest root j;
 *            flip the survivors;
 * until a pass flips nothing or max_iters passes ran.  The pass loop runs on
 * the device (a CUDA graph with a conditional while node); the host
 * synchronises once, at the end, to read the statistics.
 * Uses the calling thread's default context on the current device (created on
 * first use, default options).  stats may be NULL.
 */
int awpm_improve(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *weight,
                 const int32_t *mate_in, int32_t *mate_out, awpm_stats *stats);

/*
 * awpm_improve on an explicit context (its device, stream, options).
 * mate_in may be NULL: the paper's whole pipeline then runs -- the
 * heavy-weight greedy maximal matching (awpm_greedy), completed when it is
 * not perfect by the maximum cardinality matching (awpm_mcm), then the
 * 4-cycle phase.  When the matrix has no perfect matching,
 * AWPM_ERR_NOT_PERFECT is returned and mate_out holds a maximum matching
 * (-1 for unmatched columns).  The first two steps' statistics are not
 * reported.
 */
int awpm_improve_ctx(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                     const double *weight, const int32_t *mate_in, int32_t *mate_out,
                     awpm_stats *stats);

/*
 * Many independent problems in one solve (batched form of awpm_improve).
 * The `count` matrices are passed as one block-diagonal union in the same
 * CSC conventions: matrix b owns the columns and rows [n_off[b], n_off[b+1])
 * (n_off: count+1 non-decreasing int32 offsets from 0 to N = n_off[count]),
 * colptr[N+1], rowidx and mate_in/mate_out[N] use global indices, and every
 * stored row of a column must lie in that column's block.  No cycle crosses
 * blocks, so each pass of the union is one pass (Algorithm 2) of every
 * matrix; a matrix stops at its first empty pass (or after max_iters
 * passes) and its tiles are skipped from then on.  Each matrix's matching,
 * pass count, cycle count and weights equal those of awpm_improve on that
 * matrix alone.  All matrices run in one CUDA-graph launch.
 *   per_matrix[count] (may be NULL): iterations, converged, cycles_applied,
 *     edge_checks, weight_in, weight_out of each matrix (candidate counters
 *     are 0 there); total (may be NULL): the union (candidates, closing_found,
 *     positive summed; iterations = passes of the longest matrix; converged
 *     = every matrix converged; edge_checks summed over the matrices).
 * Errors as awpm_improve; one invalid matrix, or a row outside its column's
 * block (AWPM_ERR_INVALID_ARG), fails the whole call.
 */
int awpm_improve_batch(awpm_ctx *ctx, int32_t count, const int32_t *n_off, const int32_t *colptr,
                       const int32_t *rowidx, const double *weight, const int32_t *mate_in,
                       int32_t *mate_out, awpm_stats *per_matrix, awpm_stats *total);

/*
 * Request server (continuous batching of independent problems; the paper's
 * static-pivoting use, Section 1, where every factorisation needs its own
 * matching).  awpm_submit queues a problem and returns at once with a ticket.
 * A scheduler thread of the context runs up to opt.slots solves
 * concurrently, each on its own stream and workspace, and admits the next
 * queued request as soon as a slot is free and the device bytes held by all
 * slots stay within opt.mem_budget_bytes (a request that could never fit
 * finishes with AWPM_ERR_BUDGET).  A request's need is estimated from n and
 * nnz (nnz read from colptr[n] at admission when the caller passes -1 with a
 * device colptr); each slot solves under a budget of what the other slots
 * leave, so the slots together never hold more than opt.mem_budget_bytes,
 * and idle slots give their workspace back when a waiting request needs the
 * room.  Admission looks up to 8 requests past the head for one that fits;
 * a head overtaken 16 times is then admitted before any other request.
 * Every request is solved exactly as by
 * awpm_improve alone: the same matching, passes and statistics, whatever else
 * runs beside it.  The problem's arrays are borrowed until the request is
 * reported done; mate_out is written then.  Device arrays must hold their
 * data when submitted (the server's streams do not wait for other streams).
 *   awpm_submit: AWPM_ERR_INVALID_ARG for a bad argument; errors of the solve
 *     itself are reported by awpm_poll / awpm_wait.
 *   awpm_poll: non-blocking.  *done = 0 while queued or running (returns
 *     AWPM_OK).  Once done: *done = 1, *stats filled, the solve's own return
 *     code returned, and the ticket released (AWPM_ERR_NOT_FOUND after).
 *   awpm_wait: blocks until done, then as awpm_poll.
 * awpm_destroy drains running solves and drops queued ones.
 */
int awpm_submit(awpm_ctx *ctx, const awpm_problem *p, uint64_t *ticket);
int awpm_poll(awpm_ctx *ctx, uint64_t ticket, int *done, awpm_stats *stats);
int awpm_wait(awpm_ctx *ctx, uint64_t ticket, awpm_stats *stats);

/*
 * Cancel a request of the request server (a serving concern; the paper has
 * no counterpart).  A request still queued is removed at once: its arrays are
 * no longer borrowed, *cancelled = 1, and awpm_poll / awpm_wait report it
 * done with AWPM_ERR_CANCELLED (releasing the ticket).  A request already
 * started runs to completion and is reported as usual (*cancelled = 0).
 * Errors: AWPM_ERR_INVALID_ARG (NULL argument), AWPM_ERR_NOT_FOUND (unknown
 * or released ticket).
 */
int awpm_cancel(awpm_ctx *ctx, uint64_t ticket, int *cancelled);

/*
 * Device memory of a context (host memory is not counted): *held = the bytes
 * it holds now, its request server's slots included; *peak = the most it has
 * held at once since creation (for the server: the most all slots held
 * together, which never exceeds opt.mem_budget_bytes when a budget is set).
 * Errors: AWPM_ERR_INVALID_ARG.
 */
int awpm_memory_held(awpm_ctx *ctx, size_t *held, size_t *peak);

/*
 * Test hook for allocation failures (the paper has no counterpart): after
 * `after` more successful device allocations of this context's own
 * workspace, the next one fails as if cudaMalloc had (AWPM_ERR_OOM), once;
 * -1 switches it off.  The context stays usable: a later call allocates
 * again.  Errors: AWPM_ERR_INVALID_ARG (ctx NULL or after < -1).
 */
int awpm_inject_alloc_failure(awpm_ctx *ctx, int32_t after);

/*
 * The device bytes one solve of an n x n problem with nnz stored entries may
 * need on this context's options (lookup, selection): the request server's
 * admission estimate, an upper bound of the workspace the solve allocates.
 * host_inputs != 0 adds the staging copies of host arrays.  For planning
 * opt.mem_budget_bytes.  Errors: AWPM_ERR_INVALID_ARG (NULL, n < 0, nnz < 0).
 */
int awpm_bytes_needed(awpm_ctx *ctx, int32_t n, int32_t nnz, int32_t host_inputs,
                      size_t *bytes);

/*
 * Heavy-weight greedy maximal matching (Section 5.1: the maximal matching
 * that starts the paper's pipeline, choosing heavy edges first).  No
 * matching is given: the result is the matching greedy builds when it takes
 * the stored entries from heaviest to lightest (equal weights: lower row
 * first, then lower column) and keeps each entry whose row and column are
 * both free.  It is computed in rounds: every free column and every free row
 * names its first free entry in that order, and the entries named by both
 * ends are matched; a round that matches nothing ends the loop, and the
 * matching is then maximal.  When it is perfect (cardinality = n) it can be
 * given to awpm_improve as mate_in.
 *   colptr, rowidx, weight: the matrix as for awpm_improve (host or device).
 *   mate_out[n] (host or device): the row matched to column j, or -1.
 *   stats (may be NULL): rounds (all of them, the last one included),
 *     cardinality, the sum of the matched weights, elapsed milliseconds.
 * Errors as awpm_improve: AWPM_ERR_INVALID_ARG, _UNSORTED_OR_DUP, _NONFINITE;
 * AWPM_ERR_NOT_PERFECT when a column has no entry (no perfect matching can
 * exist then).
 */
typedef struct {
    int32_t rounds;
    int32_t cardinality;
    double weight;
    double ms_total;
    int64_t reserved[2];
} awpm_greedy_stats;

int awpm_greedy(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const double *weight, int32_t *mate_out, awpm_greedy_stats *stats);

/*
 * Maximum cardinality matching with the heavy-weight tie-break (Section 5.2:
 * augmenting paths, preferring heavier edges when several choices exist).
 * mate[n] (host or device, in/out): a matching on entry (row of column j or
 * -1, each row at most once, every pair a stored entry; all -1 is fine), a
 * maximum matching on return that keeps every column matched on entry.
 * Phases of breadth-first searches from all free columns: at each level a
 * row offered by several columns goes to the heaviest edge (equal weights:
 * lower column); a tree ends at the free row with the heaviest last edge
 * (equal weights: lower row) and stops growing; all trees with an end are
 * augmented; a phase that augments nothing ends the search.  Columns
 * without entries are allowed (they stay unmatched).  The phase and level
 * loops run on the device in one graph launch (nested conditional WHILE
 * nodes); with AWPM_FLAG_TIME_SEARCH the host drives them instead, one
 * launch per kernel (same result).
 *   stats (may be NULL): phases (the last, augmenting nothing, included),
 *     cardinality, elapsed milliseconds, search levels.
 * Errors: AWPM_ERR_INVALID_ARG, _UNSORTED_OR_DUP, _NONFINITE as for
 * awpm_improve; AWPM_ERR_NOT_PERFECT when mate is not a matching over
 * stored entries; AWPM_ERR_TIMEOUT if a search phase exceeded n + 1 levels
 * (a bound no correct search reaches).
 */
typedef struct {
    int32_t phases;
    int32_t cardinality;
    double ms_total;
    int64_t levels;        /* search levels over all phases */
    int64_t reserved;
} awpm_mcm_stats;

int awpm_mcm(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
             const double *weight, int32_t *mate, awpm_mcm_stats *stats);

/*
 * Matching weights from the values of a sparse matrix, as the paper prepares
 * its inputs (Section 6.1): the matrix is equilibrated by diagonal scaling --
 * one sweep, columns first: v_ij = |a_ij| / max_k |a_kj|, then rows:
 * w_ij = v_ij / max_l v_il, so every row's largest entry is exactly 1 and no
 * entry exceeds 1 -- and the weight is
 *   AWPM_WEIGHTS_SUM (Option A, maximise the sum of weights): w_ij,
 *   AWPM_WEIGHTS_PRODUCT (Option B, maximise the product): log(w_ij).
 * colptr, rowidx: the pattern as for awpm_improve (rows need not be sorted
 * here); values[nnz] finite and nonzero (the paper removes explicit zeros,
 * otherwise AWPM_ERR_NONFINITE); weight_out[nnz]: host or device.  Option A
 * uses only divisions and maxima, so it is bit-for-bit reproducible; Option
 * B calls the device logarithm (within its documented error of the exact
 * value).
 */
#define AWPM_WEIGHTS_SUM 0
#define AWPM_WEIGHTS_PRODUCT 1

int awpm_weights(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                 const double *values, int32_t mode, double *weight_out);

/*
 * One cycle search from a given matching without flipping anything: Steps
 * A-C of a single pass (Algorithms 3-5).  For every column j,
 * stepc_gain[j] / stepc_row[j] receive the Step-C winner rooted at j (its gain
 * and row i), or 0.0 / -1 when j has no positive-gain 4-cycle.  stepc_gain
 * and stepc_row are n-element host or device arrays.  stats (may be NULL)
 * receives candidates, closing_found and positive of this search.
 */
int awpm_search(awpm_ctx *ctx, int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const double *weight, const int32_t *mate, double *stepc_gain,
                int32_t *stepc_row, awpm_stats *stats);

/*
 * Size limits of awpm_search_noalloc (its scratch is a fixed array of about
 * 19 MB in device memory, held by every GPU that loads the library).
 */
#define AWPM_NOALLOC_MAX_N 262144
#define AWPM_NOALLOC_MAX_NNZ 4194304

/*
 * awpm_search without any memory allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example a host framework whose memory pool has already reserved the GPU's
 * memory, or code running where an allocation (which can synchronise the
 * device) is not allowed.  It computes exactly what awpm_search computes
 * (Step-C winner gain and row per column, and the request counters in stats)
 * but allocates nothing: no cudaMalloc, no cudaFree, no pinned buffers, no
 * allocating library routine.  Its scratch is one fixed __device__ array of
 * about 19 MB inside the library, which every GPU that loads the library holds
 * until the process exits.
 *   - n <= AWPM_NOALLOC_MAX_N and nnz <= AWPM_NOALLOC_MAX_NNZ, otherwise
 *     AWPM_ERR_TOO_LARGE.
 *   - colptr, rowidx, weight, mate, stepc_gain and stepc_row must be device
 *     memory of the current device (AWPM_ERR_INVALID_ARG otherwise); the
 *     caller owns them.  stream is a cudaStream_t (NULL = the default stream).
 *     stats may be NULL (host).
 *   - Every call looks up the device address of the scratch array on the
 *     current device (cudaGetSymbolAddress), so a context re-created after
 *     cudaDeviceReset gets the right address.  The call reads colptr[n] and
 *     the search's counters back to the host and synchronises `stream`
 *     before it returns, so it cannot be captured into a CUDA graph.
 *   - Every call on a device shares the one scratch array, which keeps the
 *     contents of the last call; each call clears what must start at zero.
 *     Calls whose work overlaps on the GPU (other threads, other streams)
 *     race on the array: serialise them.
 * Errors as awpm_search, plus AWPM_ERR_TOO_LARGE.
 */
int awpm_search_noalloc(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                        const double *weight, const int32_t *mate, double *stepc_gain,
                        int32_t *stepc_row, void *stream, awpm_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* AWPM_H */
