// CUDA kernels (sm_103a) of the weight-increasing alternating 4-cycle phase
// (arXiv 1801.09809, Section 5.3, Algorithms 2-6).
//
// The paper's message exchanges become arrays indexed by column in device
// memory: the A- and B-requests of Steps A and B never leave registers (one
// fused edge-parallel kernel does the lookup and the gain), Step C is a
// segmented arg-max inside each warp plus a 128-bit compare-and-swap for the
// columns that straddle a tile boundary, and Step D is one compare-and-swap
// selection per key column followed by an in-place flip.
//
// Every kernel reads the problem from a device-resident descriptor (Work) and
// runs a fixed, GPU-sized grid with grid-stride loops, so one instantiated
// CUDA graph serves every problem of a context.
#include <math.h>
#include <stdlib.h>

#include "awpm.h"
#include "awpm_internal.h"

namespace awpm {

#define FULL_MASK 0xffffffffu

// Bounded retries for the lock-free arg-max updates (each failed
// compare-and-swap means another thread stored a strictly better record, so
// the loop ends long before this; the bound only turns a broken invariant
// into an error bit instead of a hang).
constexpr int kCasRetryCap = 1 << 20;

// Closing-edge ranges longer than this go to the warp-cooperative search
// (shorter ones to a binary search per lane).  On an R-MAT graph of scale 22
// (n = 4.2 M, 69 M nonzeros) 64 measured 4.5 us per search launch faster
// than 32, and 16 was 18 us slower.
constexpr int32_t kCoopMin = 64;
// Quiet NaN: wm[j] before the entry pass finds the matched entry of column j.
constexpr unsigned long long kNaNBits = 0x7ff8000000000000ull;

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t gtid()
{
    return blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
}

__device__ __forceinline__ int64_t gstride()
{
    return (int64_t)gridDim.x * blockDim.x;
}

__device__ __forceinline__ void raise_err(Ctl *ctl, unsigned bits)
{
    atomicOr(&ctl->err, bits);
}

// Index checks of builds with AWPM_DEBUG_BOUNDS: an index derived from data
// (a row, a mate, a position) outside [0, lim) sets kErrBounds (reported as
// AWPM_ERR_INTERNAL) and the access is skipped; nothing traps.  Other builds
// compile the checks away.
#ifdef AWPM_DEBUG_BOUNDS
__device__ __noinline__ bool in_bounds(Ctl *ctl, long long i, long long lim)
{
    if (i >= 0 && i < lim)
        return true;
    atomicOr(&ctl->err, kErrBounds);
    return false;
}
#define AWPM_IN(ctl, i, lim) in_bounds((ctl), (long long)(i), (long long)(lim))
#else
#define AWPM_IN(ctl, i, lim) true
#endif

__device__ __forceinline__ bool gate(const Ctl *ctl)
{
    return *(volatile const unsigned *)&ctl->err == 0u &&
           *(volatile const int32_t *)&ctl->active != 0;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(FULL_MASK, v, o);
    return v;
}

// Sum v over the block and add it to *dst with one atomic.  All threads call.
__device__ void block_add_u64(unsigned long long v, unsigned long long *dst)
{
    __shared__ unsigned long long sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_u64(v);
    __syncthreads();
    if (lane == 0)
        sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0ull;
        v = warp_sum_u64(v);
        if (lane == 0 && v)
            atomicAdd(dst, v);
    }
}

// Deterministic block sum (fixed tree).  All threads call.
__device__ double block_sum_f64(double v)
{
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(FULL_MASK, v, o);
    __syncthreads();
    if (lane == 0)
        sm[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(FULL_MASK, v, o);
    }
    return v;
}

// Column signatures: a partitioned Bloom filter of the column's rows in 64
// bits, one bit per row in each 32-bit half, both positions taken from one
// multiplicative hash of the row (bits 27..31 select the bit of the low
// half, bits 22..26 that of the high half).  A row with either bit clear is
// not stored in the column.  With 32-bit halves the test needs no 64-bit
// shifts.
__device__ __forceinline__ unsigned long long sig_mask(int32_t r)
{
    const uint32_t h = (uint32_t)r * 0x9E3779B1u;
    return ((unsigned long long)(1u << ((h >> 22) & 31u)) << 32) | (1u << (h >> 27));
}

__device__ __forceinline__ bool sig_has(unsigned long long sig, int32_t r)
{
    const uint32_t h = (uint32_t)r * 0x9E3779B1u;
    return (((uint32_t)sig >> (h >> 27)) & ((uint32_t)(sig >> 32) >> ((h >> 22) & 31u)) & 1u) !=
           0u;
}

// Column of the lane's nonzero: c0 (column of the tile's first nonzero) plus
// the columns starting after the tile's first nonzero and up to this lane.
// Exact when no column is empty (guaranteed once the matching validated).
__device__ __forceinline__ int32_t lane_column(int32_t c0, uint32_t mask, int lane)
{
    return c0 + __popc(mask & ((2u << lane) - 1u) & ~1u);
}

// The segment of a column that starts at `lane` covers the whole column when
// the column starts here and ends inside the tile: a later start bit, the
// end of the matrix, or a column starting the next tile.
__device__ __forceinline__ bool segment_complete(uint32_t mask, int lane, int32_t base,
                                                 int32_t nnz, const uint32_t *starts, int64_t t)
{
    const bool starts_here = (mask >> lane) & 1u;
    if (!starts_here)
        return false;
    const uint32_t later = lane == 31 ? 0u : (mask >> (lane + 1));
    return later != 0u || base + kTile >= nnz || (__ldg(starts + t + 1) & 1u);
}

// ---- per-column open-addressing tables -------------------------------------
// Column c owns the 2 * deg(c) slots [2 colptr[c], 2 colptr[c+1]) of htab;
// a slot holds (position << 32 | row), all ones when empty.  Linear probing
// from slot_start(); the table is at most half full, so every probe sequence
// meets an empty slot or the row.

constexpr unsigned long long kSlotEmpty = ~0ull;

__device__ __forceinline__ uint32_t row_mix(int32_t r)
{
    uint32_t h = (uint32_t)r;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ int32_t slot_start(int32_t r, int32_t base, int32_t size)
{
    return base + (int32_t)__umulhi(row_mix(r), (uint32_t)size);
}

// ---- blocked Bloom filters of long columns (binary-search lookup) -------------
// A column with more than kBloomMin rows, stored at positions [s, e), owns the
// words [s/4, (e-1)/4] of the bloom array: one 32-bit word per 4 nonzeros (a
// word at a boundary may be shared with the neighbouring column, which only
// adds false positives).  Each row sets three bits of one word, word and bits
// picked by a hash of the row; a row with a clear bit is not in the column.
// Long columns are where the 64-bit signature fills up, so this filter keeps
// most of their absent closing entries away from the search.

// (Filters from 8 or 4 rows up took 8-12 us off a search launch on an
// R-MAT graph of scale 22, but cost a 27-point stencil of 96^3 8 % and a
// batch of 4,096 small matrices 2 % of their solve time, so the threshold
// stays at 32.)
constexpr int32_t kBloomMin = 32;

__device__ __forceinline__ void bloom_key(int32_t r, int32_t s, int32_t e, uint32_t &word,
                                          uint32_t &bits)
{
    // multiplicative hashes (top bits), with constants other than the
    // column signature's so the two filters reject different rows
    const uint32_t h = (uint32_t)r * 0x85EBCA6Bu;
    const uint32_t w0 = (uint32_t)s >> 2;
    const uint32_t nw = (((uint32_t)e - 1u) >> 2) - w0 + 1u;
    word = w0 + __umulhi(h, nw);
    const uint32_t h2 = (uint32_t)r * 0xC2B2AE35u;
    bits = (1u << (h2 >> 27)) | (1u << ((h2 >> 22) & 31u)) | (1u << ((h2 >> 17) & 31u));
}

// ---- gains as integers ----------------------------------------------------------
// FP64 instructions are scarce on this GPU, so gains are compared through
// their IEEE bit patterns.  For values in [+0, +inf] the order of the bit
// patterns read as signed 64-bit integers is the numeric order, and equal
// patterns are equal values; every stored or compared gain is either +0.0
// ("none") or a positive gain.

__device__ __forceinline__ long long gbits(double g)
{
    return __double_as_longlong(g);
}

// g > 0.0 exactly as IEEE compares it: sign clear, not zero, not NaN.
__device__ __forceinline__ bool gain_positive(double g)
{
    const long long b = gbits(g);
    return b > 0ll && b <= 0x7ff0000000000000ll;
}

// ---- lock-free arg-max records ----------------------------------------------

// (g, p) beats (cg, cp): larger gain, then lower position (gains >= +0).
__device__ __forceinline__ bool rec_better(double g, int32_t p, double cg, int32_t cp)
{
    const long long a = gbits(g), b = gbits(cg);
    return a > b || (a == b && p < cp);
}

// Maximum of (g, lowest p) into a Step-C record.
__device__ void rec_combine(Rec *addr, Rec mine, Ctl *ctl)
{
    Rec cur = *addr;
    for (int it = 0; it < kCasRetryCap; ++it) {
        if (!rec_better(mine.g, mine.p, cur.g, cur.p))
            return;
        Rec old = atomicCAS(addr, cur, mine);
        if (__double_as_longlong(old.g) == __double_as_longlong(cur.g) && old.p == cur.p &&
            old.q == cur.q)
            return;
        cur = old;
    }
    raise_err(ctl, kErrTimeout);
}

// (g, j) beats (cg, cj): larger gain, then lower root (gains >= +0).
__device__ __forceinline__ bool sel_better(double g, int32_t j, double cg, int32_t cj)
{
    const long long a = gbits(g), b = gbits(cg);
    return a > b || (a == b && j < cj);
}

// Maximum of (g, lowest root j) into a Step-D selection.
__device__ void sel_combine(Sel *addr, Sel mine, Ctl *ctl)
{
    Sel cur = *addr;
    for (int it = 0; it < kCasRetryCap; ++it) {
        if (!sel_better(mine.g, mine.j, cur.g, cur.j))
            return;
        Sel old = atomicCAS(addr, cur, mine);
        if (__double_as_longlong(old.g) == __double_as_longlong(cur.g) && old.j == cur.j &&
            old.pad == cur.pad)
            return;
        cur = old;
    }
    raise_err(ctl, kErrTimeout);
}

// ---- cache-policy loads -------------------------------------------------------

__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Row record of `row`: the signature, range and matched weight of the column
// matched to it (two arrays, so that the signature test gathers 8 bytes per
// candidate).
__device__ __forceinline__ void put_rowrec(const Work &w, int32_t row, int32_t s, int32_t e,
                                           unsigned long long sig, double wmatch)
{
    w.rsig[row] = sig;
    // one 16-byte store
    *reinterpret_cast<int4 *>(w.rrange + row) =
        make_int4(s, e, __double2loint(wmatch), __double2hiint(wmatch));
}

__device__ __forceinline__ RowRange ld_range(const RowRange *p)
{
    const int4 v = __ldg(reinterpret_cast<const int4 *>(p));
    RowRange g;
    g.s = v.x;
    g.e = v.y;
    g.w = __hiloint2double(v.w, v.z);
    return g;
}

__device__ __forceinline__ unsigned long long ld_u64_last(const unsigned long long *ptr,
                                                          unsigned long long pol)
{
    unsigned long long v;
    asm volatile("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ int32_t ld_i32_last(const int32_t *ptr, unsigned long long pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Warp-cooperative search of row `key` among the sorted rows rowidx[s, s+len)
// for one lane's request, all 32 lanes taking part: each round every lane
// reads one pivot, a ballot picks the chunk that can hold the key and the
// range shrinks 32-fold (a 100,000-row column takes 4 rounds instead of 17
// dependent probes).  Returns the position or -1.  Called by the whole warp.
__device__ __forceinline__ int32_t coop_find(const int32_t *__restrict__ rowidx, int32_t s,
                                             int32_t len, int32_t key, int lane)
{
    while (len > 32) {
        const int32_t step = (len + 31) >> 5;
        const int32_t off = lane * step;
        const int32_t v = off < len ? __ldg(rowidx + s + off) : 0x7fffffff;
        const unsigned le = __ballot_sync(FULL_MASK, v <= key);
        if (le == 0)
            return -1;
        const int c = 31 - __clz(le);
        s += c * step;
        const int32_t rest = len - c * step;
        len = rest < step ? rest : step;
    }
    const int32_t v = lane < len ? __ldg(rowidx + s + lane) : -1;
    const unsigned eq = __ballot_sync(FULL_MASK, v == key);
    return eq ? s + __ffs(eq) - 1 : -1;
}

// ---------------------------------------------------------------------------
// Initialisation and validation (before the loop of Algorithm 2)
// ---------------------------------------------------------------------------

// Clear everything a solve expects to start at zero (or empty).
__global__ void k_reset(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (gtid() == 0) {
        Ctl *c = w.ctl;
        c->err = 0u;
        c->active = 1;
        c->iterations = 0;
        c->converged = 0;
        c->live = 0;
        c->max_passes = w.max_passes;
        c->pass_flips = 0ull;
        c->flip_done = 0u;
        c->cycles = 0ull;
        c->candidates = 0ull;
        c->found = 0ull;
        c->positive = 0ull;
        c->weight_in = 0.0;
        c->weight_out = 0.0;
        if (w.bw.count > 0) {
            *w.bw.active = 0;
            *w.bw.tlist_n = 0;
        }
    }
    const bool rec = !w.rec_clean;
    for (int64_t j = gtid(); j < w.n; j += gstride()) {
        w.mr[j] = -1;
        if (rec) {
            w.best[j] = Rec{0.0, 0, 0};
            w.dsel[j] = Sel{0.0, 0, 0};
        }
        w.colsig[j] = 0ull;
        w.wm[j] = __longlong_as_double(kNaNBits);  // "no matched entry seen"
    }
    const int64_t words = ((int64_t)w.nnz + 31) / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride())
        w.starts[x] = 0u;
    for (int64_t x = gtid(); x <= w.n / 32; x += gstride())
        w.winbits[x] = 0u;
    if (w.lookup == AWPM_LOOKUP_HASH && w.htab)
        for (int64_t x = gtid(); x < 2 * (int64_t)w.nnz; x += gstride())
            w.htab[x] = kSlotEmpty;
    if (w.bloom)
        for (int64_t x = gtid(); x <= (int64_t)w.nnz / 4; x += gstride())
            w.bloom[x] = 0u;
    if (w.rowsig)
        for (int64_t x = gtid(); x < w.n; x += gstride())
            w.rowsig[x] = 0ull;
    if (w.psel) {
        for (int64_t j = gtid(); j < w.n; j += gstride())
            w.psel[j] = Sel{0.0, 0, 0};
        for (int64_t x = gtid(); x <= w.n / 32; x += gstride()) {
            w.pslive[x] = 0u;
            w.pstaken[x] = 0u;
            w.psused[x] = 0u;
        }
    }
    for (int64_t b = gtid(); b < w.bw.count; b += gstride()) {
        w.bw.mdone[b] = 0;
        w.bw.miter[b] = 0;
        w.bw.mconv[b] = 0;
        w.bw.mflips[b] = 0ull;
        w.bw.mcycles[b] = 0ull;
    }
}

// colptr[0] = 0, non-decreasing, colptr[n] = nnz.  An empty column cannot
// hold a matched entry, so it already rules out a perfect matching.
__global__ void k_check_colptr(const Work *__restrict__ W)
{
    const Work &w = *W;
    for (int64_t j = gtid(); j <= w.n; j += gstride()) {
        const int32_t c = w.colptr[j];
        const bool bad = (j == 0 && c != 0) || (j < w.n && w.colptr[j + 1] < c) ||
                         (j == w.n && c != w.nnz);
        if (bad)
            raise_err(w.ctl, kErrInvalid);
        else if (j < w.n && w.colptr[j + 1] == c)
            raise_err(w.ctl, kErrNotPerfect);
    }
}

// The column-pointer check and the start marks in one pass over colptr (the
// solve's initialisation): a column's start bit and tile entries are written
// only when its range lies inside [0, nnz], so a bad colptr (reported as
// AWPM_ERR_INVALID_ARG, which gates every later kernel) writes nothing out
// of range.
__global__ void k_check_mark(const Work *__restrict__ W)
{
    const Work &w = *W;
    for (int64_t j = gtid(); j <= w.n; j += gstride()) {
        const int32_t c = w.colptr[j];
        const int32_t e = j < w.n ? w.colptr[j + 1] : c;
        const bool bad = (j == 0 && c != 0) || (j < w.n && e < c) || (j == w.n && c != w.nnz);
        if (bad) {
            raise_err(w.ctl, kErrInvalid);
            continue;
        }
        if (j == w.n)
            continue;
        if (e == c) {
            raise_err(w.ctl, kErrNotPerfect);
            continue;
        }
        if (c < 0 || e > w.nnz)
            continue;  // (reported by the check of the last pointer)
        atomicOr(&w.starts[c >> 5], 1u << (c & 31));
        for (int64_t t = ((int64_t)c + kTile - 1) / kTile; t * kTile < e; ++t)
            w.tile_col[t] = (int32_t)j;
    }
}

// Column-start bitmap and the first column of every tile.
__global__ void k_mark_starts(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err & kErrInvalid)
        return;
    for (int64_t j = gtid(); j < w.n; j += gstride()) {
        const int32_t s = w.colptr[j], e = w.colptr[j + 1];
        if (s < e) {
            atomicOr(&w.starts[s >> 5], 1u << (s & 31));
            for (int64_t t = ((int64_t)s + kTile - 1) / kTile; t * kTile < e; ++t)
                w.tile_col[t] = (int32_t)j;
        }
    }
}

// One pass over the entries: row range, sortedness inside columns, finite
// weights, the column signatures (OR of sig_mask(row) over each column;
// lanes of one column are OR-ed in the warp, whole columns stored, columns cut
// by a tile boundary merged with atomics) and the matched weight of every
// column: the lane holding (mate_in[j], j) stores its weight as wm[j]; with
// the binary-search lookup also the Bloom filters of the long columns.  Each
// warp takes two tiles per round and issues both tiles' loads before using
// either, so twice the bytes are in flight.  Column numbers come from the
// start bitmap, exact once no column is empty (empty columns were reported by
// the column-pointer check and always stay below n).
#ifndef AWPM_ENTRIES_U
#define AWPM_ENTRIES_U 2
#endif
#ifndef AWPM_ENTRIES_MINB
#define AWPM_ENTRIES_MINB 6
#endif
__global__ void __launch_bounds__(kThreads, AWPM_ENTRIES_MINB) k_entries(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err & kErrInvalid)
        return;
    constexpr int kU = AWPM_ENTRIES_U;
    const int lane = threadIdx.x & 31;
    // 32-bit tile arithmetic: ntiles < 2^26, positions < 2^31
    const int32_t nwarps = (int32_t)(gstride() >> 5);
    const int32_t n = w.n, nnz = w.nnz, ntiles = w.ntiles;
    const int32_t *__restrict__ rowidx = w.rowidx;
    unsigned bits = 0;
    for (int32_t t0 = (int32_t)(gtid() >> 5); t0 < ntiles; t0 += kU * nwarps) {
        int32_t c0[kU], r[kU], prev[kU], mate[kU], j[kU], cs[kU], ce[kU];
        uint32_t mask[kU];
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t t = t0 + u * nwarps;
            const bool tv = t < ntiles;
            const int32_t p = tv ? t * kTile + lane : 0;
            const bool valid = tv && p < nnz;
            c0[u] = tv ? __ldg(w.tile_col + t) : 0;
            mask[u] = tv ? __ldg(w.starts + t) : 1u;
            r[u] = valid ? __ldcs(rowidx + p) : 0;
            x[u] = valid ? __ldcs(w.w + p) : 0.0;
            prev[u] = (valid && lane == 0 && p > 0) ? __ldg(rowidx + p - 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t t = t0 + u * nwarps;
            const bool valid = t < ntiles && t * kTile + lane < nnz;
            j[u] = valid ? lane_column(c0[u], mask[u], lane) : -1 - lane;
            mate[u] = valid ? __ldg(w.mate_in + j[u]) : -1;
            const bool bl = valid && w.bloom;
            cs[u] = bl ? __ldg(w.colptr + j[u]) : 0;
            ce[u] = bl ? __ldg(w.colptr + j[u] + 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t t = t0 + u * nwarps;
            const bool tv = t < ntiles;
            const int32_t base = tv ? t * kTile : 0;
            const int32_t p = base + lane;
            const bool valid = tv && p < nnz;
            const int32_t up = __shfl_up_sync(FULL_MASK, r[u], 1);
            const int32_t before = lane == 0 ? prev[u] : up;
            const bool in_range = r[u] >= 0 && r[u] < n;
            if (valid) {
                if (!in_range)
                    bits |= kErrInvalid;
                if ((__double2hiint(x[u]) & 0x7ff00000) == 0x7ff00000)  // inf or NaN
                    bits |= kErrNonfinite;
                if (p > 0 && !((mask[u] >> lane) & 1u) && before >= r[u])
                    bits |= kErrUnsorted;
                if (mate[u] == r[u])
                    w.wm[j[u]] = x[u];
                if (ce[u] - cs[u] > kBloomMin && in_range) {
                    uint32_t word, b;
                    bloom_key(r[u], cs[u], ce[u], word, b);
                    atomicOr(w.bloom + word, b);
                }
            }
            unsigned long long v = (valid && in_range) ? sig_mask(r[u]) : 0ull;
            if (mask[u] <= 1u) {
                // the whole tile lies in one column: one warp-wide OR
                const unsigned lo = __reduce_or_sync(FULL_MASK, (unsigned)v);
                const unsigned hi = __reduce_or_sync(FULL_MASK, (unsigned)(v >> 32));
                v = ((unsigned long long)hi << 32) | lo;
            } else {
                // start bits after this lane (none for lane 31)
                const uint32_t after = __funnelshift_rc(mask[u], 0u, lane + 1);
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned long long ov = __shfl_down_sync(FULL_MASK, v, off);
                    // lane + off is in the same column: no column starts in
                    // between (past lane 31 the shuffle returns the lane's own
                    // value, and OR-ing it changes nothing)
                    if ((after & ((1u << off) - 1u)) == 0u)
                        v |= ov;
                }
            }
            const bool head = valid && (lane == 0 || ((mask[u] >> lane) & 1u));
            if (head && j[u] < n) {
                if (segment_complete(mask[u], lane, base, nnz, w.starts, t))
                    w.colsig[j[u]] = v;
                else if (v)
                    atomicOr(w.colsig + j[u], v);
            }
        }
    }
    bits = __reduce_or_sync(FULL_MASK, bits);
    if (lane == 0 && bits)
        raise_err(w.ctl, bits);
}

// Initialisation of the matching in two passes, so that no record is
// written to a scattered address:
//   k_init_mates (per column j): mc[j] = mate_in[j], and mr[mate_in[j]] = j
//     (a 4-byte scattered store per column; mr stays in L2 while it fills);
//     checks that every mate_in[j] is a row number and a stored entry of
//     column j (the entry pass left wm[j] = NaN where (mate_in[j], j) is not
//     stored); and the matched weights' sum, one partial per block into
//     wpart (the grid is at most kWsumBlocks), summed by k_wsum_final;
//   k_init_rows (per row r): the row record of r from column mr[r] (gathers
//     of that column's range, signature and matched weight; the records are
//     written row by row, whole sectors at a time), and the check that every
//     row got a column: with n columns and n rows that holds exactly when
//     mate_in is a permutation.
__global__ void k_init_mates(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err) {
        if (threadIdx.x == 0)
            w.wpart[blockIdx.x] = 0.0;
        return;
    }
    constexpr int kU = 8;
    const int64_t stride = gstride();
    const int32_t n = w.n;
    unsigned bits = 0;
    double sum = 0.0;
    for (int64_t j0 = gtid(); j0 < n; j0 += kU * stride) {
        int32_t r[kU];
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t j = j0 + u * stride;
            const bool ok = j < n;
            r[u] = ok ? w.mate_in[j] : -1;
            x[u] = ok ? w.wm[j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t j = j0 + u * stride;
            if (j >= n)
                continue;
            w.mc[j] = r[u];
            if (r[u] < 0 || r[u] >= n || gbits(x[u]) == (long long)kNaNBits) {
                bits |= kErrNotPerfect;
                continue;
            }
            w.mr[r[u]] = (int32_t)j;
            sum += x[u];
        }
    }
    bits = __reduce_or_sync(FULL_MASK, bits);
    if ((threadIdx.x & 31) == 0 && bits)
        raise_err(w.ctl, bits);
    sum = block_sum_f64(sum);
    if (threadIdx.x == 0)
        w.wpart[blockIdx.x] = sum;
}

__global__ void k_init_rows(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    constexpr int kU = 4;
    const int64_t stride = gstride();
    const int32_t n = w.n;
    bool bad = false;
    for (int64_t r0 = gtid(); r0 < n; r0 += kU * stride) {
        int32_t j[kU], cs[kU], ce[kU];
        unsigned long long sig[kU];
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t r = r0 + u * stride;
            j[u] = r < n ? w.mr[r] : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t r = r0 + u * stride;
            const bool ok = r < n && j[u] >= 0;
            bad |= r < n && j[u] < 0;
            cs[u] = ok ? __ldg(w.colptr + j[u]) : 0;
            ce[u] = ok ? __ldg(w.colptr + j[u] + 1) : 0;
            sig[u] = ok ? __ldg(w.colsig + j[u]) : 0ull;
            x[u] = ok ? __ldg(w.wm + j[u]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t r = r0 + u * stride;
            if (r < n)
                put_rowrec(w, (int32_t)r, cs[u], ce[u], sig[u], x[u]);
        }
    }
    if (__any_sync(FULL_MASK, bad) && (threadIdx.x & 31) == 0)
        raise_err(w.ctl, kErrNotPerfect);
}

// Per-column hash tables (only for AWPM_LOOKUP_HASH).
__global__ void __launch_bounds__(kThreads) k_hash_build(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err || w.lookup != AWPM_LOOKUP_HASH || !w.htab)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t t = gtid() >> 5; t < w.ntiles; t += nwarps) {
        const int32_t p = (int32_t)(t * kTile) + lane;
        if (p >= w.nnz)
            continue;
        const int32_t j = lane_column(w.tile_col[t], w.starts[t], lane);
        const int32_t r = __ldcs(w.rowidx + p);
        const int32_t base = 2 * w.colptr[j];
        const int32_t size = 2 * (w.colptr[j + 1] - w.colptr[j]);
        const unsigned long long v = ((unsigned long long)(uint32_t)p << 32) | (uint32_t)r;
        int32_t pos = slot_start(r, base, size);
        int k = 0;
        for (; k < size; ++k) {
            if (atomicCAS(w.htab + pos, kSlotEmpty, v) == kSlotEmpty)
                break;
            if (++pos == base + size)
                pos = base;
        }
        if (k == size)
            raise_err(w.ctl, kErrInternal);
    }
}

__global__ void k_wsum_partial(const Work *__restrict__ W)
{
    const Work &w = *W;
    double s = 0.0;
    if (w.ctl->err == 0u)
        for (int64_t j = gtid(); j < w.n; j += gstride())
            s += w.wm[j];
    s = block_sum_f64(s);
    if (threadIdx.x == 0)
        w.wpart[blockIdx.x] = s;
}

// The sum of the first `parts` block partials (parts <= blockDim.x); 0 after
// an error.
__global__ void k_wsum_final(const Work *__restrict__ W, int out, int parts)
{
    const Work &w = *W;
    double s = block_sum_f64((int)threadIdx.x < parts ? w.wpart[threadIdx.x] : 0.0);
    if (w.ctl->err)
        s = 0.0;
    if (threadIdx.x == 0) {
        if (out)
            w.ctl->weight_out = s;
        else
            w.ctl->weight_in = s;
    }
}

// ---------------------------------------------------------------------------
// Batched solves: many matrices as one block-diagonal union
// ---------------------------------------------------------------------------
// Cycles never cross blocks (no entry joins two blocks), so every pass of
// the union is one pass of each matrix.  A matrix whose pass flips nothing
// (or that reached the pass cap) is finished: its tiles are skipped from then
// on and its counters stop, which gives each matrix exactly the passes,
// flips and result of a solve on its own.

// Offsets non-decreasing from 0 to n; matrix of every column.
__global__ void k_batch_cols(const Work *__restrict__ W)
{
    const Work &w = *W;
    const int32_t count = w.bw.count;
    const int32_t *n_off = w.bw.n_off;
    for (int64_t x = gtid(); x <= count; x += gstride()) {
        const int32_t o = n_off[x];
        if ((x == 0 && o != 0) || (x == count && o != w.n) || (x < count && n_off[x + 1] < o))
            raise_err(w.ctl, kErrInvalid);
    }
    // a warp per matrix writes the matrix number of its columns (clamped to
    // [0, n): offsets found invalid above raise the error but write nothing
    // out of range)
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t b = gtid() >> 5; b < count; b += nwarps) {
        const int32_t lo = max(n_off[b], 0), hi = min(n_off[b + 1], w.n);
        for (int32_t x = lo + lane; x < hi; x += 32)
            w.bw.colmat[x] = (int32_t)b;
    }
}

// Every stored row lies in its column's block; nonzeros per matrix; the
// matrix of each tile and whether the tile stays inside one matrix.
__global__ void __launch_bounds__(kThreads) k_batch_check(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    const BatchWork &bw = w.bw;
    unsigned bad = 0;
    // four tiles per warp round, their loads side by side (the checks are
    // chains of dependent gathers)
    constexpr int kU = 4;
    for (int64_t t0 = gtid() >> 5; t0 < w.ntiles; t0 += kU * nwarps) {
        int32_t c0[kU], b[kU], r[kU];
        uint32_t mask[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t t = t0 + u * nwarps;
            const bool tv = t < w.ntiles;
            c0[u] = tv ? w.tile_col[t] : 0;
            mask[u] = tv ? w.starts[t] : 1u;
            const int64_t p = t * kTile + lane;
            r[u] = tv && p < w.nnz ? w.rowidx[p] : -1;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            b[u] = r[u] >= 0 ? bw.colmat[lane_column(c0[u], mask[u], lane)] : 0;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t t = t0 + u * nwarps;
            if (r[u] >= 0 && (r[u] < bw.n_off[b[u]] || r[u] >= bw.n_off[b[u] + 1]))
                bad = 1;
            if (lane == 0 && t < w.ntiles) {
                const int32_t b0 = bw.colmat[c0[u]];
                const int32_t b1 =
                    (t + 1 < w.ntiles) ? bw.colmat[w.tile_col[t + 1]] : bw.colmat[w.n - 1];
                bw.tilemat[t] = b0 | (b0 == b1 ? kTileSingle : 0);
            }
        }
    }
    if (__any_sync(FULL_MASK, bad) && lane == 0)
        raise_err(w.ctl, kErrInvalid);
    for (int64_t b = gtid(); b < bw.count; b += gstride())
        bw.mnnz[b] = w.colptr[bw.n_off[b + 1]] - w.colptr[bw.n_off[b]];
}

// The tiles the next pass of a batched solve searches: those of matrices
// still running, and every tile spanning two matrices (its lanes of a
// finished matrix are skipped in the search).  Each tile at most once; the
// list's order (warp-aggregated appends) does not change any result, since
// the search's records and counters are order-free.  The count was zeroed
// by the reset (first pass) or the end-of-pass control.
__global__ void k_batch_list(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    const BatchWork &bw = w.bw;
    const int lane = threadIdx.x & 31;
    for (int64_t t0 = gtid() - lane; t0 < w.ntiles; t0 += gstride()) {
        const int64_t t = t0 + lane;
        bool keep = false;
        if (t < w.ntiles) {
            const int32_t tm = __ldg(bw.tilemat + t);
            keep = !(tm & kTileSingle) || !bw.mdone[tm & ~kTileSingle];
        }
        const unsigned m = __ballot_sync(FULL_MASK, keep);
        if (!m)
            continue;
        int32_t base = 0;
        if (lane == 0)
            base = atomicAdd(bw.tlist_n, __popc(m));
        base = __shfl_sync(FULL_MASK, base, 0);
        if (keep)
            bw.tlist[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)t;
    }
}

// One block per matrix (grid-stride over matrices): deterministic sum of its
// matched weights.
__global__ void k_batch_wsum(const Work *__restrict__ W, int out)
{
    const Work &w = *W;
    const BatchWork &bw = w.bw;
    for (int64_t b = blockIdx.x; b < bw.count; b += gridDim.x) {
        double s = 0.0;
        if (w.ctl->err == 0u)
            for (int64_t j = bw.n_off[b] + threadIdx.x; j < bw.n_off[b + 1]; j += blockDim.x)
                s += w.wm[j];
        s = block_sum_f64(s);
        if (threadIdx.x == 0)
            (out ? bw.mw_out : bw.mw_in)[b] = s;
    }
}

// ---------------------------------------------------------------------------
// Row marking (Section 4): marks of the rows' neighbourhoods and the
// transpose of the pattern, built once per solve for AWPM_LOOKUP_ROWMARK
// ---------------------------------------------------------------------------

// The mark of row i: the signature (see sig_mask) of the columns k with a
// stored (i, k), each column named by its first position colptr[k] (the
// search has that number at hand from the row record), OR-ed over the
// entries with 64-bit atomics (skipped when the bits are already set).  Runs
// after validation: no column is empty, so the start bitmap gives exact
// columns and distinct first positions.
__global__ void __launch_bounds__(kThreads) k_rm_marks(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err || !w.rowsig)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t t = gtid() >> 5; t < w.ntiles; t += nwarps) {
        const int32_t p = (int32_t)(t * kTile) + lane;
        if (p >= w.nnz)
            continue;
        const int32_t j = lane_column(__ldg(w.tile_col + t), __ldg(w.starts + t), lane);
        const int32_t i = __ldcs(w.rowidx + p);
        const unsigned long long m = sig_mask(__ldg(w.colptr + j));
        // bits only ever get set: a set bit in the (possibly stale) L1 copy
        // is set; otherwise ask the L2 copy, where the atomics land
        if ((w.rowsig[i] & m) != m && (__ldcg(w.rowsig + i) & m) != m)
            atomicOr(w.rowsig + i, m);
    }
}

// Exclusive prefix of one value per thread over a block of kRsThreads
// threads; the block's total into *total.  Called by the whole block.
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total)
{
    __shared__ int32_t s_w[kRsThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        s_w[warp] = x;
    __syncthreads();
    int32_t below = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kRsThreads / 32; ++i) {
        below += i < warp ? s_w[i] : 0;
        tot += s_w[i];
    }
    __syncthreads();
    *total = tot;
    return below + x - v;
}

// The transpose is a stable LSD radix sort of the entries (in CSC order) by
// row, 8 bits per pass: afterwards the CSC positions of each row's entries
// are contiguous and ascending, i.e. in column order.  Pass `pass` reads the
// keys of the previous pass (the row indices themselves first) and writes
// buffer pass & 1; passes at or above rs_passes do nothing.

// Digit counts of each block tile of kRsTile entries, stored digit-major
// (rs_hist[digit * rs_tiles + tile]) so one scan gives every scatter offset.
// A thread loads its 16 keys first; each warp counts into its own table.
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const Work *__restrict__ W, int pass)
{
    const Work &w = *W;
    if (w.ctl->err || pass >= w.rs_passes)
        return;
    constexpr int kWarps = kRsThreads / 32;
    __shared__ int32_t s_cnt[kWarps][kRsBins];
    const int warp = threadIdx.x >> 5;
    const int shift = 8 * pass;
    const int32_t *key = pass == 0 ? w.rowidx : w.rs_key[(pass - 1) & 1];
    for (int64_t tile = blockIdx.x; tile < w.rs_tiles; tile += gridDim.x) {
#pragma unroll
        for (int x = 0; x < kWarps; ++x)
            s_cnt[x][threadIdx.x] = 0;
        uint32_t k[kRsItems];
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            const int64_t e = tile * kRsTile + r * kRsThreads + threadIdx.x;
            k[r] = e < w.nnz ? (uint32_t)__ldcs(key + e) : 0xffffffffu;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsItems; ++r)
            if (k[r] != 0xffffffffu)
                atomicAdd(&s_cnt[warp][(k[r] >> shift) & 255u], 1);
        __syncthreads();
        int32_t c = 0;
#pragma unroll
        for (int x = 0; x < kWarps; ++x)
            c += s_cnt[x][threadIdx.x];
        w.rs_hist[(int64_t)threadIdx.x * w.rs_tiles + tile] = c;
        __syncthreads();
    }
}

// Scan of the digit counts, step 1: the total of every chunk of kScanChunk.
__global__ void __launch_bounds__(kRsThreads) k_rs_scan_a(const Work *__restrict__ W, int pass)
{
    const Work &w = *W;
    if (w.ctl->err || pass >= w.rs_passes)
        return;
    const int64_t m = (int64_t)kRsBins * w.rs_tiles;
    const int64_t chunks = (m + kScanChunk - 1) / kScanChunk;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        int32_t s = 0;
        for (int k = 0; k < kScanChunk / kRsThreads; ++k) {
            const int64_t x = c * kScanChunk + k * kRsThreads + threadIdx.x;
            if (x < m)
                s += w.rs_hist[x];
        }
        int32_t tot = 0;
        block_excl_scan(s, &tot);
        if (threadIdx.x == 0)
            w.rs_sums[c] = tot;
    }
}

// Step 2 (one block): exclusive prefix of the chunk totals, in place.
__global__ void __launch_bounds__(kRsThreads) k_rs_scan_b(const Work *__restrict__ W, int pass)
{
    const Work &w = *W;
    if (w.ctl->err || pass >= w.rs_passes)
        return;
    const int64_t m = (int64_t)kRsBins * w.rs_tiles;
    const int64_t chunks = (m + kScanChunk - 1) / kScanChunk;
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < chunks; b0 += kRsThreads) {
        const int64_t x = b0 + threadIdx.x;
        const int32_t v = x < chunks ? w.rs_sums[x] : 0;
        int32_t tot = 0;
        const int32_t pre = block_excl_scan(v, &tot);
        if (x < chunks)
            w.rs_sums[x] = carry + pre;
        carry += tot;
    }
}

// Step 3: every chunk's exclusive prefix plus the chunk's offset, in place;
// thread t takes the chunk's counts 8t .. 8t + 7.
__global__ void __launch_bounds__(kRsThreads) k_rs_scan_c(const Work *__restrict__ W, int pass)
{
    const Work &w = *W;
    if (w.ctl->err || pass >= w.rs_passes)
        return;
    constexpr int kPer = kScanChunk / kRsThreads;
    const int64_t m = (int64_t)kRsBins * w.rs_tiles;
    const int64_t chunks = (m + kScanChunk - 1) / kScanChunk;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const int64_t x0 = c * kScanChunk + (int64_t)threadIdx.x * kPer;
        int32_t v[kPer];
        int32_t s = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = x0 + k < m ? w.rs_hist[x0 + k] : 0;
            s += v[k];
        }
        int32_t tot = 0;
        int32_t run = block_excl_scan(s, &tot) + w.rs_sums[c];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (x0 + k < m)
                w.rs_hist[x0 + k] = run;
            run += v[k];
        }
    }
}

// Stable scatter of one pass.  A thread loads its kRsItems entries of the
// block tile; the tile is sorted by digit in shared memory (the entries
// placed 256 at a time, in order: within a warp, entries of equal digit --
// eight ballots -- are ranked by lane, and the warps' digit counts give each
// warp's offset; counts and running offsets alternate between two tables, so
// a round needs two barriers); then each digit's run is written to its
// global offset with consecutive threads on consecutive positions.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const Work *__restrict__ W, int pass)
{
    const Work &w = *W;
    if (w.ctl->err || pass >= w.rs_passes)
        return;
    constexpr int kWarps = kRsThreads / 32;
    __shared__ int32_t s_key[kRsTile];
    __shared__ int32_t s_val[kRsTile];
    __shared__ int32_t s_local[kRsBins];   // start of each digit's run in the tile
    __shared__ int32_t s_global[kRsBins];  // its global offset
    __shared__ int32_t s_base[2][kRsBins];
    __shared__ int32_t s_wcnt[2][kWarps][kRsBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int shift = 8 * pass;
    const int32_t *kin = pass == 0 ? w.rowidx : w.rs_key[(pass - 1) & 1];
    const int32_t *vin = pass == 0 ? nullptr : w.rs_val[(pass - 1) & 1];
    int32_t *kout = w.rs_key[pass & 1];
    int32_t *vout = w.rs_val[pass & 1];
    for (int64_t tile = blockIdx.x; tile < w.rs_tiles; tile += gridDim.x) {
        const int64_t first = tile * kRsTile;
        const int32_t count =
            (int32_t)(w.nnz - first < kRsTile ? w.nnz - first : (int64_t)kRsTile);
        int32_t kv[kRsItems], vv[kRsItems];
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            const int32_t x = r * kRsThreads + threadIdx.x;
            const bool valid = x < count;
            kv[r] = valid ? __ldcs(kin + first + x) : -1;
            vv[r] = valid ? (vin ? __ldcs(vin + first + x) : (int32_t)(first + x)) : 0;
        }
        s_base[0][threadIdx.x] = 0;  // digit counts of the tile first
#pragma unroll
        for (int x = 0; x < kWarps; ++x) {
            s_wcnt[0][x][threadIdx.x] = 0;
            s_wcnt[1][x][threadIdx.x] = 0;
        }
        s_global[threadIdx.x] = w.rs_hist[(int64_t)threadIdx.x * w.rs_tiles + tile];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsItems; ++r)
            if (kv[r] >= 0)
                atomicAdd(&s_base[0][((uint32_t)kv[r] >> shift) & 255u], 1);
        __syncthreads();
        int32_t tot = 0;
        const int32_t start = block_excl_scan(s_base[0][threadIdx.x], &tot);
        s_local[threadIdx.x] = start;
        s_base[0][threadIdx.x] = start;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            const int q = r & 1;
            const bool valid = kv[r] >= 0;
            const int d = valid ? (int)(((uint32_t)kv[r] >> shift) & 255u) : kRsBins;
            // lanes with the same digit: agree on all 8 bits and on validity
            const unsigned vm = __ballot_sync(FULL_MASK, valid);
            unsigned peers = valid ? vm : ~vm;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned m = __ballot_sync(FULL_MASK, (d >> b) & 1);
                peers &= ((d >> b) & 1) ? m : ~m;
            }
            const int rank = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank == 0)
                s_wcnt[q][warp][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                int32_t off = s_base[q][d] + rank;
                for (int x = 0; x < warp; ++x)
                    off += s_wcnt[q][x][d];
                s_key[off] = kv[r];
                s_val[off] = vv[r];
            }
            int32_t add = 0;
#pragma unroll
            for (int x = 0; x < kWarps; ++x) {
                add += s_wcnt[q][x][threadIdx.x];
                s_wcnt[q ^ 1][x][threadIdx.x] = 0;
            }
            s_base[q ^ 1][threadIdx.x] = s_base[q][threadIdx.x] + add;
            __syncthreads();
        }
        for (int32_t x = threadIdx.x; x < count; x += kRsThreads) {
            const int32_t key = s_key[x];
            const int d = (int)(((uint32_t)key >> shift) & 255u);
            const int32_t g = s_global[d] + (x - s_local[d]);
            if (g >= 0 && g < w.nnz) {
                kout[g] = key;
                vout[g] = s_val[x];
            } else {
                raise_err(w.ctl, kErrInternal);
            }
        }
        __syncthreads();
    }
}

// Row pointers of the transpose from the sorted keys: row r starts at the
// first entry whose row is >= r.
__global__ void k_rm_rowptr(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err || !w.trowptr)
        return;
    const int64_t nnz = w.nnz;
    if (nnz == 0) {
        for (int64_t r = gtid(); r <= w.n; r += gstride())
            w.trowptr[r] = 0;
        return;
    }
    const int32_t *key = w.rs_key[(w.rs_passes - 1) & 1];
    for (int64_t e = gtid(); e < nnz; e += gstride()) {
        const int32_t k = key[e];
        const int32_t prev = e > 0 ? key[e - 1] : -1;
        if (k < 0 || k >= w.n || prev > k) {  // not sorted rows: no transpose
            raise_err(w.ctl, kErrInternal);
            continue;
        }
        for (int32_t r = prev + 1; r <= k; ++r)
            w.trowptr[r] = (int32_t)e;
        if (e == nnz - 1)
            for (int64_t r = (int64_t)k + 1; r <= w.n; ++r)
                w.trowptr[r] = (int32_t)nnz;
    }
}

// Warp-cooperative search, in the ascending values arr[s, s+len), of the
// last one below `key` for one lane's request (all 32 lanes take part, as in
// coop_find).  Returns its index or -1.
__device__ __forceinline__ int32_t coop_last_below(const int32_t *__restrict__ arr, int32_t s,
                                                   int32_t len, int32_t key, int lane)
{
    while (len > 32) {
        const int32_t step = (len + 31) >> 5;
        const int32_t off = lane * step;
        const int32_t v = off < len ? __ldg(arr + s + off) : 0x7fffffff;
        const unsigned lt = __ballot_sync(FULL_MASK, v < key);
        if (lt == 0)
            return -1;
        const int c = 31 - __clz(lt);
        s += c * step;
        const int32_t rest = len - c * step;
        len = rest < step ? rest : step;
    }
    const int32_t v = lane < len ? __ldg(arr + s + lane) : 0x7fffffff;
    const unsigned lt = __ballot_sync(FULL_MASK, v < key);
    return lt ? s + 31 - __clz(lt) : -1;
}

// ---------------------------------------------------------------------------
// Steps A + B + C (Algorithms 3, 4, 5): fused edge-parallel cycle search
// ---------------------------------------------------------------------------

// Closing-entry lookups of one warp, queued across tiles (a ring of 64
// entries, struct of arrays in shared memory): a lane whose candidate passed
// the signature test leaves its request here, and the warp resolves 32
// requests at a time, one per lane, instead of searching with the one or two
// lanes of a tile that need it.
constexpr int kQueue = 64;
struct LookupQueue {
    int2 im[kQueue];  // row i, and m_j (the row looked up in column m_i)
    int2 jp[kQueue];  // root column j, and the position of (i, j)
};

// Resolve the queued requests head .. head + k - 1 (k <= 32, lane x takes
// request head + x): Bloom probe for long columns, then the column search
// (per lane up to kCoopMin rows, warp-cooperative above), or the hash probe,
// or with row marking the search of row m_j's entries (CSC positions,
// ascending) for the one inside column m_i's positions [lo, lo + len) (per
// lane, warp-cooperative above kCoopMin entries);
// a closing entry found gives the gain in the fixed order
// ((w_ij + w_q) - w(i, m_i)) - w(m_j, j), and a positive gain goes into the
// root's Step-C record (maximum gain, then lowest position; Algorithm 5).
// Called by the whole warp.
template <int kLookup, typename Queue>
__device__ __forceinline__ void resolve_lookups(
    const Queue &qu, int head, int k, int lane, const int32_t *__restrict__ rowidx,
    const double *__restrict__ wv, const double *__restrict__ wm,
    const unsigned long long *__restrict__ htab, const uint32_t *__restrict__ bloom,
    const int32_t *__restrict__ trowptr, const int32_t *__restrict__ tpos,
    const RowRange *__restrict__ rrange, int32_t nnz, int32_t nrows, Rec *__restrict__ best,
    uint32_t *winbits,
    Ctl *ctl, uint32_t &n_found, uint32_t &n_pos)
{
    const int x = (head + lane) & (kQueue - 1);
    const bool act = lane < k;
    const int2 im = act ? qu.im[x] : make_int2(0, 0);
    const int32_t mj = im.y;
    // column m_i's rows rowidx[lo, lo + len) and w(i, m_i), from the row
    // record of i
    int32_t lo = 0, len = 0;
    double wmi = 0.0;
    if (act && AWPM_IN(ctl, im.x, nrows)) {
        const RowRange rg = ld_range(rrange + im.x);
        lo = rg.s;
        len = rg.e - rg.s;
        wmi = rg.w;
        if (!(AWPM_IN(ctl, lo, (long long)nnz + 1) && AWPM_IN(ctl, len, (long long)nnz - lo + 1)))
            lo = len = 0;
    }
    int32_t q = -1;
    if (kLookup == AWPM_LOOKUP_HASH) {
        const int32_t hbase = 2 * lo;
        const int32_t hsize = 2 * len;
        int32_t pos = hsize > 0 ? slot_start(mj, hbase, hsize) : 0;
        for (int32_t left = hsize; left > 0; --left) {
            const unsigned long long v = __ldg(htab + pos);
            if ((int32_t)(uint32_t)v == mj) {
                q = (int32_t)(v >> 32);
                break;
            }
            if (v == kSlotEmpty)
                break;
            if (++pos == hbase + hsize)
                pos = hbase;
        }
    } else if (kLookup == AWPM_LOOKUP_ROWMARK) {
        // column m_i's positions are [a, b); row m_j's entries tpos[lo, lo + len)
        const int32_t a = lo, b = lo + len;
        if (act) {
            lo = __ldg(trowptr + mj);
            len = __ldg(trowptr + mj + 1) - lo;
            if (lo < 0 || len < 0 || len > nnz - lo) {
                lo = 0;
                len = 0;
                raise_err(ctl, kErrInternal);
            }
        }
        unsigned longm = __ballot_sync(FULL_MASK, len > kCoopMin);
        while (longm) {
            const int src = __ffs(longm) - 1;
            longm &= longm - 1;
            const int32_t ss = __shfl_sync(FULL_MASK, lo, src);
            const int32_t sl = __shfl_sync(FULL_MASK, len, src);
            const int32_t sb = __shfl_sync(FULL_MASK, b, src);
            const int32_t f = coop_last_below(tpos, ss, sl, sb, lane);
            if (lane == src) {
                const int32_t v = f >= 0 ? __ldg(tpos + f) : -1;
                q = v >= a ? v : -1;
                len = 0;
            }
        }
        // short rows: the last entry below column m_i's end, per lane
        const int32_t s0 = lo;
        int32_t hi = lo + len;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (__ldg(tpos + mid) < b)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (len > 0 && lo > s0) {
            const int32_t v = __ldg(tpos + lo - 1);
            if (v >= a)
                q = v;
        }
    } else {
        if (bloom && len > kBloomMin) {
            // long column: its Bloom filter rules most absent rows out first
            uint32_t word, b;
            bloom_key(mj, lo, lo + len, word, b);
            if ((__ldg(bloom + word) & b) != b)
                len = 0;
        }
        // long columns: the warp searches them together, one request at a time
        unsigned longm = __ballot_sync(FULL_MASK, len > kCoopMin);
        while (longm) {
            const int src = __ffs(longm) - 1;
            longm &= longm - 1;
            const int32_t ss = __shfl_sync(FULL_MASK, lo, src);
            const int32_t sl = __shfl_sync(FULL_MASK, len, src);
            const int32_t sk = __shfl_sync(FULL_MASK, mj, src);
            const int32_t f = coop_find(rowidx, ss, sl, sk, lane);
            if (lane == src) {
                q = f;
                len = 0;
            }
        }
        // short columns: binary search per lane (early exit on a hit)
        while (len > 0) {
            const int32_t half = len >> 1;
            const int32_t mid = lo + half;
            const int32_t v = __ldg(rowidx + mid);
            if (v == mj) {
                q = mid;
                break;
            }
            if (v < mj) {
                lo = mid + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
    }
    const int2 jp = q >= 0 ? qu.jp[x] : make_int2(0, 0);
    if (q >= 0 && !(AWPM_IN(ctl, q, nnz) && AWPM_IN(ctl, jp.y, nnz) && AWPM_IN(ctl, jp.x, nrows)))
        q = -1;
    if (q >= 0) {
        ++n_found;
        const int32_t j = jp.x;
        const int32_t p = jp.y;
        const double wij = __ldg(wv + p);
        const double wq = __ldg(wv + q);
        const double gg = ((wij + wq) - wmi) - __ldg(wm + j);
        if (gain_positive(gg)) {
            ++n_pos;
            Rec r;
            r.g = gg;
            r.p = p;
            r.q = q;
            rec_combine(best + j, r, ctl);
            atomicOr(winbits + (j >> 5), 1u << (j & 31));
        }
    }
}

// One warp per tile of kTile consecutive nonzeros (lane = one nonzero).
// The lane's column comes from the tile's first column and its word of the
// column-start bitmap (one popcount).  Lane with nonzero p = (i, j): if
// i > m_j it is an A-request (Algorithm 3); the closing entry (m_j, m_i) is
// looked up in column m_i (Algorithm 4): the row record of i gives that
// column's range and signature, so a clear signature bit settles "absent" at
// once; otherwise the request is queued and resolved with 31 others (see
// resolve_lookups).  Step-C records (Algorithm 5) are combined by a 128-bit
// compare-and-swap; `best` must be zero on entry: only positive records are
// written.  In a batched solve, tiles of finished matrices are skipped.
// Block size of the search kernels (each warp has its own lookup queue):
// 512 threads for a single problem, 256 for a batched solve.  With the grid
// one wave of resident blocks, the single problem's search measured a little
// faster with larger blocks on an R-MAT graph of scale 22 (0.267 ms per
// launch at 512 threads, 0.270 at 256, 0.271 at 128), a batch of 4,096 small
// matrices slower (21.4 ms per batch at 512, 20.0 at 256).  The minimum blocks per SM below are given
// in warps per SM, divided by the block's warps.
#ifndef AWPM_SEARCH_THREADS
#define AWPM_SEARCH_THREADS 512
#endif
template <bool kBatch>
struct SearchBlock {
    static constexpr int kThreads = kBatch ? 256 : AWPM_SEARCH_THREADS;
    static constexpr int kWarps = kThreads / 32;
};
#ifndef AWPM_SEARCH_MINB_WIDE
#define AWPM_SEARCH_MINB_WIDE (32 / SearchBlock<kBatch>::kWarps)
#endif
template <int kLookup, bool kBatch, bool kWide>
__global__ void __launch_bounds__(SearchBlock<kBatch>::kThreads,
                                  kWide ? AWPM_SEARCH_MINB_WIDE : 48 / SearchBlock<kBatch>::kWarps)
    k_search(const Work *__restrict__ W)
{
    __shared__ int s_go;
    __shared__ LookupQueue s_queue[SearchBlock<kBatch>::kWarps];
    if (threadIdx.x == 0)
        s_go = gate(W->ctl) ? 1 : 0;
    __syncthreads();
    const int32_t nnz = W->nnz;
    const int32_t ntiles = W->ntiles;
    const int32_t *__restrict__ rowidx = W->rowidx;
    const double *__restrict__ wv = W->w;
    const int32_t *__restrict__ tile_col = W->tile_col;
    const uint32_t *__restrict__ starts = W->starts;
    const int32_t *__restrict__ mc = W->mc;
    const double *__restrict__ wm = W->wm;
    const unsigned long long *__restrict__ rsig = W->rsig;
    const RowRange *__restrict__ rrange = W->rrange;
    const unsigned long long *__restrict__ htab = W->htab;
    const uint32_t *__restrict__ bloom = W->bloom;
    const unsigned long long *__restrict__ rowsig = W->rowsig;
    const int32_t *__restrict__ trowptr = W->trowptr;
    const int32_t *__restrict__ tpos = W->tpos;
    Rec *__restrict__ best = W->best;
    uint32_t *winbits = W->winbits;
    Ctl *ctl = W->ctl;
    const int32_t *__restrict__ tilemat = W->bw.tilemat;
    const int32_t *__restrict__ colmat = W->bw.colmat;
    const int32_t *__restrict__ mdone = W->bw.mdone;
    LookupQueue &qu = s_queue[threadIdx.x >> 5];

    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const int64_t nwarps = gstride() >> 5;
    const unsigned long long pol = policy_evict_last();
    // per-thread counts fit 32 bits (one nonzero per tile a warp visits)
    uint32_t n_cand = 0, n_found = 0, n_pos = 0;
    int qhead = 0, qn = 0;  // the warp's queue (warp-uniform)

    auto flush = [&](int k) {
        __syncwarp();
        resolve_lookups<kLookup>(qu, qhead, k, lane, rowidx, wv, wm, htab, bloom, trowptr,
                                 tpos, rrange, nnz, W->n, best, winbits, ctl, n_found, n_pos);
        __syncwarp();
        qhead = (qhead + k) & (kQueue - 1);
        qn -= k;
    };
    // Each round a warp takes kU tiles (t, t + nwarps, ...) and issues their
    // loads side by side, so the dependent chains (m_j, then the row record)
    // of the kU tiles overlap; the tiles of the next round have their first
    // column, start bits and row indices loaded (prefetched) meanwhile.
    constexpr int kU = kWide ? 4 : 1;
    // a batched solve walks the list of the running matrices' tiles (built
    // after every pass); a single solve walks every tile
    const int64_t steps = kBatch ? (int64_t)*W->bw.tlist_n : (int64_t)ntiles;
    const int32_t *__restrict__ tlist = W->bw.tlist;
    int64_t t = s_go ? (gtid() >> 5) : steps;
    int32_t pf_c0[kU], pf_i[kU], pf_t[kU];
    uint32_t pf_mask[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const int64_t xu = t + u * nwarps;
        pf_c0[u] = 0;
        pf_i[u] = 0;
        pf_mask[u] = 1u;
        pf_t[u] = 0;
        if (xu < steps) {
            const int64_t tu = kBatch ? (int64_t)__ldg(tlist + xu) : xu;
            if (kBatch)
                pf_t[u] = (int32_t)tu;
            pf_c0[u] = __ldg(tile_col + tu);
            pf_mask[u] = __ldg(starts + tu);
            const int32_t pp = (int32_t)(tu * kTile) + lane;
            pf_i[u] = pp < nnz ? __ldcs(rowidx + pp) : 0;
        }
    }
    for (;;) {
        const bool more = t < steps;
        if (more) {
            int32_t c0[kU], iv[kU], jv[kU], mjv[kU], pv[kU];
            uint32_t mask[kU];
            bool valid[kU], mixed[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t xu = t + u * nwarps;
                const int64_t tu = kBatch ? (int64_t)pf_t[u] : xu;
                pv[u] = (int32_t)(tu * kTile) + lane;
                valid[u] = xu < steps && pv[u] < nnz;
                mixed[u] = false;
                c0[u] = pf_c0[u];
                mask[u] = pf_mask[u];
                iv[u] = pf_i[u];
                if (kBatch && xu < steps) {
                    const int32_t tm = __ldg(tilemat + tu);
                    if (tm & kTileSingle) {
                        if (__ldg(mdone + (tm & ~kTileSingle)))
                            valid[u] = false;
                    } else {
                        mixed[u] = true;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t xn = t + (kU + u) * nwarps;
                if (xn < steps) {
                    const int64_t tn = kBatch ? (int64_t)__ldg(tlist + xn) : xn;
                    if (kBatch)
                        pf_t[u] = (int32_t)tn;
                    pf_c0[u] = __ldg(tile_col + tn);
                    pf_mask[u] = __ldg(starts + tn);
                    const int32_t pn = (int32_t)(tn * kTile) + lane;
                    pf_i[u] = pn < nnz ? __ldcs(rowidx + pn) : 0;
                }
            }
            if (kBatch) {
                // every tile of the round belongs to finished matrices: on
                // to the next round (its loads are already in flight)
                bool any = false;
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    any |= valid[u];
                if (!__any_sync(FULL_MASK, any)) {
                    t += kU * nwarps;
                    continue;
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                iv[u] = valid[u] ? iv[u] : 0;
                jv[u] = valid[u] ? lane_column(c0[u], mask[u], lane) : -1 - lane;
                if (valid[u] && !(AWPM_IN(ctl, jv[u], W->n) && AWPM_IN(ctl, iv[u], W->n))) {
                    valid[u] = false;
                    jv[u] = -1 - lane;
                }
                mjv[u] = valid[u] ? ld_i32_last(mc + jv[u], pol) : 0x7fffffff;
            }
            unsigned long long sig[kU], mark[kU];
            int32_t cs[kU];  // row marking: first position of column m_i
            bool cand[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (kBatch && mixed[u] && valid[u] && __ldg(mdone + __ldg(colmat + jv[u])))
                    mjv[u] = 0x7fffffff;  // finished matrix: no candidate
                cand[u] = valid[u] && iv[u] > mjv[u];
                sig[u] = 0ull;
                mark[u] = 0ull;
                cs[u] = 0;
                if (cand[u]) {
                    ++n_cand;
                    sig[u] = ld_u64_last(rsig + iv[u], pol);
                    if (kLookup == AWPM_LOOKUP_ROWMARK) {
                        cs[u] = __ldg(&rrange[iv[u]].s);
                        mark[u] = __ldg(rowsig + mjv[u]);  // the mark of row m_j
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                // row m_j in column m_i's signature; with row marking also
                // column m_i (first position rg.x) marked by row m_j
                const bool pass = cand[u] && sig_has(sig[u], mjv[u]) &&
                                  (kLookup != AWPM_LOOKUP_ROWMARK || sig_has(mark[u], cs[u]));
                const unsigned need = __ballot_sync(FULL_MASK, pass);
                if (pass) {
                    const int x = (qhead + qn + __popc(need & lanes_below)) & (kQueue - 1);
                    qu.im[x] = make_int2(iv[u], mjv[u]);
                    qu.jp[x] = make_int2(jv[u], pv[u]);
                }
                qn += __popc(need);
                if (qn >= 32)
                    flush(32);
            }
            t += kU * nwarps;
        }
        if (!more && qn > 0)
            flush(qn);
        if (!more)
            break;
    }
    block_add_u64((unsigned long long)n_cand, &ctl->candidates);
    block_add_u64((unsigned long long)n_found, &ctl->found);
    block_add_u64((unsigned long long)n_pos, &ctl->positive);
}

// Pipelined form of the single-problem search (the same work and results as
// k_search<kLookup, false, ...>).  A warp's tiles are taken kU at a time
// (tiles t, t + nwarps, ...), and each round advances four stages at once,
// each on loads issued one round earlier: the signature test of one round,
// the candidate test (i > m_j) and signature loads of the next, the lanes'
// columns and the loads of m_j of the one after, the tile loads (first
// column, start bits, row indices) of the one after that.  So the two
// dependent gathers of a nonzero (m_j, then the signature of its row's
// column) are each hidden behind a round of other work.  Three slot sets
// carry a round's tiles through the stages; the loop body is written out
// three times with the slots' roles rotated, so no value is copied from one
// stage's registers to the next.  Tile loads take the tile index clamped to
// ntiles (always in bounds) and a lane is valid exactly when its position is
// below nnz; a lane's request goes to its queue slot, or to a discard slot
// of its own when it does not pass, so the stores need no branch.  All tile
// arithmetic is 32-bit (ntiles < 2^26).
#ifndef AWPM_PIPE_U_WIDE
#define AWPM_PIPE_U_WIDE 2
#endif
#ifndef AWPM_PIPE_U_NARROW
#define AWPM_PIPE_U_NARROW 1
#endif
#ifndef AWPM_PIPE_WARPS_WIDE
#define AWPM_PIPE_WARPS_WIDE 32
#endif
#ifndef AWPM_PIPE_WARPS_NARROW
#define AWPM_PIPE_WARPS_NARROW 40
#endif
template <bool kWide>
struct PipeCfg {
    static constexpr int kU = kWide ? AWPM_PIPE_U_WIDE : AWPM_PIPE_U_NARROW;
    // resident warps per SM aimed at (the launch bound divides by the block's warps)
    static constexpr int kWarpsPerSM = kWide ? AWPM_PIPE_WARPS_WIDE : AWPM_PIPE_WARPS_NARROW;
};

// The lookup queue with a discard slot per lane after the 64 ring slots.
constexpr int kQueueDiscard = kQueue + 32;
struct LookupQueueD {
    int2 im[kQueueDiscard];
    int2 jp[kQueueDiscard];
};

template <int kLookup, bool kWide, bool kBatch>
__global__ void __launch_bounds__(SearchBlock<kBatch>::kThreads,
                                  PipeCfg<kWide>::kWarpsPerSM / SearchBlock<kBatch>::kWarps)
    k_search_pipe(const Work *__restrict__ W)
{
    constexpr int kU = PipeCfg<kWide>::kU;
    __shared__ int s_go;
    __shared__ LookupQueueD s_queue[SearchBlock<kBatch>::kWarps];
    if (threadIdx.x == 0)
        s_go = gate(W->ctl) ? 1 : 0;
    __syncthreads();
    const int32_t nnz = W->nnz;
    const int32_t ntiles = W->ntiles;
    const int32_t *__restrict__ rowidx = W->rowidx;
    const double *__restrict__ wv = W->w;
    const int32_t *__restrict__ tile_col = W->tile_col;
    const uint32_t *__restrict__ starts = W->starts;
    const int32_t *__restrict__ mc = W->mc;
    const double *__restrict__ wm = W->wm;
    const unsigned long long *__restrict__ rsig = W->rsig;
    const RowRange *__restrict__ rrange = W->rrange;
    const unsigned long long *__restrict__ htab = W->htab;
    const uint32_t *__restrict__ bloom = W->bloom;
    const unsigned long long *__restrict__ rowsig = W->rowsig;
    const int32_t *__restrict__ trowptr = W->trowptr;
    const int32_t *__restrict__ tpos = W->tpos;
    Rec *__restrict__ best = W->best;
    uint32_t *winbits = W->winbits;
    Ctl *ctl = W->ctl;
    LookupQueueD &qd = s_queue[threadIdx.x >> 5];
    // a batched solve walks the list of the running matrices' tiles
    const int32_t steps = kBatch ? *W->bw.tlist_n : ntiles;
    const int32_t *__restrict__ tlist = W->bw.tlist;
    const int32_t *__restrict__ tilemat = W->bw.tilemat;
    const int32_t *__restrict__ colmat = W->bw.colmat;
    const int32_t *__restrict__ mdone = W->bw.mdone;

    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const int32_t nwarps = (int32_t)(gstride() >> 5);
    const int32_t stride = kU * nwarps;
    const unsigned long long pol = policy_evict_last();
    uint32_t n_cand = 0, n_found = 0, n_pos = 0;
    int qhead = 0, qn = 0;  // the warp's queue (warp-uniform)

    auto flush = [&](int k) {
        __syncwarp();
        resolve_lookups<kLookup>(qd, qhead, k, lane, rowidx, wv, wm, htab, bloom, trowptr,
                                 tpos, rrange, nnz, W->n, best, winbits, ctl, n_found, n_pos);
        __syncwarp();
        qhead = (qhead + k) & (kQueue - 1);
        qn -= k;
    };

    // slot set s, tile u: row i, column (the tile's first column before the
    // column step), start bits then m_j, the signature, the candidate flag
    int32_t si[3][kU], sj[3][kU], sx[3][kU];
    int32_t stile[3][kU];  // batched solve: the tile of the walk's entry
    unsigned long long ssig[3][kU], smark[3][kU];
    int32_t scs[3][kU];
    bool scand[3][kU];

    // stage 1: tile loads of the round starting at tile tr into slot s
    auto st_load = [&](int s, int32_t tr) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t xu = tr + u * nwarps;
            const int32_t tu = kBatch ? (xu < steps ? __ldg(tlist + xu) : ntiles) : xu;
            if (kBatch)
                stile[s][u] = tu;
            const int32_t tl = tu < ntiles ? tu : ntiles;  // in bounds
            sj[s][u] = __ldg(tile_col + tl);
            sx[s][u] = (int32_t)__ldg(starts + tl);
            const int32_t p = tu * kTile + lane;
            si[s][u] = p < nnz ? __ldcs(rowidx + p) : 0;
        }
    };
    // stage 2: columns, and the loads of m_j
    auto st_cols = [&](int s, int32_t tr) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t tu = kBatch ? stile[s][u] : tr + u * nwarps;
            const int32_t p = tu * kTile + lane;
            bool valid = p < nnz;
            const int32_t j = lane_column(sj[s][u], (uint32_t)sx[s][u], lane);
            if (kBatch && valid) {
                // lanes of finished matrices take no part
                const int32_t tm = __ldg(tilemat + tu);
                valid = (tm & kTileSingle) ? !__ldg(mdone + (tm & ~kTileSingle))
                                           : !__ldg(mdone + __ldg(colmat + j));
            }
            const bool ok = valid && AWPM_IN(ctl, j, W->n) && AWPM_IN(ctl, si[s][u], W->n);
            sj[s][u] = ok ? j : -1;
            sx[s][u] = ok ? ld_i32_last(mc + j, pol) : 0x7fffffff;
        }
    };
    // stage 3: candidate test, and the signature loads
    auto st_cand = [&](int s) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            bool c = sj[s][u] >= 0 && si[s][u] > sx[s][u];
            if (c && !AWPM_IN(ctl, sx[s][u], W->n))
                c = false;
            scand[s][u] = c;
            ssig[s][u] = 0ull;
            if (c) {
                ++n_cand;
                ssig[s][u] = ld_u64_last(rsig + si[s][u], pol);
                if (kLookup == AWPM_LOOKUP_ROWMARK) {
                    scs[s][u] = __ldg(&rrange[si[s][u]].s);
                    smark[s][u] = __ldg(rowsig + sx[s][u]);
                }
            }
        }
    };
    // stage 4: signature test, passing requests queued
    auto st_test = [&](int s, int32_t tr) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const bool pass = scand[s][u] && sig_has(ssig[s][u], sx[s][u]) &&
                              (kLookup != AWPM_LOOKUP_ROWMARK ||
                               sig_has(smark[s][u], scs[s][u]));
            const unsigned need = __ballot_sync(FULL_MASK, pass);
            const int x = pass ? ((qhead + qn + __popc(need & lanes_below)) & (kQueue - 1))
                               : kQueue + lane;
            qd.im[x] = make_int2(si[s][u], sx[s][u]);
            qd.jp[x] = make_int2(sj[s][u], (kBatch ? stile[s][u] : tr + u * nwarps) * kTile + lane);
            qn += __popc(need);
            if (qn >= 32)
                flush(32);
        }
    };

    const int32_t t0 = s_go ? (int32_t)(gtid() >> 5) : steps;
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            scand[s][u] = false;
            ssig[s][u] = smark[s][u] = 0ull;
            scs[s][u] = 0;
        }
    // prologue: round t0 through stage 3, round t0 + stride through stage 2,
    // round t0 + 2 stride through stage 1
    st_load(0, t0);
    st_cols(0, t0);
    st_load(1, t0 + stride);
    st_cand(0);
    st_cols(1, t0 + stride);
    st_load(2, t0 + 2 * stride);
    // steady state: each step tests round tr, requests round tr + stride's
    // signatures, makes round tr + 2 stride's columns, loads round tr + 3 stride
#define AWPM_ROT_STEP(A, B, C)                                                      \
    {                                                                               \
        if (tr >= steps)                                                            \
            break;                                                                  \
        st_test(A, tr);                                                             \
        st_cand(B);                                                                 \
        st_cols(C, tr + 2 * stride);                                                \
        st_load(A, tr + 3 * stride);                                                \
        tr += stride;                                                               \
    }
    for (int32_t tr = t0;;) {
        AWPM_ROT_STEP(0, 1, 2)
        AWPM_ROT_STEP(1, 2, 0)
        AWPM_ROT_STEP(2, 0, 1)
    }
#undef AWPM_ROT_STEP
    if (qn > 0)
        flush(qn);
    block_add_u64((unsigned long long)n_cand, &ctl->candidates);
    block_add_u64((unsigned long long)n_found, &ctl->found);
    block_add_u64((unsigned long long)n_pos, &ctl->positive);
}

// ---------------------------------------------------------------------------
// Step D (Algorithm 6): conflicts, per-key selection, flip
// ---------------------------------------------------------------------------

// The winners (set bits) of the bitmap words [x0, x0 + 32), 32 at a time
// with every lane busy: the words' bit counts are scanned across the warp,
// and in each round lane l takes the winner of rank round * 32 + l (found by
// a binary search over the scan and the word's rank-th set bit).  Calls
// f(j) on every lane each round, j = -1 for lanes past the last winner.
// Called by the whole warp; `clear` zeroes the words as they are read.
template <typename F>
__device__ __forceinline__ void for_winners(uint32_t *winbits, int64_t x0, int64_t words, int lane,
                                            bool clear, F f)
{
    const uint32_t mine = x0 + lane < words ? winbits[x0 + lane] : 0u;
    if (clear && mine)
        winbits[x0 + lane] = 0u;
    const int cnt = __popc(mine);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(FULL_MASK, incl, 31);
    for (int base = 0; base < total; base += 32) {
        const int want = base + lane;
        // the last word whose first rank is <= want
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(FULL_MASK, excl, src + step);
            if (e <= want)
                src += step;
        }
        const int first = __shfl_sync(FULL_MASK, excl, src);
        const uint32_t word = __shfl_sync(FULL_MASK, mine, src);
        int32_t j = -1;
        if (want < total) {
            const int bit = (int)__fns(word, 0u, want - first + 1);
            j = (int32_t)((x0 + src) * 32 + bit);
        }
        f(j);
    }
}

// For every Step-C winner rooted at j (a set bit of the winner bitmap) with
// second matched edge at column k = m_i: drop it if column k is itself the
// root of a Step-C winner, otherwise compete for key k (maximum gain, then
// lowest root j).  The winner's key (or -1) is kept for the flip.  A warp
// takes 32 bitmap words at a time and their winners 32 at a time, a lane
// per winner.
__global__ void k_select(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t words = (int64_t)w.n / 32 + 1;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t x0 = (gtid() >> 5) * 32; x0 < words; x0 += nwarps * 32) {
        for_winners(w.winbits, x0, words, lane, false, [&](int32_t j) {
            if (j < 0 || !AWPM_IN(w.ctl, j, w.n))
                return;
            const Rec r = w.best[j];
            if (!AWPM_IN(w.ctl, r.p, w.nnz))
                return;
            const int32_t i = __ldg(w.rowidx + r.p);
            if (!AWPM_IN(w.ctl, i, w.n))
                return;
            const int32_t k = w.mr[i];
            if (!AWPM_IN(w.ctl, k, w.n))
                return;
            if ((w.winbits[k >> 5] >> (k & 31)) & 1u) {
                w.wkey[j] = -1;
                return;
            }
            w.wkey[j] = k;
            Sel sl;
            sl.g = r.g;
            sl.j = j;
            sl.pad = 0;
            sel_combine(w.dsel + k, sl, w.ctl);
        });
    }
}

// Flip every selected cycle: column j takes row i, key column k takes m_j;
// the row records of rows i and m_j follow their new mates.  The selected
// cycles are vertex-disjoint, so each lane owns its four vertices.  The
// Step-C records and winner bits visited are cleared, which leaves them
// empty for the next pass.  Winners are taken as in k_select; in a batched
// solve the flips of a round are counted per matrix with one atomic per
// matrix.
__device__ __forceinline__ unsigned long long flip_body(const Work &w)
{
    unsigned long long flips = 0;
    if (gate(w.ctl)) {
        const int lane = threadIdx.x & 31;
        const int64_t words = (int64_t)w.n / 32 + 1;
        const int64_t nwarps = gstride() >> 5;
        for (int64_t x0 = (gtid() >> 5) * 32; x0 < words; x0 += nwarps * 32) {
            for_winners(w.winbits, x0, words, lane, true, [&](int32_t j) {
                int32_t mat = -1;  // matrix of a flipped cycle (batched solve)
                if (j >= 0 && AWPM_IN(w.ctl, j, w.n)) {
                    const Rec r = w.best[j];
                    w.best[j] = Rec{0.0, 0, 0};
                    int32_t k = w.wkey[j];
                    if (k >= 0 && !(AWPM_IN(w.ctl, k, w.n) && AWPM_IN(w.ctl, r.p, w.nnz) &&
                                    AWPM_IN(w.ctl, r.q, w.nnz)))
                        k = -1;
                    const Sel sl = k >= 0 ? w.dsel[k] : Sel{0.0, 0, 0};
                    if (k >= 0 && gbits(sl.g) > 0ll && sl.j == j) {
                        w.dsel[k] = Sel{0.0, 0, 0};
                        const int32_t i = w.rowidx[r.p];
                        const int32_t mj = w.mc[j];
                        if (AWPM_IN(w.ctl, i, w.n) && AWPM_IN(w.ctl, mj, w.n)) {
                            const double wij = w.w[r.p];
                            const double wq = w.w[r.q];
                            w.mc[j] = i;
                            w.mr[i] = j;
                            w.mc[k] = mj;
                            w.mr[mj] = k;
                            w.wm[j] = wij;
                            w.wm[k] = wq;
                            put_rowrec(w, i, w.colptr[j], w.colptr[j + 1], w.colsig[j], wij);
                            put_rowrec(w, mj, w.colptr[k], w.colptr[k + 1], w.colsig[k], wq);
                            ++flips;
                            if (w.bw.count > 0)
                                mat = w.bw.colmat[k];
                        }
                    }
                }
                // every lane reaches the warp-wide match: no early exit above
                if (w.bw.count > 0) {
                    const unsigned peers = __match_any_sync(FULL_MASK, mat);
                    if (mat >= 0 && (peers & ((1u << lane) - 1u)) == 0u)
                        atomicAdd(w.bw.mflips + mat, (unsigned long long)__popc(peers));
                }
            });
        }
    }
    return flips;
}

__global__ void k_flip(const Work *__restrict__ W)
{
    const Work &w = *W;
    block_add_u64(flip_body(w), &w.ctl->pass_flips);
}

// End of a pass (Algorithm 2): count it, stop when nothing was flipped or
// the pass cap is reached.
__device__ __forceinline__ int control_step(Ctl *ctl)
{
    if (ctl->err) {
        ctl->active = 0;
        return 0;
    }
    if (!ctl->active)
        return 0;
    const unsigned long long f = ctl->pass_flips;
    ctl->pass_flips = 0;
    ctl->iterations += 1;
    ctl->cycles += f;
    if (f == 0) {
        ctl->converged = 1;
        ctl->active = 0;
    } else if (ctl->iterations >= ctl->max_passes) {
        ctl->active = 0;
    }
    return ctl->active;
}

__global__ void k_control(const Work *__restrict__ W)
{
    control_step(W->ctl);
}

__global__ void k_control_graph(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, control_step(W->ctl) ? 1u : 0u);
}

// The flip in the graph form of a single problem's pass: the block that
// finishes last (its count of finished blocks orders it after every other
// block's flip count) ends the pass and sets the WHILE condition.
__global__ void k_flip_graph(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    const Work &w = *W;
    block_add_u64(flip_body(w), &w.ctl->pass_flips);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&w.ctl->flip_done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            w.ctl->flip_done = 0u;
            cudaGraphSetConditional(h, control_step(w.ctl) ? 1u : 0u);
        }
    }
}

// End of a pass for every matrix still running: count the pass, stop the
// matrix when it flipped nothing or reached the cap; count the running ones.
__global__ void k_batch_control(const Work *__restrict__ W)
{
    const Work &w = *W;
    const BatchWork &bw = w.bw;
    const bool go = !w.ctl->err && w.ctl->active;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < bw.count;
         b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        int still = 0;
        if (go && b < bw.count && !bw.mdone[b]) {
            const unsigned long long f = bw.mflips[b];
            bw.mflips[b] = 0;
            bw.miter[b] += 1;
            bw.mcycles[b] += f;
            if (f == 0) {
                bw.mconv[b] = 1;
                bw.mdone[b] = 1;
            } else if (bw.miter[b] >= w.ctl->max_passes) {
                bw.mdone[b] = 1;
            } else {
                still = 1;
            }
        }
        still = __syncthreads_count(still);
        if (threadIdx.x == 0 && still)
            atomicAdd(bw.active, still);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *bw.tlist_n = 0;  // the list of the next pass is built after this
}

// Pass counter of the whole batch; another pass runs while any matrix runs.
__device__ __forceinline__ int batch_step(Ctl *ctl, int32_t *active)
{
    if (ctl->err || !ctl->active) {
        ctl->active = 0;
        return 0;
    }
    ctl->iterations += 1;
    const int32_t a = *active;
    *active = 0;
    ctl->cycles += ctl->pass_flips;
    ctl->pass_flips = 0;
    if (a == 0) {
        ctl->converged = 1;
        ctl->active = 0;
    }
    return ctl->active;
}

__global__ void k_batch_step(const Work *__restrict__ W)
{
    batch_step(W->ctl, W->bw.active);
}

__global__ void k_batch_step_graph(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, batch_step(W->ctl, W->bw.active) ? 1u : 0u);
}

__global__ void k_export_stepc(const Work *__restrict__ W, double *gain, int32_t *row)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    for (int64_t j = gtid(); j < w.n; j += gstride()) {
        const Rec r = w.best[j];
        const bool has = gbits(r.g) > 0ll;
        gain[j] = has ? r.g : 0.0;
        row[j] = has ? w.rowidx[r.p] : -1;
    }
}

// ---------------------------------------------------------------------------
// Greedy (Pettie-Sanders) selection of the Step-C winners (Section 4)
// ---------------------------------------------------------------------------
// Instead of Step D: the winners in order of gain, descending (equal gains:
// lower root column), each kept when its columns j and k = m_i -- hence also
// its rows m_j and i -- belong to no cycle kept before.  Computed in rounds:
// every column names the first undecided winner touching it (maximum gain,
// then lowest root, through the 128-bit compare-and-swap of the Step-D
// records); a winner named by both its columns is kept; undecided winners
// touching a kept cycle are dropped.  The first undecided winner is always
// named by both its columns, so every round decides at least one.  At the
// end the kept winners are handed to k_flip exactly as Step D hands them:
// the key column's record names the root, dropped winners get key -1.

__device__ __forceinline__ void warp_add_i32(int v, int32_t *dst)
{
    v = __reduce_add_sync(FULL_MASK, v);
    if ((threadIdx.x & 31) == 0 && v)
        atomicAdd(dst, v);
}

// Keys of all winners; every winner undecided; their number into Ctl::live.
__global__ void k_ps_begin(const Work *__restrict__ W)
{
    const Work &w = *W;
    int live = 0;
    if (gate(w.ctl)) {
        const int64_t words = (int64_t)w.n / 32 + 1;
        for (int64_t x = gtid(); x < words; x += gstride()) {
            uint32_t bits = w.winbits[x];
            w.pslive[x] = bits;
            live += __popc(bits);
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int32_t j = (int32_t)(x * 32 + b);
                w.wkey[j] = w.mr[w.rowidx[w.best[j].p]];
            }
        }
    }
    warp_add_i32(live, &w.ctl->live);
}

// Loop condition of the rounds: undecided winners remain (counter reset).
__global__ void k_ps_cond(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    Ctl *c = W->ctl;
    const int32_t live = c->live;
    c->live = 0;
    cudaGraphSetConditional(h, (live > 0 && c->err == 0u && c->active) ? 1u : 0u);
}

// Round, step 1: every undecided winner names itself at both its columns.
__global__ void k_ps_name(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int64_t words = (int64_t)w.n / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride()) {
        uint32_t bits = w.pslive[x];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int32_t j = (int32_t)(x * 32 + b);
            Sel s;
            s.g = w.best[j].g;
            s.j = j;
            s.pad = 0;
            sel_combine(w.psel + j, s, w.ctl);
            sel_combine(w.psel + w.wkey[j], s, w.ctl);
        }
    }
}

// Round, step 2: a winner named by both its columns is kept; its columns
// are marked used.
__global__ void k_ps_take(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int64_t words = (int64_t)w.n / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride()) {
        uint32_t bits = w.pslive[x];
        uint32_t kept = 0u;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int32_t j = (int32_t)(x * 32 + b);
            const int32_t k = w.wkey[j];
            const Sel a = w.psel[j], c = w.psel[k];
            if (gbits(a.g) > 0ll && a.j == j && gbits(c.g) > 0ll && c.j == j) {
                kept |= 1u << b;
                atomicOr(w.psused + (j >> 5), 1u << (j & 31));
                atomicOr(w.psused + (k >> 5), 1u << (k & 31));
            }
        }
        if (kept)
            w.pstaken[x] |= kept;
    }
}

// Round, step 3: clear the records this round touched; drop the undecided
// winners that touch a used column; count the undecided ones left.
__global__ void k_ps_prune(const Work *__restrict__ W)
{
    const Work &w = *W;
    int live = 0;
    if (gate(w.ctl)) {
        const int64_t words = (int64_t)w.n / 32 + 1;
        for (int64_t x = gtid(); x < words; x += gstride()) {
            uint32_t bits = w.pslive[x];
            if (!bits)
                continue;
            const uint32_t kept = w.pstaken[x];
            uint32_t still = 0u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int32_t j = (int32_t)(x * 32 + b);
                const int32_t k = w.wkey[j];
                w.psel[j] = Sel{0.0, 0, 0};
                w.psel[k] = Sel{0.0, 0, 0};
                if ((kept >> b) & 1u)
                    continue;
                const bool used = ((w.psused[j >> 5] >> (j & 31)) & 1u) ||
                                  ((w.psused[k >> 5] >> (k & 31)) & 1u);
                if (!used)
                    still |= 1u << b;
            }
            w.pslive[x] = still;
            live += __popc(still);
        }
    }
    warp_add_i32(live, &w.ctl->live);
}

// After the rounds: kept winners get their key column's record (the form
// k_flip reads), dropped ones key -1; the kept-set and used-column bitmaps
// are cleared for the next pass.
__global__ void k_ps_end(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int64_t words = (int64_t)w.n / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride()) {
        uint32_t bits = w.winbits[x];
        const uint32_t kept = w.pstaken[x];
        if (kept)
            w.pstaken[x] = 0u;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int32_t j = (int32_t)(x * 32 + b);
            const int32_t k = w.wkey[j];
            if ((kept >> b) & 1u) {
                Sel s;
                s.g = w.best[j].g;
                s.j = j;
                s.pad = 0;
                w.dsel[k] = s;
                atomicAnd(w.psused + (j >> 5), ~(1u << (j & 31)));
                atomicAnd(w.psused + (k >> 5), ~(1u << (k & 31)));
            } else {
                w.wkey[j] = -1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Heavy-weight greedy maximal matching (Section 5.1)
// ---------------------------------------------------------------------------
// The matching that greedy builds when it takes the stored entries from
// heaviest to lightest (equal weights: lower row, then lower column) and
// keeps each entry whose row and column are both free.  Computed in rounds:
// every free column names its first free entry in that order (largest
// weight, then lowest row), every free row names its first free entry
// (largest weight, then lowest column), and the entries named by both ends
// are matched.  Weights are compared through order keys: 64-bit integers
// ordered like the doubles, so the maxima and minima are plain 64-bit
// atomics.

constexpr long long kKeyNone = (long long)0x8000000000000000ull;

// Integer ordered like the weight (-0 taken as +0; finite weights only).
__device__ __forceinline__ long long order_key(double x)
{
    long long b = __double_as_longlong(x);
    if (b == kKeyNone)
        b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

// Clear the matching, the per-round records and the control block.
__global__ void k_gm_reset(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (gtid() == 0) {
        Ctl *c = w.ctl;
        c->err = 0u;
        c->active = 1;
        c->iterations = 0;
        c->converged = 0;
        c->live = 0;
        c->max_passes = w.max_passes;
        c->pass_flips = 0ull;
        c->flip_done = 0u;
        c->cycles = 0ull;
        c->candidates = 0ull;
        c->found = 0ull;
        c->positive = 0ull;
        c->weight_in = 0.0;
        c->weight_out = 0.0;
    }
    for (int64_t x = gtid(); x < w.n; x += gstride()) {
        w.mc[x] = -1;
        w.mr[x] = -1;
        w.wm[x] = 0.0;
        w.gckey[x] = kKeyNone;
        w.gcpos[x] = 0x7fffffff;
        w.grkey[x] = kKeyNone;
        w.grcol[x] = 0x7fffffff;
    }
    const int64_t words = ((int64_t)w.nnz + 31) / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride())
        w.starts[x] = 0u;
    for (int64_t x = gtid(); x < w.ntiles; x += gstride())
        w.gtdead[x] = 0;
}

// Entry checks of the greedy input: row range, sortedness, finite weights.
__global__ void __launch_bounds__(kThreads) k_gm_check(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err & kErrInvalid)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    unsigned bits = 0;
    for (int64_t t = gtid() >> 5; t < w.ntiles; t += nwarps) {
        const int32_t p = (int32_t)(t * kTile) + lane;
        const bool valid = p < w.nnz;
        const uint32_t mask = __ldg(w.starts + t);
        const int32_t r = valid ? __ldcs(w.rowidx + p) : 0;
        const int32_t up = __shfl_up_sync(FULL_MASK, r, 1);
        const int32_t before = lane == 0 ? ((valid && p > 0) ? __ldg(w.rowidx + p - 1) : 0) : up;
        if (valid) {
            if (r < 0 || r >= w.n)
                bits |= kErrInvalid;
            if ((__double2hiint(__ldcs(w.w + p)) & 0x7ff00000) == 0x7ff00000)
                bits |= kErrNonfinite;
            if (p > 0 && !((mask >> lane) & 1u) && before >= r)
                bits |= kErrUnsorted;
        }
    }
    bits = __reduce_or_sync(FULL_MASK, bits);
    if (lane == 0 && bits)
        raise_err(w.ctl, bits);
}

// Round, phase 1: the largest key among the free entries of every free
// column (warp maximum per column segment, then a 64-bit atomic) and of
// every free row (an atomic per entry, skipped when it cannot win).  A tile
// whose columns are all matched is marked dead and skipped from then on
// (columns never become free again).
__global__ void __launch_bounds__(kThreads) k_gm_max(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t t = gtid() >> 5; t < w.ntiles; t += nwarps) {
        if (w.gtdead[t])
            continue;
        const int32_t base = (int32_t)(t * kTile);
        const int32_t p = base + lane;
        const bool valid = p < w.nnz;
        const int32_t c0 = __ldg(w.tile_col + t);
        const uint32_t mask = __ldg(w.starts + t);
        const int32_t j = valid ? lane_column(c0, mask, lane) : 0;
        const bool cfree = valid && w.mc[j] < 0;
        if (!__any_sync(FULL_MASK, cfree)) {
            if (lane == 0)
                w.gtdead[t] = 1;
            continue;
        }
        const int32_t i = valid ? __ldcs(w.rowidx + p) : 0;
        const bool fr = cfree && w.mr[i] < 0;
        long long key = fr ? order_key(__ldcs(w.w + p)) : kKeyNone;
        if (fr && key > *(volatile const long long *)(w.grkey + i))
            atomicMax(w.grkey + i, key);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_down_sync(FULL_MASK, key, off);
            if (lane + off < 32 && ((mask >> (lane + 1)) & ((1u << off) - 1u)) == 0u && o > key)
                key = o;
        }
        const bool head = valid && (lane == 0 || ((mask >> lane) & 1u));
        if (head && key != kKeyNone && key > *(volatile const long long *)(w.gckey + j))
            atomicMax(w.gckey + j, key);
    }
}

// Round, phase 2: among the free entries holding the maximum key, the lowest
// position of every column (= lowest row) and the lowest column of every row.
__global__ void __launch_bounds__(kThreads) k_gm_min(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t t = gtid() >> 5; t < w.ntiles; t += nwarps) {
        if (w.gtdead[t])
            continue;
        const int32_t base = (int32_t)(t * kTile);
        const int32_t p = base + lane;
        const bool valid = p < w.nnz;
        const int32_t c0 = __ldg(w.tile_col + t);
        const uint32_t mask = __ldg(w.starts + t);
        const int32_t j = valid ? lane_column(c0, mask, lane) : 0;
        const int32_t i = valid ? __ldcs(w.rowidx + p) : 0;
        const bool fr = valid && w.mc[j] < 0 && w.mr[i] < 0;
        const long long key = fr ? order_key(__ldcs(w.w + p)) : kKeyNone;
        if (fr && key == w.grkey[i] && j < *(volatile const int32_t *)(w.grcol + i))
            atomicMin(w.grcol + i, j);
        int32_t pos = (fr && key == w.gckey[j]) ? p : 0x7fffffff;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t o = __shfl_down_sync(FULL_MASK, pos, off);
            if (lane + off < 32 && ((mask >> (lane + 1)) & ((1u << off) - 1u)) == 0u && o < pos)
                pos = o;
        }
        const bool head = valid && (lane == 0 || ((mask >> lane) & 1u));
        if (head && pos != 0x7fffffff)
            atomicMin(w.gcpos + j, pos);
    }
}

// Round, phase 3: a free column whose named entry is also named by its row
// is matched; the column's records are cleared for the next round.
__global__ void k_gm_match(const Work *__restrict__ W)
{
    const Work &w = *W;
    unsigned long long matched = 0;
    if (gate(w.ctl)) {
        for (int64_t j = gtid(); j < w.n; j += gstride()) {
            const int32_t p = w.gcpos[j];
            if (p == 0x7fffffff)
                continue;
            w.gckey[j] = kKeyNone;
            w.gcpos[j] = 0x7fffffff;
            const int32_t i = w.rowidx[p];
            if (w.grcol[i] == (int32_t)j) {
                w.mc[j] = i;
                w.mr[i] = (int32_t)j;
                w.wm[j] = w.w[p];
                ++matched;
            }
        }
    }
    block_add_u64(matched, &w.ctl->pass_flips);
}

// Round, phase 4: clear the rows' records for the next round.
__global__ void k_gm_rows(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!gate(w.ctl))
        return;
    for (int64_t i = gtid(); i < w.n; i += gstride()) {
        w.grkey[i] = kKeyNone;
        w.grcol[i] = 0x7fffffff;
    }
}

// ---------------------------------------------------------------------------
// Matching weights from matrix values (Section 6.1)
// ---------------------------------------------------------------------------
// One sweep of max-equilibration, columns first: v_ij = |a_ij| / max_k |a_kj|,
// w_ij = v_ij / max_l v_il, so every row's largest weight is exactly 1; the
// weight is w (Option A, sum objective) or log(w) (Option B, product
// objective).  Divisions and maxima are exact IEEE operations, so Option A
// is bit-for-bit reproducible; Option B calls the device logarithm.  A warp
// takes a column at a time.

__device__ __forceinline__ bool wt_gate(const Ctl *ctl)
{
    return (*(volatile const unsigned *)&ctl->err & (kErrInvalid | kErrNonfinite)) == 0u;
}

// The control block (the only state besides the weights' own arrays).
__global__ void k_wt_reset(const Work *__restrict__ W)
{
    Ctl *c = W->ctl;
    c->err = 0u;
    c->active = 1;
}

// Checks (rows in range; values finite and nonzero) and the column maxima;
// clears the row maxima.
__global__ void k_wt_colmax(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err & kErrInvalid)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t x = gtid(); x < w.n; x += gstride())
        w.wt_rmax[x] = 0ull;
    unsigned bits = 0;
    for (int64_t j = gtid() >> 5; j < w.n; j += nwarps) {
        const int32_t s = w.colptr[j], e = w.colptr[j + 1];
        double m = 0.0;
        for (int32_t p = s + lane; p < e; p += 32) {
            const int32_t r = __ldcs(w.rowidx + p);
            const double a = __ldcs(w.wt_a + p);
            if (r < 0 || r >= w.n)
                bits |= kErrInvalid;
            const long long b = __double_as_longlong(a) & 0x7fffffffffffffffll;
            if (b == 0ll || b >= 0x7ff0000000000000ll)
                bits |= kErrNonfinite;
            const double v = fabs(a);
            if (v > m)
                m = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(FULL_MASK, m, o);
            if (y > m)
                m = y;
        }
        if (lane == 0)
            w.wt_cmax[j] = m;
    }
    bits = __reduce_or_sync(FULL_MASK, bits);
    if (lane == 0 && bits)
        raise_err(w.ctl, bits);
}

// Row maxima of the column-scaled magnitudes (positive doubles compare like
// their bit patterns as unsigned integers).
__global__ void k_wt_rowmax(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!wt_gate(w.ctl))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t j = gtid() >> 5; j < w.n; j += nwarps) {
        const int32_t s = w.colptr[j], e = w.colptr[j + 1];
        const double cm = w.wt_cmax[j];
        for (int32_t p = s + lane; p < e; p += 32) {
            const double v = fabs(w.wt_a[p]) / cm;
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            const int32_t r = w.rowidx[p];
            if (b > *(volatile const unsigned long long *)(w.wt_rmax + r))
                atomicMax(w.wt_rmax + r, b);
        }
    }
}

// The weights.
__global__ void k_wt_out(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (!wt_gate(w.ctl))
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t j = gtid() >> 5; j < w.n; j += nwarps) {
        const int32_t s = w.colptr[j], e = w.colptr[j + 1];
        const double cm = w.wt_cmax[j];
        for (int32_t p = s + lane; p < e; p += 32) {
            const double v = fabs(w.wt_a[p]) / cm;
            const double rm = __longlong_as_double((long long)w.wt_rmax[w.rowidx[p]]);
            const double x = v / rm;
            w.wt_out[p] = w.wt_mode ? log(x) : x;
        }
    }
}

// ---------------------------------------------------------------------------
// Maximum cardinality matching with the heavy-weight tie-break (Section 5.2)
// ---------------------------------------------------------------------------
// Phases of breadth-first augmenting-path searches from every free column.
// Per level, every frontier column offers its rows not reached yet (through
// unmatched edges); a row goes to the offer with the heaviest edge, then the
// lowest column (order key and column in one 128-bit record).  A free row so reached ends a path of its tree (the tree keeps
// the heaviest last edge, then the lowest row, and stops growing); a
// matched row brings its matched column into the next frontier.  The trees
// are vertex-disjoint, so all paths found in a phase are augmented at once.
// A phase that augments nothing ends the search: the matching is maximum.
// The levels and phases are driven from the host through Ctl::live and
// Ctl::pass_flips.

// Clear the per-solve state; mr = -1; every row unreached, its offer record
// empty.
__global__ void k_mc_reset(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (gtid() == 0) {
        Ctl *c = w.ctl;
        c->err = 0u;
        c->active = 1;
        c->iterations = 0;
        c->converged = 0;
        c->live = 0;
        c->levels = 0ull;
        c->pass_flips = 0ull;
        c->cycles = 0ull;
        c->level_tiles = 0;
        c->level_listed = 0;
        c->level_done = 0u;
        c->touched = 0;
    }
    for (int64_t x = gtid(); x < w.n; x += gstride()) {
        w.mr[x] = -1;
        w.mrpar[x] = -1;
        w.mroff[x] = Off{kKeyNone, 0x7fffffff, 0};
    }
    const int64_t words = ((int64_t)w.nnz + 31) / 32 + 1;
    for (int64_t x = gtid(); x < words; x += gstride())
        w.starts[x] = 0u;
}

// A column without entries is no error for the maximum matching (it stays
// unmatched): drop that report of the column-pointer check.
__global__ void k_mc_allow_empty(const Work *__restrict__ W)
{
    Ctl *c = W->ctl;
    c->nonempty = (c->err & kErrNotPerfect) ? 0 : 1;
    atomicAnd(&c->err, ~kErrNotPerfect);
}

// The starting matching: row of every column or -1, each row once, every
// pair a stored entry (binary search in the sorted column); its size.
__global__ void k_mc_load(const Work *__restrict__ W)
{
    const Work &w = *W;
    unsigned long long have = 0;
    if (!w.ctl->err) {
        for (int64_t j = gtid(); j < w.n; j += gstride()) {
            const int32_t r = w.mmate[j];
            w.mc[j] = r < 0 ? -1 : r;
            if (r < 0)
                continue;
            if (r >= w.n || atomicCAS(&w.mr[r], -1, (int32_t)j) != -1) {
                raise_err(w.ctl, kErrNotPerfect);
                continue;
            }
            int32_t lo = w.colptr[j], len = w.colptr[j + 1] - lo;
            while (len > 0) {
                const int32_t half = len >> 1;
                if (w.rowidx[lo + half] < r) {
                    lo += half + 1;
                    len -= half + 1;
                } else {
                    len = half;
                }
            }
            if (lo >= w.colptr[j + 1] || w.rowidx[lo] != r)
                raise_err(w.ctl, kErrNotPerfect);
            ++have;
        }
    }
    block_add_u64(have, &w.ctl->cycles);
}

// The list of 32-entry tiles holding an entry of a frontier column, built
// where the frontier is made (the phase start and the end of each level):
// every frontier column appends the tiles its entries span, one atomic per
// warp.  A tile shared by two frontier columns is listed twice: the level
// steps take the same decisions however often, and in whatever order, a
// tile comes (maxima, minima and writes of equal values), so the list needs
// neither order nor uniqueness.  It holds at most min(nnz, nnz/32 + 2n)
// entries (a column spans at most len/32 + 2 tiles, and at most len); an
// append past the capacity is refused with an internal error.  Called by a
// whole warp, lane l holding the frontier bits `front` of bitmap word x.
__device__ __forceinline__ void mc_list_tiles(const Work &w, int64_t x, uint32_t front, int lane)
{
    int32_t mine = 0;
    for (uint32_t bits = front; bits; bits &= bits - 1) {
        const int64_t c = x * 32 + __ffs(bits) - 1;
        const int32_t s = __ldg(w.colptr + c), e = __ldg(w.colptr + c + 1);
        if (e > s)
            mine += ((e - 1) >> 5) - (s >> 5) + 1;
    }
    int32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    const int32_t total = __shfl_sync(FULL_MASK, incl, 31);
    if (total == 0)
        return;
    int32_t base = 0;
    if (lane == 0)
        base = atomicAdd(&w.ctl->level_tiles, total);
    base = __shfl_sync(FULL_MASK, base, 0);
    if ((int64_t)base + total > w.mtiles_cap) {
        if (lane == 0)
            raise_err(w.ctl, kErrInternal);
        return;
    }
    int32_t at = base + incl - mine;
    for (uint32_t bits = front; bits; bits &= bits - 1) {
        const int64_t c = x * 32 + __ffs(bits) - 1;
        const int32_t s = __ldg(w.colptr + c), e = __ldg(w.colptr + c + 1);
        if (e > s)
            for (int32_t t = s >> 5; t <= ((e - 1) >> 5); ++t)
                w.mtiles[at++] = t;
    }
}

// A phase: every free column roots a tree (its end record cleared) and forms
// the frontier; rows unreached, offers cleared.  Only the rows the previous
// phase reached need clearing: a row's offer record fills only at the level
// that reaches it (its parent is set at that level's join), and the reset
// cleared every row before the first phase.  End records are read only for
// the roots of the running phase.
__global__ void k_mc_phase(const Work *__restrict__ W)
{
    const Work &w = *W;
    int live = 0;
    if (!w.ctl->err) {
        for (int64_t x = gtid(); x < w.n; x += gstride()) {
            if (w.mrpar[x] != -1) {
                w.mrpar[x] = -1;
                w.mroff[x] = Off{kKeyNone, 0x7fffffff, 0};
            }
            if (w.mc[x] < 0) {
                w.mroot[x] = (int32_t)x;
                w.mtend[x] = Off{kKeyNone, 0x7fffffff, 0};
            }
        }
        // the frontier and its tile list (the list's count is zero here:
        // the reset, or the last level of the previous phase, which kept no
        // column)
        const int lane = threadIdx.x & 31;
        const int64_t words = (int64_t)w.n / 32 + 1;
        for (int64_t x0 = gtid() - lane; x0 < words; x0 += gstride()) {
            const int64_t x = x0 + lane;
            uint32_t bits = 0u;
            if (x < words) {
                for (int b = 0; b < 32; ++b) {
                    const int64_t j = x * 32 + b;
                    if (j < w.n && w.mc[j] < 0)
                        bits |= 1u << b;
                }
                w.mfront[x] = bits;
                w.mnext[x] = 0u;
                live += __popc(bits);
            }
            mc_list_tiles(w, x, bits, lane);
        }
    }
    if (gtid() == 0) {
        w.ctl->phase_levels = 0;
        w.ctl->touched = 0;
    }
    warp_add_i32(live, &w.ctl->live);
}

// Level steps 1-4 run over the listed tiles (one warp per tile): a column of
// any length, a hub included, is spread over many warps, and the work of a
// level follows the size of its frontier.  The column of an entry comes from
// the tile's first column and start bits when no column is empty, else from
// the colof array.
#define MC_TILE_LOOP_BEGIN(COUNT)                                                   \
    const int lane = threadIdx.x & 31;                                              \
    const int64_t nwarps = gstride() >> 5;                                          \
    const bool exact = w.ctl->nonempty != 0;                                        \
    const int64_t listed = (COUNT);                                                 \
    for (int64_t x = gtid() >> 5; x < listed; x += nwarps) {                        \
        const int64_t t = w.mtiles[x];                                              \
        const int32_t p = (int32_t)(t * kTile) + lane;                              \
        const bool valid = p < w.nnz;                                               \
        const int32_t c = !valid ? 0                                                \
                          : exact ? lane_column(__ldg(w.tile_col + t), __ldg(w.starts + t), lane) \
                                  : __ldg(w.mcolof + p);                            \
        const bool inf = valid && ((w.mfront[c >> 5] >> (c & 31)) & 1u);           \
        if (!__any_sync(FULL_MASK, inf))                                            \
            continue;                                                               \
        if (!inf)                                                                   \
            continue;                                                               \
        const int32_t r = w.rowidx[p];
#define MC_TILE_LOOP_END }

// (key, who) beats the record cur: heavier key, then lower index.
__device__ __forceinline__ bool off_better(long long key, int32_t who, const Off &cur)
{
    return key > cur.key || (key == cur.key && who < cur.who);
}

// Fold (key, who) into the record at addr (128-bit compare-and-swap; a
// failed exchange means another thread stored a better record, so the loop
// is short; its bound only turns a broken invariant into an error bit).  The
// first read goes to L2, where the other threads' exchanges land, so fewer
// exchanges start from a stale copy.
__device__ bool off_combine(Off *addr, long long key, int32_t who, Ctl *ctl)
{
    const int4 v = __ldcg(reinterpret_cast<const int4 *>(addr));
    Off cur;
    cur.key = (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
    cur.who = v.z;
    cur.pad = v.w;
    Off mine{key, who, 0};
    for (int k = 0; k < kCasRetryCap; ++k) {
        if (!off_better(key, who, cur))
            return false;
        const Off old = atomicCAS(addr, cur, mine);
        if (old.key == cur.key && old.who == cur.who && old.pad == cur.pad)
            return old.who == 0x7fffffff;  // this exchange replaced the empty record
        cur = old;
    }
    raise_err(ctl, kErrTimeout);
    return false;
}

// Level, step 1: per unreached row the best offer of the level: the
// heaviest edge from a frontier column, then the lowest column.
__global__ void k_mc_offer(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    // (the loop of the other level steps, written out: every lane stays to
    // the warp-wide append of the rows it lists)
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    const bool exact = w.ctl->nonempty != 0;
    const int64_t listed = w.ctl->level_tiles;
    for (int64_t x = gtid() >> 5; x < listed; x += nwarps) {
        const int64_t t = w.mtiles[x];
        const int32_t p = (int32_t)(t * kTile) + lane;
        const bool valid = p < w.nnz;
        const int32_t c = !valid ? 0
                          : exact ? lane_column(__ldg(w.tile_col + t), __ldg(w.starts + t), lane)
                                  : __ldg(w.mcolof + p);
        const bool inf = valid && ((w.mfront[c >> 5] >> (c & 31)) & 1u);
        if (!__any_sync(FULL_MASK, inf))
            continue;
        bool first = false;
        int32_t r = -1;
        if (inf) {
            r = w.rowidx[p];
            // the exchange that fills a row's empty record lists the row, once
            if (r != w.mc[c] && w.mrpar[r] == -1)
                first = off_combine(w.mroff + r, order_key(w.w[p]), c, w.ctl);
        }
        const unsigned m = __ballot_sync(FULL_MASK, first);
        if (m) {
            int32_t base = 0;
            if (lane == 0)
                base = atomicAdd(&w.ctl->touched, __popc(m));
            base = __shfl_sync(FULL_MASK, base, 0);
            if (first)
                w.mtouch[base + __popc(m & ((1u << lane) - 1u))] = r;
        }
    }
}

// Level, step 2: every row offered something at this level (listed by
// k_mc_offer) joins the tree of its best offer's column.  A free row is a
// candidate end of the tree: the tree keeps the heaviest last edge, then the
// lowest row.  A matched row brings its column into the next frontier.
__global__ void k_mc_join(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    // the next level's tile list starts empty (filled by k_mc_advance)
    if (gtid() == 0)
        w.ctl->level_tiles = 0;
    const int32_t touched = w.ctl->touched;
    for (int64_t x = gtid(); x < touched; x += gstride()) {
        const int32_t r = w.mtouch[x];
        const Off o = w.mroff[r];
        const int32_t c = o.who;
        w.mrpar[r] = c;
        const int32_t t_root = w.mroot[c];
        const int32_t c2 = w.mr[r];
        if (c2 < 0) {
            off_combine(w.mtend + t_root, o.key, r, w.ctl);
        } else {
            w.mroot[c2] = t_root;
            atomicOr(w.mnext + (c2 >> 5), 1u << (c2 & 31));
        }
    }
}

#undef MC_TILE_LOOP_BEGIN
#undef MC_TILE_LOOP_END

// Column of every entry (a warp per column), for the level kernels.
__global__ void k_mc_colof(const Work *__restrict__ W)
{
    const Work &w = *W;
    if ((w.ctl->err & kErrInvalid) || w.ctl->nonempty)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = gstride() >> 5;
    for (int64_t j = gtid() >> 5; j < w.n; j += nwarps)
        for (int32_t p = w.colptr[j] + lane; p < w.colptr[j + 1]; p += 32)
            w.mcolof[p] = (int32_t)j;
}

// Level, step 3: the next frontier without the trees that have an end; its
// size into Ctl::live.
__device__ __forceinline__ void mc_advance(const Work &w)
{
    // the next level's offered rows start empty
    if (gtid() == 0)
        w.ctl->touched = 0;
    int live = 0;
    if (!w.ctl->err) {
        // the next frontier and its tile list (the list's count was zeroed
        // by k_mc_join of this level)
        const int lane = threadIdx.x & 31;
        const int64_t words = (int64_t)w.n / 32 + 1;
        for (int64_t x0 = gtid() - lane; x0 < words; x0 += gstride()) {
            const int64_t x = x0 + lane;
            uint32_t keep = 0u;
            if (x < words) {
                uint32_t bits = w.mnext[x];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int32_t c = (int32_t)(x * 32 + b);
                    if (w.mtend[w.mroot[c]].key == kKeyNone)
                        keep |= 1u << b;
                }
                w.mfront[x] = keep;
                w.mnext[x] = 0u;
                live += __popc(keep);
            }
            mc_list_tiles(w, x, keep, lane);
        }
    }
    warp_add_i32(live, &w.ctl->live);
}

__global__ void k_mc_advance(const Work *__restrict__ W)
{
    mc_advance(*W);
}

// The level loop's condition from the live count: count the level, cap the
// levels of a phase (every level adds a row to the search forest, so n + 1
// levels mean a broken invariant), continue while a frontier is left.
__device__ __forceinline__ void mc_level_condition(const Work &w, cudaGraphConditionalHandle h)
{
    Ctl *c = w.ctl;
    const int32_t live = atomicExch(&c->live, 0);
    if (live > 0) {
        c->levels += 1;
        if (++c->phase_levels > w.n + 1)
            raise_err(c, kErrTimeout);
    }
    cudaGraphSetConditional(h, (live > 0 && *(volatile unsigned *)&c->err == 0u) ? 1u : 0u);
}

// Graph form of step 3: the block that finishes last also sets the level
// loop's condition (its count of finished blocks orders it after every
// other block's frontier count).
__global__ void k_mc_advance_graph(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    const Work &w = *W;
    mc_advance(w);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&w.ctl->level_done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            w.ctl->level_done = 0u;
            mc_level_condition(w, h);
        }
    }
}

// Graph form of the level loop's condition before a phase's first level.
__global__ void k_mc_cond_level(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    mc_level_condition(*W, h);
}

// Graph form of the end of a phase: count it and the paths it augmented;
// continue while it augmented something.
__global__ void k_mc_cond_phase(const Work *__restrict__ W, cudaGraphConditionalHandle h)
{
    Ctl *c = W->ctl;
    const unsigned long long aug = c->pass_flips;
    c->pass_flips = 0ull;
    c->cycles += aug;
    c->iterations += 1;
    const bool go = aug > 0 && c->err == 0u && c->iterations <= W->n;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Every tree with an end flips its path; their number into Ctl::pass_flips.
__global__ void k_mc_augment(const Work *__restrict__ W)
{
    const Work &w = *W;
    unsigned long long aug = 0;
    if (!w.ctl->err) {
        for (int64_t t = gtid(); t < w.n; t += gstride()) {
            if (w.mc[t] >= 0 || w.mtend[t].who == 0x7fffffff)
                continue;
            int32_t r = w.mtend[t].who;
            for (int32_t guard = 0; guard <= w.n; ++guard) {
                const int32_t c = w.mrpar[r];
                if (c < 0) {  // a broken tree: report instead of walking on
                    raise_err(w.ctl, kErrInternal);
                    break;
                }
                const int32_t old = w.mc[c];
                w.mc[c] = r;
                w.mr[r] = c;
                if (old < 0)
                    break;
                r = old;
            }
            ++aug;
        }
    }
    block_add_u64(aug, &w.ctl->pass_flips);
}

// The result back into the caller's matching array.
__global__ void k_mc_store(const Work *__restrict__ W)
{
    const Work &w = *W;
    if (w.ctl->err)
        return;
    for (int64_t j = gtid(); j < w.n; j += gstride())
        w.mmate[j] = w.mc[j];
}

// ---------------------------------------------------------------------------
// launchers: fixed grids (a multiple of the SM count)
// ---------------------------------------------------------------------------

static inline unsigned util_grid(const Shape &sh)
{
    return (unsigned)(sh.num_sms * 4);
}

static inline unsigned tile_grid(const Shape &sh)
{
    return (unsigned)(sh.num_sms * 8);
}

// The one-off initialisation kernels are chains of dependent loads per
// column (or per tile); wider grids keep more of them in flight.
static inline unsigned init_grid(const Shape &sh)
{
    return (unsigned)(sh.num_sms * 16);
}

static inline unsigned init_tile_grid(const Shape &sh)
{
    return (unsigned)(sh.num_sms * 32);
}

// The mate initialisation, which leaves one partial sum per block in wpart:
// its resident blocks (80 registers: three blocks of 256 per SM), at most
// kWsumBlocks.
#ifndef AWPM_SUM_BPS
#define AWPM_SUM_BPS 3
#endif
static inline unsigned sum_grid(const Shape &sh)
{
    const int g = sh.num_sms * AWPM_SUM_BPS;
    return (unsigned)(g < kWsumBlocks ? g : kWsumBlocks);
}

void Sink::launch(const void *func, unsigned grid, unsigned block, void **args)
{
    if (err != cudaSuccess)
        return;
    if (graph) {
        cudaKernelNodeParams p;
        p.func = const_cast<void *>(func);
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = 0;
        p.kernelParams = args;
        p.extra = nullptr;
        cudaGraphNode_t node;
        err = cudaGraphAddKernelNode(&node, graph, last ? &last : nullptr, last ? 1 : 0, &p);
        if (err == cudaSuccess)
            last = node;
    } else {
        err = cudaLaunchKernel(func, dim3(grid), dim3(block), args, 0, stream);
    }
}

void launch_init(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_reset, util_grid(sh), kThreads, a);
    k.launch((const void *)k_check_mark, init_grid(sh), kThreads, a);
    k.launch((const void *)k_entries, init_tile_grid(sh), kThreads, a);
    if (sh.batch)
        k.launch((const void *)k_batch_cols, init_grid(sh), kThreads, a);
    k.launch((const void *)k_init_mates, sum_grid(sh), kThreads, a);
    k.launch((const void *)k_init_rows, init_grid(sh), kThreads, a);
    if (sh.batch) {
        k.launch((const void *)k_batch_check, init_tile_grid(sh), kThreads, a);
        k.launch((const void *)k_batch_list, init_grid(sh), kThreads, a);
    }
    if (sh.lookup == AWPM_LOOKUP_HASH)
        k.launch((const void *)k_hash_build, init_tile_grid(sh), kThreads, a);
    if (sh.lookup == AWPM_LOOKUP_ROWMARK) {
        k.launch((const void *)k_rm_marks, init_tile_grid(sh), kThreads, a);
        // four passes cover every row index; the unneeded ones return at once.
        // Grids: the resident blocks (scatter: 48 registers, 36 KB shared)
        const unsigned rs_grid = (unsigned)sh.num_sms * 8;
        const unsigned sc_grid = (unsigned)sh.num_sms * 5;
        for (int pass = 0; pass < 4; ++pass) {
            void *ap[] = {(void *)&d, (void *)&pass};
            k.launch((const void *)k_rs_hist, rs_grid, kRsThreads, ap);
            k.launch((const void *)k_rs_scan_a, rs_grid, kRsThreads, ap);
            k.launch((const void *)k_rs_scan_b, 1, kRsThreads, ap);
            k.launch((const void *)k_rs_scan_c, rs_grid, kRsThreads, ap);
            k.launch((const void *)k_rs_scatter, sc_grid, kRsThreads, ap);
        }
        k.launch((const void *)k_rm_rowptr, init_grid(sh), kThreads, a);
    }
}

// The matched weights' sum (the input matching's when !out).  The mate
// initialisation of a single solve already left its partials in wpart;
// otherwise k_wsum_partial writes them.
void launch_weight_sum(const Work *d, const Shape &sh, bool out, Sink &k)
{
    int o = out ? 1 : 0;
    const bool from_init = !out && !sh.batch;
    int parts = from_init ? (int)sum_grid(sh) : kWsumBlocks;
    void *a[] = {(void *)&d};
    void *ao[] = {(void *)&d, (void *)&o};
    void *af[] = {(void *)&d, (void *)&o, (void *)&parts};
    if (!from_init)
        k.launch((const void *)k_wsum_partial, kWsumBlocks, kWsumThreads, a);
    k.launch((const void *)k_wsum_final, 1, kWsumBlocks, af);
    if (sh.batch)
        k.launch((const void *)k_batch_wsum, util_grid(sh), kThreads, ao);
}

bool search_pipe()
{
    const char *v = getenv("AWPM_SEARCH_PIPE");
    if (v && (v[0] == '0' || v[0] == '1') && v[1] == 0)
        return v[0] == '1';
    return true;
}

template <bool kWide>
static const void *search_fn(int lookup, bool batch)
{
    if (search_pipe()) {
        if (batch) {
            if (lookup == AWPM_LOOKUP_ROWMARK)
                return (const void *)k_search_pipe<AWPM_LOOKUP_ROWMARK, kWide, true>;
            if (lookup == AWPM_LOOKUP_HASH)
                return (const void *)k_search_pipe<AWPM_LOOKUP_HASH, kWide, true>;
            return (const void *)k_search_pipe<AWPM_LOOKUP_BSEARCH, kWide, true>;
        }
        if (lookup == AWPM_LOOKUP_ROWMARK)
            return (const void *)k_search_pipe<AWPM_LOOKUP_ROWMARK, kWide, false>;
        if (lookup == AWPM_LOOKUP_HASH)
            return (const void *)k_search_pipe<AWPM_LOOKUP_HASH, kWide, false>;
        return (const void *)k_search_pipe<AWPM_LOOKUP_BSEARCH, kWide, false>;
    }
    if (lookup == AWPM_LOOKUP_ROWMARK)
        return batch ? (const void *)k_search<AWPM_LOOKUP_ROWMARK, true, kWide>
                     : (const void *)k_search<AWPM_LOOKUP_ROWMARK, false, kWide>;
    if (lookup == AWPM_LOOKUP_HASH)
        return batch ? (const void *)k_search<AWPM_LOOKUP_HASH, true, kWide>
                     : (const void *)k_search<AWPM_LOOKUP_HASH, false, kWide>;
    return batch ? (const void *)k_search<AWPM_LOOKUP_BSEARCH, true, kWide>
                 : (const void *)k_search<AWPM_LOOKUP_BSEARCH, false, kWide>;
}

int search_blocks_per_sm(int lookup, bool batch, bool wide)
{
    const void *f = wide ? search_fn<true>(lookup, batch) : search_fn<false>(lookup, batch);
    const int threads = batch ? SearchBlock<true>::kThreads : SearchBlock<false>::kThreads;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return b < 1 ? 1 : b;
}

bool default_search_wide()
{
    const char *v = getenv("AWPM_SEARCH_WIDE");
    if (v && (v[0] == '0' || v[0] == '1') && v[1] == 0)
        return v[0] == '1';
    return true;
}

// The search grid is one wave of resident blocks: each warp walks its tiles
// to the end (two, three, four and eight waves were measured slower on an
// R-MAT graph of scale 22: the later waves' blocks start only as whole
// blocks finish).
void launch_search(const Work *d, const Shape &sh, Sink &k)
{
    const unsigned grid = (unsigned)(sh.num_sms * (sh.search_bps > 0 ? sh.search_bps : 1));
    void *a[] = {(void *)&d};
    const void *f = sh.wide ? search_fn<true>(sh.lookup, sh.batch)
                            : search_fn<false>(sh.lookup, sh.batch);
    k.launch(f, grid, sh.batch ? SearchBlock<true>::kThreads : SearchBlock<false>::kThreads, a);
}

int search_waves(int num_sms, int search_bps, int32_t ntiles)
{
    const int64_t warps =
        (int64_t)num_sms * (search_bps > 0 ? search_bps : 1) * SearchBlock<false>::kWarps;
    return (int64_t)ntiles >= 64 * warps ? 2 : 1;
}

void launch_greedy_select_begin(const Work *d, const Shape &sh, bool graph,
                                cudaGraphConditionalHandle h, Sink &k)
{
    void *a[] = {(void *)&d};
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_ps_begin, tile_grid(sh), kThreads, a);
    if (graph)
        k.launch((const void *)k_ps_cond, 1, 1, ah);
}

void launch_greedy_select_round(const Work *d, const Shape &sh, bool graph,
                                cudaGraphConditionalHandle h, Sink &k)
{
    void *a[] = {(void *)&d};
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_ps_name, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_ps_take, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_ps_prune, tile_grid(sh), kThreads, a);
    if (graph)
        k.launch((const void *)k_ps_cond, 1, 1, ah);
}

void launch_greedy_select_end_and_flip(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_ps_end, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_flip, tile_grid(sh), kThreads, a);
}

// Step D's kernels take 32 words of the winner bitmap per warp; a single
// problem of the large size class (at least 64 tiles per resident search
// warp) gets four blocks per SM (one round of words covers n up to about
// 5 M), a smaller one one block per SM.  Late
// passes have few winners, so the kernels cost about their launch and a
// read of the bitmap; blocks past the bitmap's end would only add to that.
static inline unsigned winner_grid(const Shape &sh)
{
    return sh.batch ? tile_grid(sh) : (unsigned)(sh.num_sms * (sh.search_waves > 1 ? 4 : 1));
}

void launch_select_flip_control_graph(const Work *d, const Shape &sh,
                                      cudaGraphConditionalHandle h, Sink &k)
{
    void *a[] = {(void *)&d};
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_select, winner_grid(sh), kThreads, a);
    k.launch((const void *)k_flip_graph, winner_grid(sh), kThreads, ah);
}

void launch_select_and_flip(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_select, winner_grid(sh), kThreads, a);
    k.launch((const void *)k_flip, winner_grid(sh), kThreads, a);
}

void launch_control(const Work *d, const Shape &sh, bool graph, cudaGraphConditionalHandle h,
                    Sink &k)
{
    void *a[] = {(void *)&d};
    void *ah[] = {(void *)&d, (void *)&h};
    if (sh.batch) {
        k.launch((const void *)k_batch_control, util_grid(sh), kThreads, a);
        k.launch((const void *)k_batch_list, init_grid(sh), kThreads, a);
        if (graph)
            k.launch((const void *)k_batch_step_graph, 1, 1, ah);
        else
            k.launch((const void *)k_batch_step, 1, 1, a);
        return;
    }
    if (graph)
        k.launch((const void *)k_control_graph, 1, 1, ah);
    else
        k.launch((const void *)k_control, 1, 1, a);
}

void launch_greedy_init(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_gm_reset, util_grid(sh), kThreads, a);
    k.launch((const void *)k_check_colptr, init_grid(sh), kThreads, a);
    k.launch((const void *)k_mark_starts, init_grid(sh), kThreads, a);
    k.launch((const void *)k_gm_check, init_tile_grid(sh), kThreads, a);
}

void launch_greedy_round(const Work *d, const Shape &sh, bool graph, cudaGraphConditionalHandle h,
                         Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_gm_max, init_tile_grid(sh), kThreads, a);
    k.launch((const void *)k_gm_min, init_tile_grid(sh), kThreads, a);
    k.launch((const void *)k_gm_match, util_grid(sh), kThreads, a);
    k.launch((const void *)k_gm_rows, util_grid(sh), kThreads, a);
    launch_control(d, sh, graph, h, k);
}

void launch_weights(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_wt_reset, 1, 1, a);
    k.launch((const void *)k_check_colptr, init_grid(sh), kThreads, a);
    k.launch((const void *)k_wt_colmax, init_grid(sh), kThreads, a);
    k.launch((const void *)k_wt_rowmax, init_grid(sh), kThreads, a);
    k.launch((const void *)k_wt_out, init_grid(sh), kThreads, a);
}

void launch_mcm_load(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_mc_reset, util_grid(sh), kThreads, a);
    k.launch((const void *)k_check_colptr, init_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_allow_empty, 1, 1, a);
    k.launch((const void *)k_mark_starts, init_grid(sh), kThreads, a);
    k.launch((const void *)k_gm_check, init_tile_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_load, init_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_colof, init_grid(sh), kThreads, a);
}

void launch_mcm_phase(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_mc_phase, util_grid(sh), kThreads, a);
}

void launch_mcm_level(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    // one wave of blocks: a level's work follows its frontier, and a small
    // frontier should not pay for launching idle blocks
    k.launch((const void *)k_mc_offer, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_join, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_advance, util_grid(sh), kThreads, a);
}

void launch_mcm_augment(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_mc_augment, util_grid(sh), kThreads, a);
}

void launch_mcm_level_graph(const Work *d, const Shape &sh, cudaGraphConditionalHandle h,
                            Sink &k)
{
    void *a[] = {(void *)&d};
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_mc_offer, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_join, tile_grid(sh), kThreads, a);
    k.launch((const void *)k_mc_advance_graph, util_grid(sh), kThreads, ah);
}

void launch_mcm_cond_level(const Work *d, const Shape &sh, cudaGraphConditionalHandle h, Sink &k)
{
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_mc_cond_level, 1, 1, ah);
}

void launch_mcm_cond_phase(const Work *d, const Shape &sh, cudaGraphConditionalHandle h, Sink &k)
{
    void *ah[] = {(void *)&d, (void *)&h};
    k.launch((const void *)k_mc_cond_phase, 1, 1, ah);
}

void launch_mcm_store(const Work *d, const Shape &sh, Sink &k)
{
    void *a[] = {(void *)&d};
    k.launch((const void *)k_mc_store, util_grid(sh), kThreads, a);
}

void launch_export_stepc(const Work *d, const Shape &sh, double *gain, int32_t *row, Sink &k)
{
    void *a[] = {(void *)&d, (void *)&gain, (void *)&row};
    k.launch((const void *)k_export_stepc, util_grid(sh), kThreads, a);
}

}  // namespace awpm
