// CUDA kernels (sm_103a) of the weight-increasing alternating 4-cycle phase
// (arXiv 1801.09809, Section 5.3, Algorithms 2-6).
//
// The paper's message exchanges become arrays indexed by column in device
// memory: the A- and B-requests of Steps A and B never leave registers (one
// fused edge-parallel kernel does the lookup and the gain), Step C is a
// segmented arg-max inside each warp plus a 128-bit compare-and-swap for the
// columns that straddle a tile boundary, and Step D is one compare-and-swap
// selection per key column followed by an in-place flip.
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

__device__ __forceinline__ void raise_err(Ctl *ctl, unsigned bits)
{
    atomicOr(&ctl->err, bits);
}

__device__ __forceinline__ bool gate(const Ctl *ctl)
{
    return *(volatile const unsigned *)&ctl->err == 0u &&
           *(volatile const int32_t *)&ctl->active != 0;
}

// Lower bound of row r among the sorted rows rowidx[s..e); position or -1.
__device__ __forceinline__ int32_t find_row(const int32_t *__restrict__ rowidx, int32_t s,
                                            int32_t e, int32_t r)
{
    int32_t lo = s, len = e - s;
    while (len > 0) {
        int32_t half = len >> 1;
        int32_t mid = lo + half;
        if (__ldg(rowidx + mid) < r) {
            lo = mid + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return (lo < e && __ldg(rowidx + lo) == r) ? lo : -1;
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

// ---------------------------------------------------------------------------
// Initialisation and validation (before the loop of Algorithm 2)
// ---------------------------------------------------------------------------

__global__ void k_init_ctl(Ctl *ctl, int32_t max_passes)
{
    ctl->active = 1;
    ctl->max_passes = max_passes;
}

// colptr[0] = 0, non-decreasing, colptr[n] = nnz.
__global__ void k_check_colptr(int32_t n, int32_t nnz, const int32_t *__restrict__ colptr, Ctl *ctl)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j > n)
        return;
    int32_t c = colptr[j];
    bool bad = (j == 0 && c != 0) || (j < n && colptr[j + 1] < c) || (j == n && c != nnz);
    if (bad)
        raise_err(ctl, kErrInvalid);
}

// Column-start bitmap and the first column of every tile.
__global__ void k_mark_starts(int32_t n, const int32_t *__restrict__ colptr, uint32_t *starts,
                              int32_t *tile_col, Ctl *ctl)
{
    if (ctl->err)
        return;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    int32_t s = colptr[j], e = colptr[j + 1];
    if (s < e) {
        atomicOr(&starts[s >> 5], 1u << (s & 31));
        for (int64_t t = ((int64_t)s + kTile - 1) / kTile; t * kTile < e; ++t)
            tile_col[t] = (int32_t)j;
    }
}

// Row range, sortedness inside columns, finite weights.
__global__ void k_check_entries(int32_t n, int32_t nnz, const int32_t *__restrict__ rowidx,
                                const double *__restrict__ w, const uint32_t *__restrict__ starts,
                                Ctl *ctl)
{
    if (ctl->err & kErrInvalid)
        return;
    unsigned bits = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += stride) {
        int32_t r = __ldcs(rowidx + p);
        if (r < 0 || r >= n)
            bits |= kErrInvalid;
        if (!isfinite(__ldcs(w + p)))
            bits |= kErrNonfinite;
        if (p > 0 && !((starts[p >> 5] >> (p & 31)) & 1u) && rowidx[p - 1] >= r)
            bits |= kErrUnsorted;
    }
    bits = __reduce_or_sync(FULL_MASK, bits);
    if ((threadIdx.x & 31) == 0 && bits)
        raise_err(ctl, bits);
}

// mc = mate_in, mr = its inverse, wm[j] = w(mate_in[j], j); checks that
// mate_in is a permutation over stored entries.  mr must hold -1 on entry.
__global__ void k_init_mates(int32_t n, const int32_t *__restrict__ colptr,
                             const int32_t *__restrict__ rowidx, const double *__restrict__ w,
                             const int32_t *__restrict__ mate_in, int32_t *mc, int32_t *mr,
                             double *wm, Ctl *ctl)
{
    if (ctl->err)
        return;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    int32_t r = mate_in[j];
    mc[j] = r;
    if (r < 0 || r >= n) {
        raise_err(ctl, kErrNotPerfect);
        return;
    }
    if (atomicCAS(&mr[r], -1, (int32_t)j) != -1)
        raise_err(ctl, kErrNotPerfect);
    int32_t q = find_row(rowidx, colptr[j], colptr[j + 1], r);
    if (q < 0)
        raise_err(ctl, kErrNotPerfect);
    else
        wm[j] = w[q];
}

// Deterministic two-stage sum of wm (fixed grid, fixed tree).
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

__global__ void k_wsum_partial(int32_t n, const double *__restrict__ wm, double *part, const Ctl *ctl)
{
    double s = 0.0;
    if (ctl->err == 0u) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride)
            s += wm[j];
    }
    s = block_sum_f64(s);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

__global__ void k_wsum_final(const double *__restrict__ part, Ctl *ctl, int out)
{
    double s = block_sum_f64(part[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (out)
            ctl->weight_out = s;
        else
            ctl->weight_in = s;
    }
}

// ---------------------------------------------------------------------------
// Row records (range + signature of the column matched to each row)
// ---------------------------------------------------------------------------

// Bit of row r in a column signature (multiplicative hash, top 6 bits).
__device__ __forceinline__ unsigned sig_bit(int32_t r)
{
    return ((uint32_t)r * 0x9E3779B1u) >> 26;
}

// Column of the lane's nonzero inside a tile of kTile consecutive nonzeros
// starting in column c0: the lane counts the column ends <= p among the 32
// ends colptr[c0+1 .. c0+32] held one per lane in `e` (a tile spans at most
// 32 columns when no column is empty).
__device__ __forceinline__ int32_t lane_column_offset(int32_t e, int32_t p)
{
    int32_t cnt = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        int32_t v = __shfl_sync(FULL_MASK, e, cnt + s - 1);
        if (v <= p)
            cnt += s;
    }
    int32_t v = __shfl_sync(FULL_MASK, e, cnt);
    if (v <= p)
        cnt += 1;
    return cnt;
}

// Signature of every column: OR of 1 << sig_bit(r) over its rows.  Edge
// parallel; lanes of one column are OR-ed inside the warp, then one atomic
// per column segment.  colsig must be zero on entry.
__global__ void __launch_bounds__(256)
k_colsig(int32_t n, int32_t nnz, int32_t ntiles, const int32_t *__restrict__ colptr,
         const int32_t *__restrict__ rowidx, const int32_t *__restrict__ tile_col,
         unsigned long long *colsig, const Ctl *ctl)
{
    if (ctl->err)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp0; t < ntiles; t += nwarps) {
        const int32_t base = (int32_t)(t * kTile);
        const int32_t p = base + lane;
        const bool valid = p < nnz;
        const int32_t c0 = tile_col[t];
        const int64_t ck = (int64_t)c0 + 1 + lane;
        const int32_t e = (ck <= n) ? colptr[ck] : 0x7fffffff;
        const int32_t cnt = lane_column_offset(e, p);
        const int32_t j = valid ? c0 + cnt : -1 - lane;
        unsigned long long v = valid ? (1ull << sig_bit(__ldcs(rowidx + p))) : 0ull;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long ov = __shfl_down_sync(FULL_MASK, v, off);
            const int32_t oj = __shfl_down_sync(FULL_MASK, j, off);
            if (lane + off < 32 && oj == j)
                v |= ov;
        }
        const int32_t jprev = __shfl_up_sync(FULL_MASK, j, 1);
        if (valid && (lane == 0 || jprev != j))
            atomicOr(colsig + j, v);
    }
}

// rr[r] and wmr[r] for the row r matched to column j.
__global__ void k_init_rows(int32_t n, const int32_t *__restrict__ colptr,
                            const int32_t *__restrict__ mc, const double *__restrict__ wm,
                            const unsigned long long *__restrict__ colsig, RowRec *rr, double *wmr,
                            const Ctl *ctl)
{
    if (ctl->err)
        return;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    const int32_t r = mc[j];
    RowRec x;
    x.s = colptr[j];
    x.e = colptr[j + 1];
    x.sig = colsig[j];
    rr[r] = x;
    wmr[r] = wm[j];
}

// ---------------------------------------------------------------------------
// Per-column open-addressing tables (closing-edge lookup by hashing)
// ---------------------------------------------------------------------------
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

__global__ void __launch_bounds__(256)
k_hash_build(int32_t n, int32_t nnz, int32_t ntiles, const int32_t *__restrict__ colptr,
             const int32_t *__restrict__ rowidx, const int32_t *__restrict__ tile_col,
             unsigned long long *htab, Ctl *ctl)
{
    if (ctl->err)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp0; t < ntiles; t += nwarps) {
        const int32_t p = (int32_t)(t * kTile) + lane;
        const bool valid = p < nnz;
        const int32_t c0 = tile_col[t];
        const int64_t ck = (int64_t)c0 + 1 + lane;
        const int32_t e = (ck <= n) ? colptr[ck] : 0x7fffffff;
        const int32_t cnt = lane_column_offset(e, p);
        if (!valid)
            continue;
        const int32_t j = c0 + cnt;
        const int32_t r = __ldcs(rowidx + p);
        const int32_t base = 2 * colptr[j];
        const int32_t size = 2 * (colptr[j + 1] - colptr[j]);
        const unsigned long long v = ((unsigned long long)(uint32_t)p << 32) | (uint32_t)r;
        int32_t pos = slot_start(r, base, size);
        int k = 0;
        for (; k < size; ++k) {
            if (atomicCAS(htab + pos, kSlotEmpty, v) == kSlotEmpty)
                break;
            if (++pos == base + size)
                pos = base;
        }
        if (k == size)
            raise_err(ctl, kErrInternal);
    }
}

// ---------------------------------------------------------------------------
// Steps A + B + C (Algorithms 3, 4, 5): fused edge-parallel cycle search
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool rec_better(double g, int32_t p, double cg, int32_t cp)
{
    return g > cg || (g == cg && p < cp);
}

// Lock-free maximum of (g, lowest p) into a Step-C record.
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
    raise_err(ctl, kErrInternal);
}

__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 16-byte row record through the read-only path, kept in L2 (evict last).
__device__ __forceinline__ RowRec ld_rowrec(const RowRec *ptr, unsigned long long pol)
{
    uint32_t a, b, c, d;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                 : "l"(ptr), "l"(pol));
    RowRec r;
    r.s = (int32_t)a;
    r.e = (int32_t)b;
    r.sig = ((unsigned long long)d << 32) | c;
    return r;
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

// Closing-edge ranges longer than this go to the warp-cooperative search.
constexpr int32_t kCoopMin = 32;

// One warp per tile of kTile consecutive nonzeros (lane = one nonzero).
// The lane's column comes from the tile's first column and its word of the
// column-start bitmap (one popcount).  Lane with nonzero p = (i, j): if
// i > m_j it is an A-request (Algorithm 3); the closing entry (m_j, m_i) is
// looked up in column m_i (Algorithm 4): the row record of i gives that
// column's range and signature, so a clear signature bit settles "absent" at
// once; otherwise the column is searched (binary search, warp-cooperative for
// long columns, or the column's hash table).  The gain is evaluated in the
// fixed order ((w_ij + w_q) - w(i,m_i)) - w(m_j,j).  Per column the warp
// keeps the maximum positive gain with the lowest row (Algorithm 5); columns
// cut by a tile boundary are merged across warps by a 128-bit
// compare-and-swap.  `best` must be zero on entry: only positive records are
// written.  In a batched solve, tiles of finished matrices are skipped.
template <int kLookup, bool kBatch>
__global__ void __launch_bounds__(256)
k_search(int32_t n, int32_t nnz, int32_t ntiles, const int32_t *__restrict__ rowidx,
         const double *__restrict__ w, const int32_t *__restrict__ tile_col,
         const uint32_t *__restrict__ starts, const int32_t *__restrict__ mc,
         const double *__restrict__ wm, const RowRec *__restrict__ rr,
         const double *__restrict__ wmr, const unsigned long long *__restrict__ htab,
         Rec *__restrict__ best, Ctl *ctl, const int32_t *__restrict__ tilemat,
         const int32_t *__restrict__ colmat, const int32_t *__restrict__ mdone)
{
    __shared__ int s_go;
    if (threadIdx.x == 0)
        s_go = gate(ctl) ? 1 : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t le_mask = (2u << lane) - 1u;  // lanes 0..lane
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long pol = policy_evict_last();
    unsigned long long n_cand = 0, n_found = 0, n_pos = 0;

    for (int64_t t = s_go ? warp0 : (int64_t)ntiles; t < ntiles; t += nwarps) {
        const int32_t base = (int32_t)(t * kTile);
        const int32_t p = base + lane;
        bool valid = p < nnz;
        bool mixed = false;
        const int32_t c0 = __ldg(tile_col + t);
        const uint32_t mask = __ldg(starts + t);
        if (kBatch) {
            // a tile of one finished matrix has nothing left to do
            const int32_t tm = __ldg(tilemat + t);
            if (tm & kTileSingle) {
                if (__ldg(mdone + (tm & ~kTileSingle)))
                    valid = false;
            } else {
                mixed = true;
            }
        }
        const int32_t i = valid ? __ldcs(rowidx + p) : 0;
        const int32_t j = valid ? c0 + __popc(mask & le_mask & ~1u) : -1 - lane;
        int32_t mj = valid ? ld_i32_last(mc + j, pol) : 0x7fffffff;
        if (kBatch && mixed && valid && __ldg(mdone + __ldg(colmat + j)))
            mj = 0x7fffffff;  // finished matrix: no candidate
        const bool cand = valid && i > mj;
        RowRec rec;
        rec.s = rec.e = 0;
        rec.sig = 0ull;
        if (cand) {
            ++n_cand;
            rec = ld_rowrec(rr + i, pol);
        }
        const bool pass = cand && ((rec.sig >> sig_bit(mj)) & 1ull);
        int32_t lo = rec.s;
        int32_t len = pass ? rec.e - rec.s : 0;
        int32_t q = -1;
        const double wmi = pass ? __ldg(wmr + i) : 0.0;
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
        } else {
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
        double g = 0.0;
        if (q >= 0) {
            ++n_found;
            const double wij = __ldcs(w + p);
            const double wq = __ldg(w + q);
            const double gg = ((wij + wq) - wmi) - __ldg(wm + j);
            if (gg > 0.0) {
                ++n_pos;
                g = gg;
            } else {
                q = -1;
            }
        }
        if (!__any_sync(FULL_MASK, g > 0.0))
            continue;
        // segmented arg-max over lanes of the same column (suffix direction)
        int32_t bp = valid ? p : 0x7fffffff;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double og = __shfl_down_sync(FULL_MASK, g, off);
            const int32_t op = __shfl_down_sync(FULL_MASK, bp, off);
            const int32_t oq = __shfl_down_sync(FULL_MASK, q, off);
            const int32_t oj = __shfl_down_sync(FULL_MASK, j, off);
            if (lane + off < 32 && oj == j && og > 0.0 && rec_better(og, op, g, bp)) {
                g = og;
                bp = op;
                q = oq;
            }
        }
        const bool head = valid && (lane == 0 || ((mask >> lane) & 1u));
        if (head && g > 0.0) {
            // the segment covers its whole column when the column starts here
            // and ends inside the tile (a later start bit, the end of the
            // matrix, or a column starting the next tile)
            const bool starts_here = (mask >> lane) & 1u;
            const uint32_t later = lane == 31 ? 0u : (mask >> (lane + 1));
            const bool ends_here = later != 0u || base + kTile >= nnz ||
                                   (__ldg(starts + t + 1) & 1u);
            Rec r;
            r.g = g;
            r.p = bp;
            r.q = q;
            if (starts_here && ends_here)
                best[j] = r;
            else
                rec_combine(best + j, r, ctl);
        }
    }
    block_add_u64(n_cand, &ctl->candidates);
    block_add_u64(n_found, &ctl->found);
    block_add_u64(n_pos, &ctl->positive);
}

// ---------------------------------------------------------------------------
// Step D (Algorithm 6): conflicts, per-key selection, flip
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool sel_better(double g, int32_t j, double cg, int32_t cj)
{
    return g > cg || (g == cg && j < cj);
}

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
    raise_err(ctl, kErrInternal);
}

// For every Step-C winner rooted at j with second matched edge at column
// k = m_i: drop it if column k is itself the root of a Step-C winner,
// otherwise compete for key k (maximum gain, then lowest root j).
__global__ void k_select(int32_t n, const int32_t *__restrict__ rowidx,
                         const int32_t *__restrict__ mr, const Rec *__restrict__ best, Sel *dsel,
                         Ctl *ctl)
{
    if (!gate(ctl))
        return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        const Rec r = best[j];
        if (!(r.g > 0.0))
            continue;
        const int32_t i = __ldg(rowidx + r.p);
        const int32_t k = __ldg(mr + i);
        if (best[k].g > 0.0)
            continue;
        Sel s;
        s.g = r.g;
        s.j = (int32_t)j;
        s.pad = 0;
        sel_combine(dsel + k, s, ctl);
    }
}

// Flip every selected cycle: column j takes row i, key column k takes m_j;
// the row records of rows i and m_j follow their new mates.  The selected
// cycles are vertex-disjoint, so each thread owns its four vertices.
__global__ void k_flip(int32_t n, const int32_t *__restrict__ colptr,
                       const int32_t *__restrict__ rowidx, const double *__restrict__ w,
                       const unsigned long long *__restrict__ colsig, const Rec *__restrict__ best,
                       Sel *dsel, int32_t *mc, int32_t *mr, double *wm, RowRec *rr, double *wmr,
                       Ctl *ctl, const int32_t *__restrict__ colmat, unsigned long long *mflips)
{
    unsigned long long flips = 0;
    if (gate(ctl)) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
            const Sel s = dsel[k];
            if (!(s.g > 0.0))
                continue;
            dsel[k] = Sel{0.0, 0, 0};
            const int32_t j = s.j;
            const Rec r = best[j];
            const int32_t i = rowidx[r.p];
            const int32_t mj = mc[j];
            const double wij = w[r.p];
            const double wq = w[r.q];
            mc[j] = i;
            mr[i] = j;
            mc[k] = mj;
            mr[mj] = (int32_t)k;
            wm[j] = wij;
            wm[k] = wq;
            RowRec a;
            a.s = colptr[j];
            a.e = colptr[j + 1];
            a.sig = colsig[j];
            rr[i] = a;
            wmr[i] = wij;
            RowRec b;
            b.s = colptr[k];
            b.e = colptr[k + 1];
            b.sig = colsig[k];
            rr[mj] = b;
            wmr[mj] = wq;
            ++flips;
            if (mflips)
                atomicAdd(mflips + colmat[k], 1ull);
        }
    }
    block_add_u64(flips, &ctl->pass_flips);
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

__global__ void k_control(Ctl *ctl)
{
    control_step(ctl);
}

__global__ void k_control_graph(Ctl *ctl, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, control_step(ctl) ? 1u : 0u);
}

__global__ void k_export_stepc(int32_t n, const int32_t *__restrict__ rowidx,
                               const Rec *__restrict__ best, double *gain, int32_t *row,
                               const Ctl *ctl)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n || ctl->err)
        return;
    const Rec r = best[j];
    const bool has = r.g > 0.0;
    gain[j] = has ? r.g : 0.0;
    row[j] = has ? rowidx[r.p] : -1;
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
__global__ void k_batch_cols(int32_t n, int32_t count, const int32_t *__restrict__ n_off,
                             int32_t *colmat, Ctl *ctl)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x <= count) {
        const int32_t o = n_off[x];
        if ((x == 0 && o != 0) || (x == count && o != n) || (x < count && n_off[x + 1] < o))
            raise_err(ctl, kErrInvalid);
    }
    if (x >= n)
        return;
    // last b with n_off[b] <= x (empty matrices are skipped over)
    int32_t lo = 0, len = count;
    while (len > 0) {
        const int32_t half = len >> 1;
        if (__ldg(n_off + lo + half + 1) <= x) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    colmat[x] = lo < count ? lo : count - 1;
}

// Every stored row lies in its column's block; nonzeros per matrix; the
// matrix of each tile and whether the tile stays inside one matrix.
__global__ void __launch_bounds__(256)
k_batch_check(int32_t n, int32_t nnz, int32_t ntiles, int32_t count, const int32_t *__restrict__ colptr,
              const int32_t *__restrict__ rowidx, const int32_t *__restrict__ tile_col,
              const int32_t *__restrict__ n_off, const int32_t *__restrict__ colmat,
              int32_t *tilemat, int32_t *mnnz, Ctl *ctl)
{
    if (ctl->err)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    for (int64_t t = warp0; t < ntiles; t += nwarps) {
        const int32_t p = (int32_t)(t * kTile) + lane;
        const bool valid = p < nnz;
        const int32_t c0 = tile_col[t];
        const int64_t ck = (int64_t)c0 + 1 + lane;
        const int32_t e = (ck <= n) ? colptr[ck] : 0x7fffffff;
        const int32_t cnt = lane_column_offset(e, p);
        if (valid) {
            const int32_t b = colmat[c0 + cnt];
            const int32_t r = rowidx[p];
            if (r < n_off[b] || r >= n_off[b + 1])
                bad = 1;
        }
        if (lane == 0) {
            const int32_t b0 = colmat[c0];
            const int32_t b1 = (t + 1 < ntiles) ? colmat[tile_col[t + 1]] : colmat[n - 1];
            tilemat[t] = b0 | (b0 == b1 ? kTileSingle : 0);
        }
    }
    if (__any_sync(FULL_MASK, bad) && lane == 0)
        raise_err(ctl, kErrInvalid);
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b < count)
        mnnz[b] = colptr[n_off[b + 1]] - colptr[n_off[b]];
}

// End of a pass for every matrix still running: count the pass, stop the
// matrix when it flipped nothing or reached the cap; count the running ones.
__global__ void k_batch_control(int32_t count, BatchWork bw, Ctl *ctl)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int still = 0;
    if (b < count && !ctl->err && !bw.mdone[b]) {
        const unsigned long long f = bw.mflips[b];
        bw.mflips[b] = 0;
        bw.miter[b] += 1;
        bw.mcycles[b] += f;
        if (f == 0) {
            bw.mconv[b] = 1;
            bw.mdone[b] = 1;
        } else if (bw.miter[b] >= ctl->max_passes) {
            bw.mdone[b] = 1;
        } else {
            still = 1;
        }
    }
    still = __syncthreads_count(still);
    if (threadIdx.x == 0 && still)
        atomicAdd(bw.active, still);
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

__global__ void k_batch_step(Ctl *ctl, int32_t *active)
{
    batch_step(ctl, active);
}

__global__ void k_batch_step_graph(Ctl *ctl, int32_t *active, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, batch_step(ctl, active) ? 1u : 0u);
}

// One block per matrix: deterministic sum of its matched weights.
__global__ void k_batch_wsum(int32_t count, const int32_t *__restrict__ n_off,
                             const double *__restrict__ wm, double *out, const Ctl *ctl)
{
    const int32_t b = blockIdx.x;
    double s = 0.0;
    if (ctl->err == 0u)
        for (int64_t j = n_off[b] + threadIdx.x; j < n_off[b + 1]; j += blockDim.x)
            s += wm[j];
    s = block_sum_f64(s);
    if (threadIdx.x == 0)
        out[b] = s;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(int64_t items, int threads)
{
    int64_t b = (items + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

constexpr int kSearchThreads = 256;

int default_search_u()
{
    const char *v = getenv("AWPM_SEARCH_U");
    if (v && (v[0] == '1' || v[0] == '2' || v[0] == '4') && v[1] == 0)
        return v[0] - '0';
    return 1;
}

// Resident blocks per SM of the search kernel.
template <bool kBatch>
static int search_bps(int lookup)
{
    int b = 0;
    cudaError_t e;
    const int T = kSearchThreads;
    if (lookup == AWPM_LOOKUP_HASH)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<AWPM_LOOKUP_HASH, kBatch>,
                                                          T, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, k_search<AWPM_LOOKUP_BSEARCH, kBatch>, T, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return b < 1 ? 1 : b;
}

int search_blocks_per_sm(int lookup, int u, bool batch)
{
    (void)u;
    return batch ? search_bps<true>(lookup) : search_bps<false>(lookup);
}

void launch_init(const Work &wk, int max_passes, int num_sms, cudaStream_t s)
{
    const int T = 256;
    cudaMemsetAsync(wk.ctl, 0, sizeof(Ctl), s);
    cudaMemsetAsync(wk.mr, 0xff, sizeof(int32_t) * (size_t)wk.n, s);
    cudaMemsetAsync(wk.starts, 0, sizeof(uint32_t) * (((size_t)wk.nnz + 31) / 32 + 1), s);
    cudaMemsetAsync(wk.best, 0, sizeof(Rec) * (size_t)wk.n, s);
    cudaMemsetAsync(wk.dsel, 0, sizeof(Sel) * (size_t)wk.n, s);
    cudaMemsetAsync(wk.colsig, 0, sizeof(unsigned long long) * (size_t)wk.n, s);
    k_init_ctl<<<1, 1, 0, s>>>(wk.ctl, max_passes);
    k_check_colptr<<<blocks_for((int64_t)wk.n + 1, T), T, 0, s>>>(wk.n, wk.nnz, wk.colptr, wk.ctl);
    k_mark_starts<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.starts, wk.tile_col, wk.ctl);
    int64_t want = ((int64_t)wk.nnz + T - 1) / T;
    int64_t cap = (int64_t)num_sms * 16;
    k_check_entries<<<(unsigned)(want < 1 ? 1 : (want < cap ? want : cap)), T, 0, s>>>(
        wk.n, wk.nnz, wk.rowidx, wk.w, wk.starts, wk.ctl);
    const BatchWork &bw = wk.bw;
    if (bw.count > 0) {
        cudaMemsetAsync(bw.mdone, 0, sizeof(int32_t) * (size_t)bw.count, s);
        cudaMemsetAsync(bw.miter, 0, sizeof(int32_t) * (size_t)bw.count, s);
        cudaMemsetAsync(bw.mconv, 0, sizeof(int32_t) * (size_t)bw.count, s);
        cudaMemsetAsync(bw.mflips, 0, sizeof(unsigned long long) * (size_t)bw.count, s);
        cudaMemsetAsync(bw.mcycles, 0, sizeof(unsigned long long) * (size_t)bw.count, s);
        cudaMemsetAsync(bw.active, 0, sizeof(int32_t), s);
        int64_t items = (int64_t)wk.n > (int64_t)bw.count + 1 ? (int64_t)wk.n : (int64_t)bw.count + 1;
        k_batch_cols<<<blocks_for(items, T), T, 0, s>>>(wk.n, bw.count, bw.n_off, bw.colmat, wk.ctl);
    }
    k_init_mates<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.rowidx, wk.w, wk.mate_in,
                                                    wk.mc, wk.mr, wk.wm, wk.ctl);
    int64_t twant = ((int64_t)wk.ntiles + (T / 32) - 1) / (T / 32);
    k_colsig<<<(unsigned)(twant < 1 ? 1 : (twant < cap ? twant : cap)), T, 0, s>>>(
        wk.n, wk.nnz, wk.ntiles, wk.colptr, wk.rowidx, wk.tile_col, wk.colsig, wk.ctl);
    if (bw.count > 0) {
        int64_t g = twant > blocks_for(bw.count, T) ? twant : blocks_for(bw.count, T);
        k_batch_check<<<(unsigned)(g < 1 ? 1 : g), T, 0, s>>>(wk.n, wk.nnz, wk.ntiles, bw.count,
                                                           wk.colptr, wk.rowidx, wk.tile_col,
                                                           bw.n_off, bw.colmat, bw.tilemat,
                                                           bw.mnnz, wk.ctl);
    }
    k_init_rows<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.mc, wk.wm, wk.colsig, wk.rr,
                                                   wk.wmr, wk.ctl);
    if (wk.lookup == AWPM_LOOKUP_HASH && wk.htab) {
        cudaMemsetAsync(wk.htab, 0xff, sizeof(unsigned long long) * 2 * (size_t)wk.nnz, s);
        k_hash_build<<<(unsigned)(twant < 1 ? 1 : (twant < cap ? twant : cap)), T, 0, s>>>(
            wk.n, wk.nnz, wk.ntiles, wk.colptr, wk.rowidx, wk.tile_col, wk.htab, wk.ctl);
    }
}

void launch_weight_sum(const Work &wk, bool out, cudaStream_t s)
{
    k_wsum_partial<<<kWsumBlocks, kWsumThreads, 0, s>>>(wk.n, wk.wm, wk.wpart, wk.ctl);
    k_wsum_final<<<1, kWsumBlocks, 0, s>>>(wk.wpart, wk.ctl, out ? 1 : 0);
}

void launch_reset_best(const Work &wk, cudaStream_t s)
{
    cudaMemsetAsync(wk.best, 0, sizeof(Rec) * (size_t)wk.n, s);
}

template <int kLookup, bool kBatch>
static void launch_search_k(const Work &wk, int num_sms, cudaStream_t s)
{
    const int T = kSearchThreads;
    const int64_t per_block = T / 32;
    int64_t want = ((int64_t)wk.ntiles + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms * (wk.search_bps > 0 ? wk.search_bps : 1);
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_search<kLookup, kBatch><<<grid, T, 0, s>>>(
        wk.n, wk.nnz, wk.ntiles, wk.rowidx, wk.w, wk.tile_col, wk.starts, wk.mc, wk.wm, wk.rr,
        wk.wmr, wk.htab, wk.best, wk.ctl, wk.bw.tilemat, wk.bw.colmat, wk.bw.mdone);
}

template <bool kBatch>
static void launch_search_b(const Work &wk, int num_sms, cudaStream_t s)
{
    if (wk.lookup == AWPM_LOOKUP_HASH)
        launch_search_k<AWPM_LOOKUP_HASH, kBatch>(wk, num_sms, s);
    else
        launch_search_k<AWPM_LOOKUP_BSEARCH, kBatch>(wk, num_sms, s);
}

void launch_search(const Work &wk, int num_sms, cudaStream_t s)
{
    if (wk.bw.count > 0)
        launch_search_b<true>(wk, num_sms, s);
    else
        launch_search_b<false>(wk, num_sms, s);
}

void launch_select_and_flip(const Work &wk, int num_sms, cudaStream_t s)
{
    const int T = 256;
    int64_t want = ((int64_t)wk.n + T - 1) / T;
    int64_t cap = (int64_t)num_sms * 8;
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_select<<<grid, T, 0, s>>>(wk.n, wk.rowidx, wk.mr, wk.best, wk.dsel, wk.ctl);
    k_flip<<<grid, T, 0, s>>>(wk.n, wk.colptr, wk.rowidx, wk.w, wk.colsig, wk.best, wk.dsel,
                              wk.mc, wk.mr, wk.wm, wk.rr, wk.wmr, wk.ctl, wk.bw.colmat,
                              wk.bw.count > 0 ? wk.bw.mflips : nullptr);
}

void launch_control(const Work &wk, bool graph, cudaGraphConditionalHandle h, cudaStream_t s)
{
    if (wk.bw.count > 0) {
        k_batch_control<<<blocks_for(wk.bw.count, 256), 256, 0, s>>>(wk.bw.count, wk.bw, wk.ctl);
        if (graph)
            k_batch_step_graph<<<1, 1, 0, s>>>(wk.ctl, wk.bw.active, h);
        else
            k_batch_step<<<1, 1, 0, s>>>(wk.ctl, wk.bw.active);
        return;
    }
    if (graph)
        k_control_graph<<<1, 1, 0, s>>>(wk.ctl, h);
    else
        k_control<<<1, 1, 0, s>>>(wk.ctl);
}

void launch_batch_weight_sum(const Work &wk, bool out, cudaStream_t s)
{
    if (wk.bw.count > 0)
        k_batch_wsum<<<wk.bw.count, 256, 0, s>>>(wk.bw.count, wk.bw.n_off, wk.wm,
                                                 out ? wk.bw.mw_out : wk.bw.mw_in, wk.ctl);
}

void launch_export_stepc(const Work &wk, double *gain, int32_t *row, cudaStream_t s)
{
    k_export_stepc<<<blocks_for(wk.n, 256), 256, 0, s>>>(wk.n, wk.rowidx, wk.best, gain, row, wk.ctl);
}

}  // namespace awpm
