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

// One warp per tile of kTile consecutive nonzeros (lane = one nonzero), kU
// tiles in flight per warp with their independent loads issued together.
// Lane with nonzero p = (i, j): if i > m_j it is an A-request (Algorithm 3);
// the closing entry (m_j, m_i) is looked up in column m_i (Algorithm 4): the
// row record of i gives that column's range and signature, so a clear
// signature bit settles "absent" at once, otherwise a binary search over the
// column's rows finds it.  The gain is evaluated in the fixed order
// ((w_ij + w_q) - w(i,m_i)) - w(m_j,j).  Per column the warp keeps the
// maximum positive gain with the lowest row (Algorithm 5); columns cut by a
// tile boundary are merged across warps by a 128-bit compare-and-swap.
// `best` must be zero on entry: only positive records are written.
template <int kLookup, int kU>
__global__ void __launch_bounds__(256)
k_search(int32_t n, int32_t nnz, int32_t ntiles, const int32_t *__restrict__ colptr,
         const int32_t *__restrict__ rowidx, const double *__restrict__ w,
         const int32_t *__restrict__ tile_col, const int32_t *__restrict__ mc,
         const double *__restrict__ wm, const RowRec *__restrict__ rr,
         const double *__restrict__ wmr, Rec *__restrict__ best, Ctl *ctl)
{
    __shared__ int s_go;
    if (threadIdx.x == 0)
        s_go = gate(ctl) ? 1 : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long pol = policy_evict_last();
    unsigned long long n_cand = 0, n_found = 0, n_pos = 0;

    for (int64_t t0 = s_go ? warp0 : (int64_t)ntiles; t0 < ntiles; t0 += nwarps * kU) {
        int32_t base[kU], p[kU], c0[kU], e[kU], c0s[kU], i[kU];
        bool tv[kU], valid[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t t = t0 + (int64_t)u * nwarps;
            tv[u] = t < ntiles;
            base[u] = (int32_t)(t * kTile);
            p[u] = base[u] + lane;
            valid[u] = tv[u] && p[u] < nnz;
            c0[u] = tv[u] ? __ldg(tile_col + t) : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t ck = (int64_t)c0[u] + 1 + lane;
            e[u] = (tv[u] && ck <= n) ? __ldg(colptr + ck) : 0x7fffffff;
            c0s[u] = tv[u] ? __ldg(colptr + c0[u]) : 0;
            i[u] = valid[u] ? __ldcs(rowidx + p[u]) : 0;
        }
        int32_t j[kU], colend[kU], mj[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int32_t cnt = lane_column_offset(e[u], p[u]);
            colend[u] = __shfl_sync(FULL_MASK, e[u], cnt & 31);
            j[u] = valid[u] ? c0[u] + cnt : -1 - lane;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            mj[u] = valid[u] ? ld_i32_last(mc + j[u], pol) : 0x7fffffff;
        RowRec rec[kU];
        bool cand[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            cand[u] = valid[u] && i[u] > mj[u];
            rec[u].s = rec[u].e = 0;
            rec[u].sig = 0ull;
            if (cand[u]) {
                ++n_cand;
                rec[u] = ld_rowrec(rr + i[u], pol);
            }
        }
        int32_t lo[kU], len[kU], q[kU];
        double wmi[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const bool pass = cand[u] && ((rec[u].sig >> sig_bit(mj[u])) & 1ull);
            lo[u] = rec[u].s;
            len[u] = pass ? rec[u].e - rec[u].s : 0;
            q[u] = -1;
            wmi[u] = pass ? __ldg(wmr + i[u]) : 0.0;
        }
        // merged binary searches (early exit on a hit)
        for (;;) {
            bool any = false;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (len[u] > 0) {
                    any = true;
                    const int32_t half = len[u] >> 1;
                    const int32_t mid = lo[u] + half;
                    const int32_t v = __ldg(rowidx + mid);
                    if (v == mj[u]) {
                        q[u] = mid;
                        len[u] = 0;
                    } else if (v < mj[u]) {
                        lo[u] = mid + 1;
                        len[u] -= half + 1;
                    } else {
                        len[u] = half;
                    }
                }
            }
            if (!any)
                break;
        }
        double g[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            g[u] = 0.0;
            if (q[u] >= 0) {
                ++n_found;
                const double wij = __ldcs(w + p[u]);
                const double wq = __ldg(w + q[u]);
                const double gg = ((wij + wq) - wmi[u]) - __ldg(wm + j[u]);
                if (gg > 0.0) {
                    ++n_pos;
                    g[u] = gg;
                } else {
                    q[u] = -1;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (!__any_sync(FULL_MASK, g[u] > 0.0))
                continue;
            // segmented arg-max over lanes of the same column (suffix direction)
            double gg = g[u];
            int32_t bp = valid[u] ? p[u] : 0x7fffffff;
            int32_t bq = q[u];
            const int32_t jj = j[u];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double og = __shfl_down_sync(FULL_MASK, gg, off);
                const int32_t op = __shfl_down_sync(FULL_MASK, bp, off);
                const int32_t oq = __shfl_down_sync(FULL_MASK, bq, off);
                const int32_t oj = __shfl_down_sync(FULL_MASK, jj, off);
                if (lane + off < 32 && oj == jj && og > 0.0 && rec_better(og, op, gg, bp)) {
                    gg = og;
                    bp = op;
                    bq = oq;
                }
            }
            const int32_t jprev = __shfl_up_sync(FULL_MASK, jj, 1);
            const bool head = valid[u] && (lane == 0 || jprev != jj);
            if (head && gg > 0.0) {
                const bool starts_here = (jj != c0[u]) || (c0s[u] >= base[u]);
                const bool complete = starts_here && colend[u] <= base[u] + kTile;
                Rec r;
                r.g = gg;
                r.p = bp;
                r.q = bq;
                if (complete)
                    best[jj] = r;
                else
                    rec_combine(best + jj, r, ctl);
            }
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
                       Ctl *ctl)
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

// Resident blocks per SM of the search kernel with u tiles in flight per warp.
int search_blocks_per_sm(int u)
{
    int b = 0;
    cudaError_t e;
    if (u == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<AWPM_LOOKUP_BSEARCH, 2>,
                                                          kSearchThreads, 0);
    else if (u == 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<AWPM_LOOKUP_BSEARCH, 4>,
                                                          kSearchThreads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_search<AWPM_LOOKUP_BSEARCH, 1>,
                                                          kSearchThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return b < 1 ? 1 : b;
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
    k_init_mates<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.rowidx, wk.w, wk.mate_in,
                                                    wk.mc, wk.mr, wk.wm, wk.ctl);
    int64_t twant = ((int64_t)wk.ntiles + (T / 32) - 1) / (T / 32);
    k_colsig<<<(unsigned)(twant < 1 ? 1 : (twant < cap ? twant : cap)), T, 0, s>>>(
        wk.n, wk.nnz, wk.ntiles, wk.colptr, wk.rowidx, wk.tile_col, wk.colsig, wk.ctl);
    k_init_rows<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.mc, wk.wm, wk.colsig, wk.rr,
                                                   wk.wmr, wk.ctl);
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

template <int kU>
static void launch_search_u(const Work &wk, int num_sms, cudaStream_t s)
{
    const int T = kSearchThreads;
    const int64_t per_block = (int64_t)(T / 32) * kU;
    int64_t want = ((int64_t)wk.ntiles + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms * (wk.search_bps > 0 ? wk.search_bps : 1);
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_search<AWPM_LOOKUP_BSEARCH, kU><<<grid, T, 0, s>>>(
        wk.n, wk.nnz, wk.ntiles, wk.colptr, wk.rowidx, wk.w, wk.tile_col, wk.mc, wk.wm, wk.rr,
        wk.wmr, wk.best, wk.ctl);
}

void launch_search(const Work &wk, int lookup, int num_sms, cudaStream_t s)
{
    (void)lookup;
    if (wk.search_u == 1)
        launch_search_u<1>(wk, num_sms, s);
    else if (wk.search_u == 4)
        launch_search_u<4>(wk, num_sms, s);
    else if (wk.search_u == 2)
        launch_search_u<2>(wk, num_sms, s);
    else
        launch_search_u<1>(wk, num_sms, s);
}

void launch_select_and_flip(const Work &wk, int num_sms, cudaStream_t s)
{
    const int T = 256;
    int64_t want = ((int64_t)wk.n + T - 1) / T;
    int64_t cap = (int64_t)num_sms * 8;
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_select<<<grid, T, 0, s>>>(wk.n, wk.rowidx, wk.mr, wk.best, wk.dsel, wk.ctl);
    k_flip<<<grid, T, 0, s>>>(wk.n, wk.colptr, wk.rowidx, wk.w, wk.colsig, wk.best, wk.dsel,
                              wk.mc, wk.mr, wk.wm, wk.rr, wk.wmr, wk.ctl);
}

void launch_control(const Work &wk, bool graph, cudaGraphConditionalHandle h, cudaStream_t s)
{
    if (graph)
        k_control_graph<<<1, 1, 0, s>>>(wk.ctl, h);
    else
        k_control<<<1, 1, 0, s>>>(wk.ctl);
}

void launch_export_stepc(const Work &wk, double *gain, int32_t *row, cudaStream_t s)
{
    k_export_stepc<<<blocks_for(wk.n, 256), 256, 0, s>>>(wk.n, wk.rowidx, wk.best, gain, row, wk.ctl);
}

}  // namespace awpm
