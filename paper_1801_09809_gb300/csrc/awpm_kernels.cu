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

// One warp per tile of kTile consecutive nonzeros (lane = one nonzero).
// Lane with nonzero p = (i, j): if i > m_j it is an A-request (Algorithm 3);
// the closing entry (m_j, m_i) is looked up in column m_i (Algorithm 4) and
// the gain evaluated in the fixed order ((w_ij + w_q) - w(i,m_i)) - w(m_j,j).
// The warp then keeps, per column, the maximum positive gain with the lowest
// row (Algorithm 5).
template <int kLookup>
__global__ void __launch_bounds__(256)
k_search(int32_t n, int32_t nnz, int32_t ntiles, const int32_t *__restrict__ colptr,
         const int32_t *__restrict__ rowidx, const double *__restrict__ w,
         const int32_t *__restrict__ tile_col, const int32_t *__restrict__ mc,
         const int32_t *__restrict__ mr, const double *__restrict__ wm, Rec *__restrict__ best,
         Ctl *ctl)
{
    __shared__ int s_go;
    if (threadIdx.x == 0)
        s_go = gate(ctl) ? 1 : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_cand = 0, n_found = 0, n_pos = 0;

    for (int64_t t = s_go ? warp0 : (int64_t)ntiles; t < ntiles; t += nwarps) {
        const int32_t base = (int32_t)(t * kTile);
        const int32_t p = base + lane;
        const bool valid = p < nnz;
        const int32_t c0 = __ldg(tile_col + t);
        // ends of columns c0 .. c0+31; a tile spans at most 32 columns because
        // every column holds at least its matched entry
        const int64_t ck = (int64_t)c0 + 1 + lane;
        const int32_t e = (ck <= n) ? __ldg(colptr + ck) : 0x7fffffff;
        int32_t cnt = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            int32_t v = __shfl_sync(FULL_MASK, e, cnt + s - 1);
            if (v <= p)
                cnt += s;
        }
        {
            int32_t v = __shfl_sync(FULL_MASK, e, cnt);
            if (v <= p)
                cnt += 1;
        }
        const int32_t colend = __shfl_sync(FULL_MASK, e, cnt & 31);
        const int32_t c0start = __ldg(colptr + c0);
        const int32_t j = valid ? c0 + cnt : -1 - lane;

        double g = 0.0;
        int32_t q = -1;
        if (valid) {
            const int32_t i = __ldcs(rowidx + p);
            const int32_t mj = __ldg(mc + j);
            if (i > mj) {
                ++n_cand;
                const int32_t mi = __ldg(mr + i);
                const int32_t s0 = __ldg(colptr + mi);
                const int32_t s1 = __ldg(colptr + mi + 1);
                q = find_row(rowidx, s0, s1, mj);
                if (q >= 0) {
                    ++n_found;
                    const double wij = __ldcs(w + p);
                    const double wq = __ldg(w + q);
                    g = ((wij + wq) - __ldg(wm + mi)) - __ldg(wm + j);
                    if (g > 0.0) {
                        ++n_pos;
                    } else {
                        g = 0.0;
                        q = -1;
                    }
                }
            }
        }
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
        const int32_t jprev = __shfl_up_sync(FULL_MASK, j, 1);
        const bool head = valid && (lane == 0 || jprev != j);
        if (head) {
            const bool starts_here = (j != c0) || (c0start >= base);
            const bool complete = starts_here && colend <= base + kTile;
            Rec r;
            r.g = g;
            r.p = g > 0.0 ? bp : 0;
            r.q = g > 0.0 ? q : 0;
            if (complete)
                best[j] = r;
            else if (g > 0.0)
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

// Flip every selected cycle: column j takes row i, key column k takes m_j.
// The selected cycles are vertex-disjoint, so each thread owns its four
// vertices.
__global__ void k_flip(int32_t n, const int32_t *__restrict__ rowidx, const double *__restrict__ w,
                       const Rec *__restrict__ best, Sel *dsel, int32_t *mc, int32_t *mr, double *wm,
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
            mc[j] = i;
            mr[i] = j;
            mc[k] = mj;
            mr[mj] = (int32_t)k;
            wm[j] = w[r.p];
            wm[k] = w[r.q];
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

void launch_init(const Work &wk, int max_passes, int num_sms, cudaStream_t s)
{
    const int T = 256;
    cudaMemsetAsync(wk.ctl, 0, sizeof(Ctl), s);
    cudaMemsetAsync(wk.mr, 0xff, sizeof(int32_t) * (size_t)wk.n, s);
    cudaMemsetAsync(wk.starts, 0, sizeof(uint32_t) * (((size_t)wk.nnz + 31) / 32 + 1), s);
    cudaMemsetAsync(wk.best, 0, sizeof(Rec) * (size_t)wk.n, s);
    cudaMemsetAsync(wk.dsel, 0, sizeof(Sel) * (size_t)wk.n, s);
    k_init_ctl<<<1, 1, 0, s>>>(wk.ctl, max_passes);
    k_check_colptr<<<blocks_for((int64_t)wk.n + 1, T), T, 0, s>>>(wk.n, wk.nnz, wk.colptr, wk.ctl);
    k_mark_starts<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.starts, wk.tile_col, wk.ctl);
    int64_t want = ((int64_t)wk.nnz + T - 1) / T;
    int64_t cap = (int64_t)num_sms * 16;
    k_check_entries<<<(unsigned)(want < 1 ? 1 : (want < cap ? want : cap)), T, 0, s>>>(
        wk.n, wk.nnz, wk.rowidx, wk.w, wk.starts, wk.ctl);
    k_init_mates<<<blocks_for(wk.n, T), T, 0, s>>>(wk.n, wk.colptr, wk.rowidx, wk.w, wk.mate_in,
                                                    wk.mc, wk.mr, wk.wm, wk.ctl);
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

void launch_search(const Work &wk, int lookup, int num_sms, cudaStream_t s)
{
    (void)lookup;
    const int T = 256;
    int64_t want = ((int64_t)wk.ntiles + (T / 32) - 1) / (T / 32);
    int64_t cap = (int64_t)num_sms * 8;
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_search<1><<<grid, T, 0, s>>>(wk.n, wk.nnz, wk.ntiles, wk.colptr, wk.rowidx, wk.w,
                                   wk.tile_col, wk.mc, wk.mr, wk.wm, wk.best, wk.ctl);
}

void launch_select_and_flip(const Work &wk, int num_sms, cudaStream_t s)
{
    const int T = 256;
    int64_t want = ((int64_t)wk.n + T - 1) / T;
    int64_t cap = (int64_t)num_sms * 8;
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    k_select<<<grid, T, 0, s>>>(wk.n, wk.rowidx, wk.mr, wk.best, wk.dsel, wk.ctl);
    k_flip<<<grid, T, 0, s>>>(wk.n, wk.rowidx, wk.w, wk.best, wk.dsel, wk.mc, wk.mr, wk.wm, wk.ctl);
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
