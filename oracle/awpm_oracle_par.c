/*
 * CPU ORACLE, MULTI-THREADED RESTATEMENT -- TEST AND BASELINE INFRASTRUCTURE
 * ONLY.
 *
 * The weight-increasing alternating 4-cycle phase of arXiv 1801.09809
 * (Section 5.3, Algorithms 2-6) on all host cores with OpenMP, the paper's
 * own shared-memory setting.  It is the CPU timing baseline beside the
 * single-threaded oracle (awpm_oracle.c), not a second source of truth: the
 * test suite requires its results to equal that oracle's, bit for bit.  Only
 * the test suite and the benchmark's CPU-baseline leg load it.  It shares no
 * code with the CUDA library.
 *
 * Per pass, Steps A, B and C (Algorithms 3-5) are one loop over root columns
 * j, split among threads: each column's candidates (rows i > m_j, ascending)
 * look their closing entry {m_j, m_i} up by binary search in the sorted rows
 * of column m_i, evaluate g = ((w(i,j) + w(m_j,m_i)) - w(i,m_i)) - w(m_j,j)
 * left to right, and keep the largest positive gain (the first of equal
 * gains, i.e. the lowest row).  Step D (Algorithm 6) and the flip read and
 * write the matching of other columns, so they stay sequential, in
 * ascending root order: a winner whose key column k = m_i is itself the root
 * of a Step-C winner is dropped, and per key the largest gain wins (equal
 * gains: the lowest root).  These are the readings of the single-threaded
 * oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PAR_OK 0
#define PAR_INVALID 1
#define PAR_NOT_PERFECT 2
#define PAR_OOM 5
#define PAR_PASS_CAP 65536

typedef struct {
    int32_t iterations;
    int32_t converged;
    int64_t cycles_applied;
    int64_t edge_checks;
    int64_t candidates;
    int64_t closing_found;
    int64_t positive;
    double weight_in;
    double weight_out;
} par_stats;

/* position of `row` among the sorted rows of column `col`, or -1 */
static int64_t bsearch_row(const int32_t *colptr, const int32_t *rowidx, int32_t col, int32_t row)
{
    int64_t lo = colptr[col], hi = colptr[col + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (rowidx[mid] < row)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < colptr[col + 1] && rowidx[lo] == row) ? lo : -1;
}

int oracle_par_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Whole phase from mate_in to mate_out (may alias).  The input must be valid
 * (the single-threaded oracle's validation is the reference for that); only
 * the matching is checked here.  threads <= 0: all available.
 */
int oracle_par_improve(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                       const int32_t *mate_in, int32_t *mate_out, int32_t max_iters,
                       int32_t threads, par_stats *st)
{
    if (n < 0 || max_iters < 0 || !colptr || !mate_in || !mate_out || !st)
        return PAR_INVALID;
    memset(st, 0, sizeof(*st));
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#endif
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *mc = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *mr = (int32_t *)malloc(sizeof(int32_t) * nn);
    double *wm = (double *)malloc(sizeof(double) * nn);
    double *cg = (double *)malloc(sizeof(double) * nn);   /* Step-C gain per root */
    int64_t *cp = (int64_t *)malloc(sizeof(int64_t) * nn); /* position of (i, j) */
    int64_t *cq = (int64_t *)malloc(sizeof(int64_t) * nn); /* closing entry */
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * nn); /* row i, or -1 */
    int32_t *dw = (int32_t *)malloc(sizeof(int32_t) * nn); /* Step-D root per key */
    int rc = PAR_OK;
    if (!mc || !mr || !wm || !cg || !cp || !cq || !ci || !dw) {
        rc = PAR_OOM;
        goto done;
    }
    for (int32_t i = 0; i < n; ++i)
        mr[i] = -1;
    for (int32_t j = 0; j < n; ++j) {
        int32_t r = mate_in[j];
        int64_t q = (r >= 0 && r < n) ? bsearch_row(colptr, rowidx, j, r) : -1;
        if (q < 0 || mr[r] != -1) {
            rc = PAR_NOT_PERFECT;
            goto done;
        }
        mc[j] = r;
        mr[r] = j;
        wm[j] = w[q];
    }
    double win = 0.0;
    for (int32_t j = 0; j < n; ++j)
        win += wm[j];
    st->weight_in = win;
    int32_t cap = max_iters > 0 ? max_iters : PAR_PASS_CAP;
    int64_t nnz = n > 0 ? colptr[n] : 0;
    for (;;) {
        int64_t cand = 0, found = 0, pos = 0;
        /* Steps A-C, one root column per iteration of the parallel loop */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : cand, found, pos)
        for (int32_t j = 0; j < n; ++j) {
            int32_t mj = mc[j];
            double bg = 0.0;
            int32_t bi = -1;
            int64_t bp = -1, bq = -1;
            for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                int32_t i = rowidx[p];
                if (i <= mj)
                    continue;
                ++cand;
                int32_t mi = mr[i];
                int64_t q = bsearch_row(colptr, rowidx, mi, mj);
                if (q < 0)
                    continue;
                ++found;
                double g = w[p] + w[q] - wm[mi] - wm[j];
                if (g > 0.0) {
                    ++pos;
                    if (g > bg) {
                        bg = g;
                        bi = i;
                        bp = p;
                        bq = q;
                    }
                }
            }
            cg[j] = bg;
            ci[j] = bi;
            cp[j] = bp;
            cq[j] = bq;
        }
        st->candidates += cand;
        st->closing_found += found;
        st->positive += pos;
        st->edge_checks += nnz - n;
        st->iterations += 1;
        /* Step D, ascending roots */
        for (int32_t k = 0; k < n; ++k)
            dw[k] = -1;
        for (int32_t j = 0; j < n; ++j) {
            if (ci[j] < 0)
                continue;
            int32_t k = mr[ci[j]];
            if (ci[k] >= 0)
                continue;
            if (dw[k] < 0 || cg[j] > cg[dw[k]])
                dw[k] = j;
        }
        /* flip */
        int64_t flipped = 0;
        for (int32_t k = 0; k < n; ++k) {
            int32_t j = dw[k];
            if (j < 0)
                continue;
            int32_t i = ci[j], mj = mc[j];
            mc[j] = i;
            mr[i] = j;
            mc[k] = mj;
            mr[mj] = k;
            wm[j] = w[cp[j]];
            wm[k] = w[cq[j]];
            ++flipped;
        }
        st->cycles_applied += flipped;
        if (flipped == 0) {
            st->converged = 1;
            break;
        }
        if (st->iterations >= cap)
            break;
    }
    double wout = 0.0;
    for (int32_t j = 0; j < n; ++j)
        wout += wm[j];
    st->weight_out = wout;
    for (int32_t j = 0; j < n; ++j)
        mate_out[j] = mc[j];
done:
    free(mc);
    free(mr);
    free(wm);
    free(cg);
    free(cp);
    free(cq);
    free(ci);
    free(dw);
    return rc;
}
