/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the weight-increasing
 * alternating 4-cycle algorithm (WIAC) of Azad, Buluc, Li, Wang and Langguth,
 * "A distributed-memory algorithm for computing a heavy-weight perfect matching
 * on bipartite graphs" (arXiv 1801.09809), Section 5.3, Algorithms 2-6, in
 * double precision.  Only the test suite, the package's smoke check and the
 * CPU baseline of the benchmark may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Conventions.  The matrix is n x n in CSC: colptr[n+1], rowidx[nnz] (rows
 * strictly increasing inside a column), w[nnz].  Row and column vertices are
 * both numbered 0..n-1.  mc[j] is the row matched to column j (m_j in the
 * paper), mr[i] the column matched to row i (m_i), wm[j] = w(mc[j], j), the
 * weight of the matched edge owned by column j.  A matched edge is named by
 * its column.
 *
 * Readings of the paper (where it is silent or ambiguous):
 *   - cycles are rooted at columns j and use only rows i > m_j (Section 5.3
 *     text and Algorithm 3), not all i != m_j of Algorithm 1;
 *   - the gain is evaluated left to right in IEEE double,
 *       g = ((w(i,j) + w(m_j,m_i)) - w(i,m_i)) - w(m_j,j)      (Section 3),
 *     and a cycle qualifies only if g > 0 (Algorithm 4), no epsilon;
 *   - Step C (Algorithm 5) keeps, per root column j, the maximum gain; equal
 *     gains go to the lowest row i;
 *   - Step D (Algorithm 6) drops every Step-C winner whose second matched
 *     edge {i, m_i} (column k = m_i) is itself the root edge of some Step-C
 *     winner -- whether or not that winner later survives -- and keeps, per
 *     remaining key column k, the maximum gain; equal gains go to the lowest
 *     root column j;
 *   - Algorithm 2 loops while a cycle was found: `iterations` counts passes of
 *     Steps A-D including the last one that found nothing; max_iters = 0
 *     means "until nothing is found" (with a cap of ORACLE_PASS_CAP passes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PASS_CAP 65536

/* error codes (same meaning as the library's, defined independently) */
#define OR_OK 0
#define OR_INVALID_ARG 1
#define OR_NOT_PERFECT 2
#define OR_UNSORTED_OR_DUP 3
#define OR_NONFINITE 4
#define OR_OOM 5

typedef struct {
    int32_t iterations;      /* passes of Steps A-D executed */
    int32_t converged;       /* 1 if the last pass found no weight-increasing cycle */
    int64_t cycles_applied;  /* cycles flipped in total */
    int64_t edge_checks;     /* (nnz - n) per pass */
    int64_t candidates;      /* A-requests: entries (i, j) with i > m_j */
    int64_t closing_found;   /* A-requests whose closing edge {m_j, m_i} exists */
    int64_t positive;        /* B-requests: closing edge exists and g > 0 */
    double weight_in;        /* sum over j of w(m_j, j), ascending j */
    double weight_out;
} oracle_stats;

/* One A-request of Algorithm 3, carrying the cycle's four vertices. */
typedef struct {
    int32_t i, j, mj, mi;
    double wij;
} a_request;

/* One B-request of Algorithm 4 (the closing weight rides along for the flip). */
typedef struct {
    int32_t i, j, mj, mi;
    double g;
    double wij, wq;
} b_request;

/* Position of entry (row, col) in the CSC arrays, or -1.  Linear scan. */
static int64_t find_entry(const int32_t *colptr, const int32_t *rowidx, int32_t row, int32_t col)
{
    for (int64_t p = colptr[col]; p < colptr[col + 1]; ++p)
        if (rowidx[p] == row)
            return p;
    return -1;
}

/*
 * Input checks, in priority order: malformed arguments or column pointers or
 * out-of-range rows (INVALID_ARG), rows not strictly increasing in a column
 * (UNSORTED_OR_DUP), non-finite weights (NONFINITE), matching not a perfect
 * matching over stored entries (NOT_PERFECT).
 */
/* The checks on the matrix alone (no matching), in the same priority order. */
static int validate_matrix(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                           const double *w)
{
    if (n < 0 || (n > 0 && !colptr))
        return OR_INVALID_ARG;
    if (n == 0)
        return OR_OK;
    if (colptr[0] != 0)
        return OR_INVALID_ARG;
    for (int32_t j = 0; j < n; ++j)
        if (colptr[j + 1] < colptr[j])
            return OR_INVALID_ARG;
    int64_t nnz = colptr[n];
    if (nnz > 0 && (!rowidx || !w))
        return OR_INVALID_ARG;
    for (int64_t p = 0; p < nnz; ++p)
        if (rowidx[p] < 0 || rowidx[p] >= n)
            return OR_INVALID_ARG;
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j] + 1; p < colptr[j + 1]; ++p)
            if (rowidx[p] <= rowidx[p - 1])
                return OR_UNSORTED_OR_DUP;
    for (int64_t p = 0; p < nnz; ++p)
        if (!isfinite(w[p]))
            return OR_NONFINITE;
    return OR_OK;
}

int oracle_validate(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                    const int32_t *mate)
{
    if (n < 0 || (n > 0 && (!colptr || !mate)))
        return OR_INVALID_ARG;
    int rc0 = validate_matrix(n, colptr, rowidx, w);
    if (rc0 != OR_OK || n == 0)
        return rc0;
    char *seen = (char *)calloc((size_t)n, 1);
    if (!seen)
        return OR_OOM;
    int rc = OR_OK;
    for (int32_t j = 0; j < n && rc == OR_OK; ++j) {
        int32_t r = mate[j];
        if (r < 0 || r >= n || seen[r] || find_entry(colptr, rowidx, r, j) < 0)
            rc = OR_NOT_PERFECT;
        else
            seen[r] = 1;
    }
    free(seen);
    return rc;
}

/* Sum of the matched weights, ascending column order. */
static double matching_weight(int32_t n, const double *wm)
{
    double s = 0.0;
    for (int32_t j = 0; j < n; ++j)
        s += wm[j];
    return s;
}

/*
 * One iteration of Algorithm 2: Steps A, B, C and D, then the flip.
 * mc, mr, wm are updated in place.  Optional outputs (NULL to skip):
 *   stepc_gain[j], stepc_row[j]: the Step-C winner rooted at column j
 *       (gain, row i), or (0, -1) if column j sent no C-request;
 *   stepd_root[k]: root column j of the cycle that won key column k in Step D
 *       and was flipped, or -1;
 *   counts[4]: candidates, closing_found, positive, flipped for this pass.
 * Returns the number of cycles flipped, or -1 on allocation failure.
 */
/* One Step-C winner in the order of the Pettie-Sanders selection. */
typedef struct {
    double g;
    int32_t j;
    int64_t x;  /* its B-request */
} ps_item;

/* gain descending, then root column ascending */
static int ps_cmp(const void *a, const void *b)
{
    const ps_item *p = (const ps_item *)a, *q = (const ps_item *)b;
    if (p->g > q->g)
        return -1;
    if (p->g < q->g)
        return 1;
    return (p->j > q->j) - (p->j < q->j);
}

/*
 * Row marking (Section 4): the neighbourhood of row m_j -- the columns k with
 * a stored (m_j, k) -- is marked once per root column j, and each candidate i
 * of j then finds its closing entry (m_j, m_i) by reading the mark of column
 * m_i.  The rows' neighbourhoods come from the transpose of the matrix (CSR),
 * built here by a counting sort of the entries by row, which keeps each row's
 * columns ascending.  rowptr[n+1]; rowpos[nnz], rowcol[nnz]: position in the
 * CSC arrays and column of each entry, row by row.
 */
static int transpose_by_rows(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                             int64_t **rowptr_out, int64_t **rowpos_out, int32_t **rowcol_out)
{
    int64_t nnz = n > 0 ? colptr[n] : 0;
    int64_t *rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *rowpos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *rowcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!rowptr || !rowpos || !rowcol || !fill) {
        free(rowptr); free(rowpos); free(rowcol); free(fill);
        return -1;
    }
    for (int64_t p = 0; p < nnz; ++p)
        rowptr[rowidx[p] + 1] += 1;
    for (int32_t i = 0; i < n; ++i)
        rowptr[i + 1] += rowptr[i];
    for (int32_t i = 0; i < n; ++i)
        fill[i] = rowptr[i];
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            rowpos[fill[rowidx[p]]] = p;
            rowcol[fill[rowidx[p]]++] = j;
        }
    free(fill);
    *rowptr_out = rowptr;
    *rowpos_out = rowpos;
    *rowcol_out = rowcol;
    return 0;
}

/*
 * select_mode bit 0 clear: Step D as in Algorithm 6 (above).
 * select_mode bit 0 set: the Pettie-Sanders selection the paper describes in
 * Section 4 instead of Step D: the Step-C winners S sorted by gain,
 * descending (equal gains: lower root column first), each added to D(S)
 * when none of its four vertices (columns j and k = m_i, rows i and m_j)
 * belongs to a cycle added before.
 * select_mode bit 1 set: Step B finds the closing entries by row marking
 * (above) instead of searching column m_i; the entries found, and so every
 * result, are the same.
 */
int64_t oracle_pass_mode(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                         int32_t *mc, int32_t *mr, double *wm, double *stepc_gain,
                         int32_t *stepc_row, int32_t *stepd_root, int64_t *counts,
                         int32_t select_mode)
{
    int64_t nnz = n > 0 ? colptr[n] : 0;
    a_request *areq = (a_request *)malloc(sizeof(a_request) * (size_t)(nnz > 0 ? nnz : 1));
    b_request *breq = (b_request *)malloc(sizeof(b_request) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *cwin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *dwin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!areq || !breq || !cwin || !dwin) {
        free(areq); free(breq); free(cwin); free(dwin);
        return -1;
    }
    int64_t na = 0, nb = 0, nfound = 0;
    const int row_marking = (select_mode & 2) != 0;
    select_mode &= 1;
    int64_t *rowptr = NULL, *rowpos = NULL, *mark_pos = NULL;
    int32_t *rowcol = NULL, *mark_root = NULL;
    if (row_marking) {
        mark_pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        mark_root = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!mark_pos || !mark_root || transpose_by_rows(n, colptr, rowidx, &rowptr, &rowpos, &rowcol)) {
            free(mark_pos); free(mark_root);
            free(areq); free(breq); free(cwin); free(dwin);
            return -1;
        }
        for (int32_t k = 0; k < n; ++k)
            mark_root[k] = -1;
    }

    /* Step A (Algorithm 3): every stored (i, j) with i > m_j asks the owner of
     * {m_j, m_i} to close the cycle i - j - m_j - m_i. */
    for (int32_t j = 0; j < n; ++j) {
        int32_t mj = mc[j];
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int32_t i = rowidx[p];
            if (i > mj) {
                a_request a;
                a.i = i;
                a.j = j;
                a.mj = mj;
                a.mi = mr[i];
                a.wij = w[p];
                areq[na++] = a;
            }
        }
    }

    /* Step B (Algorithm 4): if {m_j, m_i} exists, compute the gain
     *   g(i,j,m_j,m_i) = w(i,j) + w(m_i,m_j) - w(i,m_i) - w(m_j,j)
     * and forward positive ones.  w(i, m_i) is the matched weight of column m_i,
     * w(m_j, j) the matched weight of column j. */
    for (int64_t x = 0; x < na; ++x) {
        a_request a = areq[x];
        int64_t q;
        if (row_marking) {
            /* the A-requests come grouped by root column: mark row m_j's
             * neighbourhood when a new root starts */
            if (x == 0 || areq[x - 1].j != a.j)
                for (int64_t t = rowptr[a.mj]; t < rowptr[a.mj + 1]; ++t) {
                    mark_pos[rowcol[t]] = rowpos[t];
                    mark_root[rowcol[t]] = a.j;
                }
            q = mark_root[a.mi] == a.j ? mark_pos[a.mi] : -1;
        } else {
            q = find_entry(colptr, rowidx, a.mj, a.mi);
        }
        if (q < 0)
            continue;
        ++nfound;
        double wq = w[q];
        double g = a.wij + wq - wm[a.mi] - wm[a.j];
        if (g > 0.0) {
            b_request b;
            b.i = a.i;
            b.j = a.j;
            b.mj = a.mj;
            b.mi = a.mi;
            b.g = g;
            b.wij = a.wij;
            b.wq = wq;
            breq[nb++] = b;
        }
    }

    /* Step C (Algorithm 5): per matched edge {m_j, j}, i.e. per root column j,
     * keep the B-request of maximum gain (equal gains: lowest row i). */
    for (int32_t j = 0; j < n; ++j)
        cwin[j] = -1;
    for (int64_t x = 0; x < nb; ++x) {
        int32_t j = breq[x].j;
        int64_t cur = cwin[j];
        if (cur < 0 || breq[x].g > breq[cur].g ||
            (breq[x].g == breq[cur].g && breq[x].i < breq[cur].i))
            cwin[j] = x;
    }

    /* Step D (Algorithm 6): per matched edge {i, m_i}, i.e. per key column
     * k = m_i, keep the C-request of maximum gain (equal gains: lowest root j);
     * a C-request whose key column k itself sent a C-request is dropped. */
    for (int32_t k = 0; k < n; ++k)
        dwin[k] = -1;
    if (select_mode == 0) {
        for (int32_t j = 0; j < n; ++j) {
            if (cwin[j] < 0)
                continue;
            b_request *c = &breq[cwin[j]];
            int32_t k = c->mi;
            if (cwin[k] >= 0)
                continue;
            int64_t cur = dwin[k];
            if (cur < 0 || c->g > breq[cur].g || (c->g == breq[cur].g && c->j < breq[cur].j))
                dwin[k] = cwin[j];
        }
    } else {
        int64_t ns = 0;
        ps_item *items = (ps_item *)malloc(sizeof(ps_item) * (size_t)(n > 0 ? n : 1));
        char *used_col = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
        char *used_row = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
        if (!items || !used_col || !used_row) {
            free(items); free(used_col); free(used_row);
            free(areq); free(breq); free(cwin); free(dwin);
            return -1;
        }
        for (int32_t j = 0; j < n; ++j)
            if (cwin[j] >= 0) {
                items[ns].g = breq[cwin[j]].g;
                items[ns].j = j;
                items[ns].x = cwin[j];
                ++ns;
            }
        qsort(items, (size_t)ns, sizeof(ps_item), ps_cmp);
        for (int64_t t = 0; t < ns; ++t) {
            b_request *c = &breq[items[t].x];
            if (used_col[c->j] || used_col[c->mi] || used_row[c->i] || used_row[c->mj])
                continue;
            used_col[c->j] = used_col[c->mi] = 1;
            used_row[c->i] = used_row[c->mj] = 1;
            dwin[c->mi] = items[t].x;
        }
        free(items);
        free(used_col);
        free(used_row);
    }

    if (stepc_gain || stepc_row) {
        for (int32_t j = 0; j < n; ++j) {
            if (stepc_gain)
                stepc_gain[j] = cwin[j] >= 0 ? breq[cwin[j]].g : 0.0;
            if (stepc_row)
                stepc_row[j] = cwin[j] >= 0 ? breq[cwin[j]].i : -1;
        }
    }

    /* Flip M := M xor {cycle}: column j takes row i, column k = m_i takes row m_j. */
    int64_t flipped = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (stepd_root)
            stepd_root[k] = dwin[k] >= 0 ? breq[dwin[k]].j : -1;
        if (dwin[k] < 0)
            continue;
        b_request c = breq[dwin[k]];
        mc[c.j] = c.i;
        mr[c.i] = c.j;
        mc[c.mi] = c.mj;
        mr[c.mj] = c.mi;
        wm[c.j] = c.wij;
        wm[c.mi] = c.wq;
        ++flipped;
    }

    if (counts) {
        counts[0] = na;
        counts[1] = nfound;
        counts[2] = nb;
        counts[3] = flipped;
    }
    free(rowptr);
    free(rowpos);
    free(rowcol);
    free(mark_pos);
    free(mark_root);
    free(areq);
    free(breq);
    free(cwin);
    free(dwin);
    return flipped;
}

int64_t oracle_pass(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                    int32_t *mc, int32_t *mr, double *wm,
                    double *stepc_gain, int32_t *stepc_row, int32_t *stepd_root, int64_t *counts)
{
    return oracle_pass_mode(n, colptr, rowidx, w, mc, mr, wm, stepc_gain, stepc_row, stepd_root,
                            counts, 0);
}

/*
 * Whole phase (Algorithm 2): initialise mates and matched weights from
 * mate_in, run passes until one finds nothing (or max_iters passes ran),
 * write the final matching to mate_out (may alias mate_in).
 * trace_weight / trace_flips (capacity trace_cap, may be NULL) receive the
 * matching weight and the number of cycles flipped after each pass.
 */
int oracle_improve_mode(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                        const int32_t *mate_in, int32_t *mate_out, int32_t max_iters,
                        oracle_stats *st, double *trace_weight, int64_t *trace_flips,
                        int32_t trace_cap, int32_t select_mode)
{
    oracle_stats s;
    memset(&s, 0, sizeof(s));
    int rc = oracle_validate(n, colptr, rowidx, w, mate_in);
    if (rc != OR_OK)
        return rc;
    if (max_iters < 0)
        return OR_INVALID_ARG;
    int32_t nn = n > 0 ? n : 1;
    int32_t *mc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    int32_t *mr = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    double *wm = (double *)malloc(sizeof(double) * (size_t)nn);
    if (!mc || !mr || !wm) {
        free(mc); free(mr); free(wm);
        return OR_OOM;
    }
    /* Initialisation (Algorithm 2, before the loop): every owner learns the
     * mates and the matched weights. */
    for (int32_t j = 0; j < n; ++j) {
        mc[j] = mate_in[j];
        mr[mate_in[j]] = j;
        wm[j] = w[find_entry(colptr, rowidx, mate_in[j], j)];
    }
    s.weight_in = matching_weight(n, wm);
    int64_t nnz = n > 0 ? colptr[n] : 0;
    int32_t cap = max_iters > 0 ? max_iters : ORACLE_PASS_CAP;
    for (int32_t it = 1; it <= cap; ++it) {
        int64_t counts[4];
        int64_t f = oracle_pass_mode(n, colptr, rowidx, w, mc, mr, wm, NULL, NULL, NULL, counts,
                                     select_mode);
        if (f < 0) {
            rc = OR_OOM;
            break;
        }
        s.iterations = it;
        s.edge_checks += nnz - n;
        s.candidates += counts[0];
        s.closing_found += counts[1];
        s.positive += counts[2];
        s.cycles_applied += f;
        if (trace_weight && it <= trace_cap)
            trace_weight[it - 1] = matching_weight(n, wm);
        if (trace_flips && it <= trace_cap)
            trace_flips[it - 1] = f;
        if (f == 0) {
            s.converged = 1;
            break;
        }
    }
    s.weight_out = matching_weight(n, wm);
    if (rc == OR_OK)
        for (int32_t j = 0; j < n; ++j)
            mate_out[j] = mc[j];
    if (st)
        *st = s;
    free(mc);
    free(mr);
    free(wm);
    return rc;
}

int oracle_improve(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                   const int32_t *mate_in, int32_t *mate_out, int32_t max_iters,
                   oracle_stats *st, double *trace_weight, int64_t *trace_flips, int32_t trace_cap)
{
    return oracle_improve_mode(n, colptr, rowidx, w, mate_in, mate_out, max_iters, st,
                               trace_weight, trace_flips, trace_cap, 0);
}

/*
 * Step-C records of one pass from a given matching, without flipping
 * (Algorithms 3-5): stepc_gain[j], stepc_row[j] as in oracle_pass.
 */
int oracle_step_c(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                  const int32_t *mate, double *stepc_gain, int32_t *stepc_row, int64_t *counts)
{
    int rc = oracle_validate(n, colptr, rowidx, w, mate);
    if (rc != OR_OK)
        return rc;
    int32_t nn = n > 0 ? n : 1;
    int32_t *mc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    int32_t *mr = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    double *wm = (double *)malloc(sizeof(double) * (size_t)nn);
    if (!mc || !mr || !wm) {
        free(mc); free(mr); free(wm);
        return OR_OOM;
    }
    for (int32_t j = 0; j < n; ++j) {
        mc[j] = mate[j];
        mr[mate[j]] = j;
        wm[j] = w[find_entry(colptr, rowidx, mate[j], j)];
    }
    int64_t f = oracle_pass(n, colptr, rowidx, w, mc, mr, wm, stepc_gain, stepc_row, NULL, counts);
    free(mc);
    free(mr);
    free(wm);
    return f < 0 ? OR_OOM : OR_OK;
}

/*
 * Heavy-weight greedy maximal matching: the maximal matching that starts the
 * paper's pipeline (Section 5.1), with its heavy-weight preference ("we
 * select edges with heavy weights when greedily selecting edges").
 *
 * Reading: greedy takes the stored entries from heaviest to lightest (equal
 * weights: lower row first, then lower column) and keeps every entry whose
 * row and column are both still unmatched.  It is computed here in rounds, as
 * a parallel machine computes it: in each round every unmatched column names
 * its first entry in that order among the entries with an unmatched row,
 * every unmatched row names its first entry among the entries with an
 * unmatched column, and the entries named by both their row and their column
 * are matched.  The first remaining entry overall is always named twice, so
 * every round but the last matches at least one entry; the last round
 * matches none and the matching is maximal.  `rounds` counts all rounds,
 * the last one included.
 *
 * mate_out[j]: the row matched to column j, or -1.
 */
typedef struct {
    int32_t rounds;
    int32_t cardinality;   /* matched columns */
    double weight;         /* sum of the matched weights, ascending column order */
} oracle_greedy_stats;

int oracle_greedy(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
                  int32_t *mate_out, oracle_greedy_stats *st)
{
    int rc = validate_matrix(n, colptr, rowidx, w);
    if (rc != OR_OK)
        return rc;
    if (!mate_out && n > 0)
        return OR_INVALID_ARG;
    int32_t nn = n > 0 ? n : 1;
    int32_t *mc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);   /* row of column */
    int32_t *mr = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);   /* column of row */
    int64_t *cbest = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn); /* position, or -1 */
    int32_t *rbest = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn); /* column, or -1 */
    double *rbw = (double *)malloc(sizeof(double) * (size_t)nn);      /* its weight */
    if (!mc || !mr || !cbest || !rbest || !rbw) {
        free(mc); free(mr); free(cbest); free(rbest); free(rbw);
        return OR_OOM;
    }
    for (int32_t x = 0; x < n; ++x) {
        mc[x] = -1;
        mr[x] = -1;
    }
    oracle_greedy_stats s;
    memset(&s, 0, sizeof(s));
    for (;;) {
        s.rounds += 1;
        /* every unmatched column: its first entry with an unmatched row
         * (rows ascend in a column, so a strictly heavier weight wins) */
        for (int32_t j = 0; j < n; ++j) {
            cbest[j] = -1;
            if (mc[j] >= 0)
                continue;
            for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                if (mr[rowidx[p]] >= 0)
                    continue;
                if (cbest[j] < 0 || w[p] > w[cbest[j]])
                    cbest[j] = p;
            }
        }
        /* every unmatched row: its first entry with an unmatched column
         * (columns are visited in ascending order) */
        for (int32_t i = 0; i < n; ++i)
            rbest[i] = -1;
        for (int32_t j = 0; j < n; ++j) {
            if (mc[j] >= 0)
                continue;
            for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                int32_t i = rowidx[p];
                if (mr[i] >= 0)
                    continue;
                if (rbest[i] < 0 || w[p] > rbw[i]) {
                    rbest[i] = j;
                    rbw[i] = w[p];
                }
            }
        }
        /* entries named by both ends are matched */
        int32_t matched = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (cbest[j] < 0)
                continue;
            int32_t i = rowidx[cbest[j]];
            if (rbest[i] == j) {
                mc[j] = i;
                mr[i] = j;
                ++matched;
            }
        }
        s.cardinality += matched;
        if (matched == 0)
            break;
    }
    double total = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        mate_out[j] = mc[j];
        if (mc[j] >= 0)
            total += w[find_entry(colptr, rowidx, mc[j], j)];
    }
    s.weight = total;
    if (st)
        *st = s;
    free(mc); free(mr); free(cbest); free(rbest); free(rbw);
    return OR_OK;
}

/*
 * Matching weights from matrix values (Section 6.1, the experiments' setup):
 * the matrix is equilibrated by diagonal scaling so that the largest
 * magnitude in every row and column is at most 1 -- here one sweep, columns
 * first (each column divided by its largest |a|), then rows (each row divided
 * by its largest scaled magnitude), so every row's largest entry is exactly 1
 * -- and the weight is the scaled magnitude (mode 0, Option A: maximise the
 * sum) or its logarithm (mode 1, Option B: maximise the product).
 *   v_ij = |a_ij| / max_k |a_kj|,  w_ij = v_ij / max_l v_il,  mode 1: log(w_ij)
 * Values must be finite and nonzero (the paper removes explicit zeros).
 */
int oracle_weights(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *a,
                   int32_t mode, double *w)
{
    if (n < 0 || (n > 0 && !colptr) || (mode != 0 && mode != 1))
        return OR_INVALID_ARG;
    if (n == 0)
        return OR_OK;
    if (colptr[0] != 0)
        return OR_INVALID_ARG;
    for (int32_t j = 0; j < n; ++j)
        if (colptr[j + 1] < colptr[j])
            return OR_INVALID_ARG;
    int64_t nnz = colptr[n];
    if (nnz > 0 && (!rowidx || !a || !w))
        return OR_INVALID_ARG;
    for (int64_t p = 0; p < nnz; ++p)
        if (rowidx[p] < 0 || rowidx[p] >= n)
            return OR_INVALID_ARG;
    for (int64_t p = 0; p < nnz; ++p)
        if (!isfinite(a[p]) || a[p] == 0.0)
            return OR_NONFINITE;
    double *cmax = (double *)calloc((size_t)n, sizeof(double));
    double *rmax = (double *)calloc((size_t)n, sizeof(double));
    if (!cmax || !rmax) {
        free(cmax);
        free(rmax);
        return OR_OOM;
    }
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p)
            if (fabs(a[p]) > cmax[j])
                cmax[j] = fabs(a[p]);
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            double v = fabs(a[p]) / cmax[j];
            if (v > rmax[rowidx[p]])
                rmax[rowidx[p]] = v;
        }
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            double v = fabs(a[p]) / cmax[j];
            double x = v / rmax[rowidx[p]];
            w[p] = mode == 0 ? x : log(x);
        }
    free(cmax);
    free(rmax);
    return OR_OK;
}

/*
 * Maximum cardinality matching with the heavy-weight tie-break (Section 5.2):
 * augmenting paths searched from all free columns at once, breadth first,
 * choosing heavier edges when several searches reach the same row.
 *
 * Reading (the paper gives the idea, not the steps): phases; in each phase
 * every free column roots a search tree and the trees grow level by level.
 * At a level every frontier column offers each of its rows that no tree has
 * reached yet (through an unmatched edge); a row offered by several columns
 * joins the tree of the column with the heaviest edge (equal weights: lower
 * column).  A row so reached that is free ends an augmenting path of its
 * tree; a tree takes, among the free rows it reaches at that level, the one
 * with the heaviest last edge (equal weights: lower row) and stops growing.
 * A reached row that is matched brings its matched column into the next
 * frontier of its tree.  When no frontier remains, every tree with an end
 * is augmented along its path (the trees are vertex-disjoint).  A phase that
 * augments nothing ends the algorithm: no augmenting path is left, so the
 * matching is maximum (Berge).
 *
 * mate[n] in/out: row of column j or -1 (a valid matching on entry).
 */
typedef struct {
    int32_t phases;        /* phases run, the last one (augmenting nothing) included */
    int32_t cardinality;
} oracle_mcm_stats;

int oracle_mcm(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *w,
               int32_t *mate, oracle_mcm_stats *st)
{
    int rc = validate_matrix(n, colptr, rowidx, w);
    if (rc != OR_OK)
        return rc;
    if (n > 0 && !mate)
        return OR_INVALID_ARG;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *mc = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *mr = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *root = (int32_t *)malloc(sizeof(int32_t) * nn);    /* tree of a column */
    int32_t *rpar = (int32_t *)malloc(sizeof(int32_t) * nn);    /* column that reached a row */
    int32_t *front = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *tend = (int32_t *)malloc(sizeof(int32_t) * nn);    /* end row of a tree, or -1 */
    double *tw = (double *)malloc(sizeof(double) * nn);         /* its last edge's weight */
    int32_t *bestc = (int32_t *)malloc(sizeof(int32_t) * nn);   /* level: winning column */
    double *bestw = (double *)malloc(sizeof(double) * nn);      /* level: its weight */
    if (!mc || !mr || !root || !rpar || !front || !next || !tend || !tw || !bestc || !bestw) {
        rc = OR_OOM;
        goto out;
    }
    for (int32_t x = 0; x < n; ++x)
        mr[x] = -1;
    for (int32_t j = 0; j < n; ++j) {
        int32_t r = mate[j];
        if (r >= n || (r >= 0 && (mr[r] != -1 || find_entry(colptr, rowidx, r, j) < 0))) {
            rc = OR_NOT_PERFECT;   /* not a matching over stored entries */
            goto out;
        }
        mc[j] = r < 0 ? -1 : r;
        if (r >= 0)
            mr[r] = j;
    }
    oracle_mcm_stats S;
    memset(&S, 0, sizeof(S));
    for (;;) {
        S.phases += 1;
        int32_t nf = 0;
        for (int32_t x = 0; x < n; ++x) {
            rpar[x] = -1;
            tend[x] = -1;
            bestc[x] = -1;
            if (mc[x] < 0) {
                root[x] = x;
                front[nf++] = x;
            }
        }
        while (nf > 0) {
            /* offers: for every row not yet reached, the heaviest offering
             * edge, then the lowest column (frontier columns in any order) */
            for (int32_t f = 0; f < nf; ++f) {
                int32_t c = front[f];
                for (int64_t p = colptr[c]; p < colptr[c + 1]; ++p) {
                    int32_t r = rowidx[p];
                    if (r == mc[c] || rpar[r] != -1)
                        continue;
                    if (bestc[r] < 0 || w[p] > bestw[r] || (w[p] == bestw[r] && c < bestc[r])) {
                        bestc[r] = c;
                        bestw[r] = w[p];
                    }
                }
            }
            /* rows join the winning column's tree */
            int32_t nn2 = 0;
            for (int32_t f = 0; f < nf; ++f) {
                int32_t c = front[f];
                for (int64_t p = colptr[c]; p < colptr[c + 1]; ++p) {
                    int32_t r = rowidx[p];
                    if (bestc[r] != c || rpar[r] != -1)
                        continue;
                    rpar[r] = c;
                    bestc[r] = -1;
                    int32_t t = root[c];
                    if (mr[r] < 0) {
                        if (tend[t] < 0 || w[p] > tw[t] || (w[p] == tw[t] && r < tend[t])) {
                            tend[t] = r;
                            tw[t] = w[p];
                        }
                    } else {
                        int32_t c2 = mr[r];
                        root[c2] = t;
                        next[nn2++] = c2;
                    }
                }
            }
            /* trees with an end stop growing */
            nf = 0;
            for (int32_t f = 0; f < nn2; ++f)
                if (tend[root[next[f]]] < 0)
                    front[nf++] = next[f];
        }
        int32_t aug = 0;
        for (int32_t t = 0; t < n; ++t) {
            if (mc[t] >= 0 || tend[t] < 0)
                continue;
            int32_t r = tend[t];
            for (;;) {
                int32_t c = rpar[r];
                int32_t old = mc[c];
                mc[c] = r;
                mr[r] = c;
                if (old < 0)
                    break;
                r = old;
            }
            ++aug;
        }
        if (aug == 0)
            break;
    }
    S.cardinality = 0;
    for (int32_t j = 0; j < n; ++j) {
        mate[j] = mc[j];
        S.cardinality += mc[j] >= 0;
    }
    if (st)
        *st = S;
out:
    free(mc); free(mr); free(root); free(rpar); free(front); free(next);
    free(tend); free(tw); free(bestc); free(bestw);
    return rc;
}

