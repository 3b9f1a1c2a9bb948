"""Brute-force reference computations for tiny graphs (test helpers).

Everything here works from a dense view of the matrix and enumerates
exhaustively, independently of how the oracle walks the CSC arrays.
"""
from __future__ import annotations

import itertools

import numpy as np


def dense(g):
    """(W, S): dense weights and structure mask, W[row, col]."""
    n = g.n
    W = np.zeros((n, n), dtype=np.float64)
    S = np.zeros((n, n), dtype=bool)
    for j in range(n):
        for p in range(g.colptr[j], g.colptr[j + 1]):
            W[g.rowidx[p], j] = g.weight[p]
            S[g.rowidx[p], j] = True
    return W, S


def matching_weight(g, mate):
    W, _ = dense(g)
    s = 0.0
    for j in range(g.n):
        s += W[mate[j], j]
    return s


def is_perfect(g, mate):
    _, S = dense(g)
    n = g.n
    mate = np.asarray(mate)
    return (mate.shape == (n,) and sorted(mate.tolist()) == list(range(n))
            and all(S[mate[j], j] for j in range(n)))


def all_perfect_matchings(g):
    """Every perfect matching (as mate arrays, row of each column)."""
    _, S = dense(g)
    n = g.n
    for perm in itertools.permutations(range(n)):
        if all(S[perm[j], j] for j in range(n)):
            yield np.array(perm, dtype=np.int32)


def mwpm_bruteforce(g):
    best, arg = None, None
    for m in all_perfect_matchings(g):
        w = matching_weight(g, m)
        if best is None or w > best:
            best, arg = w, m
    return best, arg


def gain_fixed_order(W, i, j, mj, mi):
    """g(i, j, m_j, m_i) in the fixed left-to-right order of the method."""
    return ((W[i, j] + W[mj, mi]) - W[i, mi]) - W[mj, j]


def positive_4cycles(g, mate):
    """All alternating 4-cycles with positive gain, enumerated over every pair
    of columns (j, k): the cycle uses matched edges (mate[j], j), (mate[k], k)
    and the unmatched edges (mate[k], j), (mate[j], k).  The gain is taken from
    the root whose new row exceeds its matched row (the method's root rule)."""
    W, S = dense(g)
    n = g.n
    out = []
    for j in range(n):
        for k in range(n):
            if j == k:
                continue
            rj, rk = mate[j], mate[k]
            if not (S[rk, j] and S[rj, k]):
                continue
            if rk > rj:   # root j, new row i = rk, key column k
                gval = gain_fixed_order(W, rk, j, rj, k)
                if gval > 0:
                    out.append((j, k, gval))
    return out


def one_pass_bruteforce(g, mate, select=0):
    """One pass of Steps A-D and the flip, restated over the dense matrix with
    sets and sorting: returns (new mate, flipped cycles as (root, key)).
    select=1 replaces Step D by the Pettie-Sanders selection: the Step-C
    winners by gain, descending (equal gains: lower root), each kept when it
    shares no vertex with a cycle kept before."""
    W, S = dense(g)
    n = g.n
    mc = np.array(mate, dtype=np.int64)
    mr = np.empty(n, dtype=np.int64)
    mr[mc] = np.arange(n)
    cands = {}
    for j in range(n):
        for i in range(mc[j] + 1, n):
            if not S[i, j]:
                continue
            k = mr[i]
            if not S[mc[j], k]:
                continue
            gval = gain_fixed_order(W, i, j, mc[j], k)
            if gval > 0:
                cands.setdefault(j, []).append((gval, -i, i, k))
    # Step C: maximum gain per root, lowest row on ties
    cwin = {j: max(lst)[2:] for j, lst in cands.items()}           # j -> (i, k)
    cgain = {j: max(lst)[0] for j, lst in cands.items()}
    if select == 1:
        order = sorted(cwin, key=lambda j: (-cgain[j], j))
        used_cols, used_rows = set(), set()
        new = mc.copy()
        flips = []
        for j in order:
            i, k = cwin[j]
            verts_c, verts_r = {j, k}, {i, mc[j]}
            if verts_c & used_cols or verts_r & used_rows:
                continue
            used_cols |= verts_c
            used_rows |= verts_r
            r = mc[j]
            new[j] = i
            new[k] = r
            flips.append((j, k))
        return new.astype(np.int32), sorted(flips)
    # Step D: drop if key is a Step-C root; maximum gain per key, lowest root on ties
    bykey = {}
    for j, (i, k) in cwin.items():
        if k in cwin:
            continue
        bykey.setdefault(k, []).append((cgain[j], -j, j, i))
    new = mc.copy()
    flips = []
    for k, lst in bykey.items():
        _, _, j, i = max(lst)
        r = mc[j]
        new[j] = i
        new[k] = r
        flips.append((j, k))
    return new.astype(np.int32), sorted(flips)


def no_positive_4cycle_vectorized(g, mate):
    """Local optimality for larger graphs: True iff no stored (i, j) with
    i > mate[j] closes (via (mate[j], mate^-1[i])) a cycle of positive gain."""
    n = g.n
    cp = g.colptr.astype(np.int64)
    col = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp))
    row = g.rowidx.astype(np.int64)
    keys = col * n + row
    mc = np.asarray(mate, dtype=np.int64)
    mr = np.empty(n, dtype=np.int64)
    mr[mc] = np.arange(n)
    wm = g.weight[np.searchsorted(keys, np.arange(n, dtype=np.int64) * n + mc)]
    sel = row > mc[col]
    j = col[sel]
    i = row[sel]
    wij = g.weight[sel]
    k = mr[i]
    qk = k * n + mc[j]
    pos = np.searchsorted(keys, qk)
    pos = np.minimum(pos, keys.size - 1)
    found = keys[pos] == qk
    gain = ((wij[found] + g.weight[pos[found]]) - wm[k[found]]) - wm[j[found]]
    return not np.any(gain > 0)


def greedy_sequential(g):
    """Textbook greedy: stored entries from heaviest to lightest (equal
    weights: lower row, then lower column), each kept when its row and its
    column are both free.  Returns mate[j] (row or -1)."""
    col = np.repeat(np.arange(g.n), np.diff(g.colptr))
    order = sorted(range(len(g.rowidx)),
                   key=lambda p: (-float(g.weight[p]), int(g.rowidx[p]), int(col[p])))
    mate = np.full(g.n, -1, dtype=np.int64)
    row_used = np.zeros(g.n, dtype=bool)
    for p in order:
        i, j = int(g.rowidx[p]), int(col[p])
        if mate[j] < 0 and not row_used[i]:
            mate[j] = i
            row_used[i] = True
    return mate


def is_maximal_matching(g, mate):
    """A matching over stored entries that no stored entry between a free
    row and a free column could extend."""
    rows = [int(r) for r in mate if r >= 0]
    if len(rows) != len(set(rows)):
        return False
    free_row = np.ones(g.n, dtype=bool)
    free_row[rows] = False
    for j in range(g.n):
        seg = g.rowidx[g.colptr[j]:g.colptr[j + 1]]
        if mate[j] >= 0:
            if mate[j] not in seg:
                return False
        elif np.any(free_row[seg]):
            return False
    return True
