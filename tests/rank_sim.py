"""A literal simulation of the paper's distributed pass (Section 5.3,
Algorithms 2-6) on a virtual sqrt(p) x sqrt(p) process grid, used to pin the
oracle.

Process (a, b) owns the stored entries whose row lies in row block a and
whose column lies in column block b.  As in the paper, the matching is
replicated: every process of grid row a holds m_i and w(i, m_i) for the rows
i of block a, and every process of grid column b holds m_j and w(m_j, j) for
the columns j of block b.  One pass:

  A  (Alg. 3) each process scans its local entries (i, j) with i > m_j and
     sends an A-request carrying w(i, j) to the owner of {m_j, m_i};
  B  (Alg. 4) the owner looks {m_j, m_i} up in its local entries, evaluates
     g = ((w(i,j) + w(m_j,m_i)) - w(i,m_i)) - w(m_j,j) from its replicas
     and, if g > 0, sends a B-request to the owner of the matched edge
     {m_j, j};
  C  (Alg. 5) that owner keeps, per matched edge, the B-request of largest
     gain (equal gains: lowest row i) and sends it as a C-request to the
     owner of {i, m_i};
  D  (Alg. 6) that owner drops requests whose edge {i, m_i} it sent a
     C-request for itself (the edge is the root edge {m_k, k} of another
     Step-C winner), keeps per edge {i, m_i} the request of largest gain
     (equal gains: lowest root j), and broadcasts the flip of its cycle
     along the grid rows and columns of the four vertices.

Messages are explicit per-destination queues exchanged between the steps
(the all-to-all of the paper).  Nothing here is shared with the oracle.
"""
from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, g, mate, s):
        self.n = g.n
        self.s = s
        self.bsz = -(-g.n // s)  # block size (ceil)
        n = g.n
        self.local = {}  # (a, b) -> {(row, col): weight}
        for a in range(s):
            for b in range(s):
                self.local[(a, b)] = {}
        for j in range(n):
            for p in range(g.colptr[j], g.colptr[j + 1]):
                i = int(g.rowidx[p])
                self.local[(self.blk(i), self.blk(j))][(i, j)] = float(g.weight[p])
        # replicas: row data per (grid row a, process column b); column data
        # per (process row a, grid column b)
        w_of = {}
        for j in range(n):
            for p in range(g.colptr[j], g.colptr[j + 1]):
                w_of[(int(g.rowidx[p]), j)] = float(g.weight[p])
        self.rows = {}  # (a, b) -> {i: (m_i, w(i, m_i))}
        self.cols = {}  # (a, b) -> {j: (m_j, w(m_j, j))}
        for a in range(s):
            for b in range(s):
                self.rows[(a, b)] = {}
                self.cols[(a, b)] = {}
        for j in range(n):
            r = int(mate[j])
            for a in range(s):  # column j's data on grid column blk(j)
                self.cols[(a, self.blk(j))][j] = (r, w_of[(r, j)])
            for b in range(s):  # row r's data on grid row blk(r)
                self.rows[(self.blk(r), b)][r] = (j, w_of[(r, j)])

    def blk(self, x):
        return x // self.bsz

    def procs(self):
        return [(a, b) for a in range(self.s) for b in range(self.s)]

    def one_pass(self):
        """Run Steps A-D once; returns the number of cycles flipped."""
        s = self.s
        # Step A
        qa = {pr: [] for pr in self.procs()}
        for (a, b) in self.procs():
            for (i, j), wij in sorted(self.local[(a, b)].items(), key=lambda kv: (kv[0][1], kv[0][0])):
                mj, _ = self.cols[(a, b)][j]
                if i <= mj:
                    continue
                mi, _ = self.rows[(a, b)][i]
                qa[(self.blk(mj), self.blk(mi))].append((i, j, mj, mi, wij))
        # Step B
        qb = {pr: [] for pr in self.procs()}
        for (c, d) in self.procs():
            for (i, j, mj, mi, wij) in qa[(c, d)]:
                wq = self.local[(c, d)].get((mj, mi))
                if wq is None:
                    continue
                w_i_mi = self.cols[(c, d)][mi][1]   # matched edge of column m_i
                w_mj_j = self.rows[(c, d)][mj][1]   # matched edge of row m_j
                g = ((wij + wq) - w_i_mi) - w_mj_j
                if g > 0:
                    qb[(c, self.blk(j))].append((i, j, mj, mi, g))
        # Step C
        qc = {pr: [] for pr in self.procs()}
        sent_c = {pr: set() for pr in self.procs()}  # matched edges (m_j, j) with a C-request
        for (c, b) in self.procs():
            best = {}
            for req in qb[(c, b)]:
                i, j, mj, mi, g = req
                cur = best.get(j)
                if cur is None or g > cur[4] or (g == cur[4] and i < cur[0]):
                    best[j] = req
            for j, req in sorted(best.items()):
                i, _, mj, mi, _ = req
                sent_c[(c, b)].add((mj, j))
                qc[(self.blk(i), self.blk(mi))].append(req)
        # Step D
        flips = []
        for (a, d) in self.procs():
            win = {}
            for req in qc[(a, d)]:
                i, j, mj, mi, g = req
                if (i, mi) in sent_c[(a, d)]:
                    continue  # {i, m_i} is the root edge of another Step-C winner
                cur = win.get((i, mi))
                if cur is None or g > cur[4] or (g == cur[4] and j < cur[1]):
                    win[(i, mi)] = req
            flips.extend(win.values())
        # broadcasts of the flips along the grid rows and columns
        for (i, j, l, k, _) in flips:
            pa = self.blk(i)
            wij = self.local[(pa, self.blk(j))][(i, j)]
            wlk = self.local[(self.blk(l), self.blk(k))][(l, k)]
            for x in range(s):
                self.rows[(pa, x)][i] = (j, wij)
                self.cols[(x, self.blk(j))][j] = (i, wij)
                self.rows[(self.blk(l), x)][l] = (k, wlk)
                self.cols[(x, self.blk(k))][k] = (l, wlk)
        return len(flips)

    def matching(self):
        """Column mates, checked to agree across all replicas."""
        mate = np.full(self.n, -1, dtype=np.int64)
        for (a, b), cols in self.cols.items():
            for j, (r, _) in cols.items():
                assert mate[j] in (-1, r), "replicas of column %d disagree" % j
                mate[j] = r
        for (a, b), rows in self.rows.items():
            for i, (j, _) in rows.items():
                assert mate[j] == i, "row and column replicas disagree at row %d" % i
        return mate
