"""Seeded synthetic inputs for the weight-increasing 4-cycle phase.

This module only builds input graphs: a square sparse matrix in CSC form
(``colptr`` int32 [n+1], ``rowidx`` int32 [nnz] strictly increasing inside each
column, ``weight`` float64 [nnz]) together with a planted perfect matching
``mate`` (int32 [n], ``mate[j]`` = row matched to column j, always a stored
entry).  It holds none of the matching arithmetic, so both the CPU oracle and
the CUDA path read the very same bytes from here.

Weights follow the static-pivoting preprocessing of Section 6.1 of the paper
(arXiv 1801.09809): the value magnitudes |a_ij| are equilibrated per column so
that the largest entry of each column has magnitude 1, and the objective is
the product of magnitudes (Option B), i.e. the sum of ``log|a_ij|``.  Hence
``w_ij = log|a_ij| - max_k log|a_kj|`` (every weight <= 0, column maxima = 0).
For log-normal magnitudes ``|a| = exp(z), z ~ N(0,1)`` the logarithm is drawn
directly as ``z``.

The structures stand in for the paper's SuiteSparse test matrices (Table 2),
which are not available: uniform random sparse, 2D 5-point and 3D 27-point
stencils, banded, and R-MAT power-law graphs.  Stencils and R-MAT graphs are
randomly permuted, as the paper does before matching (Sections 5.4 and 6.3).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

SEED_BASE = 1801098090  # + config number: 1801098091 ... 1801098096


@dataclasses.dataclass
class Graph:
    n: int
    colptr: np.ndarray  # int32 [n+1]
    rowidx: np.ndarray  # int32 [nnz]
    weight: np.ndarray  # float64 [nnz]
    mate: np.ndarray    # int32 [n], planted perfect matching (row of column j)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def copy(self) -> "Graph":
        return Graph(self.n, self.colptr.copy(), self.rowidx.copy(),
                     self.weight.copy(), self.mate.copy(), self.name)


# ----------------------------------------------------------------------------
# structure helpers
# ----------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_NATIVE_SRC = os.path.join(_HERE, "gen_native.c")
_NATIVE_SO = os.path.join(_HERE, "_gen_native.so")
_native = None


def build_native(force: bool = False) -> str:
    """Compile the host helper (plain C, no CUDA) next to this file."""
    if force or not os.path.exists(_NATIVE_SO) or \
            os.path.getmtime(_NATIVE_SO) < os.path.getmtime(_NATIVE_SRC):
        tmp = _NATIVE_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _NATIVE_SRC])
        os.replace(tmp, _NATIVE_SO)
    return _NATIVE_SO


def _lib():
    global _native
    if _native is None:
        lib = ctypes.CDLL(build_native())
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gen_rmat_edges.restype = ctypes.c_int
        lib.gen_rmat_edges.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, i64p, i64p]
        lib.gen_csc_from_coo.restype = ctypes.c_int64
        lib.gen_csc_from_coo.argtypes = [ctypes.c_int64, ctypes.c_int64, i64p, i64p, i32p, i32p]
        _native = lib
    return _native


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _csc_from_coo(n: int, rows: np.ndarray, cols: np.ndarray):
    """COO (any order, duplicates allowed) -> CSC with sorted unique rows."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    m = rows.size
    if m >= 2**31:
        raise ValueError("nnz does not fit int32")
    colptr = np.empty(n + 1, dtype=np.int32)
    rowidx = np.empty(max(m, 1), dtype=np.int32)
    nnz = _lib().gen_csc_from_coo(n, m, _ptr(rows, ctypes.c_int64), _ptr(cols, ctypes.c_int64),
                                  _ptr(colptr, ctypes.c_int32), _ptr(rowidx, ctypes.c_int32))
    if nnz < 0:
        raise ValueError("bad COO input")
    return colptr, rowidx[:nnz].copy()


def _csc_from_keys(n: int, keys: np.ndarray):
    """keys = col * n + row (int64), any order, duplicates allowed."""
    cols = keys // n
    return _csc_from_coo(n, keys - cols * n, cols)


def _planted_keys(n: int, mate: np.ndarray) -> np.ndarray:
    return np.arange(n, dtype=np.int64) * n + mate.astype(np.int64)


def _col_of_nz(colptr: np.ndarray) -> np.ndarray:
    n = colptr.size - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))


def log_weights_lognormal(colptr: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """log|a_ij| with |a_ij| log-normal(0,1), transformed per column."""
    z = rng.standard_normal(int(colptr[-1]))
    return column_transform(colptr, z)


def column_transform(colptr: np.ndarray, loga: np.ndarray) -> np.ndarray:
    """w_ij = log|a_ij| - max_k log|a_kj| (equilibration, Section 6.1)."""
    deg = np.diff(colptr)
    if np.any(deg == 0):
        raise ValueError("empty column")
    cmax = np.maximum.reduceat(loga, colptr[:-1].astype(np.int64))
    return loga - np.repeat(cmax, deg)


# ----------------------------------------------------------------------------
# structures
# ----------------------------------------------------------------------------

def random_sparse(n: int, deg: int, seed: int, name: str = "") -> Graph:
    """Exactly ``deg`` distinct uniform rows per column plus the planted entry
    (pi(j), j); a planted entry that collides with a drawn one is merged."""
    rng = np.random.default_rng(seed)
    deg = min(deg, n)
    rows = rng.integers(0, n, size=(n, deg), dtype=np.int64)
    while True:
        rows.sort(axis=1)
        bad = np.nonzero((rows[:, 1:] == rows[:, :-1]).any(axis=1))[0] if deg > 1 else []
        if len(bad) == 0:
            break
        rows[bad] = rng.integers(0, n, size=(len(bad), deg), dtype=np.int64)
    mate = rng.permutation(n).astype(np.int32)
    keys = (np.arange(n, dtype=np.int64)[:, None] * n + rows).ravel()
    colptr, rowidx = _csc_from_keys(n, np.concatenate([keys, _planted_keys(n, mate)]))
    weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate, name or f"random_sparse(n={n},deg={deg})")


def _stencil_coo(side: int, dims: int, points: int):
    """Structurally symmetric stencil S on a side^dims grid, as (row, col) arrays."""
    n = side ** dims
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // side ** d) % side for d in range(dims)]
    if points == 5 and dims == 2:
        offs = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]
    elif points == 27 and dims == 3:
        offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    else:
        raise ValueError("unsupported stencil")
    rows, cols = [], []
    for off in offs:
        ok = np.ones(n, dtype=bool)
        nb = np.zeros(n, dtype=np.int64)
        for d in range(dims):
            c = coords[d] + off[d]
            ok &= (c >= 0) & (c < side)
            nb += np.clip(c, 0, side - 1) * side ** d
        rows.append(nb[ok])
        cols.append(idx[ok])
    return n, np.concatenate(rows), np.concatenate(cols)


def _permuted(n, rows, cols, rng, permute_cols: bool):
    """A[pi(r), sigma(c)] = S[r, c]; planted mate[sigma(c)] = pi(c)."""
    pi = rng.permutation(n).astype(np.int64)
    sigma = rng.permutation(n).astype(np.int64) if permute_cols else np.arange(n, dtype=np.int64)
    mate = np.empty(n, dtype=np.int32)
    mate[sigma] = pi
    colptr, rowidx = _csc_from_coo(n, pi[rows], sigma[cols])
    return colptr, rowidx, mate


def stencil_2d(side: int, seed: int, weights: str = "diag", name: str = "") -> Graph:
    """2D 5-point stencil with a random row permutation.  ``weights='diag'``:
    diagonal |a| ~ U[0.5, 1.5], off-diagonal a ~ N(0,1); ``'lognormal'``: all
    log-normal.  The planted matching is the permuted diagonal."""
    rng = np.random.default_rng(seed)
    n, rows, cols = _stencil_coo(side, 2, 5)
    colptr, rowidx, mate = _permuted(n, rows, cols, rng, permute_cols=False)
    del rows, cols
    if weights == "diag":
        weight = _diag_offdiag_weights(colptr, rowidx, mate, rng)
    else:
        weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate, name or f"stencil2d({side}x{side})")


def _diag_offdiag_weights(colptr, rowidx, mate, rng):
    nnz = rowidx.size
    col = _col_of_nz(colptr)
    diag = rowidx == mate[col]
    a = np.empty(nnz, dtype=np.float64)
    a[diag] = rng.uniform(0.5, 1.5, size=int(diag.sum()))
    off = ~diag
    vals = np.abs(rng.standard_normal(int(off.sum())))
    # an exact zero has probability 0; keep entries structurally nonzero anyway
    vals[vals == 0.0] = np.finfo(np.float64).tiny
    a[off] = vals
    return column_transform(colptr, np.log(a))


def stencil_3d(side: int, seed: int, name: str = "") -> Graph:
    """3D 27-point stencil with random row and column permutations,
    log-normal weights; the planted matching is the permuted diagonal."""
    rng = np.random.default_rng(seed)
    n, rows, cols = _stencil_coo(side, 3, 27)
    colptr, rowidx, mate = _permuted(n, rows, cols, rng, permute_cols=True)
    weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate, name or f"stencil3d({side}^3)")


def banded(n: int, bandwidth: int, seed: int, name: str = "") -> Graph:
    """Banded |i-j| <= (b-1)/2 (odd total bandwidth b), random row permutation."""
    rng = np.random.default_rng(seed)
    h = (bandwidth - 1) // 2
    idx = np.arange(n, dtype=np.int64)
    rows, cols = [], []
    for d in range(-h, h + 1):
        ok = (idx + d >= 0) & (idx + d < n)
        rows.append(idx[ok] + d)
        cols.append(idx[ok])
    colptr, rowidx, mate = _permuted(n, np.concatenate(rows), np.concatenate(cols), rng,
                                     permute_cols=False)
    weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate, name or f"banded(n={n},b={bandwidth})")


def rmat(n: int, avg_deg: float, seed: int, a=0.57, b=0.19, c=0.19, name: str = "") -> Graph:
    """R-MAT bipartite graph (recursive quadrant choice with probabilities
    a, b, c, d = 1-a-b-c), ``avg_deg * n`` sampled edges with duplicates
    removed, rows and columns randomly relabelled, plus a planted random
    permutation.  For n not a power of two, samples outside [0,n)^2 are
    rejected (scale = ceil(log2 n))."""
    rng = np.random.default_rng(seed)
    scale = max(1, int(math.ceil(math.log2(n))))
    m = int(round(avg_deg * n))
    ta = int(round(a * 65536))
    tab = int(round((a + b) * 65536))
    tabc = int(round((a + b + c) * 65536))
    rows = np.empty(m, dtype=np.int64)
    cols = np.empty(m, dtype=np.int64)
    rc = _lib().gen_rmat_edges(int(rng.integers(0, 2**63)), scale, n, m, ta, tab, tabc,
                               _ptr(rows, ctypes.c_int64), _ptr(cols, ctypes.c_int64))
    if rc != 0:
        raise RuntimeError("R-MAT sampling failed")
    prow = rng.permutation(n).astype(np.int64)
    pcol = rng.permutation(n).astype(np.int64)
    mate = rng.permutation(n).astype(np.int32)
    colptr, rowidx = _csc_from_coo(
        n, np.concatenate([prow[rows], mate.astype(np.int64)]),
        np.concatenate([pcol[cols], np.arange(n, dtype=np.int64)]))
    del rows, cols
    weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate,
                 name or f"rmat(n={n},deg={avg_deg},a={a},b={b},c={c})")


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config1() -> Graph:
    """Random sparse n = 2,000, 8 uniform rows per column + planted entry."""
    return random_sparse(2000, 8, SEED_BASE + 1, name="random_sparse_n2000")


def config2() -> Graph:
    """2D 5-point stencil on 1000 x 1000 (n = 1e6, nnz = 4,996,000)."""
    return stencil_2d(1000, SEED_BASE + 2, weights="diag", name="stencil2d_1000x1000")


def config3a() -> Graph:
    """3D 27-point stencil on 96^3 (n = 884,736, nnz = 286^3 = 23,393,656)."""
    return stencil_3d(96, SEED_BASE + 3, name="stencil3d_96")


def config3b() -> Graph:
    """R-MAT n = 2^22 = 4,194,304, 16 n samples, a = .57, b = c = .19."""
    return rmat(1 << 22, 16, SEED_BASE + 4, name="rmat_s22_ef16")


def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_spec(count: int = 4096, seed: int = SEED_BASE + 5):
    """Matrix specs of the batched workload: n log-uniform in [200, 20000],
    structure uniform over random sparse (degree U{4..16}), 2D 5-point
    (side round(sqrt n)) and banded (odd bandwidth 3..15)."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        n = _log_uniform_int(rng, 200, 20000)
        kind = int(rng.integers(0, 3))
        s = int(rng.integers(0, 2 ** 62))
        if kind == 0:
            specs.append(("random_sparse", n, int(rng.integers(4, 17)), s))
        elif kind == 1:
            specs.append(("stencil2d", max(2, int(round(math.sqrt(n)))), 0, s))
        else:
            specs.append(("banded", n, int(rng.choice(np.arange(3, 16, 2))), s))
    return specs


def build_spec(spec) -> Graph:
    kind, size, param, s = spec
    if kind == "random_sparse":
        return random_sparse(size, param, s)
    if kind == "stencil2d":
        return stencil_2d(size, s, weights="lognormal")
    if kind == "stencil3d":
        return stencil_3d(size, s)
    if kind == "banded":
        return banded(size, param, s)
    if kind == "rmat":
        return rmat(size, param, s)
    raise ValueError(kind)


def batch(count: int = 4096, seed: int = SEED_BASE + 5):
    return [build_spec(sp) for sp in batch_spec(count, seed)]


def serve_spec(count: int = 20000, seed: int = SEED_BASE + 6, n_lo=1000, n_hi=1_000_000):
    """Request specs of the served stream: n log-uniform in [n_lo, n_hi],
    structure uniform over random sparse, 2D 5-point, 3D 27-point and R-MAT,
    average degree U[4, 27] where the structure has a free degree."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        n = _log_uniform_int(rng, n_lo, n_hi)
        kind = int(rng.integers(0, 4))
        deg = int(rng.integers(4, 28))
        s = int(rng.integers(0, 2 ** 62))
        if kind == 0:
            specs.append(("random_sparse", n, deg, s))
        elif kind == 1:
            specs.append(("stencil2d", max(2, int(round(math.sqrt(n)))), 0, s))
        elif kind == 2:
            specs.append(("stencil3d", max(2, int(round(n ** (1.0 / 3.0)))), 0, s))
        else:
            specs.append(("rmat", n, deg, s))
    return specs


def poisson_arrivals(count: int, rate_per_s: float, seed: int = SEED_BASE + 6) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed ^ 0x5EED)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


# ----------------------------------------------------------------------------
# small graphs for tests
# ----------------------------------------------------------------------------

def random_small(n: int, density: float, seed: int, integer_weights: bool = False) -> Graph:
    """Tiny random graph with a planted matching (tests): each entry present
    with probability ``density``; weights either log-normal transformed or
    small integers (exact sums, for tie cases)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    mate = rng.permutation(n).astype(np.int32)
    mask[mate, np.arange(n)] = True
    rows, cols = np.nonzero(mask)
    colptr, rowidx = _csc_from_keys(n, cols.astype(np.int64) * n + rows)
    if integer_weights:
        weight = rng.integers(-4, 5, size=rowidx.size).astype(np.float64)
    else:
        weight = log_weights_lognormal(colptr, rng)
    return Graph(n, colptr, rowidx, weight, mate, f"random_small(n={n},p={density},seed={seed})")


def from_dense(w: np.ndarray, mask: np.ndarray, mate) -> Graph:
    """Graph from a dense weight matrix and a structure mask (tests)."""
    n = w.shape[0]
    rows, cols = np.nonzero(mask.astype(bool))
    colptr, rowidx = _csc_from_keys(n, cols.astype(np.int64) * n + rows)
    col = _col_of_nz(colptr)
    weight = np.ascontiguousarray(w[rowidx, col], dtype=np.float64)
    return Graph(n, colptr, rowidx, weight, np.asarray(mate, dtype=np.int32), "dense")


# ----------------------------------------------------------------------------
# batched layout
# ----------------------------------------------------------------------------

def union(graphs):
    """Pack matrices into one block-diagonal union: returns (n_off, Graph)
    where matrix b owns columns and rows [n_off[b], n_off[b+1]) and indices
    are global."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    n_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=n_off[1:])
    nnzs = np.array([g.nnz for g in graphs], dtype=np.int64)
    z_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=z_off[1:])
    N, NNZ = int(n_off[-1]), int(z_off[-1])
    if N >= 2**31 or NNZ >= 2**31:
        raise ValueError("union too large for int32 indices")
    colptr = np.empty(N + 1, dtype=np.int32)
    rowidx = np.empty(NNZ, dtype=np.int32)
    weight = np.empty(NNZ, dtype=np.float64)
    mate = np.empty(N, dtype=np.int32)
    for b, g in enumerate(graphs):
        a0, a1 = int(n_off[b]), int(n_off[b + 1])
        z0, z1 = int(z_off[b]), int(z_off[b + 1])
        colptr[a0:a1] = g.colptr[:-1] + z0
        rowidx[z0:z1] = g.rowidx + a0
        weight[z0:z1] = g.weight
        mate[a0:a1] = g.mate + a0
    colptr[N] = NNZ
    return n_off.astype(np.int32), Graph(N, colptr, rowidx, weight, mate,
                                         f"union({len(graphs)} matrices)")


def split(n_off, mate):
    """Per-matrix local matchings from a union matching."""
    return [np.asarray(mate[n_off[b]:n_off[b + 1]]) - n_off[b] for b in range(len(n_off) - 1)]
