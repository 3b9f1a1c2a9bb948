"""CPU oracle for the weight-increasing alternating 4-cycle phase.

TEST INFRASTRUCTURE ONLY: a plain C restatement of Algorithms 2-6 of
arXiv 1801.09809 (Section 5.3), loaded through ctypes.  Only the tests, the
package smoke check and the benchmark's CPU-baseline leg use it; the product
path (the CUDA library) never imports, links or runs anything from here, and
the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "awpm_oracle.c")
SO = os.path.join(HERE, "_awpm_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]

ERRORS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_PERFECT", 3: "UNSORTED_OR_DUP",
          4: "NONFINITE", 5: "OOM"}


def compile_oracle(src: str = SRC, out: str = SO) -> str:
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        compile_oracle()
    return SO



class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("cycles_applied", ctypes.c_int64), ("edge_checks", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("closing_found", ctypes.c_int64),
                ("positive", ctypes.c_int64), ("weight_in", ctypes.c_double),
                ("weight_out", ctypes.c_double)]


class _GreedyStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("cardinality", ctypes.c_int32),
                ("weight", ctypes.c_double)]


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(t))


def _arrs(g):
    return (np.ascontiguousarray(g.colptr, dtype=np.int32),
            np.ascontiguousarray(g.rowidx, dtype=np.int32),
            np.ascontiguousarray(g.weight, dtype=np.float64))


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(ERRORS.get(code, str(code)))
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Oracle:
    """ctypes front end of one compiled oracle library."""

    def __init__(self, path: str | None = None):
        self.lib = ctypes.CDLL(path or build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        L = self.lib
        L.oracle_validate.restype = ctypes.c_int
        L.oracle_validate.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p]
        L.oracle_pass.restype = ctypes.c_int64
        L.oracle_pass.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p, f64p,
                                  f64p, i32p, i32p, i64p]
        L.oracle_improve.restype = ctypes.c_int
        L.oracle_improve.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p,
                                     ctypes.c_int32, ctypes.POINTER(_Stats), f64p, i64p,
                                     ctypes.c_int32]
        L.oracle_step_c.restype = ctypes.c_int
        L.oracle_step_c.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, f64p, i32p, i64p]
        L.oracle_pass_mode.restype = ctypes.c_int64
        L.oracle_pass_mode.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p, f64p,
                                       f64p, i32p, i32p, i64p, ctypes.c_int32]
        L.oracle_improve_mode.restype = ctypes.c_int
        L.oracle_improve_mode.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p,
                                          ctypes.c_int32, ctypes.POINTER(_Stats), f64p, i64p,
                                          ctypes.c_int32, ctypes.c_int32]
        L.oracle_weights.restype = ctypes.c_int
        L.oracle_weights.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_int32, f64p]
        L.oracle_mcm.restype = ctypes.c_int
        L.oracle_mcm.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p,
                                 ctypes.POINTER(ctypes.c_int32 * 2)]
        L.oracle_greedy.restype = ctypes.c_int
        L.oracle_greedy.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p,
                                    ctypes.POINTER(_GreedyStats)]

    # -- API -----------------------------------------------------------------
    def validate(self, g, mate=None) -> str:
        cp, ri, w = _arrs(g)
        m = np.ascontiguousarray(g.mate if mate is None else mate, dtype=np.int32)
        rc = self.lib.oracle_validate(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                      _p(w, ctypes.c_double), _p(m, ctypes.c_int32))
        return ERRORS[rc]

    def improve(self, g, mate=None, max_iters: int = 0, trace_cap: int = 0, select: int = 0,
                row_marking: bool = False):
        """Run the phase; returns (mate_out, stats dict, trace) where trace is
        (weights after each pass, cycles flipped in each pass) when trace_cap>0.
        select: 0 = Step D of Algorithm 6, 1 = the Pettie-Sanders selection.
        row_marking: closing entries found by marking row m_j's neighbourhood
        (Section 4) instead of searching column m_i."""
        cp, ri, w = _arrs(g)
        m = np.ascontiguousarray(g.mate if mate is None else mate, dtype=np.int32)
        out = np.empty(max(g.n, 1), dtype=np.int32)
        st = _Stats()
        tw = np.zeros(max(trace_cap, 1), dtype=np.float64) if trace_cap else None
        tf = np.zeros(max(trace_cap, 1), dtype=np.int64) if trace_cap else None
        rc = self.lib.oracle_improve_mode(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                          _p(w, ctypes.c_double), _p(m, ctypes.c_int32),
                                          _p(out, ctypes.c_int32), max_iters, ctypes.byref(st),
                                          _p(tw, ctypes.c_double), _p(tf, ctypes.c_int64),
                                          trace_cap, select | (2 if row_marking else 0))
        if rc != 0:
            raise OracleError(rc)
        stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
        trace = None
        if trace_cap:
            k = min(st.iterations, trace_cap)
            trace = (tw[:k].copy(), tf[:k].copy())
        return out[:g.n].copy(), stats, trace

    def weights(self, n, colptr, rowidx, values, mode):
        """Equilibrated weights from matrix values: mode 0 the scaled
        magnitudes (Option A), mode 1 their logarithms (Option B)."""
        cp = np.ascontiguousarray(colptr, dtype=np.int32)
        ri = np.ascontiguousarray(rowidx, dtype=np.int32)
        a = np.ascontiguousarray(values, dtype=np.float64)
        out = np.empty(max(len(a), 1), dtype=np.float64)
        rc = self.lib.oracle_weights(int(n), _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                     _p(a, ctypes.c_double), int(mode), _p(out, ctypes.c_double))
        if rc != 0:
            raise OracleError(rc)
        return out[:len(a)].copy()

    def mcm(self, g, mate=None):
        """Maximum cardinality matching with the heavy-weight tie-break from
        the matching `mate` (-1: unmatched; default empty): (mate_out, stats
        {phases, cardinality})."""
        cp, ri, w = _arrs(g)
        m = (np.full(max(g.n, 1), -1, dtype=np.int32) if mate is None
             else np.ascontiguousarray(mate, dtype=np.int32).copy())
        st = (ctypes.c_int32 * 2)()
        rc = self.lib.oracle_mcm(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                 _p(w, ctypes.c_double), _p(m, ctypes.c_int32), ctypes.byref(st))
        if rc != 0:
            raise OracleError(rc)
        return m[:g.n], {"phases": st[0], "cardinality": st[1]}

    def greedy(self, g):
        """Heavy-weight greedy maximal matching: (mate_out with -1 for
        unmatched columns, stats dict {rounds, cardinality, weight})."""
        cp, ri, w = _arrs(g)
        out = np.empty(max(g.n, 1), dtype=np.int32)
        st = _GreedyStats()
        rc = self.lib.oracle_greedy(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                    _p(w, ctypes.c_double), _p(out, ctypes.c_int32),
                                    ctypes.byref(st))
        if rc != 0:
            raise OracleError(rc)
        return out[:g.n], {"rounds": st.rounds, "cardinality": st.cardinality,
                           "weight": st.weight}

    def step_c(self, g, mate=None):
        """Step-C winners of one pass from ``mate``: (gain[n], row[n], counts[4])."""
        cp, ri, w = _arrs(g)
        m = np.ascontiguousarray(g.mate if mate is None else mate, dtype=np.int32)
        gain = np.zeros(max(g.n, 1), dtype=np.float64)
        row = np.zeros(max(g.n, 1), dtype=np.int32)
        counts = np.zeros(4, dtype=np.int64)
        rc = self.lib.oracle_step_c(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                    _p(w, ctypes.c_double), _p(m, ctypes.c_int32),
                                    _p(gain, ctypes.c_double), _p(row, ctypes.c_int32),
                                    _p(counts, ctypes.c_int64))
        if rc != 0:
            raise OracleError(rc)
        return gain[:g.n].copy(), row[:g.n].copy(), counts

    def one_pass(self, g, mate=None, select: int = 0, row_marking: bool = False):
        """One pass of Steps A-D plus the flip; returns (new mate, step-D roots
        per key column, counts[4]).  select, row_marking as for improve()."""
        cp, ri, w = _arrs(g)
        m = np.ascontiguousarray(g.mate if mate is None else mate, dtype=np.int32)
        if self.validate(g, m) != "OK":
            raise OracleError(2)
        n = g.n
        mc = m.copy()
        mr = np.empty(max(n, 1), dtype=np.int32)
        mr[mc] = np.arange(n, dtype=np.int32)
        col = np.repeat(np.arange(n), np.diff(cp))
        keys = col.astype(np.int64) * n + ri
        wm = w[np.searchsorted(keys, np.arange(n, dtype=np.int64) * n + mc)].copy()
        droot = np.zeros(max(n, 1), dtype=np.int32)
        counts = np.zeros(4, dtype=np.int64)
        f = self.lib.oracle_pass_mode(n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                      _p(w, ctypes.c_double), _p(mc, ctypes.c_int32),
                                      _p(mr, ctypes.c_int32), _p(wm, ctypes.c_double), None,
                                      None, _p(droot, ctypes.c_int32),
                                      _p(counts, ctypes.c_int64),
                                      select | (2 if row_marking else 0))
        if f < 0:
            raise OracleError(5)
        return mc[:n].copy(), droot[:n].copy(), counts


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


PAR_SRC = os.path.join(HERE, "awpm_oracle_par.c")
PAR_SO = os.path.join(HERE, "_awpm_oracle_par.so")


def build_par(force: bool = False) -> str:
    """The multi-threaded restatement (OpenMP); raises if gcc cannot build it."""
    if force or not os.path.exists(PAR_SO) or os.path.getmtime(PAR_SO) < os.path.getmtime(PAR_SRC):
        tmp = PAR_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, PAR_SRC, "-lm"])
        os.replace(tmp, PAR_SO)
    return PAR_SO


class OraclePar:
    """ctypes front end of the multi-threaded restatement: the CPU timing
    baseline on all host cores; its results must equal the oracle's."""

    def __init__(self, path: str | None = None):
        self.lib = ctypes.CDLL(path or build_par())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        self.lib.oracle_par_improve.restype = ctypes.c_int
        self.lib.oracle_par_improve.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p,
                                                ctypes.c_int32, ctypes.c_int32,
                                                ctypes.POINTER(_Stats)]
        self.lib.oracle_par_threads.restype = ctypes.c_int
        self.lib.oracle_par_threads.argtypes = []

    def threads(self) -> int:
        return int(self.lib.oracle_par_threads())

    def improve(self, g, mate=None, max_iters: int = 0, threads: int = 0):
        """(mate_out, stats dict) of the whole phase with `threads` threads
        (0: all)."""
        cp, ri, w = _arrs(g)
        m = np.ascontiguousarray(g.mate if mate is None else mate, dtype=np.int32)
        out = np.empty(max(g.n, 1), dtype=np.int32)
        st = _Stats()
        rc = self.lib.oracle_par_improve(g.n, _p(cp, ctypes.c_int32), _p(ri, ctypes.c_int32),
                                         _p(w, ctypes.c_double), _p(m, ctypes.c_int32),
                                         _p(out, ctypes.c_int32), max_iters, threads,
                                         ctypes.byref(st))
        if rc != 0:
            raise OracleError(rc)
        return out[:g.n], {k: getattr(st, k) for k, _ in _Stats._fields_}
