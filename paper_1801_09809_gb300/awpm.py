"""Python binding of libawpm (ctypes): argument marshalling only.

Same names and argument order as the C ABI in include/awpm.h.  Arrays may be
numpy arrays (host) or torch tensors (host or CUDA); the library tells host and
device memory apart itself.  Every computation runs in the CUDA library; if
it is not built this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# AWPM_LIBRARY names another build of the same library (for example one
# compiled with AWPM_DEBUG_BOUNDS); the default is the in-tree libawpm.so.
LIB_PATH = os.environ.get("AWPM_LIBRARY") or os.path.join(HERE, "libawpm.so")

AWPM_OK = 0
ERRORS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_PERFECT", 3: "UNSORTED_OR_DUP", 4: "NONFINITE",
          5: "OOM", 6: "BUDGET", 7: "CUDA", 8: "TIMEOUT", 9: "NOT_FOUND", 10: "TOO_LARGE",
          11: "INTERNAL", 12: "CANCELLED"}
LOOKUP_AUTO, LOOKUP_BSEARCH, LOOKUP_HASH, LOOKUP_ROWMARK = 0, 1, 2, 3
SELECT_STEP_D, SELECT_GREEDY = 0, 1
FLAG_TIME_SEARCH = 1
PASS_CAP = 65536


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("lookup", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("mem_budget_bytes", ctypes.c_size_t),
                ("slots", ctypes.c_int32), ("select", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("mate_in", ctypes.c_void_p), ("mate_out", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("cycles_applied", ctypes.c_int64), ("edge_checks", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("closing_found", ctypes.c_int64),
                ("positive", ctypes.c_int64), ("weight_in", ctypes.c_double),
                ("weight_out", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_search", ctypes.c_double), ("lookup_used", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class GreedyStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("cardinality", ctypes.c_int32),
                ("weight", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 2)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class McmStats(ctypes.Structure):
    _fields_ = [("phases", ctypes.c_int32), ("cardinality", ctypes.c_int32),
                ("ms_total", ctypes.c_double), ("levels", ctypes.c_int64),
                ("reserved", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class AwpmError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        self.code = code
        self.name = ERRORS.get(code, str(code))
        super().__init__(f"awpm error {self.name}" + (f": {detail}" if detail else ""))


_lib_handle = None

# (name, restype, argtypes) of every exported entry point
_VP = ctypes.c_void_p
SIGNATURES = [
    ("awpm_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("awpm_last_error", ctypes.c_char_p, []),
    ("awpm_default_options", None, [ctypes.POINTER(Options)]),
    ("awpm_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(Options)]),
    ("awpm_destroy", ctypes.c_int, [_VP]),
    ("awpm_improve", ctypes.c_int, [ctypes.c_int32, _VP, _VP, _VP, _VP, _VP,
                                    ctypes.POINTER(Stats)]),
    ("awpm_improve_ctx", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP,
                                        ctypes.POINTER(Stats)]),
    ("awpm_search", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP,
                                   ctypes.POINTER(Stats)]),
    ("awpm_improve_batch", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP,
                                          ctypes.POINTER(Stats), ctypes.POINTER(Stats)]),
    ("awpm_submit", ctypes.c_int, [_VP, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_uint64)]),
    ("awpm_poll", ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(Stats)]),
    ("awpm_wait", ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(Stats)]),
    ("awpm_cancel", ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    ("awpm_memory_held", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_size_t)]),
    ("awpm_inject_alloc_failure", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("awpm_bytes_needed", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_size_t)]),
    ("awpm_search_noalloc", ctypes.c_int, [ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                           ctypes.POINTER(Stats)]),
    ("awpm_greedy", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP,
                                   ctypes.POINTER(GreedyStats)]),
    ("awpm_weights", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32, _VP]),
    ("awpm_mcm", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP,
                                ctypes.POINTER(McmStats)]),
]
NOALLOC_MAX_N = 262144
NOALLOC_MAX_NNZ = 4194304


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1801_09809_gb300.build.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib_handle = L
    return _lib_handle


def _check(rc: int):
    if rc != AWPM_OK:
        detail = ""
        if ERRORS.get(rc) in ("CUDA", "OOM"):
            detail = (lib().awpm_last_error() or b"").decode()
        raise AwpmError(rc, detail)


_DT = {"int32": (np.int32, "torch.int32"), "float64": (np.float64, "torch.float64")}


def _ptr(a, kind: str):
    """Address of a C-contiguous numpy array or torch tensor of the given kind."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != _DT[kind][0] or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {kind} array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != _DT[kind][1] or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {kind} tensor")
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


class Context:
    def __init__(self, handle: int):
        self.handle = handle

    def __repr__(self):
        return f"<awpm_ctx 0x{self.handle:x}>"


def awpm_create(device: int = -1, max_iters: int = 0, lookup: int = LOOKUP_AUTO,
                flags: int = 0, stream=None, mem_budget_bytes: int = 0, slots: int = 0,
                select: int = 0) -> Context:
    L = lib()
    o = Options()
    L.awpm_default_options(ctypes.byref(o))
    o.device, o.max_iters, o.lookup, o.flags = device, max_iters, lookup, flags
    o.stream = _stream_handle(stream)
    o.mem_budget_bytes = mem_budget_bytes
    o.slots = slots
    o.select = select
    h = _VP()
    _check(L.awpm_create(ctypes.byref(h), ctypes.byref(o)))
    return Context(h.value)


def awpm_destroy(ctx: Context) -> None:
    if ctx is not None and ctx.handle:
        _check(lib().awpm_destroy(ctx.handle))
        ctx.handle = 0


def awpm_improve(n, colptr, rowidx, weight, mate_in, mate_out) -> dict:
    st = Stats()
    _check(lib().awpm_improve(int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                              _ptr(weight, "float64"), _ptr(mate_in, "int32"),
                              _ptr(mate_out, "int32"), ctypes.byref(st)))
    return st.as_dict()


def awpm_improve_ctx(ctx: Context, n, colptr, rowidx, weight, mate_in, mate_out) -> dict:
    st = Stats()
    _check(lib().awpm_improve_ctx(ctx.handle, int(n), _ptr(colptr, "int32"),
                                  _ptr(rowidx, "int32"), _ptr(weight, "float64"),
                                  _ptr(mate_in, "int32"), _ptr(mate_out, "int32"),
                                  ctypes.byref(st)))
    return st.as_dict()


def awpm_improve_batch(ctx: Context, count, n_off, colptr, rowidx, weight, mate_in, mate_out,
                       per_matrix: bool = True):
    """Batched solve of a block-diagonal union; returns (total stats, list of
    per-matrix stats or None)."""
    tot = Stats()
    pm = (Stats * max(int(count), 1))() if per_matrix else None
    _check(lib().awpm_improve_batch(ctx.handle, int(count), _ptr(n_off, "int32"),
                                    _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                                    _ptr(weight, "float64"), _ptr(mate_in, "int32"),
                                    _ptr(mate_out, "int32"), pm, ctypes.byref(tot)))
    return tot.as_dict(), ([pm[b].as_dict() for b in range(int(count))] if per_matrix else None)


def awpm_search(ctx: Context, n, colptr, rowidx, weight, mate, stepc_gain, stepc_row) -> dict:
    st = Stats()
    _check(lib().awpm_search(ctx.handle, int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                             _ptr(weight, "float64"), _ptr(mate, "int32"),
                             _ptr(stepc_gain, "float64"), _ptr(stepc_row, "int32"),
                             ctypes.byref(st)))
    return st.as_dict()


def awpm_greedy(ctx: Context, n, colptr, rowidx, weight, mate_out) -> dict:
    """Heavy-weight greedy maximal matching into mate_out (-1: unmatched)."""
    st = GreedyStats()
    _check(lib().awpm_greedy(ctx.handle, int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                             _ptr(weight, "float64"), _ptr(mate_out, "int32"),
                             ctypes.byref(st)))
    return st.as_dict()


def awpm_mcm(ctx: Context, n, colptr, rowidx, weight, mate) -> dict:
    """Maximum cardinality matching (heavy-weight tie-break) in place in
    `mate` (-1: unmatched)."""
    st = McmStats()
    _check(lib().awpm_mcm(ctx.handle, int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                          _ptr(weight, "float64"), _ptr(mate, "int32"), ctypes.byref(st)))
    return st.as_dict()


WEIGHTS_SUM, WEIGHTS_PRODUCT = 0, 1


def awpm_weights(ctx: Context, n, colptr, rowidx, values, mode, weight_out) -> None:
    """Equilibrated matching weights from matrix values into weight_out
    (mode WEIGHTS_SUM: scaled magnitudes; WEIGHTS_PRODUCT: their logs)."""
    _check(lib().awpm_weights(ctx.handle, int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                              _ptr(values, "float64"), int(mode), _ptr(weight_out, "float64")))


def awpm_search_noalloc(n, colptr, rowidx, weight, mate, stepc_gain, stepc_row,
                        stream=None) -> dict:
    """awpm_search for callers that cannot allocate device memory: device
    arrays only, n <= NOALLOC_MAX_N, nnz <= NOALLOC_MAX_NNZ; scratch is a fixed
    array inside the library shared by all calls on a device."""
    st = Stats()
    _check(lib().awpm_search_noalloc(int(n), _ptr(colptr, "int32"), _ptr(rowidx, "int32"),
                                     _ptr(weight, "float64"), _ptr(mate, "int32"),
                                     _ptr(stepc_gain, "float64"), _ptr(stepc_row, "int32"),
                                     _stream_handle(stream), ctypes.byref(st)))
    return st.as_dict()


def awpm_submit(ctx: Context, n, colptr, rowidx, weight, mate_in, mate_out, nnz=None) -> int:
    """Queue one problem on the context's request server; returns the ticket.
    The arrays must stay alive until awpm_poll/awpm_wait reports it done."""
    p = Problem(int(n), int(nnz) if nnz is not None else -1, _ptr(colptr, "int32"),
                _ptr(rowidx, "int32"), _ptr(weight, "float64"), _ptr(mate_in, "int32"),
                _ptr(mate_out, "int32"))
    t = ctypes.c_uint64()
    _check(lib().awpm_submit(ctx.handle, ctypes.byref(p), ctypes.byref(t)))
    return t.value


def awpm_poll(ctx: Context, ticket: int):
    """(done, stats or None); raises AwpmError if the finished solve failed."""
    d = ctypes.c_int(0)
    st = Stats()
    _check(lib().awpm_poll(ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(st)))
    return (True, st.as_dict()) if d.value else (False, None)


def awpm_wait(ctx: Context, ticket: int) -> dict:
    st = Stats()
    _check(lib().awpm_wait(ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(st)))
    return st.as_dict()


def awpm_cancel(ctx: Context, ticket: int) -> bool:
    """Cancel a queued request; True if it had not started (it is then
    reported done with CANCELLED), False if it runs to completion."""
    c = ctypes.c_int(0)
    _check(lib().awpm_cancel(ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(c)))
    return bool(c.value)


def awpm_memory_held(ctx: Context):
    """(device bytes held now, most held at once) by the context and its
    request server's slots."""
    h, p = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib().awpm_memory_held(ctx.handle, ctypes.byref(h), ctypes.byref(p)))
    return h.value, p.value


def awpm_inject_alloc_failure(ctx: Context, after: int) -> None:
    """Test hook: the context's next device allocation after `after`
    successful ones fails (OOM), once; -1 switches it off."""
    _check(lib().awpm_inject_alloc_failure(ctx.handle, int(after)))


def awpm_bytes_needed(ctx: Context, n: int, nnz: int, host_inputs: bool = False) -> int:
    """Admission estimate of one solve's device workspace on this context."""
    b = ctypes.c_size_t(0)
    _check(lib().awpm_bytes_needed(ctx.handle, int(n), int(nnz), int(bool(host_inputs)),
                                   ctypes.byref(b)))
    return b.value


def awpm_strerror(code: int) -> str:
    return lib().awpm_strerror(code).decode()
