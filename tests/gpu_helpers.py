"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
compare it with the CPU oracle."""
from __future__ import annotations

import numpy as np

from paper_1801_09809_gb300 import awpm


def matched_abs_sum(g, mate):
    col = np.arange(g.n)
    cp = g.colptr.astype(np.int64)
    keys = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(cp)) * g.n + g.rowidx
    pos = np.searchsorted(keys, col.astype(np.int64) * g.n + np.asarray(mate, dtype=np.int64))
    return float(np.abs(g.weight[pos]).sum())


def weight_tol(g, mate):
    """|W_gpu - W_oracle| <= 1e-12 * sum_j |w(m_j, j)| (the two sums differ only
    in the order of n double additions)."""
    return 1e-12 * matched_abs_sum(g, mate) + 1e-300


def to_device(g, torch):
    dev = torch.device("cuda")
    return (torch.from_numpy(g.colptr).to(dev), torch.from_numpy(g.rowidx).to(dev),
            torch.from_numpy(g.weight).to(dev), torch.from_numpy(np.ascontiguousarray(g.mate)).to(dev))


def run_gpu(ctx, g, mate=None, torch=None, host=False):
    """Solve on the GPU; returns (mate_out as numpy, stats)."""
    mate = g.mate if mate is None else np.ascontiguousarray(mate, dtype=np.int32)
    if host or torch is None:
        out = np.empty(g.n, dtype=np.int32)
        st = awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, mate, out)
        return out, st
    cp, ri, w, _ = to_device(g, torch)
    m = torch.from_numpy(mate).to(cp.device)
    out = torch.empty_like(m)
    st = awpm.awpm_improve_ctx(ctx, g.n, cp, ri, w, m, out)
    return out.cpu().numpy(), st


def assert_same_as_oracle(g, got, st, ref, rst, what=""):
    assert np.array_equal(got, ref), f"{what}: matching differs ({int(np.sum(got != ref))} columns)"
    assert st["iterations"] == rst["iterations"], (what, st, rst)
    assert st["converged"] == rst["converged"], (what, st, rst)
    assert st["cycles_applied"] == rst["cycles_applied"], (what, st, rst)
    assert st["candidates"] == rst["candidates"], (what, st, rst)
    assert st["closing_found"] == rst["closing_found"], (what, st, rst)
    assert st["positive"] == rst["positive"], (what, st, rst)
    assert st["edge_checks"] == rst["edge_checks"], (what, st, rst)
    tol = weight_tol(g, ref)
    assert abs(st["weight_in"] - rst["weight_in"]) <= weight_tol(g, g.mate), (what, st, rst)
    assert abs(st["weight_out"] - rst["weight_out"]) <= tol, (what, st, rst)
