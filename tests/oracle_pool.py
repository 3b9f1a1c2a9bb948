"""The CPU oracle over many generated problems at once (test infrastructure).

Workers are started with the `spawn` method, so a pool made after the test
process has touched the GPU never inherits a CUDA context.  Each worker builds
its problems from their seeded specs itself (the generators are
deterministic), runs the oracle and returns the matching and the statistics.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _solve(spec):
    import oracle
    from paper_1801_09809_gb300 import gen
    g = gen.build_spec(spec)
    out, st, _ = oracle.get().improve(g)
    return out, st


def improve_specs(specs, processes=None):
    """oracle.improve on gen.build_spec(s) for every spec, in order:
    a list of (mate_out, stats)."""
    import oracle
    oracle.build()  # compiled once here, not by every worker
    procs = processes or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        # the largest problems first, so that none starts last
        order = sorted(range(len(specs)), key=lambda k: -_size_hint(specs[k]))
        res = pool.map(_solve, [specs[k] for k in order], chunksize=1 if len(specs) < 64 else 8)
    out = [None] * len(specs)
    for k, r in zip(order, res):
        out[k] = r
    return out


def _size_hint(spec):
    kind, size, param, _ = spec
    if kind == "stencil2d":
        return size * size * 5
    if kind == "stencil3d":
        return size ** 3 * 27 * 4  # more passes than the others
    return size * max(param, 4)
