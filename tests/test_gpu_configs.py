"""The batched and served workloads at their configured scale against the CPU
oracle, matrix by matrix (needs a GPU).

- Batched: all 4,096 matrices of the batched mix (n log-uniform in
  [200, 20000]; random sparse, 2D 5-point, banded) in one awpm_improve_batch
  call, the launch the bench times.
- Served: the first 28 problems of the served pool (n log-uniform in
  [1e3, 1e6]; random sparse, 2D, 3D 27-point, R-MAT; five of them above
  n = 3e5), submitted together to the request server and solved alone.

The oracle runs in a process pool (spawn), one problem per task.
"""
import numpy as np
import pytest

import oracle_pool
from gpu_helpers import weight_tol
from paper_1801_09809_gb300 import awpm, gen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09809_gb300 import build
    build.build()
    return _t


def _same(g, got, st, ref, rst, what):
    assert np.array_equal(got, ref), f"{what}: {int(np.sum(got != ref))} columns differ"
    for k in ("iterations", "converged", "cycles_applied", "edge_checks"):
        assert st[k] == rst[k], (what, k, st[k], rst[k])
    assert abs(st["weight_in"] - rst["weight_in"]) <= weight_tol(g, g.mate), what
    assert abs(st["weight_out"] - rst["weight_out"]) <= weight_tol(g, ref), what


def test_batched_4096_matrices(torch):
    specs = gen.batch_spec(4096)
    refs = oracle_pool.improve_specs(specs)
    graphs = [gen.build_spec(sp) for sp in specs]
    n_off, u = gen.union(graphs)
    assert u.nnz > 10**8
    d = torch.device("cuda")
    t = [torch.from_numpy(a).to(d) for a in (n_off, u.colptr, u.rowidx, u.weight, u.mate)]
    out = torch.empty_like(t[4])
    ctx = awpm.awpm_create(device=0)
    try:
        for rep in range(2):  # the second call reuses the context's graph
            tot, pm = awpm.awpm_improve_batch(ctx, len(graphs), *t, out)
            mates = gen.split(n_off, out.cpu().numpy())
            for b, g in enumerate(graphs):
                ref, rst = refs[b]
                _same(g, mates[b], pm[b], ref, rst, f"rep {rep} matrix {b} {g.name}")
            assert tot["iterations"] == max(r[1]["iterations"] for r in refs)
    finally:
        awpm.awpm_destroy(ctx)


def test_served_pool_large_requests(torch):
    specs = gen.serve_spec(28, seed=gen.SEED_BASE + 6)
    graphs = [gen.build_spec(sp) for sp in specs]
    assert sum(g.n > 300_000 for g in graphs) >= 2
    refs = oracle_pool.improve_specs(specs)
    d = torch.device("cuda")
    ctx = awpm.awpm_create(device=0, slots=4, mem_budget_bytes=100 * 10**9)
    solo = awpm.awpm_create(device=0)
    try:
        # all submitted at once, largest first, alternating host and device inputs
        order = sorted(range(len(graphs)), key=lambda k: -graphs[k].nnz)
        outs, keep, tickets = {}, {}, {}
        for r, k in enumerate(order):
            g = graphs[k]
            if r % 2:
                arrs = [torch.from_numpy(a).to(d) for a in (g.colptr, g.rowidx, g.weight, g.mate)]
                outs[k] = torch.empty(g.n, dtype=torch.int32, device=d)
            else:
                arrs = [g.colptr, g.rowidx, g.weight, g.mate]
                outs[k] = np.empty(g.n, dtype=np.int32)
            keep[k] = arrs
            tickets[k] = awpm.awpm_submit(ctx, g.n, *arrs, outs[k], nnz=g.nnz)
        for k in order:
            st = awpm.awpm_wait(ctx, tickets[k])
            g = graphs[k]
            got = outs[k].cpu().numpy() if hasattr(outs[k], "cpu") else outs[k]
            ref, rst = refs[k]
            _same(g, got, st, ref, rst, f"served {k} {g.name}")
            # the same problem alone on its own context
            o = np.empty(g.n, dtype=np.int32)
            st1 = awpm.awpm_improve_ctx(solo, g.n, g.colptr, g.rowidx, g.weight, g.mate, o)
            _same(g, o, st1, ref, rst, f"alone {k} {g.name}")
    finally:
        awpm.awpm_destroy(ctx)
        awpm.awpm_destroy(solo)
