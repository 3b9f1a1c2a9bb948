"""Batched solves (block-diagonal union, one graph launch) against the CPU
oracle run on each matrix alone (needs a GPU)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import weight_tol
from paper_1801_09809_gb300 import awpm, gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09809_gb300 import build
    build.build()
    return _t


def run_batch(ctx, graphs, torch, host=False):
    n_off, u = gen.union(graphs)
    if host:
        out = np.empty(u.n, dtype=np.int32)
        tot, pm = awpm.awpm_improve_batch(ctx, len(graphs), n_off, u.colptr, u.rowidx, u.weight,
                                          u.mate, out)
        return gen.split(n_off, out), tot, pm
    d = torch.device("cuda")
    t = [torch.from_numpy(a).to(d) for a in (n_off, u.colptr, u.rowidx, u.weight, u.mate)]
    out = torch.empty_like(t[4])
    tot, pm = awpm.awpm_improve_batch(ctx, len(graphs), *t, out)
    return gen.split(n_off, out.cpu().numpy()), tot, pm


def check_batch(ctx, graphs, torch, max_iters=0, host=False, select=0):
    mates, tot, pm = run_batch(ctx, graphs, torch, host=host)
    orc = oracle.get()
    passes = 0
    for b, g in enumerate(graphs):
        ref, rst, _ = orc.improve(g, max_iters=max_iters, select=select)
        assert np.array_equal(mates[b], ref), (b, g.name)
        assert pm[b]["iterations"] == rst["iterations"], (b, g.name, pm[b], rst)
        assert pm[b]["converged"] == rst["converged"], (b, g.name)
        assert pm[b]["cycles_applied"] == rst["cycles_applied"], (b, g.name)
        assert pm[b]["edge_checks"] == rst["edge_checks"], (b, g.name)
        assert abs(pm[b]["weight_in"] - rst["weight_in"]) <= weight_tol(g, g.mate)
        assert abs(pm[b]["weight_out"] - rst["weight_out"]) <= weight_tol(g, ref)
        passes = max(passes, rst["iterations"])
    assert tot["iterations"] == passes
    return tot, pm


def test_batch_mixed_structures(torch):
    specs = gen.batch_spec(48, seed=424242)
    graphs = [gen.build_spec(sp) for sp in specs]
    for lookup in (awpm.LOOKUP_BSEARCH, awpm.LOOKUP_HASH, awpm.LOOKUP_ROWMARK):
        ctx = awpm.awpm_create(device=0, lookup=lookup)
        try:
            check_batch(ctx, graphs, torch)
        finally:
            awpm.awpm_destroy(ctx)


def test_batch_alone_equals_mixed(torch):
    """A matrix gives the same result alone, in a small batch and in a large
    one (different neighbours, different tile boundaries)."""
    target = gen.stencil_3d(9, 777)
    others = [gen.build_spec(sp) for sp in gen.batch_spec(30, seed=31337)]
    ctx = awpm.awpm_create(device=0)
    try:
        alone, _, pa = run_batch(ctx, [target], torch)
        mid, _, pm = run_batch(ctx, others[:5] + [target] + others[5:9], torch)
        big, _, pb = run_batch(ctx, others + [target], torch)
        assert np.array_equal(alone[0], mid[5]) and np.array_equal(alone[0], big[-1])
        assert pa[0]["iterations"] == pm[5]["iterations"] == pb[-1]["iterations"]
        # and equal to the single-matrix entry point
        out = np.empty(target.n, dtype=np.int32)
        st = awpm.awpm_improve_ctx(ctx, target.n, target.colptr, target.rowidx, target.weight,
                                   target.mate, out)
        assert np.array_equal(out, alone[0]) and st["iterations"] == pa[0]["iterations"]
    finally:
        awpm.awpm_destroy(ctx)


@pytest.mark.parametrize("max_iters", [1, 3])
def test_batch_pass_cap(torch, max_iters):
    graphs = [gen.stencil_3d(8, 900 + k) for k in range(6)] + [gen.stencil_2d(20, 950)]
    ctx = awpm.awpm_create(device=0, max_iters=max_iters)
    try:
        check_batch(ctx, graphs, torch, max_iters=max_iters)
    finally:
        awpm.awpm_destroy(ctx)


def test_batch_host_arrays_and_timed_mode(torch):
    graphs = [gen.build_spec(sp) for sp in gen.batch_spec(12, seed=5150)]
    ctx = awpm.awpm_create(device=0, flags=awpm.FLAG_TIME_SEARCH)
    try:
        check_batch(ctx, graphs, torch, host=True)
        check_batch(ctx, graphs, torch, host=False)
    finally:
        awpm.awpm_destroy(ctx)


def test_batch_tiny_and_degenerate(torch):
    """Many tiny matrices: several per tile, a 1x1, a diagonal-only one."""
    graphs = [gen.random_small(2 + k % 5, 0.6, 60 + k, integer_weights=True) for k in range(40)]
    graphs.insert(7, gen.from_dense(np.array([[0.5]]), np.ones((1, 1), bool), [0]))
    graphs.insert(20, gen.from_dense(np.diag([-1.0, -2.0, -3.0]), np.eye(3, dtype=bool), [0, 1, 2]))
    ctx = awpm.awpm_create(device=0)
    try:
        check_batch(ctx, graphs, torch)
    finally:
        awpm.awpm_destroy(ctx)


def test_batch_rejects_cross_block_entries(torch):
    g1, g2 = gen.stencil_2d(6, 1), gen.stencil_2d(6, 2)
    n_off, u = gen.union([g1, g2])
    bad = u.copy()
    # move one off-diagonal entry of block 0 to a row of block 1 (keeps the
    # column sorted: the last entry of column 0 gets the largest row)
    last = int(u.colptr[1]) - 1
    if u.rowidx[last] != u.mate[0]:
        bad.rowidx[last] = u.n - 1
        ctx = awpm.awpm_create(device=0)
        try:
            with pytest.raises(awpm.AwpmError) as ei:
                awpm.awpm_improve_batch(ctx, 2, n_off, bad.colptr, bad.rowidx, bad.weight,
                                        bad.mate, np.empty(u.n, np.int32))
            assert ei.value.name == "INVALID_ARG"
        finally:
            awpm.awpm_destroy(ctx)


def test_batch_greedy_selection(torch):
    """The Pettie-Sanders selection on a batch: cycles of different matrices
    never share a column, so the union's selection is each matrix's own."""
    graphs = [gen.build_spec(sp) for sp in gen.batch_spec(24, seed=6060)]
    graphs += [gen.random_small(40, 0.2, 6100 + k, integer_weights=True) for k in range(8)]
    ctx = awpm.awpm_create(device=0, select=awpm.SELECT_GREEDY)
    try:
        check_batch(ctx, graphs, torch, select=1)
    finally:
        awpm.awpm_destroy(ctx)

