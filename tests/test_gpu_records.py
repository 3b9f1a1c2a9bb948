"""A solve skips clearing the Step-C and Step-D records when the previous
solve on the context left them empty (a single solve with Step D's
selection that ended without error), and clears them otherwise.  Sequences
of solves on one context -- smaller and larger problems, a failed solve, a
search-only call (which leaves its records behind), a batched solve, a
pass-capped solve and the greedy selection in between -- each give the
oracle's result (needs a GPU)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import assert_same_as_oracle, run_gpu
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


def check(ctx, g, torch, max_iters=0, select=0, host=False):
    ref, rst, _ = oracle.get().improve(g, max_iters=max_iters, select=select)
    got, st = run_gpu(ctx, g, torch=torch, host=host)
    assert_same_as_oracle(g, got, st, ref, rst, g.name)


def test_sequence_on_one_context(torch):
    a = gen.rmat(1 << 13, 12, 9801)
    b = gen.rmat(1 << 12, 12, 9802)
    c = gen.rmat(1 << 14, 12, 9803)
    s = gen.stencil_2d(60, 9804)
    ctx = awpm.awpm_create(device=0, lookup=awpm.LOOKUP_BSEARCH)
    try:
        check(ctx, a, torch)
        check(ctx, b, torch)               # smaller: records left empty by the solve before
        check(ctx, c, torch, host=True)    # larger: cleared
        check(ctx, a, torch)
        bad = np.array(b.mate, dtype=np.int32)
        bad[1] = bad[0]                    # a row matched twice
        with pytest.raises(awpm.AwpmError):
            awpm.awpm_improve_ctx(ctx, b.n, b.colptr, b.rowidx, b.weight, bad,
                                  np.empty(b.n, np.int32))
        check(ctx, a, torch)               # after an error: cleared
        gain = np.empty(c.n, np.float64)
        row = np.empty(c.n, np.int32)
        awpm.awpm_search(ctx, c.n, c.colptr, c.rowidx, c.weight, c.mate, gain, row)
        assert np.any(gain > 0)            # records written and not flipped
        check(ctx, c, torch)               # after a search-only call: cleared
        check(ctx, b, torch)
        graphs = [gen.build_spec(sp) for sp in gen.batch_spec(12, seed=9805)]
        n_off, u = gen.union(graphs)
        out = np.empty(u.n, np.int32)
        awpm.awpm_improve_batch(ctx, len(graphs), n_off, u.colptr, u.rowidx, u.weight, u.mate,
                                out)
        orc = oracle.get()
        for k, m in enumerate(gen.split(n_off, out)):
            assert np.array_equal(m, orc.improve(graphs[k])[0]), k
        awpm.awpm_improve_batch(ctx, len(graphs), n_off, u.colptr, u.rowidx, u.weight, u.mate,
                                out)                 # its records left empty by the first
        for k, m in enumerate(gen.split(n_off, out)):
            assert np.array_equal(m, orc.improve(graphs[k])[0]), k
        check(ctx, s, torch)               # after a batched solve: left empty
        check(ctx, s, torch, host=True)
    finally:
        awpm.awpm_destroy(ctx)


def test_pass_cap_and_greedy_selection(torch):
    a = gen.rmat(1 << 13, 12, 9806)
    s = gen.stencil_2d(50, 9807)
    capped = awpm.awpm_create(device=0, lookup=awpm.LOOKUP_BSEARCH, max_iters=1)
    greedy = awpm.awpm_create(device=0, lookup=awpm.LOOKUP_BSEARCH, select=1)
    try:
        for g in (a, s, a):
            check(capped, g, torch, max_iters=1)
            check(greedy, g, torch, select=1)
    finally:
        awpm.awpm_destroy(capped)
        awpm.awpm_destroy(greedy)
