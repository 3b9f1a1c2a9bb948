"""Full-size workloads on the GPU against the CPU oracle, element by element
(needs a GPU; the oracle finishes each of these in well under two minutes).

Launch configuration as in bench.py: device-resident inputs, one context, the
default (graph) pass loop, and the timed (event) loop for the largest graph.
"""
import numpy as np
import pytest

import brute
import oracle
from gpu_helpers import assert_same_as_oracle, run_gpu
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


@pytest.mark.parametrize("maker", [gen.config2, gen.config3a, gen.config3b],
                         ids=["stencil2d_1000", "stencil3d_96", "rmat_s22"])
def test_full_size(torch, maker):
    g = maker()
    ref, rst, _ = oracle_improve(g)
    modes = [0, awpm.FLAG_TIME_SEARCH] if g.n > 4_000_000 else [0]
    for flags in modes:
        c = awpm.awpm_create(device=0, flags=flags)
        try:
            got, st = run_gpu(c, g, torch=torch)
            assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} flags={flags}")
            # run twice: the cached graph gives the same result
            got2, st2 = run_gpu(c, g, torch=torch)
            assert np.array_equal(got2, got) and st2["weight_out"] == st["weight_out"]
        finally:
            awpm.awpm_destroy(c)
    assert rst["converged"] == 1
    assert brute.no_positive_4cycle_vectorized(g, got)


_ORACLE = {}


def oracle_improve(g, **kw):
    """The oracle's phase on a full-size graph, computed once per module."""
    key = (g.name, tuple(sorted(kw.items())))
    if key not in _ORACLE:
        _ORACLE[key] = oracle.get().improve(g, **kw)
    return _ORACLE[key]


@pytest.fixture(scope="module")
def rmat22():
    return gen.config3b()


@pytest.mark.parametrize("lookup", [awpm.LOOKUP_HASH, awpm.LOOKUP_ROWMARK], ids=["hash", "rowmark"])
def test_full_size_lookups(torch, rmat22, lookup):
    """The per-column hash tables and row marking (transpose of 69 M entries,
    three radix passes) on the largest graph, element by element."""
    g = rmat22
    ref, rst, _ = oracle_improve(g)
    c = awpm.awpm_create(device=0, lookup=lookup)
    try:
        got, st = run_gpu(c, g, torch=torch)
        assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} lookup={lookup}")
        assert st["lookup_used"] == lookup
    finally:
        awpm.awpm_destroy(c)


def test_full_size_pipeline(torch, rmat22):
    """The whole pipeline from no matching on the largest graph: the GPU's
    greedy matching, its maximum matching from that start (19 phases) and
    the 4-cycle phase each equal the oracle's."""
    g = rmat22
    orc = oracle.get()
    gm, gst = orc.greedy(g)
    mm, mst = orc.mcm(g, gm)
    assert mst["cardinality"] == g.n
    ref, rst, _ = orc.improve(g, mate=mm)
    d = torch.device("cuda")
    cp, ri, w = (torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (g.colptr, g.rowidx, g.weight))
    m = torch.empty(g.n, dtype=torch.int32, device=d)
    c = awpm.awpm_create(device=0)
    try:
        st = awpm.awpm_greedy(c, g.n, cp, ri, w, m)
        assert np.array_equal(m.cpu().numpy(), gm) and st["cardinality"] == gst["cardinality"]
        st = awpm.awpm_mcm(c, g.n, cp, ri, w, m)
        assert np.array_equal(m.cpu().numpy(), mm)
        assert (st["phases"], st["cardinality"]) == (mst["phases"], mst["cardinality"])
        out = torch.empty_like(m)
        st = awpm.awpm_improve_ctx(c, g.n, cp, ri, w, None, out)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert st["iterations"] == rst["iterations"]
        assert st["cycles_applied"] == rst["cycles_applied"]
    finally:
        awpm.awpm_destroy(c)


def test_full_size_pettie_sanders(torch):
    """The Pettie-Sanders selection on the 27-point stencil (16 passes, many
    competing cycles), element by element."""
    g = gen.config3a()
    ref, rst, _ = oracle_improve(g, select=1)
    c = awpm.awpm_create(device=0, select=awpm.SELECT_GREEDY)
    try:
        got, st = run_gpu(c, g, torch=torch)
        assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} select=greedy")
    finally:
        awpm.awpm_destroy(c)
