"""Maximum cardinality matching on the GPU against the CPU oracle, through
the C ABI (needs a GPU): matchings, phases and cardinality bit-exact."""
import numpy as np
import pytest

import oracle
import pins
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


@pytest.fixture(scope="module")
def ctx(torch):
    c = awpm.awpm_create(device=0)
    yield c
    awpm.awpm_destroy(c)


def mcm_gpu(ctx, g, start, torch, host=False):
    m = np.full(g.n, -1, dtype=np.int32) if start is None else np.array(start, dtype=np.int32)
    if host:
        st = awpm.awpm_mcm(ctx, g.n, g.colptr, g.rowidx, g.weight, m)
        return m, st
    d = torch.device("cuda")
    cp, ri, w, dm = (torch.from_numpy(np.ascontiguousarray(x)).to(d)
                     for x in (g.colptr, g.rowidx, g.weight, m))
    st = awpm.awpm_mcm(ctx, g.n, cp, ri, w, dm)
    return dm.cpu().numpy(), st


def check(ctx, g, torch, start=None, host=False):
    ref, rst = oracle.get().mcm(g, start)
    got, st = mcm_gpu(ctx, g, start, torch, host)
    assert got.tolist() == ref.tolist(), g.name
    assert st["phases"] == rst["phases"] and st["cardinality"] == rst["cardinality"], (st, rst)
    return got, st


def test_from_empty_and_from_greedy(ctx, torch):
    orc = oracle.get()
    graphs = [pins.random_pattern(80 + 60 * s, 1 + s % 3, 9100 + s, integer_weights=(s % 2 == 0))
              for s in range(8)]
    graphs += [gen.rmat(1 << 12, 8, 9200), gen.random_small(500, 0.01, 9201),
               gen.stencil_2d(60, 9202)]
    for k, g in enumerate(graphs):
        check(ctx, g, torch, None, host=(k % 2 == 0))
        check(ctx, g, torch, orc.greedy(g)[0], host=(k % 2 == 1))


def test_hand_tie_breaks(ctx, torch):
    h = gen.from_dense(np.array([[1.0, 0.0], [5.0, 0.0]]),
                       np.array([[True, False], [True, False]]), [0, 1])
    got, _ = check(ctx, h, torch)
    assert got.tolist() == [1, -1]
    h2 = gen.from_dense(np.array([[1.0, 5.0], [0.0, 0.0]]),
                        np.array([[True, True], [False, False]]), [0, 1])
    got, _ = check(ctx, h2, torch)
    assert got.tolist() == [-1, 0]


def test_bad_start(ctx, torch):
    g = pins.random_pattern(200, 3, 9300)
    m = np.full(g.n, -1, dtype=np.int32)
    m[0] = g.rowidx[g.colptr[0]]
    m[1] = m[0]  # one row twice
    with pytest.raises(awpm.AwpmError) as ei:
        mcm_gpu(ctx, g, m, torch, host=True)
    assert ei.value.name == "NOT_PERFECT"
    check(ctx, g, torch)


def test_graph_and_host_loop_agree(torch):
    """The search as one graph launch (loops on the device) and with levels and
    phases driven from the host (AWPM_FLAG_TIME_SEARCH): same matching, same
    phase and level counts, twice in a row on one context (the cached graph)."""
    ch = awpm.awpm_create(device=0, flags=awpm.FLAG_TIME_SEARCH)
    cg = awpm.awpm_create(device=0)
    try:
        for g in (gen.rmat(1 << 13, 8, 9400), pins.random_pattern(700, 2, 9401),
                  gen.stencil_2d(50, 9402)):
            a, sa = mcm_gpu(ch, g, None, torch)
            for _ in range(2):
                b, sb = mcm_gpu(cg, g, None, torch)
                assert a.tolist() == b.tolist()
                assert (sa["phases"], sa["levels"], sa["cardinality"]) == \
                    (sb["phases"], sb["levels"], sb["cardinality"])
    finally:
        awpm.awpm_destroy(ch)
        awpm.awpm_destroy(cg)


def test_hand_cases_equal_weights(ctx, torch):
    """The hand-derived cases of tests/golden/mcm_cases.txt (equal offers to
    the lower column, equal ends to the lower row, a tree with an end stops
    growing): the GPU gives the expected matchings and phase counts."""
    import os
    for c in pins.load_hand_cases(os.path.join(pins.GOLDEN, "mcm_cases.txt")):
        g = pins.graph_of_case(c)
        for host in (False, True):
            got, st = mcm_gpu(ctx, g, c["mate"], torch, host=host)
            assert got.tolist() == c["expect_mate"], (c["name"], got)
            assert st["phases"] == c["expect_phases"], (c["name"], st)
            assert st["cardinality"] == c["expect_cardinality"], (c["name"], st)
