"""The greedy maximal matching on the GPU against the CPU oracle, through
the C ABI (needs a GPU): matchings, rounds and cardinality bit-exact, the
matched weight within 1e-12 of the sum of |matched weights|."""
import numpy as np
import pytest

import brute
import oracle
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


def greedy_gpu(ctx, g, torch, host=False):
    if host:
        out = np.empty(g.n, dtype=np.int32)
        st = awpm.awpm_greedy(ctx, g.n, g.colptr, g.rowidx, g.weight, out)
        return out, st
    cp, ri, w = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
                 for a in (g.colptr, g.rowidx, g.weight))
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st = awpm.awpm_greedy(ctx, g.n, cp, ri, w, out)
    return out.cpu().numpy(), st


def check(ctx, g, torch, host=False):
    ref, rst = oracle.get().greedy(g)
    got, st = greedy_gpu(ctx, g, torch, host)
    assert got.tolist() == ref.tolist(), g.name
    assert st["rounds"] == rst["rounds"] and st["cardinality"] == rst["cardinality"], (st, rst)
    scale = float(np.abs(g.weight).sum()) + 1.0
    assert abs(st["weight"] - rst["weight"]) <= 1e-12 * scale
    return got, st


def test_small_and_ties(ctx, torch):
    for s in range(12):
        g = gen.random_small(20 + 37 * s, 0.05 + 0.03 * (s % 4), 8100 + s,
                             integer_weights=(s % 2 == 0))
        check(ctx, g, torch, host=(s % 3 == 0))


def test_structures(ctx, torch):
    for g in (gen.stencil_2d(120, 8201), gen.stencil_3d(18, 8202), gen.banded(20000, 11, 8203),
              gen.rmat(1 << 15, 16, 8204), gen.config1()):
        got, st = check(ctx, g, torch)
        assert brute.is_maximal_matching(g, got) or g.n > 5000


def test_long_columns_and_equal_weights(ctx, torch):
    """Columns spanning many tiles (cross-warp maxima) and all-equal weights
    (every choice decided by the row and column order)."""
    rng = np.random.default_rng(8301)
    n = 5000
    rows, cols = [], []
    for hub in (7, 2500, 4999):
        r = rng.choice(n, size=3000, replace=False)
        rows.append(r)
        cols.append(np.full(r.size, hub))
    rows.append(rng.integers(0, n, 4 * n))
    cols.append(rng.integers(0, n, 4 * n))
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    colptr, rowidx = gen._csc_from_coo(n, np.concatenate(rows), np.concatenate(cols))
    w = gen.log_weights_lognormal(colptr, rng)
    g = gen.Graph(n, colptr, rowidx, w, np.arange(n, dtype=np.int32), "hubs")
    check(ctx, g, torch)
    g.weight = np.round(g.weight)  # few distinct values: ties everywhere
    check(ctx, g, torch)
    g.weight = np.zeros_like(g.weight)
    g.weight[::3] = -0.0
    check(ctx, g, torch)


def test_errors(ctx, torch):
    g = gen.random_small(30, 0.3, 8401)
    b = g.copy()
    b.weight[3] = np.nan
    with pytest.raises(awpm.AwpmError) as ei:
        greedy_gpu(ctx, b, torch)
    assert ei.value.name == "NONFINITE"
    b = g.copy()
    c = 11
    s0, e0 = int(g.colptr[c]), int(g.colptr[c + 1])
    b.rowidx = np.delete(g.rowidx, np.arange(s0, e0))
    b.weight = np.delete(g.weight, np.arange(s0, e0))
    b.colptr = g.colptr.copy()
    b.colptr[c + 1:] -= e0 - s0
    with pytest.raises(awpm.AwpmError) as ei:
        greedy_gpu(ctx, b, torch, host=True)
    assert ei.value.name == "NOT_PERFECT"
    check(ctx, g, torch)  # the context stays usable


def blocks_for_pipeline(nb, seed):
    """2x2 blocks [[10+u, 6+v], [6+x, 1+y]] (u, v, x, y in [0, 0.2]) along the
    diagonal plus light entries (-100) scattered off the blocks: greedy takes
    the heavy corner, then the light one, and is perfect; every block then
    has a weight-increasing 4-cycle (gain 1 + v + x - u - y > 0) and the
    off-block cycles all lose."""
    rng = np.random.default_rng(seed)
    n = 2 * nb
    rows, cols, vals = [], [], []
    for b in range(nb):
        u, v, x, y = rng.uniform(0.0, 0.2, 4)
        r0, c0 = 2 * b, 2 * b
        rows += [r0, r0, r0 + 1, r0 + 1]
        cols += [c0, c0 + 1, c0, c0 + 1]
        vals += [10 + u, 6 + v, 6 + x, 1 + y]
    extra = 3 * n
    er, ec = rng.integers(0, n, extra), rng.integers(0, n, extra)
    off = (er // 2) != (ec // 2)
    rows += er[off].tolist()
    cols += ec[off].tolist()
    vals += [-100.0] * int(off.sum())
    W = {}
    for r, c, v in zip(rows, cols, vals):
        W.setdefault((r, c), v)
    keys = sorted(W, key=lambda rc: (rc[1], rc[0]))
    colptr = np.zeros(n + 1, dtype=np.int32)
    for _, c in keys:
        colptr[c + 1] += 1
    colptr = np.cumsum(colptr).astype(np.int32)
    rowidx = np.array([r for r, _ in keys], dtype=np.int32)
    weight = np.array([W[k] for k in keys], dtype=np.float64)
    return gen.Graph(n, colptr, rowidx, weight, np.arange(n, dtype=np.int32), "blocks_pipeline")


def test_greedy_then_improve(ctx, torch):
    """Greedy from scratch, then the 4-cycle phase from its (perfect) result:
    both steps equal the oracle's, and the phase improves every block."""
    g = blocks_for_pipeline(2000, 8501)
    got, st = check(ctx, g, torch)
    assert st["cardinality"] == g.n
    ref, rst, _ = oracle.get().improve(g, mate=got)
    assert rst["cycles_applied"] == g.n // 2
    out = np.empty(g.n, dtype=np.int32)
    s2 = awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, got, out)
    assert out.tolist() == ref.tolist() and s2["iterations"] == rst["iterations"]


def test_improve_without_matching(ctx, torch):
    """awpm_improve with no matching runs the pipeline: greedy, then the
    maximum matching when greedy is not perfect, then the 4-cycle phase;
    NOT_PERFECT with a maximum matching when no perfect one exists."""
    orc = oracle.get()
    g = blocks_for_pipeline(500, 8601)
    gm, _ = orc.greedy(g)
    ref, rst, _ = orc.improve(g, mate=gm)
    out = np.empty(g.n, dtype=np.int32)
    st = awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, None, out)
    assert out.tolist() == ref.tolist() and st["cycles_applied"] == rst["cycles_applied"]
    h = gen.rmat(1 << 12, 8, 8602)            # greedy is not perfect here, the maximum is
    hm, hst = orc.greedy(h)
    assert hst["cardinality"] < h.n
    mm, mst = orc.mcm(h, hm)
    assert mst["cardinality"] == h.n
    ref, rst, _ = orc.improve(h, mate=mm)
    out = np.empty(h.n, dtype=np.int32)
    st = awpm.awpm_improve_ctx(ctx, h.n, h.colptr, h.rowidx, h.weight, None, out)
    assert out.tolist() == ref.tolist() and st["iterations"] == rst["iterations"]
    import pins
    z = pins.random_pattern(2000, 2, 8603)   # no perfect matching
    zm, zst = orc.greedy(z)
    zm, zst = orc.mcm(z, zm)
    assert zst["cardinality"] < z.n
    out = np.empty(z.n, dtype=np.int32)
    with pytest.raises(awpm.AwpmError) as ei:
        awpm.awpm_improve_ctx(ctx, z.n, z.colptr, z.rowidx, z.weight, None, out)
    assert ei.value.name == "NOT_PERFECT"
    assert out.tolist() == zm.tolist()


def test_host_loop_mode(torch):
    """Rounds launched from the host (AWPM_FLAG_TIME_SEARCH) give the graph's
    result."""
    c = awpm.awpm_create(device=0, flags=awpm.FLAG_TIME_SEARCH)
    try:
        for g in (gen.rmat(1 << 13, 16, 8701), gen.random_small(500, 0.05, 8702, integer_weights=True)):
            check(c, g, torch)
    finally:
        awpm.awpm_destroy(c)

