"""CUDA path against the CPU oracle, through the C ABI (needs a GPU).

Matchings, pass counts and request counters must be bit-exact; total weights
agree within 1e-12 of the sum of |matched weights| (only the summation order
differs).
"""
import numpy as np
import pytest

import brute
import oracle
import pins
from gpu_helpers import assert_same_as_oracle, run_gpu, to_device, weight_tol
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


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


def check(ctx, orc, g, torch, mate=None, max_iters=0, host=False, what=""):
    ref, rst, _ = orc.improve(g, mate=mate, max_iters=max_iters)
    got, st = run_gpu(ctx, g, mate=mate, torch=torch, host=host)
    assert_same_as_oracle(g, got, st, ref, rst, what or g.name)
    return got, st


def test_hand_cases(ctx, orc, torch):
    for c in pins.load_hand_cases():
        g = pins.graph_of_case(c)
        got, st = run_gpu(ctx, g, torch=torch)
        assert got.tolist() == c["expect_mate"], c["name"]
        assert st["iterations"] == c["expect_iterations"], c["name"]
        assert st["cycles_applied"] == c["expect_cycles"], c["name"]
        assert st["weight_out"] == c["expect_weight"], c["name"]
        check(ctx, orc, g, torch, what=c["name"])


def test_2x2_closed_form(ctx, orc, torch):
    rng = np.random.default_rng(3)
    for _ in range(40):
        w00, w01, w10, w11 = rng.choice([-2.0, -1.0, -0.5, 0.0, 1.0], 4)
        g = pins.full2(w00, w01, w10, w11)
        got, st = run_gpu(ctx, g, torch=torch)
        flip = (w01 + w10) > (w00 + w11)
        assert got.tolist() == ([1, 0] if flip else [0, 1])


@pytest.mark.parametrize("integer", [False, True], ids=["lognormal", "integer_ties"])
def test_random_small(ctx, orc, torch, integer):
    for s in range(150):
        n = 2 + (s * 7) % 90
        g = gen.random_small(n, (0.05, 0.2, 0.5, 0.9)[s % 4], 5000 + s, integer_weights=integer)
        check(ctx, orc, g, torch, what=f"seed {s}")


@pytest.mark.parametrize("maker", [
    lambda: gen.config1(),
    lambda: gen.stencil_2d(97, 11, weights="diag"),
    lambda: gen.stencil_2d(64, 12, weights="lognormal"),
    lambda: gen.stencil_3d(13, 13),
    lambda: gen.banded(7001, 9, 14),
    lambda: gen.banded(3000, 15, 15),
    lambda: gen.random_sparse(30001, 12, 16),
    lambda: gen.rmat(1 << 14, 16, 17),
    lambda: gen.rmat(20011, 9, 18),
], ids=["config1", "st2d_97", "st2d_64_ln", "st3d_13", "band_7001_9", "band_3000_15",
        "rs_30001", "rmat_s14", "rmat_20011"])
def test_medium_graphs(ctx, orc, torch, maker):
    g = maker()
    check(ctx, orc, g, torch)


def test_stepc_records(ctx, orc, torch):
    """Step-C winners of one search (gain and row per root column), element by
    element, from the planted matching and from intermediate matchings."""
    for g in (gen.stencil_2d(80, 21), gen.stencil_3d(11, 22), gen.rmat(1 << 13, 16, 23),
              gen.random_small(60, 0.5, 24, integer_weights=True)):
        mates = [g.mate]
        for t in (1, 2):
            m, st, _ = orc.improve(g, max_iters=t)
            mates.append(m)
        for m in mates:
            rg, rr, cnt = orc.step_c(g, m)
            cp, ri, w, _ = to_device(g, torch)
            md = torch.from_numpy(np.ascontiguousarray(m)).cuda()
            gg = torch.empty(g.n, dtype=torch.float64, device="cuda")
            rw = torch.empty(g.n, dtype=torch.int32, device="cuda")
            st = awpm.awpm_search(ctx, g.n, cp, ri, w, md, gg, rw)
            assert np.array_equal(rw.cpu().numpy(), rr), g.name
            assert np.array_equal(gg.cpu().numpy(), rg), g.name  # bit-exact gains
            assert st["candidates"] == cnt[0] and st["closing_found"] == cnt[1]
            assert st["positive"] == cnt[2]
            # host output arrays give the same
            hg = np.empty(g.n, dtype=np.float64)
            hr = np.empty(g.n, dtype=np.int32)
            awpm.awpm_search(ctx, g.n, g.colptr, g.rowidx, g.weight, np.ascontiguousarray(m), hg, hr)
            assert np.array_equal(hr, rr) and np.array_equal(hg, rg)


def test_host_and_device_pointers_agree(ctx, orc, torch):
    g = gen.stencil_2d(50, 31)
    a, sa = run_gpu(ctx, g, torch=torch, host=False)
    b, sb = run_gpu(ctx, g, torch=torch, host=True)
    assert np.array_equal(a, b) and sa["iterations"] == sb["iterations"]
    assert sa["weight_out"] == sb["weight_out"]


def test_timed_mode_same_result(torch, orc):
    c = awpm.awpm_create(device=0, flags=awpm.FLAG_TIME_SEARCH)
    try:
        for g in (gen.stencil_3d(12, 41), gen.rmat(1 << 12, 8, 42), gen.config1()):
            got, st = run_gpu(c, g, torch=torch)
            ref, rst, _ = orc.improve(g)
            assert_same_as_oracle(g, got, st, ref, rst, g.name)
            assert st["ms_search"] > 0.0
    finally:
        awpm.awpm_destroy(c)


@pytest.mark.parametrize("max_iters", [1, 2, 3, 10])
def test_max_iters(torch, orc, max_iters):
    c = awpm.awpm_create(device=0, max_iters=max_iters)
    try:
        for g in (gen.stencil_3d(12, 51), gen.stencil_2d(60, 52)):
            ref, rst, _ = orc.improve(g, max_iters=max_iters)
            got, st = run_gpu(c, g, torch=torch)
            assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} max_iters={max_iters}")
    finally:
        awpm.awpm_destroy(c)


def test_resume_from_intermediate(ctx, orc, torch):
    g = gen.stencil_3d(12, 61)
    full, fst = run_gpu(ctx, g, torch=torch)
    c1 = awpm.awpm_create(device=0, max_iters=2)
    try:
        mid, mst = run_gpu(c1, g, torch=torch)
    finally:
        awpm.awpm_destroy(c1)
    fin, st2 = run_gpu(ctx, g, mate=mid, torch=torch)
    assert np.array_equal(fin, full)
    assert mst["iterations"] + st2["iterations"] == fst["iterations"]


def test_mate_out_aliases_mate_in(ctx, orc, torch):
    g = gen.stencil_2d(40, 71)
    ref, rst, _ = orc.improve(g)
    cp, ri, w, m = to_device(g, torch)
    st = awpm.awpm_improve_ctx(ctx, g.n, cp, ri, w, m, m)
    assert np.array_equal(m.cpu().numpy(), ref)


def test_default_context_entry_point(orc, torch):
    g = gen.stencil_2d(30, 81)
    ref, rst, _ = orc.improve(g)
    cp, ri, w, m = to_device(g, torch)
    out = torch.empty_like(m)
    st = awpm.awpm_improve(g.n, cp, ri, w, m, out)
    assert np.array_equal(out.cpu().numpy(), ref) and st["iterations"] == rst["iterations"]


@pytest.mark.parametrize("lookup", [awpm.LOOKUP_AUTO, awpm.LOOKUP_ROWMARK], ids=["auto", "rowmark"])
def test_degenerate_sizes(orc, torch, lookup):
    """n = 0, n = 1, and diagonal-only matrices (no candidate at all), also
    through row marking (a transpose of one entry; 1 to 2 radix passes)."""
    ctx = awpm.awpm_create(device=0, lookup=lookup)
    try:
        out = np.empty(0, dtype=np.int32)
        st = awpm.awpm_improve_ctx(ctx, 0, np.zeros(1, np.int32), np.zeros(0, np.int32),
                                   np.zeros(0), np.zeros(0, np.int32), out)
        assert st["iterations"] == 1 and st["converged"] == 1
        for n in (1, 2, 7, 257, 1000):
            W = np.diag(np.arange(n, dtype=np.float64) * -0.5)
            g = gen.from_dense(W, np.eye(n, dtype=bool), np.arange(n))
            check(ctx, orc, g, torch, what=f"diag n={n}")
        # a full 2 x 2 (one flip) and a full 3 x 3
        for n in (2, 3):
            W = np.arange(n * n, dtype=np.float64).reshape(n, n) % 5 - 2.0
            g = gen.from_dense(W, np.ones((n, n), dtype=bool), np.arange(n))
            check(ctx, orc, g, torch, what=f"full n={n}")
    finally:
        awpm.awpm_destroy(ctx)


def test_skewed_columns(ctx, orc, torch):
    """A few very long columns (thousands of tiles) among tiny ones: columns
    that straddle many tiles are combined across warps."""
    rng = np.random.default_rng(91)
    n = 20000
    rows, cols = [], []
    for hub in (3, 777, 15000):
        r = rng.choice(n, size=12000, replace=False)
        rows.append(r)
        cols.append(np.full(r.size, hub))
    rows.append(rng.integers(0, n, 3 * n))
    cols.append(rng.integers(0, n, 3 * n))
    mate = rng.permutation(n)
    rows.append(mate)
    cols.append(np.arange(n))
    colptr, rowidx = gen._csc_from_coo(n, np.concatenate(rows), np.concatenate(cols))
    w = gen.log_weights_lognormal(colptr, rng)
    g = gen.Graph(n, colptr, rowidx, w, mate.astype(np.int32), "skewed")
    check(ctx, orc, g, torch)
    # hub rows too: a dense row makes many roots share one key column
    W = np.zeros((300, 300))
    S = rng.random((300, 300)) < 0.05
    S[5, :] = True
    S[:, 9] = True
    p = rng.permutation(300)
    S[p, np.arange(300)] = True
    W[S] = np.round(rng.standard_normal(int(S.sum())) * 4) / 4
    check(ctx, orc, gen.from_dense(W, S, p), torch, what="dense row+col, ties")


def test_long_columns_bloom(ctx, orc, torch):
    """Columns longer than 32 rows carry Bloom filters in front of the binary
    search: long columns next to each other (filter words shared at their
    boundaries), closing entries mostly absent (sparse) or mostly present
    (dense, integer weights with ties)."""
    rng = np.random.default_rng(171)
    n = 6000
    deg = np.where(rng.random(n) < 0.5, rng.integers(33, 400, size=n), rng.integers(1, 9, size=n))
    rows = [rng.choice(n, size=int(d), replace=False) for d in deg]
    cols = [np.full(int(d), c) for c, d in enumerate(deg)]
    mate = rng.permutation(n)
    rows.append(mate)
    cols.append(np.arange(n))
    colptr, rowidx = gen._csc_from_coo(n, np.concatenate(rows), np.concatenate(cols))
    w = gen.log_weights_lognormal(colptr, rng)
    g = gen.Graph(n, colptr, rowidx, w, mate.astype(np.int32), "long_columns")
    assert np.mean(np.diff(g.colptr) > 32) > 0.4
    check(ctx, orc, g, torch)
    check(ctx, orc, gen.random_small(400, 0.3, 172, integer_weights=True), torch,
          what="dense, integer ties")


@pytest.mark.parametrize("kind,expect", [
    ("dup_mate", "NOT_PERFECT"), ("mate_out_of_range", "NOT_PERFECT"),
    ("mate_not_stored", "NOT_PERFECT"), ("inf_weight", "NONFINITE"), ("nan_weight", "NONFINITE"),
    ("row_out_of_range", "INVALID_ARG"), ("bad_colptr", "INVALID_ARG"),
    ("unsorted", "UNSORTED_OR_DUP"), ("duplicate_row", "UNSORTED_OR_DUP"),
    ("unsorted_and_nonfinite", "UNSORTED_OR_DUP"), ("empty_column", "NOT_PERFECT"),
])
def test_validation_errors(ctx, orc, torch, kind, expect):
    g = gen.random_small(30, 0.3, 101)
    W, S = brute.dense(g)
    b = g.copy()
    j = int(np.argmax(np.diff(g.colptr)))
    a0 = int(g.colptr[j])
    if kind == "dup_mate":
        b.mate[0] = b.mate[1]
    elif kind == "mate_out_of_range":
        b.mate[3] = 30
    elif kind == "mate_not_stored":
        for c in range(g.n):
            miss = [r for r in range(g.n) if not S[r, c]]
            if miss:
                other = int(np.nonzero(b.mate == miss[0])[0][0])
                b.mate[c], b.mate[other] = miss[0], b.mate[c]
                break
    elif kind == "inf_weight":
        b.weight[5] = -np.inf
    elif kind == "nan_weight":
        b.weight[7] = np.nan
    elif kind == "row_out_of_range":
        b.rowidx[4] = 31
    elif kind == "bad_colptr":
        b.colptr[10] = b.colptr[11] + 1
    elif kind == "unsorted":
        b.rowidx[a0], b.rowidx[a0 + 1] = g.rowidx[a0 + 1], g.rowidx[a0]
    elif kind == "duplicate_row":
        b.rowidx[a0 + 1] = g.rowidx[a0]
    elif kind == "unsorted_and_nonfinite":
        b.rowidx[a0], b.rowidx[a0 + 1] = g.rowidx[a0 + 1], g.rowidx[a0]
        b.weight[0] = np.nan
    elif kind == "empty_column":
        c = 11
        s0, e0 = int(g.colptr[c]), int(g.colptr[c + 1])
        b.rowidx = np.delete(g.rowidx, np.arange(s0, e0))
        b.weight = np.delete(g.weight, np.arange(s0, e0))
        b.colptr = g.colptr.copy()
        b.colptr[c + 1:] -= e0 - s0
    assert orc.validate(b) == expect
    for host in (False, True):
        with pytest.raises(awpm.AwpmError) as ei:
            run_gpu(ctx, b, torch=torch, host=host)
        assert ei.value.name == expect, (kind, host)
    # the context stays usable after an error
    check(ctx, orc, g, torch, what="after error")


def test_invalid_host_arguments(ctx, torch):
    g = gen.random_small(10, 0.4, 111)
    out = np.empty(g.n, dtype=np.int32)
    with pytest.raises(awpm.AwpmError) as ei:
        awpm.awpm_improve_ctx(ctx, -1, g.colptr, g.rowidx, g.weight, g.mate, out)
    assert ei.value.name == "INVALID_ARG"
    with pytest.raises(awpm.AwpmError) as ei:
        awpm.awpm_improve_ctx(ctx, g.n, None, g.rowidx, g.weight, g.mate, out)
    assert ei.value.name == "INVALID_ARG"


def test_memory_budget(torch):
    c = awpm.awpm_create(device=0, mem_budget_bytes=1 << 16)
    try:
        g = gen.stencil_2d(100, 121)
        with pytest.raises(awpm.AwpmError) as ei:
            run_gpu(c, g, torch=torch)
        assert ei.value.name == "BUDGET"
    finally:
        awpm.awpm_destroy(c)


def test_context_reuse_across_sizes(ctx, orc, torch):
    """Workspace growth and graph re-capture across problem sizes and back."""
    for g in (gen.stencil_2d(20, 131), gen.stencil_2d(150, 132), gen.stencil_2d(20, 131),
              gen.rmat(5000, 6, 133), gen.stencil_2d(150, 132)):
        check(ctx, orc, g, torch)


@pytest.mark.parametrize("lookup", [awpm.LOOKUP_BSEARCH, awpm.LOOKUP_HASH, awpm.LOOKUP_ROWMARK],
                         ids=["bsearch", "hash", "rowmark"])
def test_lookup_strategies(torch, orc, lookup):
    """The three closing-edge lookups (binary search, per-column hash table,
    row marking) give the oracle's result, ties and dense columns included."""
    c = awpm.awpm_create(device=0, lookup=lookup)
    try:
        graphs = [gen.stencil_3d(14, 141), gen.rmat(1 << 14, 16, 142), gen.config1(),
                  gen.random_small(300, 0.2, 143, integer_weights=True),
                  gen.banded(5000, 13, 144)]
        for g in graphs:
            ref, rst, _ = orc.improve(g)
            got, st = run_gpu(c, g, torch=torch)
            assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} lookup={lookup}")
            assert st["lookup_used"] == lookup
    finally:
        awpm.awpm_destroy(c)


def test_autotuner_trials_are_exact(torch, orc):
    """lookup AUTO: the first solves of a problem class try each launch
    configuration (each a full solve), then one is kept; every result equals
    the oracle's."""
    c = awpm.awpm_create(device=0)  # lookup AUTO
    try:
        g = gen.rmat(1 << 13, 16, 151)
        ref, rst, _ = orc.improve(g)
        used = []
        for _ in range(6):
            got, st = run_gpu(c, g, torch=torch)
            assert_same_as_oracle(g, got, st, ref, rst, "autotuned")
            used.append(st["lookup_used"])
        assert set(used[:3]) == {awpm.LOOKUP_BSEARCH, awpm.LOOKUP_HASH}
        assert len(set(used[3:])) == 1
        # a different size class starts its own trials
        g2 = gen.stencil_2d(40, 152)
        ref2, rst2, _ = orc.improve(g2)
        got2, st2 = run_gpu(c, g2, torch=torch)
        assert_same_as_oracle(g2, got2, st2, ref2, rst2, "autotuned 2")
    finally:
        awpm.awpm_destroy(c)


@pytest.mark.parametrize("flags", [0, awpm.FLAG_TIME_SEARCH], ids=["graph", "timed"])
def test_greedy_selection(torch, orc, flags):
    """The Pettie-Sanders selection instead of Step D (rounds of winners named
    by both their columns; a WHILE node nested in the pass graph, or rounds
    driven from the host): the oracle's result in that mode, ties included."""
    c = awpm.awpm_create(device=0, select=awpm.SELECT_GREEDY, flags=flags)
    try:
        graphs = [gen.random_small(300, 0.2, 161, integer_weights=True), gen.config1(),
                  gen.stencil_2d(60, 162), gen.stencil_3d(12, 163), gen.rmat(1 << 13, 16, 164),
                  gen.banded(4000, 9, 165)]
        graphs += [gen.random_small(8 + s, 0.7, 170 + s, integer_weights=True) for s in range(10)]
        for g in graphs:
            ref, rst, _ = orc.improve(g, select=1)
            got, st = run_gpu(c, g, torch=torch)
            assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} select=greedy")
        for mi in (1, 2):
            g = gen.stencil_3d(10, 166)
            c2 = awpm.awpm_create(device=0, select=awpm.SELECT_GREEDY, flags=flags, max_iters=mi)
            try:
                ref, rst, _ = orc.improve(g, select=1, max_iters=mi)
                got, st = run_gpu(c2, g, torch=torch)
                assert_same_as_oracle(g, got, st, ref, rst, f"max_iters={mi}")
            finally:
                awpm.awpm_destroy(c2)
    finally:
        awpm.awpm_destroy(c)



def arrow_graph(n, seed):
    """Planted diagonal plus a full row 0 and a full column 0: row 0's
    neighbourhood is long (warp-cooperative search) and every other row is
    short."""
    rng = np.random.default_rng(seed)
    rows = np.concatenate([np.arange(n), np.zeros(n, dtype=np.int64), np.arange(n)])
    cols = np.concatenate([np.arange(n), np.arange(n), np.zeros(n, dtype=np.int64)])
    colptr, rowidx = gen._csc_from_coo(n, rows, cols)
    w = rng.standard_normal(len(rowidx))
    return gen.Graph(n, colptr, rowidx, w, np.arange(n, dtype=np.int32), f"arrow_{n}")


@pytest.mark.parametrize("flags", [0, awpm.FLAG_TIME_SEARCH], ids=["graph", "timed"])
def test_row_marking_transpose_and_selections(torch, orc, flags):
    """Row marking (Section 4) on the shapes its transpose must handle: one,
    two and three radix passes (n up to 256, up to 65,536, above), a row with
    thousands of entries, hub rows, empty-free ragged tails; under Step D
    and the Pettie-Sanders selection; every result equals the oracle's row
    marking mode and its column-search mode."""
    graphs = [gen.random_small(200, 0.05, 161), gen.stencil_2d(300, 162),
              gen.rmat(1 << 17, 8, 163), arrow_graph(3000, 164), gen.banded(70001, 7, 165)]
    for sel in (awpm.SELECT_STEP_D, awpm.SELECT_GREEDY):
        c = awpm.awpm_create(device=0, lookup=awpm.LOOKUP_ROWMARK, select=sel, flags=flags)
        try:
            for g in graphs:
                ref, rst, _ = orc.improve(g, select=sel, row_marking=True)
                ref2, _, _ = orc.improve(g, select=sel)
                assert ref.tolist() == ref2.tolist()
                got, st = run_gpu(c, g, torch=torch)
                assert_same_as_oracle(g, got, st, ref, rst, f"{g.name} rowmark sel={sel}")
                assert st["lookup_used"] == awpm.LOOKUP_ROWMARK
        finally:
            awpm.awpm_destroy(c)
