"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each pin takes an oracle instance and raises AssertionError when the oracle
disagrees.  They are collected in PINS so that the same suite can be run
against deliberately broken copies of the oracle (tests/test_oracle_mutants.py):
every plausible mistake must trip at least one pin.
"""
from __future__ import annotations

import os

import numpy as np

import brute
from paper_1801_09809_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------
# fixtures
# ----------------------------------------------------------------------------

def load_hand_cases(path=os.path.join(GOLDEN, "hand_cases.txt")):
    cases, cur = [], None
    for raw in open(path):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest, "entries": []}
            cases.append(cur)
        elif key == "cite":
            cur["cite"] = rest
        elif key == "n":
            cur["n"] = int(rest)
        elif key == "mate":
            cur["mate"] = [int(x) for x in rest.split()]
        elif key == "e":
            r, c, w = rest.split()
            cur["entries"].append((int(r), int(c), float(w)))
        elif key == "expect_mate":
            cur["expect_mate"] = [int(x) for x in rest.split()]
        elif key in ("expect_iterations", "expect_cycles", "expect_phases", "expect_cardinality"):
            cur[key] = int(rest)
        elif key == "expect_weight":
            cur[key] = float(rest)
        else:
            raise ValueError(line)
    return cases


def graph_of_case(c):
    n = c["n"]
    W = np.zeros((n, n))
    S = np.zeros((n, n), dtype=bool)
    for r, col, w in c["entries"]:
        W[r, col] = w
        S[r, col] = True
    return gen.from_dense(W, S, c["mate"])


def full2(w00, w01, w10, w11, mate=(0, 1)):
    W = np.array([[w00, w01], [w10, w11]], dtype=np.float64)
    return gen.from_dense(W, np.ones((2, 2), dtype=bool), list(mate))


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------

def pin_hand_cases(orc):
    """Hand-derived outcomes (tests/golden/hand_cases.txt)."""
    for c in load_hand_cases():
        g = graph_of_case(c)
        out, st, _ = orc.improve(g)
        assert out.tolist() == c["expect_mate"], (c["name"], out)
        assert st["iterations"] == c["expect_iterations"], (c["name"], st)
        assert st["cycles_applied"] == c["expect_cycles"], (c["name"], st)
        assert st["converged"] == 1, c["name"]
        assert st["weight_out"] == c["expect_weight"], (c["name"], st)


def pin_2x2_closed_form(orc):
    """n = 2, full pattern.  The only alternating 4-cycle swaps the two matched
    edges; by the gain definition (Section 3) it flips exactly when
    w01 + w10 > w00 + w11 (identity start), strictly (Algorithm 4)."""
    vals = [-3.0, -1.5, -1.0, -0.25, 0.0, 0.5, 2.0]
    rng = np.random.default_rng(7)
    for _ in range(300):
        w00, w01, w10, w11 = rng.choice(vals, 4)
        for mate in ((0, 1), (1, 0)):
            g = full2(w00, w01, w10, w11, mate)
            out, st, _ = orc.improve(g)
            if mate == (0, 1):
                flip = (w01 + w10) > (w00 + w11)
                expect = [1, 0] if flip else [0, 1]
            else:
                flip = (w00 + w11) > (w01 + w10)
                expect = [0, 1] if flip else [1, 0]
            assert out.tolist() == expect, (w00, w01, w10, w11, mate, out)
            assert st["cycles_applied"] == int(flip)
            assert st["iterations"] == (2 if flip else 1)
            wexp = (w10 + w01) if expect == [1, 0] else (w00 + w11)
            assert st["weight_out"] == wexp


def pin_block_diagonal(orc):
    """k independent full 2x2 blocks: one pass flips every block with positive
    gain (they are vertex-disjoint and rooted at different columns), the
    second pass finds nothing, and the result is the maximum-weight perfect
    matching of each block (assignment problem on 2 x 2)."""
    rng = np.random.default_rng(11)
    k = 40
    n = 2 * k
    W = np.zeros((n, n))
    S = np.zeros((n, n), dtype=bool)
    mate = np.arange(n)
    nflip = 0
    expect = np.arange(n)
    for b in range(k):
        blk = rng.integers(-8, 9, size=(2, 2)).astype(np.float64) / 4.0
        W[2 * b:2 * b + 2, 2 * b:2 * b + 2] = blk
        S[2 * b:2 * b + 2, 2 * b:2 * b + 2] = True
        if blk[0, 1] + blk[1, 0] > blk[0, 0] + blk[1, 1]:
            nflip += 1
            expect[2 * b], expect[2 * b + 1] = 2 * b + 1, 2 * b
    g = gen.from_dense(W, S, mate)
    out, st, trace = orc.improve(g, trace_cap=8)
    assert out.tolist() == expect.tolist()
    assert st["cycles_applied"] == nflip
    assert st["iterations"] == (2 if nflip else 1)
    assert trace[1][0] == nflip


def pin_six_cycle(orc):
    """Section 4: an alternating 6-cycle has no 4-cycle, so the phase cannot
    improve it although a far heavier perfect matching exists."""
    c = [x for x in load_hand_cases() if x["name"] == "six_cycle_counterexample"][0]
    g = graph_of_case(c)
    out, st, _ = orc.improve(g)
    best, arg = brute.mwpm_bruteforce(g)
    assert out.tolist() == [0, 1, 2] and st["cycles_applied"] == 0
    assert best == 30.0 and arg.tolist() == [1, 2, 0]


def _small_graphs(count=60, integer=False):
    for s in range(count):
        n = 2 + s % 6
        dens = (0.3, 0.5, 0.8)[s % 3]
        yield gen.random_small(n, dens, 1000 + s, integer_weights=integer)


def pin_bruteforce_small(orc):
    """n <= 7: the output is a perfect matching over stored entries; the weight
    never decreases from pass to pass; every pass but the last flips >= 1
    cycle; at exit no positive-gain alternating 4-cycle remains (exhaustive
    enumeration of column pairs); and the weight is at most the maximum over
    all perfect matchings (exhaustive enumeration)."""
    for integer in (False, True):
        for g in _small_graphs(integer=integer):
            out, st, trace = orc.improve(g, trace_cap=64)
            assert brute.is_perfect(g, out)
            assert st["converged"] == 1
            ws, fs = trace
            prev = st["weight_in"]
            for t in range(len(ws)):
                assert ws[t] >= prev
                prev = ws[t]
                if t < len(ws) - 1:
                    assert fs[t] >= 1
                    assert ws[t] > ws[t - 1] if t > 0 else ws[t] > st["weight_in"]
            assert fs[-1] == 0
            assert brute.positive_4cycles(g, out) == []
            best, _ = brute.mwpm_bruteforce(g)
            assert st["weight_out"] <= best + 1e-12
            assert abs(brute.matching_weight(g, out) - st["weight_out"]) <= 1e-12


def pin_one_pass_bruteforce(orc):
    """One pass from random matchings equals the dense set-and-sort restatement
    of Steps A-D (integer weights make ties frequent)."""
    rng = np.random.default_rng(5)
    for s in range(80):
        n = 3 + s % 6
        g = gen.random_small(n, 0.7, 2000 + s, integer_weights=(s % 2 == 0))
        mats = list(brute.all_perfect_matchings(g))
        for m in [mats[x] for x in rng.choice(len(mats), size=min(4, len(mats)), replace=False)]:
            new, flips = brute.one_pass_bruteforce(g, m)
            got, droot, counts = orc.one_pass(g, m)
            assert got.tolist() == new.tolist(), (s, m, got, new)
            assert sorted((int(droot[k]), k) for k in range(n) if droot[k] >= 0) == flips
            assert counts[3] == len(flips)


def pin_local_optimality_midsize(orc):
    """Random sparse n = 2000 (the small workload): perfect output, no
    positive-gain 4-cycle at exit (vectorised exhaustive check), weight at
    most the exact maximum-weight perfect matching (LAPJVsp, scipy)."""
    from scipy.optimize import linear_sum_assignment  # noqa: F401 (availability)
    from scipy.sparse import csc_matrix
    from scipy.sparse.csgraph import min_weight_full_bipartite_matching
    g = gen.config1()
    out, st, trace = orc.improve(g, trace_cap=256)
    assert st["converged"] == 1
    assert sorted(out.tolist()) == list(range(g.n))
    assert brute.no_positive_4cycle_vectorized(g, out)
    assert np.all(np.diff(np.concatenate([[st["weight_in"]], trace[0]])) >= 0)
    # exact optimum: shift weights to be > 0 (zeros would vanish from the
    # sparse pattern); a constant shift moves every perfect matching equally
    shift = 1.0 - g.weight.min()
    A = csc_matrix((g.weight + shift, g.rowidx, g.colptr), shape=(g.n, g.n))
    r, c = min_weight_full_bipartite_matching(A, maximize=True)
    opt = float(np.sum(np.asarray(A[r, c]).ravel())) - shift * g.n
    assert st["weight_out"] <= opt + 1e-9 * abs(opt)
    assert st["weight_out"] > st["weight_in"]
    # the quality report: gap to the optimum for these (log, <= 0) weights,
    # and the ratio w(M) / w(M*) for the positive weights exp(w) on the same
    # pattern (Option A), where a ratio is meaningful
    ga = g.copy()
    ga.weight = np.exp(g.weight)
    outa, sta, _ = orc.improve(ga)
    B = csc_matrix((ga.weight, ga.rowidx, ga.colptr), shape=(g.n, g.n))
    ra, ca = min_weight_full_bipartite_matching(B, maximize=True)
    opta = float(np.sum(np.asarray(B[ra, ca]).ravel()))
    ratio = sta["weight_out"] / opta
    assert 0.0 < ratio <= 1.0 + 1e-12
    # the paper's whole pipeline from no matching: greedy (Section 5.1), then
    # the maximum matching (Section 5.2), then the 4-cycle phase; each stage
    # keeps a perfect matching at most the optimum, the phase never loses weight
    pipe = {}
    for name, gg, best in (("log", g, opt), ("exp", ga, opta)):
        gm, _ = orc.greedy(gg)
        mm, mst = orc.mcm(gg, gm)
        assert mst["cardinality"] == gg.n
        outp, stp, _ = orc.improve(gg, mate=mm.astype(np.int32))
        assert stp["converged"] == 1 and brute.no_positive_4cycle_vectorized(gg, outp)
        assert stp["weight_in"] <= stp["weight_out"] <= best + 1e-9 * abs(best)
        pipe[name] = stp["weight_out"]
    print(f"\nquality n={g.n}: log weights gap {opt - st['weight_out']:.6g} "
          f"(w {st['weight_out']:.6g}, optimum {opt:.6g}); exp weights ratio {ratio:.6f}; "
          f"from greedy + maximum matching: log gap {opt - pipe['log']:.6g}, "
          f"exp ratio {pipe['exp'] / opta:.6f}")
    return {"gap_log": opt - st["weight_out"], "ratio_exp": ratio,
            "pipeline_gap_log": opt - pipe["log"], "pipeline_ratio_exp": pipe["exp"] / opta}


def pin_rank_simulation(orc):
    """The paper's distributed pass simulated literally on virtual process
    grids of 1, 4 and 9 processes (explicit A/B/C request queues, replicated
    matching, broadcast flips; Section 5.3, Algorithms 2-6) gives the
    oracle's matching after every pass, ties included."""
    import rank_sim
    for s in range(12):
        n = 20 + 15 * s
        g = gen.random_small(n, 0.06 + 0.01 * (s % 4), 4100 + s, integer_weights=(s % 3 == 0))
        for side in (1, 2, 3):
            grid = rank_sim.Grid(g, g.mate, side)
            cur = g.mate.copy()
            for it in range(200):
                flips = grid.one_pass()
                ref, _, counts = orc.one_pass(g, cur)
                got = grid.matching()
                assert got.tolist() == ref.tolist(), (s, side, it)
                assert flips == counts[3], (s, side, it)
                cur = ref
                if flips == 0:
                    break
            out, st, _ = orc.improve(g)
            assert cur.tolist() == out.tolist() and it + 1 == st["iterations"], (s, side)


def pin_pettie_sanders_selection(orc):
    """The Pettie-Sanders selection mode (Section 4: Step-C winners by gain,
    each kept when disjoint from those kept before): one pass equals the
    dense set-and-sort restatement (integer weights: ties); the kept cycles
    are disjoint and maximal among the Step-C winners; whole runs end with
    no positive-gain 4-cycle and a non-decreasing weight."""
    rng = np.random.default_rng(6)
    for s in range(60):
        n = 3 + s % 6
        g = gen.random_small(n, 0.7, 2600 + s, integer_weights=(s % 2 == 0))
        mats = list(brute.all_perfect_matchings(g))
        for m in [mats[x] for x in rng.choice(len(mats), size=min(4, len(mats)), replace=False)]:
            new, flips = brute.one_pass_bruteforce(g, m, select=1)
            got, droot, counts = orc.one_pass(g, m, select=1)
            assert got.tolist() == new.tolist(), (s, m)
            assert sorted((int(droot[k]), k) for k in range(n) if droot[k] >= 0) == flips
    for s in range(6):
        g = gen.random_small(150 + 50 * s, 0.05, 2700 + s, integer_weights=(s % 2 == 0))
        gain, row, _ = orc.step_c(g)
        _, droot, counts = orc.one_pass(g, select=1)
        mc = g.mate
        mr = np.empty(g.n, dtype=np.int64)
        mr[mc] = np.arange(g.n)
        roots = [j for j in range(g.n) if row[j] >= 0]
        key = {j: int(mr[row[j]]) for j in roots}
        kept = {int(droot[k]) for k in range(g.n) if droot[k] >= 0}
        used = set()
        for j in kept:
            assert not ({j, key[j]} & used)
            used |= {j, key[j]}
        for j in roots:
            if j not in kept:
                assert {j, key[j]} & used, (s, j)
        out, st, trace = orc.improve(g, select=1, trace_cap=64)
        assert st["converged"] == 1 and brute.no_positive_4cycle_vectorized(g, out)
        assert np.all(np.diff(np.concatenate([[st["weight_in"]], trace[0]])) >= 0)


def pin_row_marking(orc):
    """Row marking (Section 4: the neighbourhood of row m_j marked once per
    root, each candidate reads the mark of column m_i): one pass equals the
    dense set-and-sort restatement under both selections (the dense view looks
    entries up by (row, column), neither by column search nor by marks); a
    whole run reaches the same matching, passes and counts as the column
    search, on graphs with short and long rows."""
    rng = np.random.default_rng(7)
    for s in range(40):
        n = 3 + s % 6
        g = gen.random_small(n, 0.7, 2800 + s, integer_weights=(s % 2 == 0))
        mats = list(brute.all_perfect_matchings(g))
        for m in [mats[x] for x in rng.choice(len(mats), size=min(3, len(mats)), replace=False)]:
            for sel in (0, 1):
                new, flips = brute.one_pass_bruteforce(g, m, select=sel)
                got, droot, counts = orc.one_pass(g, m, select=sel, row_marking=True)
                assert got.tolist() == new.tolist(), (s, sel, m)
                assert sorted((int(droot[k]), k) for k in range(n) if droot[k] >= 0) == flips
    graphs = [gen.random_small(300 + 70 * s, 0.03, 2900 + s, integer_weights=(s % 2 == 0))
              for s in range(4)]
    graphs += [gen.rmat(1 << 10, 8, 2910), gen.stencil_2d(24, 2911)]
    for g in graphs:
        for sel in (0, 1):
            a, sa, _ = orc.improve(g, select=sel)
            b, sb, _ = orc.improve(g, select=sel, row_marking=True)
            assert a.tolist() == b.tolist(), g.name
            for f in ("iterations", "candidates", "closing_found", "positive",
                      "cycles_applied"):
                assert sa[f] == sb[f], (g.name, f)


def pin_greedy_matching(orc):
    """Heavy-weight greedy maximal matching (Section 5.1): the round-based
    matching equals the textbook sequential greedy over the entries sorted by
    weight (ties by row, then column), is maximal, and its statistics add up;
    integer weights (ties), signed zeros and empty columns included."""
    cases = []
    for s in range(30):
        n = 5 + 13 * s
        cases.append(gen.random_small(n, 0.05 + 0.04 * (s % 4), 5100 + s,
                                      integer_weights=(s % 2 == 0)))
    cases.append(gen.stencil_2d(12, 5200))
    cases.append(full2(3.0, 2.0, 2.0, 1.0))
    cases.append(full2(1.0, 3.0, 3.0, 1.0))
    z = full2(0.0, -0.0, -0.0, 0.0)
    cases.append(z)
    # empty columns: drop every entry of two columns
    e = gen.random_small(40, 0.2, 5300)
    keep = np.ones(e.nnz, dtype=bool)
    for c in (3, 17):
        keep[e.colptr[c]:e.colptr[c + 1]] = False
    counts = np.diff(e.colptr) - np.add.reduceat(~keep, e.colptr[:-1])
    e.rowidx, e.weight = e.rowidx[keep], e.weight[keep]
    e.colptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    cases.append(e)
    for g in cases:
        got, st = orc.greedy(g)
        ref = brute.greedy_sequential(g)
        assert got.tolist() == ref.tolist(), g.name
        assert brute.is_maximal_matching(g, got), g.name
        assert st["cardinality"] == int(np.sum(got >= 0))
        assert st["rounds"] >= 1 + (1 if st["cardinality"] else 0)
        wsum = sum(float(g.weight[g.colptr[j] + int(np.nonzero(
            g.rowidx[g.colptr[j]:g.colptr[j + 1]] == got[j])[0][0])])
            for j in range(g.n) if got[j] >= 0)
        assert abs(st["weight"] - wsum) <= 1e-12 * max(1.0, abs(wsum))
    # 2x2 by hand: the heaviest entry first
    assert orc.greedy(full2(3.0, 2.0, 2.0, 1.0))[0].tolist() == [0, 1]
    assert orc.greedy(full2(1.0, 3.0, 3.0, 1.0))[0].tolist() == [1, 0]
    assert orc.greedy(full2(1.0, 3.0, 2.0, 1.0))[0].tolist() == [1, 0]


def pin_weights(orc):
    """Equilibrated weights (Section 6.1, Options A and B): a 2x2 by hand;
    every row's largest weight is exactly 1 (log: 0) and no weight exceeds
    it; scaling a column by a power of two changes nothing (exact in
    binary floating point; columns are normalised first, so this holds for
    column scalings); a diagonal matrix gives all ones; Option B is the
    logarithm of Option A; zeros and non-finite values are rejected."""
    import math
    W = np.array([[2.0, 1.0], [4.0, -8.0]])
    g = gen.from_dense(W, np.ones((2, 2), dtype=bool), [0, 1])
    wa = orc.weights(2, g.colptr, g.rowidx, g.weight, 0)
    assert wa.tolist() == [1.0, 1.0, 0.25, 1.0]      # column-major: (0,0),(1,0),(0,1),(1,1)
    rng = np.random.default_rng(7)
    for s in range(8):
        h = gen.random_small(60 + 30 * s, 0.08, 3100 + s)
        a = rng.standard_normal(h.nnz) * np.exp(rng.uniform(-20, 20, h.nnz))
        wa = orc.weights(h.n, h.colptr, h.rowidx, a, 0)
        wb = orc.weights(h.n, h.colptr, h.rowidx, a, 1)
        col = np.repeat(np.arange(h.n), np.diff(h.colptr))
        rowmax = np.full(h.n, -np.inf)
        np.maximum.at(rowmax, h.rowidx, wa)
        assert np.all(rowmax == 1.0) and np.all(wa <= 1.0) and np.all(wa > 0.0)
        assert np.allclose(wb, np.log(wa), rtol=0, atol=1e-15)
        sc = a * np.exp2(rng.integers(-30, 30, h.n))[col]
        assert np.array_equal(orc.weights(h.n, h.colptr, h.rowidx, sc, 0), wa)
    d = gen.from_dense(np.diag([3.0, -0.5, 7.0]), np.eye(3, dtype=bool), [0, 1, 2])
    assert orc.weights(3, d.colptr, d.rowidx, d.weight, 0).tolist() == [1.0, 1.0, 1.0]
    assert orc.weights(3, d.colptr, d.rowidx, d.weight, 1).tolist() == [0.0, 0.0, 0.0]
    for bad in (0.0, math.inf, math.nan):
        z = d.weight.copy()
        z[1] = bad
        try:
            orc.weights(3, d.colptr, d.rowidx, z, 0)
            raise AssertionError("bad value accepted")
        except Exception as e:  # noqa: BLE001
            assert getattr(e, "name", "") == "NONFINITE", e


def random_pattern(n, per_col, seed, integer_weights=False):
    """Random sparse pattern without a planted matching (so possibly without
    a perfect one): per_col uniform rows per column, duplicates merged."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, n, n * per_col)
    cols = np.repeat(np.arange(n), per_col)
    colptr, rowidx = gen._csc_from_coo(n, rows, cols)
    w = (rng.integers(0, 4, len(rowidx)).astype(np.float64) if integer_weights
         else rng.standard_normal(len(rowidx)))
    return gen.Graph(n, colptr, rowidx, w, np.arange(n, dtype=np.int32), f"pattern_{seed}")


def pin_mcm(orc):
    """Maximum cardinality matching (Section 5.2): its cardinality equals the
    maximum from scipy's bipartite matching, from an empty start and from the
    greedy matching; it is a matching over stored entries; columns matched on
    entry stay matched; with one free column and two free rows, and with two
    free columns offering one free row, the heavier edge is taken."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_bipartite_matching
    cases = [random_pattern(60 + 40 * s, 1 + s % 3, 4200 + s, integer_weights=(s % 2 == 0))
             for s in range(10)]
    cases += [gen.rmat(1 << 11, 4, 4300), gen.random_small(300, 0.01, 4301)]
    for g in cases:
        A = csr_matrix((np.ones(g.nnz), g.rowidx, g.colptr), shape=(g.n, g.n))  # A^T as CSR
        best = int(np.sum(maximum_bipartite_matching(A, perm_type="column") >= 0))
        for start in (None, orc.greedy(g)[0]):
            m, st = orc.mcm(g, start)
            assert st["cardinality"] == best == int(np.sum(m >= 0)), (g.name, st, best)
            rows = m[m >= 0]
            assert len(set(rows.tolist())) == len(rows)
            for j in np.nonzero(m >= 0)[0]:
                assert m[j] in g.rowidx[g.colptr[j]:g.colptr[j + 1]]
            if start is not None:
                assert np.all(m[start >= 0] >= 0)
    h = gen.from_dense(np.array([[1.0, 0.0], [5.0, 0.0]]), np.array([[True, False], [True, False]]),
                       [0, 1])
    m, _ = orc.mcm(h)
    assert m.tolist() == [1, -1]
    # two free columns offer the same free row: the heavier edge wins it
    h2 = gen.from_dense(np.array([[1.0, 5.0], [0.0, 0.0]]),
                        np.array([[True, True], [False, False]]), [0, 1])
    m, _ = orc.mcm(h2)
    assert m.tolist() == [-1, 0]


def pin_mcm_hand_cases(orc):
    """Hand-derived maximum matchings (tests/golden/mcm_cases.txt): equal
    offers go to the lower column, equal tree ends to the lower row, and a
    tree that found its end stops growing (the readings of Section 5.2)."""
    cases = load_hand_cases(os.path.join(GOLDEN, "mcm_cases.txt"))
    assert len(cases) >= 3
    for c in cases:
        g = graph_of_case(c)
        m, st = orc.mcm(g, np.asarray(c["mate"], dtype=np.int32))
        assert m.tolist() == c["expect_mate"], (c["name"], m)
        assert st["phases"] == c["expect_phases"], (c["name"], st)
        assert st["cardinality"] == c["expect_cardinality"], (c["name"], st)


def pin_validation(orc):
    """Input checks: error classes for malformed inputs."""
    g = gen.random_small(5, 0.6, 3)
    assert orc.validate(g) == "OK"
    bad = g.copy(); bad.mate[0] = bad.mate[1]
    assert orc.validate(bad) == "NOT_PERFECT"
    bad = g.copy(); bad.mate[0] = g.n
    assert orc.validate(bad) == "NOT_PERFECT"
    # a mate that is not a stored entry
    W, S = brute.dense(g)
    for j in range(g.n):
        missing = [r for r in range(g.n) if not S[r, j]]
        if missing:
            bad = g.copy()
            other = int(np.nonzero(bad.mate == missing[0])[0][0])
            bad.mate[j], bad.mate[other] = missing[0], bad.mate[j]
            assert orc.validate(bad) == "NOT_PERFECT"
            break
    bad = g.copy(); bad.weight[2] = np.inf
    assert orc.validate(bad) == "NONFINITE"
    bad = g.copy(); bad.weight[1] = np.nan
    assert orc.validate(bad) == "NONFINITE"
    bad = g.copy(); bad.rowidx[0] = -1
    assert orc.validate(bad) == "INVALID_ARG"
    bad = g.copy(); bad.colptr[1] = bad.colptr[2] + 1
    assert orc.validate(bad) == "INVALID_ARG"
    j = int(np.argmax(np.diff(g.colptr)))
    bad = g.copy(); a, b = g.colptr[j], g.colptr[j] + 1
    bad.rowidx[a], bad.rowidx[b] = g.rowidx[b], g.rowidx[a]
    assert orc.validate(bad) == "UNSORTED_OR_DUP"


def pin_resume(orc):
    """Each pass is a function of (graph, matching) alone: stopping after t
    passes and restarting from that matching gives the same final matching
    and the same total number of passes."""
    g = gen.config1()
    full, st, _ = orc.improve(g)
    for t in (1, 2, 3):
        if t >= st["iterations"]:
            break
        mid, st1, _ = orc.improve(g, max_iters=t)
        assert st1["iterations"] == t and st1["converged"] == 0
        fin, st2, _ = orc.improve(g, mate=mid)
        assert fin.tolist() == full.tolist()
        assert t + st2["iterations"] == st["iterations"]


def pin_paper_maxiters(orc):
    """Algorithm 2 with maxiters = 10: at most 10 passes; converged only when
    the last pass found nothing."""
    g = gen.config1()
    out, st, trace = orc.improve(g, max_iters=10, trace_cap=10)
    assert st["iterations"] <= 10
    assert st["converged"] == int(trace[1][-1] == 0)


PINS = [pin_hand_cases, pin_2x2_closed_form, pin_block_diagonal, pin_six_cycle,
        pin_bruteforce_small, pin_one_pass_bruteforce, pin_rank_simulation,
        pin_local_optimality_midsize, pin_validation, pin_resume, pin_paper_maxiters,
        pin_pettie_sanders_selection, pin_row_marking, pin_greedy_matching, pin_weights,
        pin_mcm, pin_mcm_hand_cases]
