"""Planted mistakes in the CPU oracle must each be caught by a pin (no GPU).

Each mutant is a copy of oracle/awpm_oracle.c with one plausible mistake
(a dropped term, a wrong sign or index, a transposed operand, a wrong
tie-break, a missing rule); it is compiled into a temporary library and the
whole pin suite is run against it in a child process.  The test passes when at
least one pin fails for every mutant.
"""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

MUTANTS = [
    ("closing weight sign", "double g = a.wij + wq - wm[a.mi] - wm[a.j];",
     "double g = a.wij - wq - wm[a.mi] - wm[a.j];"),
    ("dropped root matched weight", "double g = a.wij + wq - wm[a.mi] - wm[a.j];",
     "double g = a.wij + wq - wm[a.mi];"),
    ("matched weight indexed by row", "double g = a.wij + wq - wm[a.mi] - wm[a.j];",
     "double g = a.wij + wq - wm[a.mj] - wm[a.j];"),
    ("closing weight replaced by own weight", "double g = a.wij + wq - wm[a.mi] - wm[a.j];",
     "double g = a.wij + a.wij - wm[a.mi] - wm[a.j];"),
    ("transposed closing lookup", "find_entry(colptr, rowidx, a.mj, a.mi);",
     "find_entry(colptr, rowidx, a.mi, a.mj);"),
    ("root filter dropped", "if (i > mj) {", "if (i != mj) {"),
    ("root filter reversed", "if (i > mj) {", "if (i < mj) {"),
    ("non-strict positivity", "if (g > 0.0) {", "if (g >= 0.0) {"),
    ("step C keeps minimum", "breq[x].g > breq[cur].g ||", "breq[x].g < breq[cur].g ||"),
    ("step C tie to highest row", "breq[x].i < breq[cur].i", "breq[x].i > breq[cur].i"),
    ("step D tie to highest root", "c->j < breq[cur].j", "c->j > breq[cur].j"),
    ("step D keeps minimum", "c->g > breq[cur].g ||", "c->g < breq[cur].g ||"),
    ("step D discard rule dropped",
     "if (cwin[k] >= 0)\n                continue;\n            int64_t cur = dwin[k];",
     "int64_t cur = dwin[k];"),
    ("flip gives key column the wrong row", "mc[c.mi] = c.mj;", "mc[c.mi] = c.i;"),
    ("flip forgets the row side", "mr[c.mj] = c.mi;", "mr[c.mj] = c.j;"),
    ("flip keeps stale matched weight", "wm[c.mi] = c.wq;", "wm[c.mi] = c.wij;"),
    ("stops one pass early", "if (f == 0) {", "if (f <= 1) {"),
    ("duplicate mates accepted", "if (r < 0 || r >= n || seen[r] ||", "if (r < 0 || r >= n ||"),
    ("non-finite weights accepted", "if (!isfinite(w[p]))", "if (0)"),
    ("row marking reads the root's own row", "for (int64_t t = rowptr[a.mj]; t < rowptr[a.mj + 1]; ++t) {",
     "for (int64_t t = rowptr[a.i]; t < rowptr[a.i + 1]; ++t) {"),
    ("row marking keeps stale marks", "q = mark_root[a.mi] == a.j ? mark_pos[a.mi] : -1;",
     "q = mark_root[a.mi] >= 0 ? mark_pos[a.mi] : -1;"),
    ("row marking marks once per pass", "if (x == 0 || areq[x - 1].j != a.j)", "if (x == 0)"),
    ("transpose records the previous column", "rowpos[fill[rowidx[p]]] = p;\n            rowcol[fill[rowidx[p]]++] = j;",
     "rowpos[fill[rowidx[p]]] = p;\n            rowcol[fill[rowidx[p]]++] = j > 0 ? j - 1 : j;"),
    ("Pettie-Sanders order ascending", "    if (p->g > q->g)\n        return -1;",
     "    if (p->g < q->g)\n        return -1;"),
    ("Pettie-Sanders tie to the highest root", "return (p->j > q->j) - (p->j < q->j);",
     "return (p->j < q->j) - (p->j > q->j);"),
    ("Pettie-Sanders ignores the key column",
     "if (used_col[c->j] || used_col[c->mi] || used_row[c->i] || used_row[c->mj])",
     "if (used_col[c->j] || used_row[c->mj])"),
    ("weights skip the row normalisation", "double x = v / rmax[rowidx[p]];", "double x = v;"),
    ("weights take the column maximum of signed values", "if (fabs(a[p]) > cmax[j])\n                cmax[j] = fabs(a[p]);",
     "if (a[p] > cmax[j])\n                cmax[j] = fabs(a[p]);"),
    ("weights accept zeros", "if (!isfinite(a[p]) || a[p] == 0.0)", "if (!isfinite(a[p]))"),
    ("maximum matching offers prefer the lighter edge",
     "if (bestc[r] < 0 || w[p] > bestw[r] || (w[p] == bestw[r] && c < bestc[r])) {",
     "if (bestc[r] < 0 || w[p] < bestw[r] || (w[p] == bestw[r] && c < bestc[r])) {"),
    ("maximum matching ends at the lowest free row",
     "if (tend[t] < 0 || w[p] > tw[t] || (w[p] == tw[t] && r < tend[t])) {",
     "if (tend[t] < 0 || r < tend[t]) {"),
    ("maximum matching equal offers to the higher column",
     "if (bestc[r] < 0 || w[p] > bestw[r] || (w[p] == bestw[r] && c < bestc[r])) {",
     "if (bestc[r] < 0 || w[p] > bestw[r] || (w[p] == bestw[r] && c > bestc[r])) {"),
    ("maximum matching equal ends to the higher row",
     "if (tend[t] < 0 || w[p] > tw[t] || (w[p] == tw[t] && r < tend[t])) {",
     "if (tend[t] < 0 || w[p] > tw[t] || (w[p] == tw[t] && r > tend[t])) {"),
    ("maximum matching trees with an end keep growing",
     "if (tend[root[next[f]]] < 0)\n                    front[nf++] = next[f];",
     "front[nf++] = next[f];"),
    ("maximum matching stops after one phase", "        if (aug == 0)\n            break;",
     "        break;"),
    ("greedy column keeps the lightest", "if (cbest[j] < 0 || w[p] > w[cbest[j]])",
     "if (cbest[j] < 0 || w[p] < w[cbest[j]])"),
    ("greedy column tie to the highest row", "if (cbest[j] < 0 || w[p] > w[cbest[j]])",
     "if (cbest[j] < 0 || w[p] >= w[cbest[j]])"),
    ("greedy row tie to the highest column", "if (rbest[i] < 0 || w[p] > rbw[i]) {",
     "if (rbest[i] < 0 || w[p] >= rbw[i]) {"),
    ("greedy ignores the row's choice", "if (rbest[i] == j) {", "if (mr[i] < 0) {"),
]

RUNNER = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle, pins
    orc = oracle.Oracle({so!r})
    failed = []
    for pin in pins.PINS:
        try:
            pin(orc)
        except Exception as e:  # any failure of the pin counts
            failed.append(pin.__name__)
            break
    print("FAILED_PINS", failed)
    sys.exit(0 if failed else 3)
""")


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = str(tmp_path / "mutant.so")
    oracle.compile_oracle(str(mpath), so)
    root = os.path.dirname(oracle.HERE)
    tests = os.path.dirname(os.path.abspath(__file__))
    code = RUNNER.format(root=root, tests=tests, so=so)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    # exit 0: a pin failed (caught); a crash (negative code) is caught too
    assert r.returncode != 3, f"mutant '{name}' passed every pin:\n{r.stdout}\n{r.stderr}"
