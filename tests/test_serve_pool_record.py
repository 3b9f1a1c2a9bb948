"""The stored oracle results of the served pool (tests/golden/
serve_pool_oracle.json, written by make_serve_oracle.py from the oracle
alone) are reproducible: the smallest problems are generated again, their
input digests compared, and the oracle run again on them (no GPU)."""
import json
import os

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_record_matches_generator_and_oracle():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_serve_oracle", os.path.join(HERE, "golden", "make_serve_oracle.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    data = json.load(open(os.path.join(HERE, "golden", "serve_pool_oracle.json")))
    recs = data["records"]
    assert data["pool_size"] == len(recs) >= 128
    from paper_1801_09809_gb300 import gen
    specs = gen.serve_spec(len(recs), seed=data["seed"])
    assert [list(s) for s in specs] == [r["spec"] for r in recs]
    smallest = sorted(range(len(recs)), key=lambda k: recs[k]["nnz"])[:6]
    orc = oracle.get()
    for k in smallest:
        g = gen.build_spec(specs[k])
        assert (g.n, g.nnz) == (recs[k]["n"], recs[k]["nnz"])
        assert mk.input_digest(g) == recs[k]["input"]
        out, st, _ = orc.improve(g)
        assert mk.mate_digest(out) == recs[k]["mate"]
        assert st["iterations"] == recs[k]["iterations"]
        assert st["cycles_applied"] == recs[k]["cycles_applied"]
