"""The search's tuning switches, environment variables the library reads
(AWPM_SEARCH_PIPE=0: the former four-tiles-per-round search kernel instead
of the pipelined one; AWPM_SEARCH_WIDE=0: the narrow form; AWPM_BLOOM=0: no
Bloom filters of the long columns), change speed only: with each setting a
single solve and a batched solve give the oracle's matchings and statistics
(needs a GPU).  Each setting runs in a child process, since the library
reads some of the variables once per process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import weight_tol
from paper_1801_09809_gb300 import gen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# R-MAT graphs have long columns (Bloom filters, warp-cooperative searches);
# the stencil has only short ones
SINGLE = [("rmat", 1 << 14, 16, 9701), ("rmat", 1 << 13, 8, 9702), ("stencil", 70, 0, 9703)]
BATCH_SEED = 9704


def make(spec):
    kind, a, b, seed = spec
    if kind == "rmat":
        return gen.rmat(a, b, seed)
    return gen.stencil_2d(a, seed)


CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from paper_1801_09809_gb300 import awpm, gen
import test_gpu_switches as T
ctx = awpm.awpm_create(device=0, lookup=awpm.LOOKUP_BSEARCH)
res = {"single": [], "batch": None}
keys = ("iterations", "converged", "cycles_applied", "candidates", "closing_found",
        "positive", "weight_in", "weight_out")
for spec in T.SINGLE:
    g = T.make(spec)
    out = np.empty(g.n, np.int32)
    st = awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, out)
    res["single"].append({"mate": out.tolist(), **{k: st[k] for k in keys}})
graphs = [gen.build_spec(sp) for sp in gen.batch_spec(24, seed=T.BATCH_SEED)]
n_off, u = gen.union(graphs)
out = np.empty(u.n, np.int32)
tot, pm = awpm.awpm_improve_batch(ctx, len(graphs), n_off, u.colptr, u.rowidx, u.weight,
                                  u.mate, out)
res["batch"] = {"mates": [m.tolist() for m in gen.split(n_off, out)],
                "iterations": [p["iterations"] for p in pm],
                "cycles": [p["cycles_applied"] for p in pm]}
awpm.awpm_destroy(ctx)
print(json.dumps(res))
"""


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09809_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def expected():
    orc = oracle.get()
    single = []
    for spec in SINGLE:
        g = make(spec)
        ref, rst, _ = orc.improve(g)
        single.append((g, ref, rst))
    graphs = [gen.build_spec(sp) for sp in gen.batch_spec(24, seed=BATCH_SEED)]
    batch = [(g,) + tuple(orc.improve(g)[:2]) for g in graphs]
    return single, batch


@pytest.mark.parametrize("env", [
    {"AWPM_SEARCH_PIPE": "0"},
    {"AWPM_SEARCH_PIPE": "0", "AWPM_SEARCH_WIDE": "0"},
    {"AWPM_SEARCH_WIDE": "0"},
    {"AWPM_BLOOM": "0"},
    {"AWPM_SEARCH_PIPE": "0", "AWPM_BLOOM": "0"},
], ids=lambda e: ",".join(f"{k}={v}" for k, v in e.items()))
def test_switch_matches_oracle(built, expected, env):
    full = dict(os.environ)
    full.update(env)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=full, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    single, batch = expected
    for (g, ref, rst), res in zip(single, got["single"]):
        assert res["mate"] == ref.tolist(), (env, g.name)
        for k in ("iterations", "converged", "cycles_applied", "candidates", "closing_found",
                  "positive"):
            assert res[k] == rst[k], (env, g.name, k, res[k], rst[k])
        assert abs(res["weight_out"] - rst["weight_out"]) <= weight_tol(g, ref)
    for b, (g, ref, rst) in enumerate(batch):
        assert got["batch"]["mates"][b] == ref.tolist(), (env, b)
        assert got["batch"]["iterations"][b] == rst["iterations"], (env, b)
        assert got["batch"]["cycles"][b] == rst["cycles_applied"], (env, b)
    assert np.all(np.array(got["batch"]["iterations"]) >= 1)
