"""The AWPM_DEBUG_BOUNDS build (device index checks that report
AWPM_ERR_INTERNAL and skip the access, never trap) gives the oracle's
results on the parity cases with no check firing (needs a GPU).  The library
is compiled with the flag into a temporary directory and loaded in a child
process through AWPM_LIBRARY."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))

CHILD = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import numpy as np
    import oracle, pins
    from gpu_helpers import assert_same_as_oracle
    from paper_1801_09809_gb300 import awpm, gen
    assert awpm.LIB_PATH == {lib!r}
    orc = oracle.get()
    graphs = [pins.graph_of_case(c) for c in pins.load_hand_cases()]
    graphs += [gen.random_small(40, 0.15, 71, integer_weights=True), gen.config1(),
               gen.stencil_2d(60, 72), gen.stencil_3d(12, 73), gen.rmat(1 << 13, 8, 74)]
    for lookup in (awpm.LOOKUP_BSEARCH, awpm.LOOKUP_HASH, awpm.LOOKUP_ROWMARK):
        for flags in (0, awpm.FLAG_TIME_SEARCH):
            ctx = awpm.awpm_create(device=0, lookup=lookup, flags=flags)
            for g in graphs:
                out = np.empty(g.n, np.int32)
                st = awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, out)
                ref, rst, _ = orc.improve(g)
                assert_same_as_oracle(g, out, st, ref, rst, g.name)
            awpm.awpm_destroy(ctx)
    specs = gen.batch_spec(24, seed=99)
    bg = [gen.build_spec(sp) for sp in specs]
    n_off, u = gen.union(bg)
    ctx = awpm.awpm_create(device=0)
    out = np.empty(u.n, np.int32)
    tot, pm = awpm.awpm_improve_batch(ctx, len(bg), n_off, u.colptr, u.rowidx, u.weight,
                                      u.mate, out)
    for b, (g, m) in enumerate(zip(bg, gen.split(n_off, out))):
        ref, rst, _ = orc.improve(g)
        assert np.array_equal(m, ref) and pm[b]["iterations"] == rst["iterations"]
    awpm.awpm_destroy(ctx)
    print("DEBUG_BOUNDS_OK")
""")


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def test_debug_bounds_build_matches_oracle(torch, tmp_path):
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    from paper_1801_09809_gb300 import build
    lib = str(tmp_path / "libawpm_debug.so")
    build.build_debug(lib, str(tmp_path / "obj"))
    env = dict(os.environ, AWPM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=TESTS, lib=lib)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "DEBUG_BOUNDS_OK" in r.stdout, r.stdout + r.stderr
