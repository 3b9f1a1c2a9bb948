"""NVTX ranges of the library (needs a GPU): a small NVTX tool
(tests/nvtx_log.c) records every range pushed while a child process calls
the entry points; each call appears as a balanced range with the steps it
runs on the host nested inside."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}]
    import numpy as np
    from paper_1801_09809_gb300 import awpm, gen
    g = gen.stencil_2d(30, 5)
    ctx = awpm.awpm_create(device=0)
    out = np.empty(g.n, np.int32)
    awpm.awpm_improve_ctx(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, out)
    m = np.full(g.n, -1, np.int32)
    awpm.awpm_greedy(ctx, g.n, g.colptr, g.rowidx, g.weight, m)
    m = np.full(g.n, -1, np.int32)
    awpm.awpm_mcm(ctx, g.n, g.colptr, g.rowidx, g.weight, m)
    t = awpm.awpm_submit(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, out)
    awpm.awpm_wait(ctx, t)
    awpm.awpm_destroy(ctx)
    timed = awpm.awpm_create(device=0, flags=awpm.FLAG_TIME_SEARCH)
    awpm.awpm_improve_ctx(timed, g.n, g.colptr, g.rowidx, g.weight, g.mate, out)
    awpm.awpm_destroy(timed)
""")


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09809_gb300 import build
    build.build()
    return _t


def test_ranges_are_recorded(torch, tmp_path):
    inc = "/usr/local/cuda/include"
    if shutil.which("gcc") is None or not os.path.isdir(os.path.join(inc, "nvtx3")):
        pytest.skip("gcc or NVTX headers missing")
    tool = tmp_path / "libnvtx_log.so"
    subprocess.check_call(["gcc", "-shared", "-fPIC", "-O1", "-I" + inc,
                           os.path.join(HERE, "nvtx_log.c"), "-o", str(tool)])
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(tool), AWPM_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, check=True,
                   timeout=600)
    events = log.read_text().split()
    pushed = [e[1:] for e in events if e.startswith("+")]
    for name in ("awpm_improve", "awpm_greedy", "awpm_mcm", "awpm_submit", "admit",
                 "enqueue", "finish", "pass"):
        assert name in pushed, (name, pushed)
    # balanced; a whole solve nests its enqueue and finish
    depth = 0
    for e in events:
        depth += 1 if e.startswith("+") else -1
        assert depth >= 0
    assert depth == 0
    i = events.index("+awpm_improve")
    assert events[i + 1] == "+enqueue"
