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
    ref, rst, _ = oracle.get().improve(g)
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
