"""The multi-threaded restatement of the oracle (the CPU timing baseline on
all host cores) gives the oracle's results exactly: matchings, pass counts,
counters and weights (no GPU)."""
import subprocess

import numpy as np
import pytest

import oracle
from paper_1801_09809_gb300 import gen


@pytest.fixture(scope="module")
def par():
    try:
        return oracle.OraclePar()
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip(f"OpenMP restatement not buildable here: {e}")


@pytest.mark.parametrize("threads", [1, 3, 0])
def test_same_as_oracle(par, threads):
    orc = oracle.get()
    graphs = [gen.random_small(40 + 37 * s, 0.05 + 0.03 * (s % 3), 7100 + s,
                               integer_weights=(s % 2 == 0)) for s in range(8)]
    graphs += [gen.rmat(1 << 13, 16, 7201), gen.stencil_2d(60, 7202),
               gen.stencil_3d(10, 7203), gen.banded(3000, 9, 7204), gen.config1()]
    for g in graphs:
        for max_iters in (0, 2):
            a, sa, _ = orc.improve(g, max_iters=max_iters)
            b, sb = par.improve(g, max_iters=max_iters, threads=threads)
            assert np.array_equal(a, b), (g.name, max_iters)
            assert sa == sb, (g.name, max_iters, sa, sb)


def test_bad_matching_is_rejected(par):
    g = gen.random_small(30, 0.3, 7301)
    b = g.copy()
    b.mate[0] = b.mate[1]
    with pytest.raises(oracle.OracleError):
        par.improve(b)
