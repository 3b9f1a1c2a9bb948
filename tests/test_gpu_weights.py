"""Matching weights from matrix values on the GPU against the CPU oracle
(needs a GPU): Option A bit-exact, Option B within a few units in the last
place (device logarithm against the host one)."""
import numpy as np
import pytest

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


def values_for(g, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(g.nnz) * np.exp(rng.uniform(-30, 30, g.nnz))


def gpu_weights(ctx, g, a, mode, torch, host=False):
    if host:
        out = np.empty(g.nnz, dtype=np.float64)
        awpm.awpm_weights(ctx, g.n, g.colptr, g.rowidx, a, mode, out)
        return out
    d = torch.device("cuda")
    cp, ri, av = (torch.from_numpy(np.ascontiguousarray(x)).to(d) for x in (g.colptr, g.rowidx, a))
    out = torch.empty(g.nnz, dtype=torch.float64, device=d)
    awpm.awpm_weights(ctx, g.n, cp, ri, av, mode, out)
    return out.cpu().numpy()


@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_option_a_bit_exact(ctx, torch, host):
    orc = oracle.get()
    for k, g in enumerate([gen.config1(), gen.stencil_2d(80, 901), gen.rmat(1 << 14, 16, 902),
                           gen.banded(3000, 7, 903), gen.stencil_3d(12, 904)]):
        a = values_for(g, 910 + k)
        ref = orc.weights(g.n, g.colptr, g.rowidx, a, 0)
        got = gpu_weights(ctx, g, a, awpm.WEIGHTS_SUM, torch, host)
        assert np.array_equal(got, ref), g.name


def test_option_b_within_ulps(ctx, torch):
    orc = oracle.get()
    for k, g in enumerate([gen.config1(), gen.rmat(1 << 14, 16, 920), gen.stencil_3d(12, 921)]):
        a = values_for(g, 930 + k)
        ref = orc.weights(g.n, g.colptr, g.rowidx, a, 1)
        got = gpu_weights(ctx, g, a, awpm.WEIGHTS_PRODUCT, torch)
        assert np.all(got[ref == 0.0] == 0.0)
        assert np.all(np.abs(got - ref) <= 4 * np.spacing(np.abs(ref))), g.name


def test_errors(ctx, torch):
    g = gen.random_small(40, 0.2, 940)
    a = values_for(g, 941)
    for bad, name in ((0.0, "NONFINITE"), (np.nan, "NONFINITE"), (np.inf, "NONFINITE")):
        b = a.copy()
        b[5] = bad
        with pytest.raises(awpm.AwpmError) as ei:
            gpu_weights(ctx, g, b, awpm.WEIGHTS_SUM, torch)
        assert ei.value.name == name
    h = g.copy()
    h.rowidx = h.rowidx.copy()
    h.rowidx[3] = g.n
    with pytest.raises(awpm.AwpmError) as ei:
        gpu_weights(ctx, h, a, awpm.WEIGHTS_SUM, torch, host=True)
    assert ei.value.name == "INVALID_ARG"
    assert np.array_equal(gpu_weights(ctx, g, a, awpm.WEIGHTS_SUM, torch),
                          oracle.get().weights(g.n, g.colptr, g.rowidx, a, 0))


def test_weights_then_improve(ctx, torch):
    """Values -> Option B weights on the GPU -> the 4-cycle phase: equal to
    the oracle's phase on those weights."""
    g = gen.stencil_3d(14, 950)
    a = values_for(g, 951)
    w = gpu_weights(ctx, g, a, awpm.WEIGHTS_PRODUCT, torch)
    h = g.copy()
    h.weight = w
    ref, rst, _ = oracle.get().improve(h)
    out = np.empty(h.n, dtype=np.int32)
    st = awpm.awpm_improve_ctx(ctx, h.n, h.colptr, h.rowidx, h.weight, h.mate, out)
    assert out.tolist() == ref.tolist() and st["iterations"] == rst["iterations"]
