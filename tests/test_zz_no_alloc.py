"""awpm_search_noalloc, the search entry point that allocates nothing (needs a GPU).

It serves callers that cannot call cudaMalloc (a framework whose memory pool
already holds the GPU's memory, or code where an allocation is not allowed):
its scratch is a fixed array inside the library.  Its Step-C output must equal
that of awpm_search, which uses the context's allocated workspace, on two
calls in a row (the second call reuses the scratch left by the first).  This
file is collected last so that a run stopping at the first failure has run
everything else first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1801_09809_gb300 import awpm, gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09809_gb300 import build
    build.build()
    _t.cuda.set_device(0)
    return _t


def _device(g, torch, mate):
    d = torch.device("cuda", 0)
    return (torch.from_numpy(g.colptr).to(d), torch.from_numpy(g.rowidx).to(d),
            torch.from_numpy(g.weight).to(d), torch.from_numpy(np.ascontiguousarray(mate)).to(d))


def test_noalloc_matches_search(torch):
    graphs = [gen.stencil_2d(300, 7001), gen.rmat(1 << 16, 16, 7002), gen.stencil_3d(20, 7003),
              gen.random_small(200, 0.1, 7004, integer_weights=True)]
    ctx = awpm.awpm_create(device=0)
    try:
        for g in graphs:
            assert g.n <= awpm.NOALLOC_MAX_N and g.nnz <= awpm.NOALLOC_MAX_NNZ
            cp, ri, w, m = _device(g, torch, g.mate)
            ref_g = torch.empty(g.n, dtype=torch.float64, device="cuda")
            ref_r = torch.empty(g.n, dtype=torch.int32, device="cuda")
            ref_st = awpm.awpm_search(ctx, g.n, cp, ri, w, m, ref_g, ref_r)
            for call in range(2):
                out_g = torch.full((g.n,), -7.0, dtype=torch.float64, device="cuda")
                out_r = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
                st = awpm.awpm_search_noalloc(g.n, cp, ri, w, m, out_g, out_r)
                torch.cuda.synchronize()
                # Step-C records are exact (same gain arithmetic, same tie rule)
                assert torch.equal(out_r, ref_r), (g.name, call)
                assert torch.equal(out_g, ref_g), (g.name, call)
                for k in ("candidates", "closing_found", "positive", "edge_checks"):
                    assert st[k] == ref_st[k], (g.name, call, k)
    finally:
        awpm.awpm_destroy(ctx)


def test_noalloc_alternating_sizes(torch):
    """A small problem after a large one still clears the shared scratch."""
    big = gen.stencil_2d(400, 7011)
    small = gen.stencil_2d(30, 7012)
    ctx = awpm.awpm_create(device=0)
    try:
        for g in (big, small, big, small):
            cp, ri, w, m = _device(g, torch, g.mate)
            a_g = torch.empty(g.n, dtype=torch.float64, device="cuda")
            a_r = torch.empty(g.n, dtype=torch.int32, device="cuda")
            awpm.awpm_search(ctx, g.n, cp, ri, w, m, a_g, a_r)
            b_g = torch.empty_like(a_g)
            b_r = torch.empty_like(a_r)
            awpm.awpm_search_noalloc(g.n, cp, ri, w, m, b_g, b_r)
            assert torch.equal(a_r, b_r) and torch.equal(a_g, b_g)
    finally:
        awpm.awpm_destroy(ctx)


def test_noalloc_rejects_oversize_and_host_arrays(torch):
    g = gen.stencil_2d(600, 7021)  # n = 360,000 > NOALLOC_MAX_N
    cp, ri, w, m = _device(g, torch, g.mate)
    og = torch.empty(g.n, dtype=torch.float64, device="cuda")
    orow = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(awpm.AwpmError) as ei:
        awpm.awpm_search_noalloc(g.n, cp, ri, w, m, og, orow)
    assert ei.value.name == "TOO_LARGE"
    s = gen.stencil_2d(20, 7022)
    hg = np.empty(s.n, dtype=np.float64)
    hr = np.empty(s.n, dtype=np.int32)
    with pytest.raises(awpm.AwpmError) as ei:
        awpm.awpm_search_noalloc(s.n, s.colptr, s.rowidx, s.weight, s.mate, hg, hr)
    assert ei.value.name == "INVALID_ARG"
