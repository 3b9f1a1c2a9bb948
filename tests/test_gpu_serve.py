"""Request server (continuous batching): every request gives the result it
gives alone, whatever runs beside it (needs a GPU)."""
import time

import numpy as np
import pytest

import oracle
from gpu_helpers import weight_tol
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


def request_pool(count, seed, n_lo=200, n_hi=20000):
    specs = gen.serve_spec(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    return [gen.build_spec(sp) for sp in specs]


def test_served_results_equal_alone(torch):
    graphs = request_pool(24, 777)
    orc = oracle.get()
    refs = [orc.improve(g) for g in graphs]
    ctx = awpm.awpm_create(device=0, slots=4)
    try:
        # half host arrays, half device arrays
        outs, keep, tickets = [], [], []
        for k, g in enumerate(graphs):
            if k % 2:
                d = torch.device("cuda")
                arrs = [torch.from_numpy(a).to(d) for a in (g.colptr, g.rowidx, g.weight, g.mate)]
                out = torch.empty(g.n, dtype=torch.int32, device=d)
                nnz = g.nnz
            else:
                arrs = [g.colptr, g.rowidx, g.weight, g.mate]
                out = np.empty(g.n, dtype=np.int32)
                nnz = None
            keep.append(arrs)
            outs.append(out)
            tickets.append(awpm.awpm_submit(ctx, g.n, *arrs, out, nnz=nnz))
        pending = set(range(len(graphs)))
        stats = {}
        deadline = time.time() + 120
        while pending and time.time() < deadline:
            for k in list(pending):
                done, st = awpm.awpm_poll(ctx, tickets[k])
                if done:
                    stats[k] = st
                    pending.discard(k)
        assert not pending, "requests did not finish"
        for k, g in enumerate(graphs):
            ref, rst, _ = refs[k]
            got = outs[k].cpu().numpy() if hasattr(outs[k], "cpu") else outs[k]
            assert np.array_equal(got, ref), (k, g.name)
            assert stats[k]["iterations"] == rst["iterations"], (k, g.name)
            assert stats[k]["cycles_applied"] == rst["cycles_applied"]
            assert abs(stats[k]["weight_out"] - rst["weight_out"]) <= weight_tol(g, ref)
            # the ticket is released once reported
            with pytest.raises(awpm.AwpmError) as ei:
                awpm.awpm_poll(ctx, tickets[k])
            assert ei.value.name == "NOT_FOUND"
    finally:
        awpm.awpm_destroy(ctx)


def test_budget_admission_and_oversize(torch):
    graphs = request_pool(10, 4242, n_lo=2000, n_hi=30000)
    need = max(g.n * 120 + g.nnz * 40 for g in graphs)
    ctx = awpm.awpm_create(device=0, slots=3, mem_budget_bytes=int(need * 1.5))
    try:
        outs = [np.empty(g.n, dtype=np.int32) for g in graphs]
        tickets = [awpm.awpm_submit(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, o)
                   for g, o in zip(graphs, outs)]
        orc = oracle.get()
        for g, o, t in zip(graphs, outs, tickets):
            st = awpm.awpm_wait(ctx, t)
            ref, rst, _ = orc.improve(g)
            assert np.array_equal(o, ref) and st["iterations"] == rst["iterations"]
        big = gen.stencil_2d(700, 99)
        ob = np.empty(big.n, dtype=np.int32)
        t = awpm.awpm_submit(ctx, big.n, big.colptr, big.rowidx, big.weight, big.mate, ob)
        with pytest.raises(awpm.AwpmError) as ei:
            awpm.awpm_wait(ctx, t)
        assert ei.value.name == "BUDGET"
    finally:
        awpm.awpm_destroy(ctx)


def test_invalid_request_reports_its_error(torch):
    good = gen.stencil_2d(30, 5)
    bad = good.copy()
    bad.mate[0] = bad.mate[1]
    ctx = awpm.awpm_create(device=0, slots=2)
    try:
        o1 = np.empty(good.n, dtype=np.int32)
        o2 = np.empty(bad.n, dtype=np.int32)
        t1 = awpm.awpm_submit(ctx, good.n, good.colptr, good.rowidx, good.weight, good.mate, o1)
        t2 = awpm.awpm_submit(ctx, bad.n, bad.colptr, bad.rowidx, bad.weight, bad.mate, o2)
        with pytest.raises(awpm.AwpmError) as ei:
            awpm.awpm_wait(ctx, t2)
        assert ei.value.name == "NOT_PERFECT"
        awpm.awpm_wait(ctx, t1)
        ref, _, _ = oracle.get().improve(good)
        assert np.array_equal(o1, ref)
    finally:
        awpm.awpm_destroy(ctx)


def test_destroy_with_queued_requests(torch):
    graphs = request_pool(12, 1234)
    ctx = awpm.awpm_create(device=0, slots=1)
    outs = [np.empty(g.n, dtype=np.int32) for g in graphs]
    for g, o in zip(graphs, outs):
        awpm.awpm_submit(ctx, g.n, g.colptr, g.rowidx, g.weight, g.mate, o)
    awpm.awpm_destroy(ctx)  # drains the running solve, drops the queued ones
