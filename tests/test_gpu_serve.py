"""The request server (continuous batching) through the C ABI.

A request must give the same result alone and among others: the server runs every request
with the same kernels (the cluster-variant Newton kernel, fixed-order reductions), so the
result is bitwise the same however many requests share the device.  The FP64 results are
also held to the FP64 bar (1e-10 relative, max norm) against solo fmg_solve calls, which use
the cooperative Newton kernel (a different reduction order).  Admission by memory is checked
with a budget that holds one hierarchy at a time, and a request larger than the budget is
refused with FMG_ERR_OOM.
"""
import numpy as np
import pytest

from paper_1611_05677_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def fmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_05677_gb300 import fmg as F

    F.load()
    return F


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def requests():
    out = []
    for i, (dim, H, r, f, a) in enumerate([(2, 4, 4, "cubic", 1.0), (2, 8, 3, "expm1", 1.0),
                                           (3, 4, 2, "cubic", 1.0), (2, 4, 2, "expm1", 1.0),
                                           (2, 4, 4, "cubic", 1.7), (3, 4, 1, "expm1", 1.0),
                                           (2, 4, 4, "cubic", 1.0), (2, 4, 5, "expm1", 0.6)]):
        modes = [((1,) * dim, 1.0), ((2,) + (1,) * (dim - 1), 0.5 - 0.1 * i)]
        out.append(W.Problem(dim=dim, coarse_cells=H, refinements=r, f=f, a=a, modes=modes,
                             name=f"req{i}"))
    return out


def pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    return t


def run(fmg, server, probs, precision, together):
    """Submits the requests (all at once, or one after the other) and returns their results."""
    gs = [pinned(p.g_nodal()) for p in probs]
    us = [torch.zeros(gs[i].shape, dtype=torch.float64).pin_memory() for i in range(len(probs))]
    params = [fmg.make_params(p, precision=precision) for p in probs]
    results = {}
    tickets = []
    for i in range(len(probs)):
        tickets.append(server.submit(params[i], gs[i], us[i]))
        if not together:
            server.drain(120.0)
            for r in server.poll():
                results[r.ticket] = r
    server.drain(120.0)
    for r in server.poll():
        results[r.ticket] = r
    out = []
    for i, t in enumerate(tickets):
        r = results[t]
        assert r.status == fmg.FMG_OK, (probs[i].name, r.status)
        assert r.stats.flags == 0
        assert r.latency_ms >= r.queue_ms >= 0.0
        out.append(us[i].numpy().copy())
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_are_the_same_alone_and_in_the_mix(fmg, precision):
    probs = requests()
    server = fmg.Server(max_inflight=4)
    alone = run(fmg, server, probs, precision, together=False)
    mixed_in = run(fmg, server, probs, precision, together=True)
    # twice over, interleaved with itself, to keep several contexts of a shape busy at once
    again = run(fmg, server, probs + probs, precision, together=True)
    for i, p in enumerate(probs):
        assert np.array_equal(alone[i], mixed_in[i]), p.name
        assert np.array_equal(alone[i], again[i]), p.name
        assert np.array_equal(alone[i], again[i + len(probs)]), p.name
    info = server.info()
    assert info.completed == info.submitted == 4 * len(probs)
    assert info.in_flight == 0 and info.queued == 0
    # hierarchies are kept: far fewer contexts than requests
    assert info.contexts_created <= 2 * len(probs)
    server.close()
    if precision == "fp64":
        for i, p in enumerate(probs):
            s = fmg.Solver(fmg.make_params(p, precision="fp64"), p.g_nodal())
            ref = s.solve().cpu().numpy()
            s.close()
            assert rel(alone[i], ref) <= FP64_TOL, p.name


def test_admission_by_memory_budget(fmg):
    probs = requests()
    need = max(fmg.fmg_workspace_bytes(fmg.make_params(p, precision="mixed")) for p in probs)
    ref_server = fmg.Server(max_inflight=4)
    ref = run(fmg, ref_server, probs, "mixed", together=True)
    ref_server.close()
    # room for the largest hierarchy only: requests wait for memory, idle contexts are evicted
    server = fmg.Server(hbm_budget=need, max_inflight=4)
    got = run(fmg, server, probs, "mixed", together=True)
    info = server.info()
    assert info.bytes_held <= need
    assert info.contexts_evicted > 0
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    server.close()


def test_request_larger_than_budget_is_refused(fmg):
    small = W.Problem(dim=2, coarse_cells=4, refinements=2, f="cubic", modes=[((1, 1), 1.0)])
    big = W.Problem(dim=2, coarse_cells=4, refinements=5, f="cubic", modes=[((1, 1), 1.0)])
    budget = fmg.fmg_workspace_bytes(fmg.make_params(small, precision="fp64"))
    server = fmg.Server(hbm_budget=budget, max_inflight=2)
    g = pinned(big.g_nodal())
    u = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
    t = server.submit(fmg.make_params(big, precision="fp64"), g, u)
    gs = pinned(small.g_nodal())
    us = torch.zeros(gs.shape, dtype=torch.float64).pin_memory()
    t2 = server.submit(fmg.make_params(small, precision="fp64"), gs, us)
    server.drain(60.0)
    res = {r.ticket: r for r in server.poll()}
    assert res[t].status == fmg.FMG_ERR_OOM
    assert res[t2].status == fmg.FMG_OK
    server.close()
