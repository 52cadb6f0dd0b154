"""Continuous-batching server: each request's result is the same alone and
in a mix of concurrent requests, requests overlap on the device, and
admission by HBM footprint holds the reservations under the budget."""
import numpy as np
import pytest

from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    return stb.Context(0)


def _req(level, slabs, nrhs, seed):
    m = inputs.sphere_mesh(level, slabs, 4.0, 0.2, seed=seed)
    return m, inputs.pulse_params(nrhs, seed=seed + 100)


def test_server_same_alone_and_in_mix(ctx):
    import paper_2103_16841_gb300 as stb
    srv = stb.Server(ctx, max_slots=3, precision="mixed", inner="fp32", tol=1e-8, restart=50, maxit=1000)
    a = _req(1, 8, 2, 1)
    ta = srv.submit(a[0], params=a[1])
    alone = srv.wait([ta])[ta]
    assert alone["status"] == 0 and alone["rel_residual"] <= 1e-8
    mix = [_req(1, 16, 4, 2), a, _req(2, 8, 1, 3), _req(1, 8, 1, 4), _req(2, 8, 4, 5)]
    tickets = [srv.submit(m, params=p) for m, p in mix]
    res = srv.wait(tickets)
    assert all(res[t]["status"] == 0 for t in tickets)
    again = res[tickets[1]]
    assert np.array_equal(again["w"], alone["w"])       # bit for bit
    st = srv.stats()
    print("server mix:", st)
    assert st["completed"] == 1 + len(mix) and st["failed"] == 0
    assert st["peak_running"] >= 2                       # requests overlapped on the device
    srv.close()
    # the same request through the direct API path
    mesh = stb.Mesh.from_spacetime(ctx, a[0])
    op = stb.Operator(ctx, mesh, "mixed", store_fp32=True)
    b = op.rhs(stb.DATA_PULSE, a[1])
    w, _ = op.solve(b, tol=1e-8, restart=50, maxit=1000, inner="fp32", max_refine=10)
    assert np.abs(w.T - alone["w"]).max() <= 1e-12 * np.abs(w).max()


def test_server_admission_by_hbm(ctx):
    import paper_2103_16841_gb300 as stb
    reqs = [_req(1, 8, 1, 10 + k) for k in range(4)]
    big = stb.Server(ctx, max_slots=2, precision="mixed", inner="fp32")
    t = big.submit(reqs[0][0], params=reqs[0][1])
    need = big.wait([t])[t]["reserved_bytes"]
    big.close()
    assert need > 0
    slots, share = 4, 64 << 20
    # a pool that holds one of these requests at a time
    srv = stb.Server(ctx, hbm_budget=slots * share + int(1.6 * need), max_slots=slots, precision="mixed",
                     inner="fp32")
    tickets = [srv.submit(m, params=p) for m, p in reqs]
    res = srv.wait(tickets)
    st = srv.stats()
    print("admission:", st, "need", need)
    assert all(res[t]["status"] == 0 for t in tickets)
    assert st["peak_running"] == 1
    assert st["peak_reserved_bytes"] <= int(1.6 * need)
    srv.close()
    # a request that can never fit completes with BEM_ERR_OUT_OF_MEMORY
    small = stb.Server(ctx, hbm_budget=slots * share + need // 2, max_slots=slots, precision="mixed", inner="fp32")
    t = small.submit(reqs[0][0], params=reqs[0][1])
    r = small.wait([t])[t]
    assert r["status"] == 2 and r["w"] is None
    small.close()


def test_server_resident_operators(ctx):
    """With cache_operators the assembled operator of a mesh stays resident:
    later requests on the same mesh skip the assembly (cache hits) and give the
    same densities as a fresh assembly and solve; when the pool is short,
    idle resident operators are evicted least recently used."""
    import paper_2103_16841_gb300 as stb
    m1, p1 = _req(1, 8, 1, 31)
    m2, p2 = _req(1, 16, 2, 32)
    srv = stb.Server(ctx, max_slots=2, precision="mixed", inner="fp32", tol=1e-8, cache_operators=True)
    t0 = srv.submit(m1, params=p1)
    first = srv.wait([t0])[t0]
    assert first["status"] == 0 and not first["cache_hit"]
    prm = [inputs.pulse_params(2, seed=40 + k) for k in range(3)]
    ts = [srv.submit(m1, params=p) for p in prm] + [srv.submit(m2, params=p2)]
    res = srv.wait(ts)
    assert all(res[t]["status"] == 0 for t in ts)
    assert sum(res[t]["cache_hit"] for t in ts[:3]) >= 2     # at most one may overlap the busy entry
    st = srv.stats()
    assert st["cache_hits"] >= 2 and st["cached_operators"] == 2   # one per mesh
    srv.close()
    mesh = stb.Mesh.from_spacetime(ctx, m1)
    op = stb.Operator(ctx, mesh, "mixed", store_fp32=True)
    for t, p in zip(ts[:3], prm):
        w, _ = op.solve(op.rhs(stb.DATA_PULSE, p), tol=1e-8, restart=50, maxit=2000, inner="fp32", max_refine=10)
        assert np.abs(w.T - res[t]["w"]).max() <= 1e-12 * np.abs(w).max()
    # eviction: a pool that holds one resident operator at a time
    need = first["reserved_bytes"]
    slots, share = 2, 64 << 20
    small = stb.Server(ctx, hbm_budget=slots * share + int(1.5 * need), max_slots=slots, precision="mixed",
                       inner="fp32", tol=1e-8, cache_operators=True)
    m3, p3 = _req(1, 8, 1, 33)                 # the same shape as m1, another jitter
    order = [(m1, p1), (m3, p3), (m1, p1)]
    for mm, pp in order:
        t = small.submit(mm, params=pp)
        r = small.wait([t])[t]
        assert r["status"] == 0
    st = small.stats()
    assert st["cached_operators"] <= 1 and st["peak_reserved_bytes"] <= int(1.5 * need)
    small.close()
