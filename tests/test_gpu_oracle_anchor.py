"""Batched and served solves against the FP64 oracle.

A small scatterer (the icosahedron scaled to an ellipsoid, T = 4, 8 jittered
slabs: 480 panels, two pulse right-hand sides) is small enough for the
oracle's dense assembly and LU. It is solved as one member of a batch of
scatterers (one persistent assembly launch over all operators, one
block-diagonal GMRES) and as one request among concurrent requests of the
continuous-batching server; each result is compared with the oracle's
solution of the same discrete system: FP64 within 1e-10, the mixed form
(FP32 quadrature values, FP32 inner solves, FP64 refinement) within 1e-6.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NT = os.cpu_count()

CASES = [("fp64", "fp64", 1e-10), ("mixed", "fp32", 1e-6)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    return stb.Context(0)


@pytest.fixture(scope="module")
def anchor():
    v, f = inputs.ellipsoid(0, np.array([1.2, 0.8, 0.6]))
    m = inputs.prism_mesh(v, f, 8, 4.0, 0.2, seed=11)
    prm = inputs.pulse_params(2, seed=12)
    om = oracle.Mesh.from_spacetime(m)
    A = om.matrix(nthreads=NT)
    W = oracle.lu_solve(A, om.rhs(inputs.DATA_PULSE, prm))
    return m, prm, W


def _rel(w, W):
    return np.linalg.norm(w - W, axis=0) / np.linalg.norm(W, axis=0)


@pytest.mark.parametrize("precision,inner,tol", CASES)
def test_batch_member_matches_oracle_lu(ctx, anchor, precision, inner, tol):
    import paper_2103_16841_gb300 as stb
    m, prm, W = anchor
    probs = [(m, prm)] + inputs.scatterer_meshes(3, seed=5)
    meshes = [stb.Mesh.from_spacetime(ctx, mm) for mm, _ in probs]
    batch = stb.Batch(ctx, meshes, precision=precision)
    ws, infos = batch.solve([p for _, p in probs], tol=1e-12, restart=50, maxit=3000, inner=inner, max_refine=15)
    assert all(i["converged"] for inf in infos for i in inf)
    rel = _rel(ws[0], W)
    print("batch member vs oracle LU (%s):" % precision, rel)
    assert rel.max() <= tol
    batch.close()


@pytest.mark.parametrize("precision,inner,tol", CASES)
def test_served_request_matches_oracle_lu(ctx, anchor, precision, inner, tol):
    import paper_2103_16841_gb300 as stb
    m, prm, W = anchor
    srv = stb.Server(ctx, max_slots=3, precision=precision, inner=inner, tol=1e-12, restart=50, maxit=3000,
                     max_refine=15)
    others = [inputs.sphere_mesh(1, 8, 4.0, 0.2, seed=21), inputs.sphere_mesh(1, 16, 4.0, 0.2, seed=22)]
    tickets = [srv.submit(others[0], params=inputs.pulse_params(3, seed=23)), srv.submit(m, params=prm),
               srv.submit(others[1], params=inputs.pulse_params(1, seed=24))]
    res = srv.wait(tickets)
    assert all(res[t]["status"] == 0 for t in tickets)
    w = res[tickets[1]]["w"].T                 # [n_tet, nrhs]
    rel = _rel(w, W)
    print("served request vs oracle LU (%s):" % precision, rel)
    assert rel.max() <= tol
    srv.close()
