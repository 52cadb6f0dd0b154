"""The problem statement's boundary calls through the C ABI (Sec. 2: Dirichlet
data g -> density): right-hand sides from samples of arbitrary data at the
library's face quadrature points, the asynchronous solve with its bounded wait
and cancellation, and the trial-space option.

Right-hand sides and solutions are checked against the FP64 oracle (its own
face rule and dense LU) on the 960-panel sphere (icosphere level 1, T = 2,
4 slabs)."""
import os

import numpy as np
import pytest

import oracle
from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NT = os.cpu_count()


def pulse(pts, prm):
    """g = exp(-((t - <x, d> - c) / w)^2) at points (t, x, y, z)."""
    d, c, w = prm[:3], prm[3], prm[4]
    return np.exp(-(((pts[:, 0] - pts[:, 1:] @ d - c) / w) ** 2))


@pytest.fixture(scope="module")
def c1():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    ctx = stb.Context(0)
    m = inputs.workload_c1()
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "fp64")
    return ctx, m, mesh, op


def test_rhs_points_weights_sum_to_the_projected_areas(c1):
    """Per face the weights integrate dA over the spatial triangle: their sum is
    |K|, so sum over all faces = sum over faces of the areas of their triangles."""
    ctx, m, mesh, op = c1
    for level, ng in [(0, 1), (1, 3), (2, 8)]:
        pts, w = op.rhs_points(level, ng)
        npps = 4 ** level * ng * ng
        assert pts.shape == (mesh.n_surfaces * npps, 4)
        per_face = w.reshape(mesh.n_surfaces, npps).sum(axis=1)
        assert np.all(per_face > 0)
        # every face of a column has the same |K|: constant within runs of equal spatial centroids
        xyz = pts[:, 1:].reshape(mesh.n_surfaces, npps, 3).mean(axis=1)
        key = np.round(xyz, 9)
        _, inv = np.unique(key, axis=0, return_inverse=True)
        for g in np.unique(inv)[:50]:
            v = per_face[inv == g]
            assert np.ptp(v) <= 1e-14 * v.max()


def test_rhs_from_samples_matches_oracle(c1):
    """b_i = int_K g(P_lo(y), y) - g(P_hi(y), y) dA from samples of a pulse at
    the library's points against the oracle's own face rule."""
    ctx, m, mesh, op = c1
    prm = inputs.pulse_params(3, seed=2)
    om = oracle.Mesh.from_spacetime(m)
    b_or = om.rhs(inputs.DATA_PULSE, prm, nrhs=3)
    pts, w = op.rhs_points(3, 8)
    g = np.stack([pulse(pts, p) for p in prm], axis=1)
    b = op.rhs_from_samples(g, 3, 8)
    err = np.abs(b - b_or).max() / np.abs(b_or).max()
    print("rhs from samples vs oracle: %.3e" % err)
    assert err <= 1e-10
    # one right-hand side at a time gives the same bits
    b0 = op.rhs_from_samples(g[:, 0], 3, 8)
    assert np.array_equal(b0, b[:, 0])


def test_solve_for_sampled_data_matches_oracle_lu(c1):
    ctx, m, mesh, op = c1
    prm = inputs.pulse_params(1, seed=5)
    om = oracle.Mesh.from_spacetime(m)
    A = om.matrix(nthreads=NT)
    w_ref = oracle.lu_solve(A, om.rhs(inputs.DATA_PULSE, prm)[:, 0])
    pts, _ = op.rhs_points(3, 8)
    b = op.rhs_from_samples(pulse(pts, prm[0]), 3, 8)
    w, info = op.solve(b, tol=1e-13, restart=100, maxit=3000)
    assert info[0]["converged"]
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    print("solve for sampled data vs oracle LU: %.3e" % rel)
    assert rel <= 1e-9


def test_rhs_points_reject_bad_rules(c1):
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, op = c1
    for level, ng in [(-1, 8), (5, 8), (0, 0), (0, 17)]:
        with pytest.raises(stb.BemError) as e:
            op.rhs_points(level, ng)
        assert e.value.status == 1


def test_trial_space_p1_is_unsupported(c1):
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, op = c1
    with pytest.raises(stb.BemError) as e:
        stb.Operator(ctx, mesh, "fp64", trial_space="p1")
    assert e.value.status == 6


@pytest.fixture(scope="module")
def l2x8():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    ctx = stb.Context(0)
    m = inputs.sphere_mesh(2, 8, 2.0, 0.2, seed=3)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "fp64")
    b = op.rhs(stb.DATA_PULSE, inputs.pulse_params(2, seed=2))
    return ctx, op, b


def test_solve_async_matches_solve(l2x8):
    """The asynchronous solve returns the same density as the blocking one (the
    same kernels in the same order); a zero-time wait on the just-started
    request runs out with BEM_ERR_DEVICE_TIMEOUT and leaves it valid."""
    ctx, op, b = l2x8
    w_sync, info_sync = op.solve(b, tol=1e-12, restart=50, maxit=2000)
    s = torch.cuda.Stream()
    bd = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
    wd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    req = op.solve_async(bd, wd, tol=1e-12, restart=50, maxit=2000, stream=s)
    assert req.wait(0.0) is None                 # still running: the wait ran out
    out = req.wait(120.0)
    assert out is not None
    st, infos = out
    assert st == 0 and all(i["converged"] for i in infos)
    req.close()
    w = wd.cpu().numpy().T
    assert np.abs(w - w_sync).max() <= 1e-14 * np.abs(w_sync).max()
    assert [i["iterations"] for i in infos] == [i["iterations"] for i in info_sync]


def test_solve_async_cancel(l2x8):
    """A cancelled solve stops at its next poll with BEM_ERR_CANCELLED."""
    ctx, op, b = l2x8
    s = torch.cuda.Stream()
    bd = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
    wd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    req = op.solve_async(bd, wd, tol=1e-15, restart=20, maxit=100000, stream=s)
    req.cancel()
    out = req.wait(120.0)
    assert out is not None and out[0] == 9
    req.close()
    assert torch.isfinite(wd).all()


def test_request_destroy_stops_a_running_solve(l2x8):
    ctx, op, b = l2x8
    s = torch.cuda.Stream()
    bd = torch.tensor(np.ascontiguousarray(b.T), device="cuda")
    wd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    req = op.solve_async(bd, wd, tol=1e-15, restart=20, maxit=100000, stream=s)
    req.close()                                  # cancels and joins the worker
    torch.cuda.synchronize()
