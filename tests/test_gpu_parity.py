"""GPU parity: the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: FP64 entries and inner potentials within 1e-11 relative to the
largest entry of the compared set (normwise; tiny entries are compared in
absolute terms at that scale); the sparsity pattern bit-exact; the mixed
(FP32 arc quadrature) path within 1e-6 relative.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = os.cpu_count()


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    return stb.Context(0)


def _pairs(m, n, seed, near_frac=0.5):
    X = m.stv_xyzt()
    rng = np.random.default_rng(seed)
    ncol = 3 * m.n_slabs
    xs, tets, svs = [], [], []
    while len(xs) < n:
        i = int(rng.integers(0, m.n_tet))
        if rng.uniform() < near_frac:
            j = int(np.clip(i + rng.integers(-2 * ncol, 3), 0, m.n_tet - 1))
        else:
            j = int(rng.integers(0, m.n_tet))
        Ti = X[m.tets[i]]
        w = rng.dirichlet([1, 1, 1])
        face = [0, 1, 2] if rng.uniform() < 0.5 else [1, 2, 3]
        x = w[0] * Ti[face[0]] + w[1] * Ti[face[1]] + w[2] * Ti[face[2]]
        x[0] += rng.choice([0.0, rng.uniform(0, 0.4)])
        xs.append(x)
        tets.append(X[m.tets[j]])
        svs.append(m.stv_sv[m.tets[j]])
    return np.array(xs), np.array(tets), np.array(svs)


def _oracle_inner(xs, tets):
    return np.array([oracle.inner(x, t) for x, t in zip(xs, tets)])


@pytest.mark.parametrize("mesh", ["c1", "l2j"])
def test_inner_potentials_fp64(ctx, mesh):
    import paper_2103_16841_gb300 as stb
    m = inputs.workload_c1() if mesh == "c1" else inputs.sphere_mesh(2, 8, 2.0, 0.2, seed=3)
    xs, tets, svs = _pairs(m, 400, 1)
    g = stb.inner_potentials(ctx, xs, tets, svs, "fp64")
    r = _oracle_inner(xs, tets)
    scale = np.abs(r).max()
    assert scale > 0
    err = np.abs(g - r) / scale
    assert err.max() <= 1e-11, (err.max(), int(np.argmax(err)))


def test_inner_potentials_appendix(ctx):
    """Appendix example panels (corner and edge approach), GPU vs closed form."""
    import math
    import paper_2103_16841_gb300 as stb
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "appendix_closed_forms.txt")
    rows = [l.split() for l in open(gold) if not l.startswith("#")]
    xs, tets, vals = [], [], []
    for case, t, r, val in rows:
        t, r, val = float(t), float(r), float(val)
        h, eps = 10 * t, float(r) * t
        tets.append([[h, 0, 0, 0], [0, h, 0, 0], [0, 0, h, 0], [0, 0, 0, 0.0]])
        xs.append([t, -eps / math.sqrt(2), -eps / math.sqrt(2), 0.0] if case == "corner" else [t, -eps, 5 * t, 0.0])
        vals.append(val)
    sv = np.tile(np.array([0, 1, 2, 0]), (len(xs), 1))
    g = stb.inner_potentials(ctx, np.array(xs), np.array(tets), sv, "fp64") * 4 * math.pi
    vals = np.array(vals)
    ts = np.array([float(r[1]) for r in rows])
    # FP64: relative to each value, with a floor at 1% of the example's time
    # scale t (the grazing case eps/t = 0.999 has I ~ 5e-7 t)
    scale = np.maximum(np.abs(vals), 0.01 * ts)
    assert (np.abs(g - vals) / scale).max() <= 1e-11, (np.abs(g - vals) / scale).max()
    # mixed: normwise, relative to the largest value of the set, as for entries
    gm = stb.inner_potentials(ctx, np.array(xs), np.array(tets), sv, "mixed") * 4 * math.pi
    assert (np.abs(gm - vals) / np.abs(vals).max()).max() <= 1e-6


def test_inner_potentials_mixed(ctx):
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(2, 8, 2.0, 0.2, seed=3)
    xs, tets, svs = _pairs(m, 300, 2)
    g = stb.inner_potentials(ctx, xs, tets, svs, "mixed")
    r = _oracle_inner(xs, tets)
    assert (np.abs(g - r) / np.abs(r).max()).max() <= 1e-6


@pytest.fixture(scope="module")
def small(ctx):
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(0, 3, 1.5, 0.2, seed=5)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "fp64")
    om = oracle.Mesh.from_spacetime(m)
    A_or = om.matrix(nthreads=NT)
    return m, mesh, op, om, A_or


def test_pattern_bitexact_small(small):
    m, mesh, op, om, _ = small
    rowptr, cols = op.export_pattern()
    P = om.pattern()
    assert op.stats()["nnz"] == int(P.sum())
    assert np.array_equal(np.diff(rowptr), P.sum(axis=1))
    assert np.array_equal(cols, np.nonzero(P)[1])


def test_matrix_parity_small(small):
    m, mesh, op, om, A_or = small
    A = op.export_dense()
    scale = np.abs(A_or).max()
    assert np.abs(A - A_or).max() <= 1e-11 * scale
    P = om.pattern()
    assert np.all(A[P == 0] == 0.0)      # exact zeros outside the pattern


def test_matvec_parity_small(small):
    m, mesh, op, om, A_or = small
    x = np.random.default_rng(0).normal(size=(2, m.n_tet))
    y = op.matvec(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = x @ A_or.T
    assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()


def test_rhs_parity(small):
    m, mesh, op, om, _ = small
    prm = inputs.pulse_params(3, seed=2)
    for kind, p in [(inputs.DATA_SIN2_UNIFORM, None), (inputs.DATA_PULSE, prm)]:
        g = op.rhs(kind, p)
        r = om.rhs(kind, p)
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def test_solve_small_vs_oracle_lu(small):
    m, mesh, op, om, A_or = small
    b = om.rhs(inputs.DATA_SIN2_UNIFORM)[:, 0]
    w_ref = oracle.lu_solve(A_or, b)
    w, info = op.solve(op.rhs(inputs.DATA_SIN2_UNIFORM)[:, 0], tol=1e-13, restart=100, maxit=2000)
    assert info[0]["converged"]
    assert np.linalg.norm(w - w_ref) <= 1e-10 * np.linalg.norm(w_ref)


@pytest.fixture(scope="module")
def c1(ctx):
    import paper_2103_16841_gb300 as stb
    m = inputs.workload_c1()
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "fp64")
    om = oracle.Mesh.from_spacetime(m)
    return m, mesh, op, om


def test_pattern_bitexact_c1(c1):
    m, mesh, op, om = c1
    rowptr, cols = op.export_pattern()
    P = om.pattern()
    assert np.array_equal(np.diff(rowptr), P.sum(axis=1))
    assert np.array_equal(cols, np.nonzero(P)[1])


def test_entries_parity_c1(c1):
    m, mesh, op, om = c1
    rng = np.random.default_rng(4)
    P = om.pattern()
    ij = np.argwhere(P)
    pick = ij[rng.choice(ij.shape[0], 3000, replace=False)]
    rows = rng.choice(m.n_tet, 2, replace=False)
    full = np.array([(i, j) for i in rows for j in range(m.n_tet)])
    pick = np.concatenate([pick, full])
    g = op.entries(pick)
    r = om.entries(pick, nthreads=NT)
    scale = np.abs(r).max()
    assert np.abs(g - r).max() <= 1e-11 * scale


def test_c1_sphere_closed_form_and_solver(c1):
    """P1 at C1: GMRES converges; the solution follows phi = pi sin(pi t)."""
    m, mesh, op, om = c1
    b = op.rhs(inputs.DATA_SIN2_UNIFORM)[:, 0]
    w, info = op.solve(b, tol=1e-12, restart=100, maxit=3000)
    assert info[0]["converged"], info
    X = m.stv_xyzt()
    tm = np.array([X[m.tets[j]][:, 0].mean() for j in range(m.n_tet)])
    ex = np.pi * np.sin(np.pi * tm)
    e = np.linalg.norm(w - ex) / np.linalg.norm(ex)
    assert e < 0.3, e
