"""Edge cases of the GPU path: the smallest meshes (one prism, one column of
many slabs), ragged columns (different slab counts side by side), the
column-size limit, rejected meshes and arguments, empty calls."""
import os
import types

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


def _merge(ms, shifts):
    """Space-time meshes side by side (spatial shift per part), one array set."""
    sv, stv_sv, stv_t, tets = [], [], [], []
    nsv = nstv = 0
    for m, d in zip(ms, shifts):
        sv.append(m.svert + np.asarray(d)[None, :])
        stv_sv.append(m.stv_sv + nsv)
        stv_t.append(m.stv_t)
        tets.append(m.tets + nstv)
        nsv += m.svert.shape[0]
        nstv += m.stv_t.shape[0]
    out = types.SimpleNamespace(svert=np.concatenate(sv), stv_sv=np.concatenate(stv_sv).astype(np.int32),
                                stv_t=np.concatenate(stv_t), tets=np.concatenate(tets).astype(np.int32))
    out.n_tet = out.tets.shape[0]
    out.stv_xyzt = lambda: np.column_stack([out.stv_t, out.svert[out.stv_sv]])
    return out


def _tri(scale=1.0):
    return np.array([[0.0, 0.0, 0.0], [scale, 0.0, 0.1], [0.2, scale, 0.0]]), np.array([[0, 1, 2]])


def _full_parity(ctx, m, tol=1e-11):
    import paper_2103_16841_gb300 as stb
    mesh = stb.Mesh.from_tets(ctx, m.svert, m.stv_sv, m.stv_t, m.tets)
    op = stb.Operator(ctx, mesh, "fp64")
    om = oracle.Mesh(m.stv_xyzt(), m.stv_sv, m.tets)
    P = om.pattern()
    rowptr, cols = op.export_pattern()
    assert np.array_equal(np.diff(rowptr), P.sum(axis=1)) and np.array_equal(cols, np.nonzero(P)[1])
    A = op.export_dense()
    R = om.matrix(nthreads=NT)
    assert np.abs(A - R).max() <= tol * np.abs(R).max()
    assert np.all(A[P == 0] == 0.0)
    return op, A


def test_single_prism(ctx):
    v, f = _tri()
    m = inputs.prism_mesh(v, f, 1, 1.0)
    _full_parity(ctx, m)


def test_one_column_many_slabs(ctx):
    v, f = _tri(0.3)
    m = inputs.prism_mesh(v, f, 40, 4.0, 0.2, seed=9)
    _full_parity(ctx, m)


def test_ragged_columns(ctx):
    """Columns with 3, 7 and 12 slabs next to each other (rows per column differ)."""
    import paper_2103_16841_gb300 as stb
    v, f = _tri(0.5)
    parts = [inputs.prism_mesh(v, f, n, 3.0, 0.2, seed=n) for n in (3, 7, 12)]
    m = _merge(parts, [(0, 0, 0), (0.9, 0.1, 0.0), (0.2, 0.8, 0.3)])
    op, A = _full_parity(ctx, m)
    x = np.random.default_rng(1).normal(size=(5, m.n_tet))
    for dt, tol in [("fp64", 1e-12), ("fp32", 1e-5), ("tf32", 4e-3), ("bf16", 3e-2)]:
        y = op.matvec(torch.tensor(x, device="cuda"), dtype=dt).cpu().numpy()
        ref = x @ A.T
        assert np.abs(y - ref).max() <= tol * (np.abs(x) @ np.abs(A).T).max(), dt


def test_column_size_limit(ctx):
    import paper_2103_16841_gb300 as stb
    v, f = _tri(0.3)
    m = inputs.prism_mesh(v, f, 64, 4.0)                   # 192 panels over one triangle: the limit
    mesh = stb.Mesh.from_tets(ctx, m.svert, m.stv_sv, m.stv_t, m.tets)
    op = stb.Operator(ctx, mesh, "mixed")
    assert op.check()[0] == 0
    m2 = inputs.prism_mesh(v, f, 65, 4.0)
    with pytest.raises(stb.BemError):
        stb.Mesh.from_tets(ctx, m2.svert, m2.stv_sv, m2.stv_t, m2.tets)


def test_rejected_meshes(ctx):
    import paper_2103_16841_gb300 as stb
    v, f = _tri()
    m = inputs.prism_mesh(v, f, 2, 1.0)
    bad_id = m.tets.copy()
    bad_id[0, 0] = 10_000
    not_flat = m.tets.copy()
    not_flat[0] = [0, 1, 3, 4]                             # two spatial vertices only: not a panel of Gamma_K x R
    flat_v = v.copy()
    flat_v[2] = 0.5 * (v[0] + v[1])                        # collinear spatial triangle
    for sv, tets in [(m.svert, bad_id), (m.svert, not_flat), (flat_v, m.tets)]:
        with pytest.raises(stb.BemError) as e:
            stb.Mesh.from_tets(ctx, sv, m.stv_sv, m.stv_t, tets)
        assert e.value.status == 7                         # BEM_ERR_BAD_MESH
    zero_dt = m.stv_t.copy()
    zero_dt[1] = zero_dt[0]                                # a vertical edge of zero length
    with pytest.raises(stb.BemError) as e:
        stb.Mesh.from_tets(ctx, m.svert, m.stv_sv, zero_dt, m.tets)
    assert e.value.status == 7


def test_rejected_arguments_and_empty_calls(ctx):
    import paper_2103_16841_gb300 as stb
    v, f = _tri()
    m = inputs.prism_mesh(v, f, 2, 1.0)
    mesh = stb.Mesh.from_tets(ctx, m.svert, m.stv_sv, m.stv_t, m.tets)
    with pytest.raises(stb.BemError) as e:
        stb.Operator(ctx, mesh, "fp64", m_q=5)
    assert e.value.status == 6                             # BEM_ERR_UNSUPPORTED
    with pytest.raises(stb.BemError) as e:
        stb.Operator(ctx, mesh, "fp64", n_theta=3)
    assert e.value.status == 1
    op = stb.Operator(ctx, mesh, "fp64")
    with pytest.raises(stb.BemError) as e:
        op.entries(np.array([[0, m.n_tet]], dtype=np.int32))
    assert e.value.status == 1
    with pytest.raises(stb.BemError):
        op.pattern_rows(np.array([m.n_tet], dtype=np.int32))
    assert op.entries(np.zeros((0, 2), dtype=np.int32)).shape == (0,)
    out = stb.inner_potentials(ctx, np.zeros((0, 4)), np.zeros((0, 4, 4)), np.zeros((0, 4), dtype=np.int32))
    assert out.shape == (0,)
    # a data pulse that never reaches the surface before T: b = 0, w = 0
    prm = np.array([[1.0, 0.0, 0.0, 50.0, 0.25]])
    b = op.rhs(stb.DATA_PULSE, prm)
    assert np.all(b == 0.0)
    w, info = op.solve(b, tol=1e-10)
    assert np.all(w == 0.0) and info[0]["converged"]


def test_cone_grazing_a_corner_of_timelike_faces(ctx):
    """Two ellipsoids of the 512-scatterer batch where the cone grazes a
    corner of faces steeper than the light cone (|grad P| > 1): the two arc
    events lie ~3e-8 apart, below what FP32 event positions resolve; the
    mixed operator must stay finite (the face is recomputed in FP64) and agree
    with the FP64 operator."""
    import paper_2103_16841_gb300 as stb
    grazing_row = {0: 6510, 1: 5744}        # a row holding the grazing pair in each mesh
    for k, (m, _) in enumerate(inputs.scatterer_meshes(512, seed=3, only=[174, 460])):
        mesh = stb.Mesh.from_spacetime(ctx, m)
        om = stb.Operator(ctx, mesh, "mixed")
        assert om.check()[0] == 0
        o64 = stb.Operator(ctx, mesh, "fp64")
        rng = np.random.default_rng(7)
        rows = np.unique(np.append(rng.choice(m.n_tet, 8, replace=False), grazing_row[k])).astype(np.int32)
        cols = o64.pattern_rows(rows)
        ij = np.array([(r, c) for r, cs in zip(rows, cols) for c in cs], dtype=np.int32)
        a64, am = o64.entries(ij), om.entries(ij)
        err = np.abs(am - a64).max() / np.abs(a64).max()
        print("grazing ellipsoid %d: mixed vs FP64 entries, normwise %.3e" % (k, err))
        assert err <= 1e-6
