"""Host-side lit-panel search of Sec. 3.3 (bem_cluster_tree_*, no GPU needed):
the cluster tree's structure, X_N(x) as a superset of the lit panels
(exact lit set from the oracle's inner integral: V 1_sigma(x) > 0), and the
cardinality study of Sec. 4.1 (experiment 1) on a sequence of sphere meshes
with dt proportional to h: |Sigma_N^Xi(x)| and |X_N(x)| grow like N^(2/3)
and stay within a bounded factor of each other."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_16841_gb300 import inputs


def _lit_exact(m, x):
    T = m.stv_xyzt()[m.tets]
    return {j for j in range(m.n_tet) if oracle.inner(x, T[j]) > 0.0}


def _points(m, k, seed):
    """Apexes on the mesh's spatial vertices (t in (0, T]) and off the surface."""
    rng = np.random.default_rng(seed)
    sv = m.svert[rng.choice(len(m.svert), k)]
    t = rng.uniform(0.2, 1.0, k) * m.T
    pts = np.column_stack([t, sv])
    off = np.column_stack([rng.uniform(0.2, 1.0, k) * m.T, rng.normal(size=(k, 3)) * 0.8])
    return np.vstack([pts, off])


def test_tree_structure():
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(1, 4, 2.0, 0.2, seed=3)
    for n_min in (1, 8, 32):
        tr = stb.ClusterTree(m, n_min=n_min)
        info = tr.info()
        assert info["nodes"] == 2 * info["leaves"] - 1          # binary: every inner node has two sons
        assert info["leaves"] >= math.ceil(m.n_tet / n_min)
        # a point far in the past of every panel lights nothing; a point
        # far in the future lights nothing either (the cone has passed by)
        assert len(tr.query([-10.0, 0.0, 0.0, 0.0])[0]) == 0
        assert len(tr.query([100.0, 0.0, 0.0, 0.0])[0]) == 0
        tr.close()


def test_candidates_contain_the_lit_panels():
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(1, 4, 2.0, 0.2, seed=3)
    for n_min in (1, 8):
        tr = stb.ClusterTree(m, n_min=n_min)
        for x in _points(m, 6, seed=n_min):
            cand, _ = tr.query(x)
            assert len(set(cand.tolist())) == len(cand)           # each panel at most once
            lit = _lit_exact(m, x)
            assert lit <= set(cand.tolist()), (x, len(lit - set(cand.tolist())))
        tr.close()


def test_cardinality_study():
    """Experiment 1: points on the sphere at t = T. Exact lit sets on levels
    1-2 (oracle), candidate sets on levels 1-3 (tree, n_min = 8)."""
    import paper_2103_16841_gb300 as stb
    T = 2.0
    rows = []
    for level, slabs in [(1, 4), (2, 8), (3, 16)]:
        m = inputs.sphere_mesh(level, slabs, T, 0.0)
        tr = stb.ClusterTree(m, n_min=8)
        xs = [np.array([T, 0.0, 0.0, 1.0]), np.array([T, 0.6, 0.0, 0.8])]
        cand = [tr.query(x) for x in xs]
        n_x = np.mean([len(c) for c, _ in cand])
        n_vis = np.mean([v for _, v in cand])
        n_lit = np.mean([len(_lit_exact(m, x)) for x in xs]) if level <= 2 else float("nan")
        rows.append((m.n_tet, n_lit, n_x, n_vis))
        tr.close()
    print("N, |lit|, |X_N|, clusters tested:", rows)
    (N1, l1, x1, v1), (N2, l2, x2, v2), (N3, _, x3, v3) = rows
    # N grows 8x per level; a 2D intersection grows like N^(2/3), 4x
    for a, b, Na, Nb in [(l1, l2, N1, N2), (x1, x2, N1, N2), (x2, x3, N2, N3)]:
        p = math.log(b / a) / math.log(Nb / Na)
        assert 0.5 <= p <= 0.8, p
    # X_N is a bounded multiple of the lit set, and the search touches far fewer clusters than panels
    assert x1 <= 4.0 * l1 and x2 <= 4.0 * l2
    assert v3 < 0.25 * N3


def test_rejects_bad_input():
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(0, 2, 1.0, 0.0)
    with pytest.raises(stb.BemError) as e:
        stb.ClusterTree(m, n_min=0)
    assert e.value.status == 1
    bad = inputs.sphere_mesh(0, 2, 1.0, 0.0)
    bad.tets = bad.tets.copy()
    bad.tets[0, 0] = 10 ** 6                                # vertex id out of range
    with pytest.raises(stb.BemError) as e:
        stb.ClusterTree(bad, n_min=4)
    assert e.value.status == 1
