"""Batches of small scatterers: one persistent launch per assembly pass over
all operators, one block-diagonal GMRES (CUDA graphs); every scatterer's
result against the same problem assembled and solved on its own."""
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


@pytest.mark.parametrize("precision,inner", [("mixed", "fp32"), ("fp64", "fp64")])
def test_batch_matches_single_operators(ctx, precision, inner):
    import paper_2103_16841_gb300 as stb
    probs = inputs.scatterer_meshes(6, seed=3)
    meshes = [stb.Mesh.from_spacetime(ctx, m) for m, _ in probs]
    batch = stb.Batch(ctx, meshes, precision=precision)
    st = batch.stats()
    ws, infos = batch.solve([p for _, p in probs], tol=1e-10, restart=50, maxit=2000, inner=inner, max_refine=12)
    nnz = 0
    for (m, prm), mesh, wb, inf in zip(probs, meshes, ws, infos):
        op = stb.Operator(ctx, mesh, precision, store_fp32=True)
        nnz += op.stats()["nnz"]
        b = op.rhs(stb.DATA_PULSE, prm)
        w, _ = op.solve(b, tol=1e-10, restart=50, maxit=2000, inner=inner, max_refine=12)
        assert all(i["converged"] for i in inf)
        err = np.abs(wb - w).max() / np.abs(w).max()
        assert err <= 1e-7, err
        op.close()
    assert st["nnz"] == nnz
    print("batch of %d: %s" % (len(probs), st))
    batch.close()
