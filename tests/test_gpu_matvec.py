"""Products with the assembled operator in every arithmetic (FP64, FP32,
tensor-core TF32 and BF16), against the FP64 product, on a small mesh with
the exported dense matrix, and at full size (level-3 sphere, 32 slabs, 64
right-hand sides) in the launch configuration the solver uses."""
import numpy as np
import pytest

from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# unit roundoff of the rounded operands (values and x) per arithmetic
U = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    return stb.Context(0)


@pytest.fixture(scope="module")
def small(ctx):
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(1, 6, 2.0, 0.2, seed=5)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "fp64")
    return m, op, op.export_dense()


@pytest.mark.parametrize("dtype", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 13, 64, 70])
def test_product_error_bound_small(small, dtype, nrhs):
    """|y - A x| <= (2 u + W u_fp32) (|A| |x|) row by row, W the row's nonzeros."""
    m, op, A = small
    x = np.random.default_rng(nrhs).normal(size=(nrhs, m.n_tet))
    y = op.matvec(torch.tensor(x, device="cuda"), dtype=dtype).cpu().numpy()
    ref = x @ A.T
    absb = np.abs(x) @ np.abs(A).T
    nnz_row = (A != 0).sum(axis=1)
    bound = (2 * U[dtype] + 2 * U[dtype] ** 2 + (nnz_row + 2) * 2.0 ** -24) * absb + 1e-300
    ratio = np.abs(y - ref) / bound
    assert ratio.max() <= 1.0, (dtype, nrhs, ratio.max())


@pytest.mark.parametrize("dtype", ["fp32", "tf32", "bf16"])
def test_product_columns_exact_rounding_small(small, dtype):
    """x = unit vectors: every y entry is one value rounded to the arithmetic
    (after the FP64 -> FP32 rounding of the stored copy), so each entry of the
    chosen columns of A comes back within those two roundings."""
    m, op, A = small
    cols = np.random.default_rng(1).choice(m.n_tet, 64, replace=False)
    x = np.zeros((64, m.n_tet))
    x[np.arange(64), cols] = 1.0
    y = op.matvec(torch.tensor(x, device="cuda"), dtype=dtype).cpu().numpy()
    ref = A[:, cols].T
    assert np.all(np.abs(y - ref) <= (U[dtype] + 2.0 ** -24) * np.abs(ref) * (1 + 1e-9))
    assert np.all((ref == 0) == (y == 0))


@pytest.fixture(scope="module")
def c2(ctx):
    import paper_2103_16841_gb300 as stb
    m = inputs.workload_c2()
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "mixed")
    return m, op


@pytest.mark.parametrize("dtype", ["tf32", "bf16"])
def test_c2_spmm_64_columns_exact_rounding(c2, dtype):
    m, op = c2
    cols = np.random.default_rng(2).choice(m.n_tet, 64, replace=False)
    x = torch.zeros((64, m.n_tet), dtype=torch.float64, device="cuda")
    x[torch.arange(64), torch.tensor(cols)] = 1.0
    ref = op.matvec(x, dtype="fp64")
    y = op.matvec(x, dtype=dtype)
    err = (y - ref).abs() - U[dtype] * ref.abs() * (1 + 1e-9)
    assert err.max().item() <= 0.0
    assert torch.equal(ref == 0, y == 0)


@pytest.mark.parametrize("dtype", ["fp32", "tf32", "bf16"])
def test_c2_spmm_64_dense(c2, dtype):
    """Dense x in [0.5, 1]: per right-hand side, the relative 2-norm error
    against the FP64 product. Rounding values and x costs about 2u per
    product; cancellation between entries of mixed sign can enlarge it for a
    row sum, so the thresholds allow a factor of about 4 over 2u (the columns
    test above checks every fragment position exactly)."""
    m, op = c2
    g = torch.Generator(device="cuda").manual_seed(3)
    x = 0.5 + 0.5 * torch.rand((64, m.n_tet), dtype=torch.float64, device="cuda", generator=g)
    ref = op.matvec(x, dtype="fp64")
    y = op.matvec(x, dtype=dtype)
    rel = ((y - ref).norm(dim=1) / ref.norm(dim=1)).max().item()
    print("C2 64-RHS %s product, largest per-RHS relative 2-norm error: %.3e" % (dtype, rel))
    assert rel <= {"fp32": 1e-5, "tf32": 4e-3, "bf16": 3e-2}[dtype]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-12)])
def test_matrix_free_product_matches_assembled(ctx, precision, tol):
    """The matrix-free product (quadrature summed against x, no stored values)
    against the assembled operator's FP64-accumulated product: the same
    entries, so equal up to summation order."""
    import paper_2103_16841_gb300 as stb
    m = inputs.sphere_mesh(1, 8, 4.0, 0.2, seed=6)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, precision)
    mf = stb.Operator(ctx, mesh, precision, matrix_free=True)
    assert mf.stats()["nnz"] == op.stats()["nnz"] and mf.stats()["stored"] == 0
    x = torch.tensor(np.random.default_rng(3).normal(size=(3, m.n_tet)), device="cuda")
    y = op.matvec(x, dtype="fp64")
    yf = mf.matvec(x)
    err = ((yf - y).abs().max() / y.abs().max()).item()
    print("matrix-free vs assembled (%s): %.3e" % (precision, err))
    assert err <= tol
    # a solve through the matrix-free operator
    b = op.rhs(stb.DATA_PULSE, inputs.pulse_params(1, seed=2))[:, 0]
    w, info = op.solve(b, tol=1e-10, restart=50, maxit=1000)
    wf, infof = mf.solve(b, tol=1e-10, restart=50, maxit=1000)
    assert infof[0]["converged"]
    assert np.abs(wf - w).max() <= 1e-8 * np.abs(w).max()


def test_bounded_wait_gives_up_and_leaves_the_context_usable(ctx, small):
    """The tensor-core product's mbarrier waits are bounded: a wait on a
    barrier that nothing completes returns after its budget with
    BEM_ERR_DEVICE_TIMEOUT (the product then flags the operator), and the
    context runs products afterwards."""
    st, ms = ctx.selftest_bounded_wait()
    assert st == 5 and 0.0 < ms < 1000.0
    m, op, A = small
    x = np.random.default_rng(0).normal(size=(4, m.n_tet))
    y = op.matvec(torch.tensor(x, device="cuda"), dtype="bf16").cpu().numpy()
    assert np.all(np.isfinite(y))
    assert op.check()[0] == 0          # no product of this operator gave up
