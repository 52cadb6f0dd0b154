"""Solver pins on the 960-panel sphere (icosphere level 1, T = 2, 4 uniform
slabs, sin^2 data): GPU GMRES in FP64, and the mixed-precision operator with
FP32 inner solves and FP64 refinement, against the oracle's dense LU
solution of the same discrete system."""
import os

import numpy as np
import pytest

import oracle
from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NT = os.cpu_count()


@pytest.fixture(scope="module")
def c1_lu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    ctx = stb.Context(0)
    m = inputs.workload_c1()
    om = oracle.Mesh.from_spacetime(m)
    A = om.matrix(nthreads=NT)
    b = om.rhs(inputs.DATA_SIN2_UNIFORM)[:, 0]
    w_ref = oracle.lu_solve(A, b)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    return ctx, m, mesh, w_ref


def test_c1_fp64_gmres_vs_oracle_lu(c1_lu):
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, w_ref = c1_lu
    op = stb.Operator(ctx, mesh, "fp64")
    w, info = op.solve(op.rhs(stb.DATA_SIN2_UNIFORM)[:, 0], tol=1e-13, restart=100, maxit=3000)
    assert info[0]["converged"]
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    print("C1 FP64 GMRES vs oracle LU: %.3e" % rel)
    assert rel <= 1e-10


def test_c1_mixed_refined_vs_oracle_lu(c1_lu):
    """Mixed-precision form (FP32 quadrature values, FP32 inner GMRES, FP64
    refinement on the outer residual) against the FP64 oracle: <= 1e-6."""
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, w_ref = c1_lu
    op = stb.Operator(ctx, mesh, "mixed")
    w, info = op.solve(op.rhs(stb.DATA_SIN2_UNIFORM)[:, 0], tol=1e-12, restart=100, maxit=2000,
                       inner="fp32", max_refine=12)
    assert info[0]["converged"]
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    print("C1 mixed + refinement vs oracle LU: %.3e" % rel)
    assert rel <= 1e-6


@pytest.mark.parametrize("inner", ["tf32", "bf16"])
def test_c1_tensor_core_inner_solves_vs_oracle_lu(c1_lu, inner):
    """Inner GMRES with tensor-core products (TF32 or BF16 values and
    vectors, FP32 accumulation) inside the FP64 refinement reaches the same
    solution as FP32 inner solves: the bar of the mixed form, <= 1e-6."""
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, w_ref = c1_lu
    op = stb.Operator(ctx, mesh, "mixed")
    w, info = op.solve(op.rhs(stb.DATA_SIN2_UNIFORM)[:, 0], tol=1e-12, restart=100, maxit=2000,
                       inner=inner, max_refine=40)
    assert info[0]["converged"]
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    print("C1 mixed, %s inner + FP64 refinement (%d refinements) vs oracle LU: %.3e"
          % (inner, info[0]["refinements"], rel))
    assert rel <= 1e-6


@pytest.mark.parametrize("inner", ["fp32", "tf32", "bf16"])
def test_c1_refinement_with_fp64_residual_vs_oracle_lu(c1_lu, inner):
    """bem_solve_refined: the outer residual from the FP64 operator, the inner
    solves on the mixed operator; the refinement converges to the FP64
    operator's solution, so it matches the oracle LU to FP64 solver accuracy
    although the inner operator carries the FP32 quadrature error."""
    import paper_2103_16841_gb300 as stb
    ctx, m, mesh, w_ref = c1_lu
    op64 = stb.Operator(ctx, mesh, "fp64", store_fp32=False)
    opm = stb.Operator(ctx, mesh, "mixed")
    b = op64.rhs(stb.DATA_SIN2_UNIFORM)[:, 0]
    w, info = opm.solve_refined(op64, b, tol=1e-13, restart=100, maxit=2000, inner=inner, max_refine=30)
    assert info[0]["converged"]
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    print("C1 refinement with the FP64 residual (%s inner) vs oracle LU: %.3e" % (inner, rel))
    assert rel <= 1e-10
