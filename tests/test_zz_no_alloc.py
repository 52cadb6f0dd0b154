"""The allocation-free matrix-vector product (bem_matvec_noalloc) against the
regular one (bem_matvec), through the C ABI.

Callers that cannot let a library allocate device memory while they run (a
serving runtime that reserves device memory up front, or a loop on a latency
budget where cudaMalloc/cudaFree cost time and cudaFree synchronizes) use the
allocation-free entry point; its temporaries live in a fixed device array of
the library. This file runs last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def op():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    ctx = stb.Context(0)
    m = inputs.sphere_mesh(1, 4, 2.0, 0.2, seed=2)
    mesh = stb.Mesh.from_spacetime(ctx, m)
    o = stb.Operator(ctx, mesh, "fp64")
    yield o
    o.close()
    mesh.close()


def test_noalloc_matches_matvec_two_calls(op):
    g = torch.Generator(device="cuda").manual_seed(7)
    for nrhs in (1, 3):
        shape = (op.n,) if nrhs == 1 else (nrhs, op.n)
        for _ in range(2):                       # two calls in a row share the fixed scratch
            x = torch.randn(shape, dtype=torch.float64, device="cuda", generator=g)
            ref = op.matvec(x)
            y = op.matvec_noalloc(x)
            torch.cuda.synchronize()
            scale = ref.abs().max().item()
            assert scale > 0
            assert (y - ref).abs().max().item() <= 1e-11 * scale


def test_noalloc_rejects_oversized(op):
    import paper_2103_16841_gb300 as stb
    nrhs = (1 << 20) // op.n + 1
    x = torch.zeros((nrhs, op.n), dtype=torch.float64, device="cuda")
    with pytest.raises(stb.BemError) as e:
        op.matvec_noalloc(x)
    assert e.value.status == 1
