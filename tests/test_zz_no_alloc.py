"""The allocation-free matrix-vector product (bem_matvec_noalloc) against the
regular one (bem_matvec), through the C ABI.

Callers that cannot let a library allocate device memory while they run (a
serving runtime that reserves device memory up front, or a loop on a latency
budget where cudaMalloc/cudaFree cost time and cudaFree synchronizes) use the
allocation-free entry point; its temporaries live in a fixed device array of
the library. Both products are enqueued on torch's current stream, the stream
that wrote x. This file runs last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# operator kind -> (constructor arguments, tolerance relative to max |A x|):
# assembled products are the same kernel on the same values (bit-identical up
# to FP64 rounding); the matrix-free product adds rows with atomics, so the
# order of its last bits varies between runs
KINDS = {
    "fp64": (dict(precision="fp64"), 1e-11),
    "mixed": (dict(precision="mixed"), 1e-11),
    "fp64_matrix_free": (dict(precision="fp64", matrix_free=True), 1e-12),
}


@pytest.fixture(scope="module")
def mesh():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    ctx = stb.Context(0)
    m = inputs.sphere_mesh(1, 4, 2.0, 0.2, seed=2)
    me = stb.Mesh.from_spacetime(ctx, m)
    yield ctx, me
    me.close()


@pytest.fixture(scope="module", params=list(KINDS))
def op(request, mesh):
    import paper_2103_16841_gb300 as stb
    ctx, me = mesh
    kw, tol = KINDS[request.param]
    o = stb.Operator(ctx, me, **kw)
    yield o, tol
    o.close()


def test_noalloc_matches_matvec_two_calls(op):
    o, tol = op
    s = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(7)
    for nrhs in (1, 3):
        shape = (o.n,) if nrhs == 1 else (nrhs, o.n)
        for _ in range(2):                       # two calls in a row share the fixed scratch
            x = torch.randn(shape, dtype=torch.float64, device="cuda", generator=g)
            ref = o.matvec(x, stream=s)
            y = o.matvec_noalloc(x, stream=s)
            torch.cuda.synchronize()
            scale = ref.abs().max().item()
            assert scale > 0
            assert (y - ref).abs().max().item() <= tol * scale


def test_noalloc_keeps_current_device(op):
    o, _ = op
    before = torch.cuda.current_device()
    x = torch.ones(o.n, dtype=torch.float64, device="cuda")
    o.matvec_noalloc(x, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == before


def test_noalloc_rejects_oversized(op):
    import paper_2103_16841_gb300 as stb
    o, _ = op
    nrhs = (1 << 20) // o.n + 1
    x = torch.zeros((nrhs, o.n), dtype=torch.float64, device="cuda")
    with pytest.raises(stb.BemError) as e:
        o.matvec_noalloc(x, stream=torch.cuda.current_stream())
    assert e.value.status == 1
