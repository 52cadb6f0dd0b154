"""Launch-shape autotuning of the persistent quadrature: the first assembly
of a shape class times the candidates and records the choice (process and
cache file); later operators of the class, in this process or another one
reading the file, take it without timing; tuned and untuned assemblies give
the same bits."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2103_16841_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _values(op, n):
    x = torch.tensor(np.random.default_rng(0).normal(size=(2, n)), device="cuda")
    return op.matvec(x, dtype="fp64").cpu().numpy()


def test_tuning_records_and_reuses_the_launch_shape(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2103_16841_gb300 as stb
    cache = tmp_path / "tune.txt"
    m = inputs.sphere_mesh(2, 12, 3.0, 0.2, seed=9)
    ctx = stb.Context(0)
    ctx.set_tuning(1, str(cache))
    mesh = stb.Mesh.from_spacetime(ctx, m)
    op = stb.Operator(ctx, mesh, "mixed")
    t = op.tuning()
    assert t["tuned"] == "timed"
    chosen = "b%dx%d" % (t["budget_ctas"], t["ctas_per_sm"])
    assert chosen in t["sample_ms"] and len(t["sample_ms"]) >= 2
    assert t["sample_ms"][chosen] == min(t["sample_ms"].values())
    cache_code = 4 * (t["budget_ctas"] == 2) + t["ctas_per_sm"] - 1
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("stbem-tune-v2 ") and lines[0].endswith(" %d" % cache_code)
    # the same class again on another context: from the cache, no timing
    ctx2 = stb.Context(0)
    ctx2.set_tuning(1, str(cache))
    op2 = stb.Operator(ctx2, stb.Mesh.from_spacetime(ctx2, m), "mixed")
    t2 = op2.tuning()
    assert t2["tuned"] == "cache" and (t2["ctas_per_sm"], t2["budget_ctas"]) == (t["ctas_per_sm"], t["budget_ctas"])
    # an untuned operator: the build's shape, the same values
    ctx3 = stb.Context(0)
    op3 = stb.Operator(ctx3, stb.Mesh.from_spacetime(ctx3, m), "mixed")
    assert op3.tuning()["tuned"] == "default"
    assert np.array_equal(_values(op, m.n_tet), _values(op3, m.n_tet))
    # another process reads the file
    code = ("import json, sys; sys.path.insert(0, %r); import paper_2103_16841_gb300 as stb; "
            "from paper_2103_16841_gb300 import inputs; c = stb.Context(0); c.set_tuning(1, %r); "
            "m = inputs.sphere_mesh(2, 12, 3.0, 0.2, seed=9); "
            "o = stb.Operator(c, stb.Mesh.from_spacetime(c, m), 'mixed'); print(json.dumps(o.tuning()))"
            % (ROOT, str(cache)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    t4 = json.loads(out.stdout.strip().splitlines()[-1])
    assert t4["tuned"] == "cache" and (t4["ctas_per_sm"], t4["budget_ctas"]) == (t["ctas_per_sm"], t["budget_ctas"])
    assert len(cache.read_text().splitlines()) == 1
