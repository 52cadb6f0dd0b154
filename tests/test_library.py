"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports
every symbol that include/stbem.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2103_16841_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "stbem.h")).read()
    return sorted(set(re.findall(r"\b(bem_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(_lib.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_no_gpu_gives_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2103_16841_gb300 as stb
    with pytest.raises(stb.BemError) as e:
        stb.Context(0)
    assert e.value.status == 3
