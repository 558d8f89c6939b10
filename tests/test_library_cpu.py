"""CPU-side checks of the C-ABI library: it builds, loads, and exports every symbol that
include/poslo.h declares (no compute calls: there is no GPU here)."""
import os
import re
import subprocess

import pytest

from paper_2506_08781_gb300 import build, poslo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "poslo.h")).read()
    return sorted(set(re.findall(r"\b(poslo_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    try:
        build.build()
    except RuntimeError as e:   # nvcc missing: the library cannot exist
        pytest.skip(str(e))
    return poslo.load_library()


def test_header_and_binding_agree():
    assert sorted(poslo.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (poslo_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    for s in _declared():
        assert hasattr(lib, s)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(poslo.PosloError):
        poslo.Context(device=0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(poslo, "_lib", None)
    with pytest.raises(ImportError):
        poslo.load_library(str(tmp_path / "nope.so"))
