"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point declared in include/lt.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(lt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1409_2556_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    from paper_1409_2556_gb300 import _lib
    assert set(_lib.EXPORTS) == set(declared)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1409_2556_gb300 import _lib
    # the loader must not silently fall back: a missing library raises
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1409_2556_gb300 import Engine, LtError
    with pytest.raises(LtError):
        Engine(0)
