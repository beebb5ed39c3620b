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


@pytest.mark.parametrize("t", [10.0, 137.0, 1.0e4])
@pytest.mark.parametrize("Nz", [8, 16, 32, 64])
def test_library_contour_matches_the_oracle(t, Nz):
    """Host-side arithmetic of the library (no device call): the Talbot nodes and quadrature weights
    that every solve uses (Sec. 2.2) equal the oracle's independent contour to rounding, and the
    projected nodes (reading of Sec. 3: tau in the closed right half-plane) differ only in Re z."""
    import numpy as np

    from oracle import contour
    from paper_1409_2556_gb300 import _lib
    lib = _lib.load()
    z = np.zeros(Nz)
    w = np.zeros(Nz)
    assert lib.lt_contour_nodes(t, Nz, 0, z.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)) == 0
    zc, wc = z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]
    zo, wo = contour.nodes_weights(t, Nz)
    assert np.max(np.abs(zc - zo) / np.abs(zo)) < 1e-13
    assert np.max(np.abs(wc - wo)) / np.max(np.abs(wo)) < 1e-13
    zp = np.zeros(Nz)
    assert lib.lt_contour_nodes(t, Nz, 1, zp.ctypes.data_as(ctypes.c_void_p), None) == 0
    assert np.array_equal(zp[1::2], z[1::2])
    assert np.array_equal(zp[0::2], np.maximum(z[0::2], 0.0))
    assert lib.lt_contour_nodes(t, Nz + 1, 0, z.ctypes.data_as(ctypes.c_void_p), None) == -1   # odd Nz refused
