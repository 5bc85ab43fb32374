"""CPU checks of the C ABI: the library loads, exports every declared symbol, and its
pure host functions behave (no GPU compute is called here)."""
import re
import os

import numpy as np
import pytest

import paper_2310_14746_gb300 as hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hlbm_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2310_14746_gb300 import build
    build.build()
    return hb.library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the binding wraps each declared call under the same name
    assert names <= set(hb.SIGNATURES)
    for n in names:
        assert callable(getattr(hb, n)), n


def test_strerror(lib):
    for code in (hb.HLBM_OK, hb.HLBM_ERR_INVALID_ARG, hb.HLBM_ERR_OOM, hb.HLBM_ERR_CUDA,
                 hb.HLBM_ERR_NOT_CONVERGED, hb.HLBM_ERR_TIMEOUT, hb.HLBM_ERR_BUSY, hb.HLBM_ERR_IO,
                 hb.HLBM_ERR_STATE):
        assert hb.hlbm_strerror(code) != "unknown status"
    assert hb.hlbm_strerror(12345) == "unknown status"


def test_porosity_from_permeability_host(lib, oracle):
    """The pure host conversion varpi = 1 - nu tau / K (eq. d definition) agrees with the
    oracle's, including the clamps."""
    K = np.array([1e-4, 1e-3, 0.02, 0.5, 3.0, np.inf, 0.0, -2.0, np.nan], dtype=np.float32)
    nu, tau = 0.1 / 3, 0.6
    got = hb.hlbm_porosity_from_permeability(K, nu, tau)
    ref = oracle.porosity_from_permeability(K.astype(np.float64), nu, tau)
    np.testing.assert_allclose(got, ref.astype(np.float32), rtol=1e-6, atol=1e-7)
    assert got.min() >= 0 and got.max() <= 1


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument checks run before any device call."""
    import ctypes
    h = ctypes.c_void_p()
    L = lib
    assert L.hlbm_create(ctypes.byref(h), 7, 4, 4, 4, 1, 0, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_create(ctypes.byref(h), 9, 4, 4, 2, 1, 0, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_create(ctypes.byref(h), 19, 0, 4, 4, 1, 0, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_create(ctypes.byref(h), 19, 4, 4, 4, 9, 0, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_create(ctypes.byref(h), 19, 4, 4, 4, 1, 5, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_create(None, 19, 4, 4, 4, 1, 0, None) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_set_relaxation(None, 0.6) == hb.HLBM_ERR_INVALID_ARG
    assert L.hlbm_step(None, 1) == hb.HLBM_ERR_INVALID_ARG
    L.hlbm_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: a missing shared library raises on first use."""
    monkeypatch.setattr(hb, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(hb, "_L", None)
    with pytest.raises(RuntimeError):
        hb.library()
