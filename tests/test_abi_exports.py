"""The C ABI library builds here (nvcc cross-compiles for sm_103a without a GPU), loads, and
exports every function that include/rp.h declares; no compute call is made."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rp_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    from paper_1810_01780_gb300 import _abi, build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "rp_trace" in names and "rp_find_paths" in names and "rp_trace_static" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding knows the same entry points
    assert set(names) <= set(_abi.SIGNATURES), sorted(set(names) - set(_abi.SIGNATURES))
    assert lib.rp_version  # a symbol lookup only


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the library absent every entry point of the binding raises."""
    import pytest

    from paper_1810_01780_gb300 import _abi, api, workloads as W

    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        api.Medium(W.ice_with_surface())
    with pytest.raises(RuntimeError, match="not built"):
        api.Surrogate(seed=0)
    with pytest.raises(RuntimeError, match="not built"):
        _abi.lib()
