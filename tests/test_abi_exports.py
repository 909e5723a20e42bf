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


def _prototypes():
    txt = open(os.path.join(ROOT, "include", "rp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\n(int|const char \*)\s*(rp_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() not in ("", "void")]
        out[m.group(2)] = (m.group(1), params)
    return out


def _c_kind(decl):
    if "*" in decl or re.match(r"(const\s+)?rp_(medium|surrogate)_t\b", decl):
        return "ptr"
    for kind in ("int64_t", "int32_t", "size_t", "float", "double", "int"):
        if re.match(rf"(const\s+)?{kind}\b", decl):
            return {"int": "int32_t"}.get(kind, kind)
    raise AssertionError(decl)


def _ctypes_kind(t):
    import ctypes as C

    if t in (C.c_void_p, C.c_char_p) or hasattr(t, "_type_") and t.__name__.startswith("LP_"):
        return "ptr"
    return {C.c_int64: "int64_t", C.c_int32: "int32_t", C.c_size_t: "size_t",
            C.c_float: "float", C.c_double: "double"}[t]


def test_binding_signatures_match_the_header():
    """Argument kinds (pointer, int64, int32, size_t, float, double) of every prototype in
    include/rp.h against the ctypes signatures the binding installs."""
    import ctypes as C

    from paper_1810_01780_gb300 import _abi

    protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, (ret, params) in protos.items():
        res, args = _abi.SIGNATURES[name]
        assert (res is C.c_char_p) == (ret == "const char *"), name
        assert [_c_kind(p) for p in params] == [_ctypes_kind(a) for a in args], name
