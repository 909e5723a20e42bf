"""The oracle and the CUDA path share no code: no source of the package (Python binding, CUDA
kernels, C ABI) names the oracle, and no source of the oracle imports the package, includes
its headers or reads its CUDA sources.  Only the tests, the smoke check and the benchmark's
CPU legs load the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1810_01780_gb300")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_loads_the_oracle():
    bad = []
    for path in list(_sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp"))) + \
            [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]:
        text = open(path).read()
        if re.search(r"^\s*(import|from)\s+oracle\b|rp_oracle|librp_oracle|or_trace", text, re.M):
            bad.append(os.path.relpath(path, ROOT))
    assert not bad, bad


def test_oracle_does_not_use_the_product():
    bad = []
    for path in _sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        text = open(path).read()
        if re.search(r"^\s*(import|from)\s+paper_1810_01780_gb300\b|#include\s+[<\"].*(rp\.h|csrc|"
                     r"trace_core|rp_internal)|libradiopropa", text, re.M):
            bad.append(os.path.relpath(path, ROOT))
    assert not bad, bad


def _repo_python_files():
    """The repository's Python files: those git tracks (working files that .gitignore lists are
    not part of the repository), or, without git, every file outside hidden and
    underscore-prefixed top-level folders."""
    import subprocess

    try:
        out = subprocess.run(["git", "ls-files", "--cached", "--others", "--exclude-standard",
                              "*.py"], cwd=ROOT, capture_output=True, text=True, check=True)
        return [os.path.join(ROOT, f) for f in out.stdout.split()]
    except (OSError, subprocess.CalledProcessError):
        return [p for p in _sources(ROOT, (".py",))
                if not os.path.relpath(p, ROOT).startswith((".", "_"))]


def test_only_tests_smoke_and_bench_load_the_oracle():
    users = []
    for path in _repo_python_files():
        rel = os.path.relpath(path, ROOT)
        if rel.startswith(("oracle" + os.sep, "tests" + os.sep)):
            continue
        if re.search(r"^\s*(import|from)\s+oracle\b", open(path).read(), re.M):
            users.append(rel)
    assert sorted(users) == ["__graft_entry__.py", "bench.py"], users
