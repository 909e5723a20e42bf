"""The oracle's Python mirrors of its C structs (ctypes for the medium and the parameters,
numpy dtypes for the ray, hit and solution records) against oracle/rp_oracle.h: a C program
built from the header prints each struct's size and every field's offset."""
import ctypes as C
import os
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fields(obj):
    if isinstance(obj, type) and issubclass(obj, C.Structure):
        return C.sizeof(obj), {f[0]: getattr(obj, f[0]).offset for f in obj._fields_}
    return obj.itemsize, {k: obj.fields[k][1] for k in obj.names}


PAIRS = [("or_medium", oracle.Medium), ("or_params", oracle.Params),
         ("or_ray", oracle.RAY_DTYPE), ("or_hit", oracle.HIT_DTYPE),
         ("or_solution", oracle.SOL_DTYPE)]


def test_oracle_mirrors_match_the_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rp_oracle.h"',
             'int main(void) {']
    for cname, obj in PAIRS:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in _fields(obj)[1]:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['return 0;', '}']
    src, exe = tmp_path / "olayout.c", tmp_path / "olayout"
    src.write_text("\n".join(lines))
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "oracle"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("layout program does not build:\n" + r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}
    for cname, obj in PAIRS:
        size, offs = _fields(obj)
        assert got[(cname, "size")] == size, cname
        for f, off in offs.items():
            assert got[(cname, f)] == off, (cname, f)
