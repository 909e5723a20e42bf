"""The ctypes mirrors of the C ABI's structs (paper_1810_01780_gb300/_abi.py) against the
header itself: a C program built from include/rp.h prints every struct's size and each field's
offset, which must equal the ctypes layout (field names are the same on both sides)."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1810_01780_gb300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [("rp_layer", A.Layer), ("rp_sphere", A.Sphere), ("rp_surface", A.Surface),
         ("rp_medium_desc", A.MediumDesc),
         ("rp_rays", A.Rays), ("rp_receivers", A.Receivers), ("rp_trace_params", A.TraceParams),
         ("rp_ray_out", A.RayOut), ("rp_hits", A.Hits), ("rp_stats", A.Stats),
         ("rp_path_params", A.PathParams), ("rp_solutions", A.Solutions),
         ("rp_train_params", A.TrainParams), ("rp_surrogate_params", A.SurrogateParams),
         ("rp_surrogate_stats", A.SurrogateStats), ("rp_peaks", A.Peaks)]


def _c_layout(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rp.h"', 'int main(void) {']
    for cname, cls in PAIRS:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("layout program does not build:\n" + r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    return got


def test_ctypes_structs_match_the_header(tmp_path):
    got = _c_layout(tmp_path)
    for cname, cls in PAIRS:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])


def test_binding_constants_match_the_header(tmp_path):
    """Every enum value and limit the binding mirrors, printed by a C program built from the
    header."""
    want = {"RP_OK": A.RP_OK, "RP_MAX_LAYERS": A.MAX_LAYERS, "RP_MAX_SPHERES": A.MAX_SPHERES}
    want.update({name: code for code, name in A.ERRORS.items()})
    want.update({f"RP_MEDIUM_{k.upper()}": v for k, v in A.MEDIUM_KIND.items()})
    want.update({"RP_FP64": A.PRECISION["fp64"], "RP_FP32_MIXED": A.PRECISION["fp32"]})
    want.update({f"RP_POL_{k.upper()}": v for k, v in A.POLARIZATION.items()})
    want.update({f"RP_RHS_{k.upper()}": v for k, v in A.RHS_FORM.items()})
    want.update({f"RP_ST_{k}": v for k, v in A.STATUS.items()})
    want.update({f"RP_SOL_{k}": v for k, v in A.SOL_TYPE.items()})
    lines = ['#include <stdio.h>', '#include "rp.h"', 'int main(void) {']
    lines += [f'printf("{n} %lld\\n", (long long)({n}));' for n in want]
    lines += ['return 0;', '}']
    src, exe = tmp_path / "consts.c", tmp_path / "consts"
    src.write_text("\n".join(lines))
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("constants program does not build:\n" + r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}
    assert got == want
