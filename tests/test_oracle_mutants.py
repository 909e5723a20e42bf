"""Planted mistakes: each entry plants one plausible error (a flipped sign, a dropped term,
a swapped index or operand, a wrong constant) in a fresh copy of the oracle and runs the pin
named beside it, which must then fail; the unchanged copy passes every named pin.  This is
what shows that the pins fix the oracle's arithmetic rather than restate it.  The copies live
in pytest's temporary folder; the repository's oracle is never touched."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what is planted, file, original text, planted text, the pin that must fail)
MUTANTS = [
    ('ck a43 sign', 'oracle/rp_oracle.c',
     '{3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0}',
     '{3.0 / 10.0, 9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0}',
     'tests/test_oracle_pins.py::test_tableau_order_conditions'),
    ('ck b5 typo', 'oracle/rp_oracle.c',
     '250.0 / 621.0',
     '250.0 / 612.0',
     'tests/test_oracle_pins.py::test_tableau_order_conditions'),
    ('rhs drop projection', 'oracle/rp_oracle.c',
     'k[3 + i] = (g[i] - gt * y[3 + i]) / n;',
     'k[3 + i] = g[i] / n;',
     'tests/test_oracle_pins.py::test_rhs_projection_and_index'),
    ('rhs projection sign', 'oracle/rp_oracle.c',
     'k[3 + i] = (g[i] - gt * y[3 + i]) / n;',
     'k[3 + i] = (g[i] + gt * y[3 + i]) / n;',
     'tests/test_oracle_pins.py::test_rhs_projection_and_index'),
    ("rhs momentum r' unnormalised", 'oracle/rp_oracle.c',
     'k[i] = y[3 + i] / q;',
     'k[i] = y[3 + i];',
     'tests/test_oracle_pins.py::test_snell_invariant_conserved[momentum]'),
    ('momentum stages on t', 'oracle/rp_oracle.c',
     'for (int c = 3; c < 6; ++c) y0[c] = n0 * y0_in[c];',
     'for (int c = 3; c < 6; ++c) y0[c] = y0_in[c];',
     'tests/test_oracle_pins.py::test_snell_invariant_conserved[momentum]'),
    ('dn/dz missing 1/z0', 'oracle/rp_oracle.c',
     '*dndz = dn / z0 * e;',
     '*dndz = dn * e;',
     'tests/test_oracle_pins.py::test_ray_step_local_order'),
    ('propagate 4th order', 'oracle/rp_oracle.c',
     's5 += or_ck_b5[i] * k[i][c];',
     's5 += or_ck_b4[i] * k[i][c];',
     'tests/test_oracle_pins.py::test_ray_step_local_order'),
    ('layer offset dropped', 'oracle/rp_oracle.c',
     '*n = n0 - dn * e + off;',
     '*n = n0 - dn * e;',
     'tests/test_oracle_pins.py::test_layer_offset_shifts_the_profile'),
    ('dn==0 branch drops off', 'oracle/rp_oracle.c',
     '*n = n0 + off;',
     '*n = n0;',
     'tests/test_oracle_pins.py::test_layer_offset_shifts_the_profile'),
    ('layer_of boundary', 'oracle/rp_oracle.c',
     'if (z >= m->z_top[j]) k = j;',
     'if (z > m->z_top[j] + 1.0) k = j;',
     'tests/test_oracle_pins.py::test_start_layer_from_depth'),
    ('reflection sign', 'oracle/rp_oracle.c',
     't_refl[a] = t[a] + 2.0 * cos_i * nrm[a];',
     't_refl[a] = t[a] - 2.0 * cos_i * nrm[a];',
     'tests/test_oracle_pins.py::test_start_layer_from_depth'),
    ('error norm h scaling', 'oracle/rp_oracle.c',
     'er2 += d * d;',
     'er2 += (h * d) * (h * d);',
     'tests/test_oracle_pins.py::test_error_measure_is_per_unit_step[60.0]'),
    ('reject exponent', 'oracle/rp_oracle.c',
     'double fac = 0.9 * pow(e, -0.25);',
     'double fac = 0.9 * pow(e, 0.25);',
     'tests/test_oracle_pins.py::test_grid_ray_in_random_field_obeys_fermat'),
    ('no max_path truncation', 'oracle/rp_oracle.c',
     'h_try = p->max_path - s;',
     'h_try = h;',
     'tests/test_oracle_pins.py::test_straight_lines_constant_index'),
    ('fresnel rs swapped', 'oracle/rp_oracle.c',
     'double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);',
     'double rs = (n2 * cos_i - n1 * cos_t) / (n1 * cos_i + n2 * cos_t);',
     'tests/test_oracle_pins.py::test_fresnel_energy_conservation[s]'),
    ('fresnel ts numerator', 'oracle/rp_oracle.c',
     'double ts = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);',
     'double ts = 2.0 * n2 * cos_i / (n1 * cos_i + n2 * cos_t);',
     'tests/test_oracle_pins.py::test_fresnel_energy_conservation[s]'),
    ('fresnel tp denominator', 'oracle/rp_oracle.c',
     'double tp = 2.0 * n1 * cos_i / (n2 * cos_i + n1 * cos_t);',
     'double tp = 2.0 * n1 * cos_i / (n1 * cos_i + n2 * cos_t);',
     'tests/test_oracle_pins.py::test_fresnel_energy_conservation[p]'),
    ('fresnel rp swapped', 'oracle/rp_oracle.c',
     'double rp = (n2 * cos_i - n1 * cos_t) / (n2 * cos_i + n1 * cos_t);',
     'double rp = (n1 * cos_i - n2 * cos_t) / (n2 * cos_i + n1 * cos_t);',
     'tests/test_oracle_pins.py::test_fresnel_energy_conservation[p]'),
    ('unpol no half', 'oracle/rp_oracle.c',
     'double R = 0.5 * (rs * rs + rp * rp);',
     'double R = (rs * rs + rp * rp);',
     'tests/test_oracle_pins.py::test_fresnel_energy_conservation[unpol]'),
    ('snell refraction sign', 'oracle/rp_oracle.c',
     't_refr[a] = eta * t[a] + (eta * cos_i - cos_t) * nrm[a];',
     't_refr[a] = eta * t[a] + (eta * cos_i + cos_t) * nrm[a];',
     'tests/test_oracle_pins.py::test_step_growth_and_inherited_step'),
    ('secondary path reset', 'oracle/rp_oracle.c',
     'sec.s = s;',
     'sec.s = 0.0;',
     'tests/test_oracle_pins.py::test_step_growth_and_inherited_step'),
    ('snell eta not squared', 'oracle/rp_oracle.c',
     'double sin2_t = eta * eta * (1.0 - cos_i * cos_i);',
     'double sin2_t = eta * (1.0 - cos_i * cos_i);',
     'tests/test_oracle_pins.py::test_snell_vector_refraction_and_tir'),
    ('tir threshold', 'oracle/rp_oracle.c',
     'if (sin2_t > 1.0) {',
     'if (sin2_t > 0.98) {',
     'tests/test_oracle_pins.py::test_snell_vector_refraction_and_tir'),
    ('split n1 n2 swapped', 'oracle/rp_oracle.c',
     'or_split_dirs(y + 3, nrm, n1, n2,',
     'or_split_dirs(y + 3, nrm, n2, n1,',
     'tests/test_oracle_pins.py::test_boundary_split_constant_layers'),
    ('secondary amp uses r', 'oracle/rp_oracle.c',
     'sec.A = A * tau;',
     'sec.A = A * rr;',
     'tests/test_oracle_pins.py::test_boundary_split_constant_layers'),
    ('secondary time reset', 'oracle/rp_oracle.c',
     'sec.T = y[6];',
     'sec.T = 0.0;',
     'tests/test_oracle_pins.py::test_sphere_entry_reflection_refraction_exact'),
    ('receiver exit point', 'oracle/rp_oracle.c',
     'double lam = (-qb - sqrt(disc)) / (2.0 * qa);',
     'double lam = (-qb + sqrt(disc)) / (2.0 * qa);',
     'tests/test_oracle_pins.py::test_receiver_entry_point'),
    ('receiver time not interpolated', 'oracle/rp_oracle.c',
     'hp->time = y0[6] + lam * (y1[6] - y0[6]);',
     'hp->time = y1[6];',
     'tests/test_oracle_pins.py::test_receiver_entry_point'),
    ('grid weight index', 'oracle/rp_oracle.c',
     'e[dz][dy] = a0 + w[0] * (a1 - a0);',
     'e[dz][dy] = a0 + w[1] * (a1 - a0);',
     'tests/test_oracle_pins.py::test_grid_trilinear_exact_on_linear_field'),
    ('grid z weight', 'oracle/rp_oracle.c',
     'v[c] = f0 + w[2] * (f1 - f0);',
     'v[c] = f0 + w[1] * (f1 - f0);',
     'tests/test_oracle_pins.py::test_grid_trilinear_exact_on_linear_field'),
    ('grid inside bound', 'oracle/rp_oracle.c',
     'double hi = m->origin[a] + m->spacing * (double)(dims[a] - 1);',
     'double hi = m->origin[a] + m->spacing * (double)(dims[a] + 1);',
     'tests/test_oracle_pins.py::test_grid_leaves_domain'),
    ('pf type swap', 'oracle/rp_oracle.c',
     'if (r->n_refl > 0) return OR_SOL_REFLECTED;\n    if (r->n_turn > 0) return OR_SOL_REFRACTED;',
     'if (r->n_turn > 0) return OR_SOL_REFLECTED;\n    if (r->n_refl > 0) return OR_SOL_REFRACTED;',
     'tests/test_oracle_pins.py::test_path_finding_reproduces_paper_accuracy'),
    ('pf receive angle x', 'oracle/rp_oracle.c',
     's->receive = acos(fmax(-1.0, fmin(1.0, r->dir[2])));',
     's->receive = acos(fmax(-1.0, fmin(1.0, r->dir[0])));',
     'tests/test_oracle_pins.py::test_path_finding_reproduces_paper_accuracy'),
    ('max_time compares path', 'oracle/rp_oracle.c',
     '} else if (p->max_time > 0.0 && y[6] >= p->max_time) {',
     '} else if (p->max_time > 0.0 && s >= p->max_time * 299792458.0) {',
     'tests/test_oracle_pins.py::test_break_conditions'),
    ('min_amp vs current A', 'oracle/rp_oracle.c',
     '} else if (p->min_amp > 0.0 && fabs(A) < p->min_amp * fabs(st->A0)) {',
     '} else if (p->min_amp > 0.0 && fabs(A) < p->min_amp) {',
     'tests/test_oracle_pins.py::test_break_conditions'),
    ('mlp gelu sign', 'oracle/mlp.py',
     'return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))',
     'return 0.5 * x * (1.0 - _erf(x / math.sqrt(2.0)))',
     'tests/test_mlp_oracle_pins.py::test_gradients_match_finite_differences'),
    ('mlp gelu_grad term', 'oracle/mlp.py',
     '+ x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)',
     '+ np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)',
     'tests/test_mlp_oracle_pins.py::test_gradients_match_finite_differences'),
    ('mlp adam bias correction', 'oracle/mlp.py',
     'vh = v / (1.0 - beta2**step)',
     'vh = v',
     'tests/test_mlp_oracle_pins.py::test_adam_first_step_is_signed_lr'),
    ('mlp adam beta1 mix', 'oracle/mlp.py',
     'm = beta1 * m + (1.0 - beta1) * g',
     'm = beta1 * m + (1.0 - beta2) * g',
     'tests/test_mlp_oracle_pins.py::test_adam_first_step_is_signed_lr'),
    ('mlp bf16 truncation', 'oracle/mlp.py',
     'r = ((u + 0x7FFF + lsb) >> 16) << 16',
     'r = (u >> 16) << 16',
     'tests/test_mlp_oracle_pins.py::test_bf16_round'),
    ('earliest event -> latest', 'oracle/rp_oracle.c',
     'if (fr < ev_frac) {',
     'if (ev == EV_NONE || fr > ev_frac) {',
     'tests/test_oracle_pins.py::test_earliest_of_two_surfaces_in_one_step'),
    ('sphere exit region', 'oracle/rp_oracle.c',
     'other = inside ? or_layer_of(m, y[2]) : OR_MAX_LAYERS + j;',
     'other = inside ? 0 : OR_MAX_LAYERS + j;',
     'tests/test_oracle_pins.py::test_sphere_exit_into_the_layer_below_and_start_region'),
    ('sphere region strict', 'oracle/rp_oracle.c',
     'if (d2 < m->sph_R[j] * m->sph_R[j]) return OR_MAX_LAYERS + j;',
     'if (d2 < 0.9 * m->sph_R[j] * m->sph_R[j]) return OR_MAX_LAYERS + j;',
     'tests/test_oracle_pins.py::test_sphere_exit_into_the_layer_below_and_start_region'),
    ('h_max clamp dropped', 'oracle/rp_oracle.c',
     'if (h_next > p->h_max) h_next = p->h_max;',
     '',
     'tests/test_oracle_pins.py::test_closed_form_range_path_time[projected]'),
    ('analytic I0 sign', 'oracle/analytic.py',
     'return -(1.0 / self.b) * math.log(n + w)',
     'return (1.0 / self.b) * math.log(n + w)',
     'tests/test_oracle_pins.py::test_closed_form_range_path_time[projected]'),
    ('receiver amp parent', 'oracle/rp_oracle.c',
     'hp->amp = A;',
     'hp->amp = st->A0;',
     'tests/test_oracle_pins.py::test_receiver_hit_carries_the_current_amplitude'),
    ('pf vertical direction', 'oracle/rp_oracle.c',
     'double th = (zr[i] >= zs[i]) ? 0.0 : pi;',
     'double th = (zr[i] >= zs[i]) ? pi : 0.0;',
     'tests/test_oracle_pins.py::test_path_finder_vertical_pairs'),
    ('pf miss sign', 'oracle/rp_oracle.c',
     'if (r->status == OR_ST_MAX_PATH) return INFINITY;',
     'if (r->status == OR_ST_MAX_PATH) return -INFINITY;',
     'tests/test_oracle_pins.py::test_path_finder_matches_closed_forms_on_workload_pairs'),
]


def _copy_tree(dst):
    skip = shutil.ignore_patterns("*.so", "*.o", "__pycache__", "csrc", "_build*", "*.tmp*")
    for sub in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(dst, sub), ignore=skip)
    shutil.copytree(os.path.join(ROOT, "paper_1810_01780_gb300"),
                    os.path.join(dst, "paper_1810_01780_gb300"), ignore=skip)


def _run_pins(root, nodes):
    env = {k: v for k, v in os.environ.items() if not k.startswith("PYTEST_")}
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"] + nodes,
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_every_planted_mistake_fails_its_pin(tmp_path):
    base = tmp_path / "base"
    _copy_tree(str(base))
    nodes = sorted({m[4] for m in MUTANTS})
    rc, out = _run_pins(str(base), nodes)
    assert rc == 0, "the unchanged copy must pass every named pin:\n" + out

    def one(i):
        name, path, old, new, node = MUTANTS[i]
        d = tmp_path / f"m{i:02d}"
        shutil.copytree(str(base), str(d), ignore=shutil.ignore_patterns("*.so", "__pycache__"))
        p = d / path
        text = p.read_text()
        if text.count(old) != 1:
            return name, "the original text is not found exactly once in " + path
        p.write_text(text.replace(old, new))
        rc, out = _run_pins(str(d), [node])
        shutil.rmtree(str(d))
        return name, None if rc != 0 else "survived: " + node

    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        bad = [(n, why) for n, why in ex.map(one, range(len(MUTANTS))) if why]
    assert not bad, bad
