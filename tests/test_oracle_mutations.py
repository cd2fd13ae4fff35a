"""Planted mistakes in the FP64 oracle, each of which one of its pins must catch.

Every entry below rewrites one spot of a copy of ``oracle/sph_oracle.c``.  The spots are
a wrong coefficient, a dropped self term, a wrong periodic image, a sign or bracket error
in the h update, a closed bound where the rule has an open one, and so on.  The copy is
compiled and the pin named beside the entry is run against it; the pin must fail.  The
unmodified copy passes every named pin, so a failure comes from the planted mistake.
The CUDA path is not involved.

Three rewrites are left out because they do not change any result:
- a periodic bucket row whose search span equals the row length, scanned as the span;
- a non-periodic extent that is not enlarged, since the bucket index is clamped anyway;
- a Newton step tried at zero slope, since the infinite point fails the bracket test.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

IP = "test_oracle_interact_pins.py::"  # pins in that file; the rest are in test_oracle_pins.py

# (what the mistake is, the original text, the planted text, the pin that must fail)
MUTANTS = [
    ("w: cubic coefficient",
     "double t = 6.0 * q - 6.0;",
     "double t = 6.0 * q - 5.0;",
     "test_kernel_normalisation_is_one"),
    ("w: knot moved",
     "    if (q <= 0.5) {\n        double t",
     "    if (q <= 0.45) {\n        double t",
     "test_kernel_normalisation_is_one"),
    ("w: outer piece squared",
     "return 2.0 * (a * a * a);",
     "return 2.0 * (a * a);",
     "test_kernel_normalisation_is_one"),
    ("mqdw: inner slope",
     "(12.0 - 18.0 * q)",
     "(12.0 - 16.0 * q)",
     "test_mqdw_is_minus_q_times_derivative_of_w"),
    ("mqdw: outer power",
     "return (6.0 * q) * (a * a);",
     "return (6.0 * q) * a;",
     "test_mqdw_is_minus_q_times_derivative_of_w"),
    ("c6: polynomial",
     "q * (25.0 + q * 32.0)",
     "q * (24.0 + q * 32.0)",
     "test_wendland_c6_normalisation_and_shape"),
    ("c6: power 8 -> 7",
     "return a8 * p;",
     "return a4 * a2 * a * p;",
     "test_wendland_c6_normalisation_and_shape"),
    ("c6 mqdw: prefactor",
     "return 22.0 * (q * q)",
     "return 20.0 * (q * q)",
     "test_wendland_c6_mqdw_is_minus_q_derivative"),
    ("c6 mqdw: polynomial",
     "q * (7.0 + q * 16.0)",
     "q * (7.0 + q * 15.0)",
     "test_wendland_c6_mqdw_is_minus_q_derivative"),
    ("min image: no wrap",
     "if (dx > 0.5 * L) return dx - L;",
     "if (dx > L) return dx - L;",
     "test_fixed_h_matches_numpy_brute_force"),
    ("min image: wrong sign",
     "if (dx < -0.5 * L) return dx + L;",
     "if (dx < -0.5 * L) return dx - L;",
     "test_fixed_h_matches_numpy_brute_force"),
    ("pair: r <= h",
     "if (r2 < h2) {\n        double r = sqrt(r2);\n        double q = r / h;",
     "if (r2 <= h2) {\n        double r = sqrt(r2);\n        double q = r / h;",
     "test_adversarial_positions_on_cell_faces_and_box_edges"),
    ("pair: self excluded",
     "    double r2 = dx * dx + dy * dy + dz * dz;\n    if (near_rel",
     "    double r2 = dx * dx + dy * dy + dz * dz;\n    if (i == j) return;\n    if (near_rel",
     "test_fixed_h_matches_numpy_brute_force"),
    ("pair: dy from x",
     "double dy = ps->y[j] - ps->y[i];\n    double dz = ps->z[j] - ps->z[i];\n    if (ps->periodic) {\n        dx = min_image(dx, ps->box[0]);",
     "double dy = ps->y[j] - ps->x[i];\n    double dz = ps->z[j] - ps->z[i];\n    if (ps->periodic) {\n        dx = min_image(dx, ps->box[0]);",
     "test_fixed_h_matches_numpy_brute_force"),
    ("pair: target mass",
     "a->sum_mw += ps->m[j] * w;",
     "a->sum_mw += ps->m[i] * w;",
     "test_adversarial_positions_on_cell_faces_and_box_edges"),
    ("pair: q = r2/h",
     "double q = r / h;\n        double w = ps->kernel",
     "double q = r2 / h;\n        double w = ps->kernel",
     "test_fixed_h_matches_numpy_brute_force"),
    ("pair: y image uses x box",
     "dy = min_image(dy, ps->box[1]);\n        dz = min_image(dz, ps->box[2]);\n    }\n    double r2",
     "dy = min_image(dy, ps->box[0]);\n        dz = min_image(dz, ps->box[2]);\n    }\n    double r2",
     "test_non_cubic_periodic_box_matches_brute_force"),
    ("finish: rho h^-2",
     "*rho = a->sum_mw * (8.0 / (pi * h * h * h));",
     "*rho = a->sum_mw * (8.0 / (pi * h * h));",
     "test_fixed_h_matches_numpy_brute_force"),
    ("finish: nw 16/3",
     "*nw = (32.0 / 3.0) * a->sum_w;",
     "*nw = (16.0 / 3.0) * a->sum_w;",
     "test_fixed_h_matches_numpy_brute_force"),
    ("finish: dnw no 1/h",
     "*dnw = (32.0 / 3.0) * a->sum_dw / h;",
     "*dnw = (32.0 / 3.0) * a->sum_dw;",
     "test_fixed_h_matches_numpy_brute_force"),
    ("finish: c6 rho 32 pi",
     "(1365.0 / (64.0 * pi * h * h * h))",
     "(1365.0 / (32.0 * pi * h * h * h))",
     "test_wendland_c6_matches_brute_force_and_finite_difference"),
    ("finish: c6 nw",
     "*nw = (1365.0 / 48.0) * a->sum_w;",
     "*nw = (1365.0 / 64.0) * a->sum_w;",
     "test_wendland_c6_matches_brute_force_and_finite_difference"),
    ("finish: c6 dnw",
     "*dnw = (1365.0 / 48.0) * a->sum_dw / h;",
     "*dnw = (1365.0 / 48.0) * a->sum_dw / (h * h);",
     "test_wendland_c6_matches_brute_force_and_finite_difference"),
    ("grid: half-width search",
     "int64_t a0 = (int64_t)floor((xi[d] - h - ps->origin[d]) / c);",
     "int64_t a0 = (int64_t)floor((xi[d] - 0.5 * h - ps->origin[d]) / c);",
     "test_fixed_h_matches_numpy_brute_force"),
    ("grid: open clamp drops last",
     "if (a1 > g - 1) a1 = g - 1;",
     "if (a1 > g - 2) a1 = g - 2;",
     "test_non_periodic_matches_brute_force"),
    ("solve: band strict",
     "if (fabs(nw - nngb) <= tol) {",
     "if (fabs(nw - nngb) < tol) {",
     "test_band_edges_are_inclusive"),
    ("solve: bracket swapped",
     "if (nw < nngb) *hlo = hc;\n    else *hhi = hc;",
     "if (nw < nngb) *hhi = hc;\n    else *hlo = hc;",
     "test_update_rule_along_trajectories"),
    ("solve: bracket not updated",
     "if (nw < nngb) *hlo = hc;\n    else *hhi = hc;",
     "",
     "test_single_particle_grows_until_box_limit"),
    ("solve: newton sign",
     "double hn = hc - (nw - nngb) / dnw;",
     "double hn = hc + (nw - nngb) / dnw;",
     "test_update_rule_along_trajectories"),
    ("solve: step limit 1/4",
     "hn >= 0.5 * hc && hn <= 2.0 * hc",
     "hn >= 0.25 * hc && hn <= 2.0 * hc",
     "test_update_rule_along_trajectories"),
    ("solve: step limit 4",
     "hn >= 0.5 * hc && hn <= 2.0 * hc",
     "hn >= 0.5 * hc && hn <= 4.0 * hc",
     "test_update_rule_along_trajectories"),
    ("solve: step limits open",
     "hn >= 0.5 * hc && hn <= 2.0 * hc",
     "hn > 0.5 * hc && hn < 2.0 * hc",
     "test_h_update_branches"),
    ("solve: no bracket test",
     "if (hn > *hlo && hn < *hhi && hn >= 0.5 * hc",
     "if (hn >= 0.5 * hc",
     "test_h_update_branches"),
    ("solve: bracket closed",
     "if (hn > *hlo && hn < *hhi && hn >= 0.5 * hc",
     "if (hn >= *hlo && hn <= *hhi && hn >= 0.5 * hc",
     "test_h_update_branches"),
    ("solve: bisection geometric",
     "return 0.5 * (*hlo + *hhi);",
     "return sqrt(*hlo * *hhi);",
     "test_h_update_branches"),
    ("solve: growth swapped",
     "if (has_lo) return hc * ORACLE_GROWTH;\n    return hc / ORACLE_GROWTH;",
     "if (has_lo) return hc / ORACLE_GROWTH;\n    return hc * ORACLE_GROWTH;",
     "test_single_particle_grows_until_box_limit"),
    ("solve: growth 1.25",
     "if (has_lo) return hc * ORACLE_GROWTH;",
     "if (has_lo) return hc * 1.25;",
     "test_single_particle_grows_until_box_limit"),
    ("solve: box limit >",
     "if (ps->periodic && hn >= half_box) {",
     "if (ps->periodic && hn > half_box) {",
     "test_a_proposal_of_half_the_box_stops_the_particle"),
    ("solve: box limit missing",
     "if (ps->periodic && hn >= half_box) {",
     "if (0) {",
     "test_single_particle_grows_until_box_limit"),
    ("solve: output next h",
     "h[t] = hn;\n            again[t] = 1;",
     "h[t] = hn;\n            h_inout[t] = hn;\n            again[t] = 1;",
     "test_update_rule_along_trajectories"),
    ("solve: todo loses order",
     "if (again[todo[k]]) todo[nn++] = todo[k];",
     "if (again[todo[ntodo - 1 - k]]) todo[nn++] = todo[ntodo - 1 - k];",
     "test_lattice_root_by_refined_solve"),
    ("solve: pair count not summed",
     "pairs += a.count;",
     "pairs += 0;",
     "test_update_rule_along_trajectories"),
    ("knn: K-th off by one",
     "h_out[t] = sqrt(r2[k - 1]);",
     "h_out[t] = sqrt(r2[k]);",
     "test_knn_lattice_shells_closed_form"),
    ("knn: self excluded",
     "qsort(r2, (size_t)n, sizeof(double), cmp_double);\n            h_out[t] = sqrt(r2[k - 1]);",
     "r2[i] = HUGE_VAL;\n            qsort(r2, (size_t)n, sizeof(double), cmp_double);\n            h_out[t] = sqrt(r2[k - 1]);",
     "test_knn_lattice_shells_closed_form"),
    ("knn: no min image",
     "dx = min_image(dx, ps.box[0]);",
     "dx = dx;",
     "test_knn_lattice_shells_closed_form"),
    ("knn: exceeds >",
     "if (h_out[t] >= half) status_out[t]",
     "if (h_out[t] > half) status_out[t]",
     "test_knn_exceeds_box_and_argument_range"),
    ("batch: group mass offset",
     "setup_pset(&ps, e - s, x + s, y + s, z + s, m + s, nobox, 0, kernel);",
     "setup_pset(&ps, e - s, x + s, y + s, z + s, m, nobox, 0, kernel);",
     "test_batch_equals_groups_solved_alone"),
    ("batch: passes summed",
     "if (gs.passes > st->passes) st->passes = gs.passes;",
     "st->passes += gs.passes;",
     "test_batch_equals_groups_solved_alone"),
    ("interact: gradient sign",
     "double wp = -(kernel ? oracle_mqdw_c6(q) : oracle_mqdw(q)) / q;",
     "double wp = (kernel ? oracle_mqdw_c6(q) : oracle_mqdw(q)) / q;",
     IP + "test_two_particles_closed_form"),
    ("interact: gradient h^-3",
     "double dWdr = sigma / (hi * hi * hi * hi) * wp;",
     "double dWdr = sigma / (hi * hi * hi) * wp;",
     IP + "test_linear_field_on_a_lattice"),
    ("interact: gradient not a unit vector",
     "gW[d] = dWdr * (L.e[k].d[d] / r);",
     "gW[d] = dWdr * L.e[k].d[d];",
     IP + "test_two_particles_closed_form"),
    ("interact: curl operands swapped",
     "const double u[3] = {-dvel[0], -dvel[1], -dvel[2]};",
     "const double u[3] = {dvel[0], dvel[1], dvel[2]};",
     IP + "test_linear_field_on_a_lattice"),
    ("interact: curl y component",
     "cv[1] += ps.m[j] * (u[2] * gW[0] - u[0] * gW[2]);",
     "cv[1] += ps.m[j] * (u[0] * gW[2] - u[2] * gW[0]);",
     IP + "test_two_particles_closed_form"),
    ("interact: dispersion about v_i",
     "e[d] = v[d][j] - vb[d];",
     "e[d] = v[d][j] - v[d][i];",
     IP + "test_two_particles_closed_form"),
    ("interact: mean not normalised",
     "for (int d = 0; d < 3; d++) vb[d] = vb[d] / rh;",
     "for (int d = 0; d < 3; d++) vb[d] = vb[d] / (rh * hi);",
     IP + "test_uniform_field_and_galilean_boost"),
    ("interact: divergence of v_i - v_j",
     "dv_sum += ps.m[j] * (dvel[0] * gW[0] + dvel[1] * gW[1] + dvel[2] * gW[2]);",
     "dv_sum -= ps.m[j] * (dvel[0] * gW[0] + dvel[1] * gW[1] + dvel[2] * gW[2]);",
     IP + "test_linear_field_on_a_lattice"),
    ("interact: target mass",
     "r_sum += ps.m[L.e[k].j] * W;",
     "r_sum += ps.m[i] * W;",
     IP + "test_matches_numpy_brute_force"),
    ("interact: self pair dropped",
     "    if (r2 < h2) {\n        const double d[3] = {-s[0], -s[1], -s[2]};",
     "    if (r2 < h2 && i != j) {\n        const double d[3] = {-s[0], -s[1], -s[2]};",
     IP + "test_matches_numpy_brute_force"),
    ("interact: z image uses y box",
     "s[k] = min_image(s[k], ps->box[k]);",
     "s[k] = min_image(s[k], ps->box[k > 1 ? 1 : k]);",
     IP + "test_matches_numpy_brute_force"),
]


def _copy(dst, source):
    os.makedirs(os.path.join(dst, "oracle"))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(dst, "oracle"))
    with open(os.path.join(dst, "oracle", "sph_oracle.c"), "w") as f:
        f.write(source)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "test_gpu_*", "test_zz_*"))
    os.symlink(os.path.join(ROOT, "paper_1612_06090_gb300"), os.path.join(dst, "paper_1612_06090_gb300"))


def _run_pins(cwd, pins):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [f"tests/{p}" if "::" in p else f"tests/test_oracle_pins.py::{p}" for p in pins]
    return subprocess.run(cmd, cwd=cwd, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.slow
def test_every_planted_mistake_fails_its_pin(tmp_path):
    with open(os.path.join(ROOT, "oracle", "sph_oracle.c")) as f:
        source = f.read()
    for name, old, new, _ in MUTANTS:
        assert source.count(old) == 1, f"{name}: the original text must occur exactly once"
    pins = sorted({pin for *_, pin in MUTANTS})
    control = str(tmp_path / "control")
    _copy(control, source)
    r = _run_pins(control, pins)
    assert r.returncode == 0, r.stdout[-2000:]

    def one(k):
        name, old, new, pin = MUTANTS[k]
        d = str(tmp_path / f"m{k:02d}")
        _copy(d, source.replace(old, new))
        return name, pin, _run_pins(d, [pin])

    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
        results = list(ex.map(one, range(len(MUTANTS))))
    # exit code 1: the pin ran and failed (not a collection or usage error)
    survivors = [(name, pin, r.returncode) for name, pin, r in results if r.returncode != 1]
    assert not survivors, survivors
