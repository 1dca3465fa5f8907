"""Mutation test of the oracle's pins: each plausible mistake (a dropped term, a
wrong sign or index, a transposed operand), planted in a copy of the C oracle on
the CPU, must make at least one pin fail."""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle_pins import PINS

# cheap pins first: a mutant stops at its first failing pin
ORDER = ["pin_ndc_worked_example", "pin_ndc_shorter_side_spans_unit_square",
         "pin_camera_distance", "pin_primary_ray", "pin_ray_sphere_closed_forms",
         "pin_ties_lowest_index", "pin_phong_closed_forms", "pin_single_sphere_lit_side", "pin_blinn_closed_form",
         "pin_plane_horizon", "pin_occlusion_invariant", "pin_philox_kat", "pin_rgba8",
         "pin_margin_grazing", "pin_margin_closest_terms", "pin_margin_shadow_terms", "pin_margin_light_gate",
         "pin_counters", "pin_area_samples_stratified", "pin_vogel_sunflower",
         "pin_reflection_mixing_closed_form", "pin_coupled_reflectivity",
         "pin_depth_reductions", "pin_area_light", "pin_mirror_symmetry",
         "pin_sky_invariants", "pin_sky_on_misses", "pin_verlet_free_fall", "pin_verlet_ground_contact",
         "pin_recursion_equals_loop", "pin_path_geometry_invariants", "pin_occlusion_brute_force",
         "pin_closest_hit_brute_force"]

MUTANTS = {
    "ndc_v_sign": ("*v = -(y / h * 2.0 - 1.0);", "*v = (y / h * 2.0 - 1.0);"),
    "ndc_swap_wh": ("*u = (x - w / 2.0 + h / 2.0) / h * 2.0 - 1.0;",
                    "*u = (x - h / 2.0 + w / 2.0) / h * 2.0 - 1.0;"),
    "cam_dist_full_angle": ("1.0 / tan(fov_rad / 2.0)", "1.0 / tan(fov_rad)"),
    "dir_c_minus_p": ("nrm(sub(P, C))", "nrm(sub(C, P))"),
    "pitch_sign": ("r.y * cp + r.z * sp", "r.y * cp - r.z * sp"),
    "yaw_transposed": ("r.x * cyw + r.z * syw", "r.x * cyw - r.z * syw"),
    "far_root_first": ("double tn = -b - s;", "double tn = -b + s;"),
    "tangent_miss": ("if (disc < 0.0) return 0;", "if (disc <= 0.0) return 0;"),
    "plane_sign": ("double tt = -(dot(o, n) + pd) / den;", "double tt = (dot(o, n) + pd) / den;"),
    "ties_last_index": ("&& t < tb) { tb = t; best = i; }", "&& t <= tb) { tb = t; best = i; }"),
    "shadow_ignores_distance": ("if (sphere_root(o, dir, s->g, s->r, &t) && t < dist) hit = 1;",
                                "if (sphere_root(o, dir, s->g, s->r, &t)) hit = 1;"),
    "no_ambient": ("double a = cx->ka, s = 0.0;", "double a = 0.0, s = 0.0;"),
    "reflect_light_half": ("v3 r = sub(scl(n, 2.0 * ndl), lh);", "v3 r = sub(scl(n, ndl), lh);"),
    "blinn_minus": ("v3 h = nrm(add(lh, view));", "v3 h = nrm(sub(lh, view));"),
    "no_ndl_gate": ("if (ndl <= 0.0) continue;", ""),
    "diffuse_ignores_shadow": ("a += L->I * vis * ndl;", "a += L->I * ndl;"),
    "spec_ignores_ks": ("s += L->I * vis * m->ks * sp;", "s += L->I * vis * sp;"),
    "face_forward_flipped": ("if (dot(*n, d) > 0.0) *n = scl(*n, -1.0);",
                             "if (dot(*n, d) < 0.0) *n = scl(*n, -1.0);"),
    "mix_ratio_swapped": ("col[c] = m->alb[c] * (1.0 - m->rho) + rc[c] * m->rho;",
                          "col[c] = m->alb[c] * m->rho + rc[c] * (1.0 - m->rho);"),
    "mix_unshaded_reflection": ("for (int c = 0; c < 3; ++c) out[c] = col[c] * A + S;",
                                "for (int c = 0; c < 3; ++c) out[c] = (depth ? m->alb[c] * (1.0 - m->rho) * A + S + (col[c] - m->alb[c] * (1.0 - m->rho)) : col[c] * A + S);"),
    "throughput_no_A": ("T *= m->rho * A;", "T *= m->rho;"),
    "depth_off_by_one": ("if (depth == 0) {", "if (depth <= 1) {"),
    "reflect_sign": ("v3 rd = sub(d, scl(n, 2.0 * dot(d, n)));", "v3 rd = add(d, scl(n, 2.0 * dot(d, n)));"),
    "philox_key_bump": ("k0 += W0; k1 += W1;", "k0 += W1; k1 += W0;"),
    "philox_word_swap": ("uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c3 ^ k0;"),
    "u01_bits": ("(double)(w >> 8) * (1.0 / 16777216.0)", "(double)(w >> 9) * (1.0 / 16777216.0)"),
    "area_offset": ("((i + xi1) / g - 0.5) * L->area", "((i + xi1) / g) * L->area"),
    "area_strata_transposed": ("int i = s % g, j = s / g;", "int i = s / g, j = s % g;"),
    "rgba_truncate": ("floorf(v * 255.0f + 0.5f)", "floorf(v * 255.0f)"),
    "rgba_channel_order": ("px |= q << (8 * c);", "px |= q << (8 * (2 - c));"),
    "no_eps_offset": ("v3 po = add(p, scl(n, cx->eps));", "v3 po = p;"),
    "vogel_double_radius": ("double r = L->srad * sqrt((double)i / (double)n);",
                            "double r = 2.0 * L->srad * sqrt((double)i / (double)n);"),
    "vogel_angle": ("double phi = M_PI * (3.0 - sqrt(5.0));", "double phi = M_PI * (3.0 - sqrt(3.0));"),
    "coupled_uncapped": ("p->rho = fmin(p->ex / in->max_reflectivity, 1.0);", "p->rho = p->ex / in->max_reflectivity;"),
    "sky_u_sign": ("const double u = 0.5 + atan2(d.z, d.x) / (2.0 * M_PI);",
                   "const double u = 0.5 + atan2(-d.z, d.x) / (2.0 * M_PI);"),
    "sky_u_full_turn_half": ("const double u = 0.5 + atan2(d.z, d.x) / (2.0 * M_PI);",
                             "const double u = 0.5 + atan2(d.z, d.x) / M_PI;"),
    "sky_no_half_texel": ("const double x = u * W - 0.5, y = v * H - 0.5;",
                          "const double x = u * W, y = v * H - 0.5;"),
    "sky_v_flipped": ("const double v = 0.5 - asin(dy) / M_PI;", "const double v = 0.5 + asin(dy) / M_PI;"),
    "sky_u_clamped": ("const int i1 = (i0 + 1) % W;", "const int i1 = i0 + 1 < W ? i0 + 1 : W - 1;"),
    "sky_lerp_swapped": ("out[c] = (1.0 - fy) * top + fy * bot;", "out[c] = fy * top + (1.0 - fy) * bot;"),
    "miss_black_forward": ("for (int c = 0; c < 3; ++c) out[c] += T * sk[c];", ""),
    "miss_black_recursive": ("if (id < 0) { miss_color(cx, d, out); return; }",
                             "if (id < 0) { out[0] = out[1] = out[2] = 0.0; return; }"),
    "verlet_no_inertia": ("v3 xn = add(add(x, sub(x, xp)), V(0.0, -gdt2, 0.0));", "v3 xn = add(x, V(0.0, -gdt2, 0.0));"),
    "verlet_half_gravity": ("const double gdt2 = g * dt * dt;", "const double gdt2 = 0.5 * g * dt * dt;"),
    "verlet_restitution_ignored": ("(1.0 + e) * vn", "2.0 * vn"),
    "verlet_no_pushout": ("xn = sub(xn, scl(nn, sd));", ""),
    "verlet_no_rest_contact": ("-vn <= 2.0 * gdt2 ? vn : (1.0 + e) * vn", "(1.0 + e) * vn"),
    "verlet_prev_not_reset": ("xq = sub(xn, v);", "xq = x;"),
    "sphere_normal_over_radius": ("*n = nrm(sub(*p, cx->prim[id].g));",
                                  "*n = scl(sub(*p, cx->prim[id].g), 1.0 / cx->prim[id].r);"),
    # margins (the exemption from the colour tolerance is decided by them)
    "margin_gap_dropped": ("if (best >= 0 && t2 < INFINITY) m = fmin(m, t2 - tb);", ""),
    "margin_plane_gap_dropped": ("if (best != cx->ns && tp > 0.0) t2 = fmin(t2, tp);", ""),
    "margin_horizon_dropped": ("if (best == cx->ns || best < 0) m = fmin(m, fabs(den) * cx->S);", ""),
    "margin_horizon_unscaled": ("m = fmin(m, fabs(den) * cx->S);", "m = fmin(m, fabs(den));"),
    "margin_horizon_only_on_plane_hits": ("if (best == cx->ns || best < 0) m", "if (best == cx->ns) m"),
    "margin_closest_plane_root_dropped": ("if (P->origin != cx->ns) m = fmin(m, fabs(tp));\n            if (best",
                                          "if (best"),
    "margin_closest_roots_dropped": ("m = fmin(m, fabs(tca - sq));\n            m = fmin(m, fabs(tca + sq));", ""),
    "margin_closest_origin_not_skipped": ("if (disc >= 0.0 && i != P->origin) {", "if (disc >= 0.0) {"),
    "margin_silhouette_behind_hit": ("(best < 0 || tca - s->r < tb)", "(1)"),
    "margin_silhouette_behind_origin": ("if (tca + s->r > 0.0 && ", "if ("),
    "margin_shadow_endpoints_dropped": ("m = fmin(m, fabs(r1 - dist));\n                m = fmin(m, fabs(r2 - dist));",
                                        ""),
    "margin_shadow_far_endpoint_dropped": ("m = fmin(m, fabs(r2 - dist));", ""),
    "margin_shadow_origin_roots_dropped": ("if (i != P->origin) m = fmin(m, fmin(fabs(r1), fabs(r2)));", ""),
    "margin_shadow_origin_not_skipped": ("if (i != P->origin) m = fmin(m, fmin(fabs(r1), fabs(r2)));",
                                         "m = fmin(m, fmin(fabs(r1), fabs(r2)));"),
    "margin_shadow_silhouette_dropped": ("if (tca >= 0.0 && tca <= dist) m = fmin(m, fabs(ld - s->r));", ""),
    "margin_shadow_silhouette_beyond_light": ("if (tca >= 0.0 && tca <= dist)", "if (tca >= 0.0)"),
    "margin_shadow_plane_endpoint_dropped": ("m = fmin(m, fabs(tp - dist));", ""),
    "margin_shadow_plane_origin_dropped": (
        "m = fmin(m, fabs(tp - dist));\n                if (P->origin != cx->ns) m = fmin(m, fabs(tp));",
        "m = fmin(m, fabs(tp - dist));"),
    "margin_light_gate_dropped": ("if (P->want_margin) P->margin = fmin(P->margin, fabs(ndl) * cx->S);", ""),
    "margin_light_gate_unscaled": ("fabs(ndl) * cx->S", "fabs(ndl)"),
}


@pytest.fixture(scope="module")
def src():
    with open(oracle.oracle.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(src, name, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    path = tmp_path / "rt_oracle.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                    "-fvisibility=hidden", "-ffp-contract=off", "-o", str(so), str(path), "-lm"],
                   check=True)
    caught = None
    with oracle.using_library(str(so)):
        for pin in ORDER:
            try:
                PINS[pin](oracle)
            except (AssertionError, ValueError, TypeError, ZeroDivisionError, IndexError):
                caught = pin
                break
    assert caught, f"mutant {name} survived every pin"


def test_every_pin_is_ordered():
    assert sorted(ORDER) == sorted(PINS)
