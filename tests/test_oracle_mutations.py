"""Plant one plausible mistake at a time in a private copy of the oracle
source, compile it, and check that at least one pin catches it (CPU only)."""
import os

import pytest

import oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pba_oracle.c")

MUTATIONS = {
    "rotation_jacobian_skew_sign": ("acc += M[3 * r + k] * (-2.0 * Spu[3 * k + c]);",
                                    "acc += M[3 * r + k] * (2.0 * Spu[3 * k + c]);"),
    "target_translation_jacobian_sign": ("dPj[6 * r + c] = -RoT[3 * r + c];", "dPj[6 * r + c] = RoT[3 * r + c];"),
    "normal_cue_uses_Rj_not_RjT": ("mat3_vec(RjT, Rn, RjTRn);", "mat3_vec(Rj, Rn, RjTRn);"),
    "image_gradient_axes_swapped": ("gu[ci] += w[t] * 0.5 * (tval(prm, Ir, ci) - tval(prm, Il, ci));",
                                    "gu[ci] += w[t] * 0.5 * (tval(prm, Id, ci) - tval(prm, Iu, ci));"),
    "huber_weight_dropped": ("*w = prm->huber_delta / chi;", "*w = 1.0;"),
    "omega_dropped_from_b": ("s_b += J[r][a] * om[r] * e[r];", "s_b += J[r][a] * e[r];"),
    "depth_cue_jacobian_dropped": ("map_i += dz[k] * dPi[6 * k + col];", "map_i += 0.0 * dPi[6 * k + col];"),
    "cholesky_off_by_one": ("for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];",
                            "for (int k = 1; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];"),
    "spherical_jacobian_transposed": ("for (int k = 0; k < 3; ++k) acc += K12[3 * r + k] * D[3 * k + c];",
                                      "for (int k = 0; k < 3; ++k) acc += K12[3 * r + k] * D[3 * c + k];"),
    "boxplus_translation_not_rotated": ("mat3_vec(R, dx, Rdt);", "Rdt[0] = dx[0]; Rdt[1] = dx[1]; Rdt[2] = dx[2];"),
    "pinhole_principal_point_swapped": ("double vy = s->fy * p[1] + s->cy * p[2];\n        double vz = p[2];\n        uv[0]",
                                        "double vy = s->fy * p[1] + s->cx * p[2];\n        double vz = p[2];\n        uv[0]"),
    "assembly_block_transposed": ("+= H12[12 * (6 * ba + a) + 6 * bb + c];", "+= H12[12 * (6 * bb + a) + 6 * ba + c];"),
    "offset_rotation_not_transposed": ("mat3_vec(RoT, tmp, pb);", "mat3_vec(Ro, tmp, pb);"),
    "offset_translation_sign": ("for (int a = 0; a < 3; ++a) tmp[a] = q[a] - to[a];",
                                "for (int a = 0; a < 3; ++a) tmp[a] = q[a] + to[a];"),
    "bilinear_weight_swapped": ("const double w[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};",
                                "const double w[4] = {(1 - a) * (1 - b), (1 - a) * b, a * (1 - b), a * b};"),
    "offset_map_translation_factor": ("A[6 * r + 3 + c] = 2.0 * x[r];", "A[6 * r + 3 + c] = x[r];"),
    "offset_jacobian_drops_target": ("s += (Ji[6 * r + k] + Jj[6 * r + k]) * A[6 * k + c];",
                                     "s += Ji[6 * r + k] * A[6 * k + c];"),
    "offset_map_rotation_transposed": ("A[6 * r + c] = Ro[3 * r + c];", "A[6 * r + c] = Ro[3 * c + r];"),
    "huber_rho_constant_sign": ("*rho = 2.0 * prm->huber_delta * chi - prm->huber_delta * prm->huber_delta;",
                                "*rho = 2.0 * prm->huber_delta * chi + prm->huber_delta * prm->huber_delta;"),
    "occlusion_relative_term_dropped": ("double thr = prm->occ_abs + prm->occ_rel * zd;", "double thr = prm->occ_abs;"),
    "target_normal_threshold_squared": ("if (nt < 0.5 && ", "if (nt < 0.25 && "),
    "z_min_ignored": ("if (!(zd > prm->z_min) && ", "if (!(zd > 0.0) && "),
    "stencil_corner_for_edge_texel": ("{1, -1}, {1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 1}};",
                                      "{1, -1}, {1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 2}};"),
    "pinhole_window_one_column_short": ("u >= 1.0 && u < (double)(s->width - 2)", "u >= 1.0 && u < (double)(s->width - 3)"),
    "boxplus_large_step_not_normalised": ("qw = 1.0 / n; qx /= n; qy /= n; qz /= n;", "qw = 0.0;"),
    "omega_dropped_from_H": ("for (int r = 0; r < 5; ++r) s_h += J[r][a] * om[r] * J[r][c];",
                             "for (int r = 0; r < 5; ++r) s_h += J[r][a] * J[r][c];"),
    "huber_weight_dropped_from_H": ("H12[12 * a + c] += w * s_h;", "H12[12 * a + c] += s_h;"),
    "huber_weight_squared_in_H": ("H12[12 * a + c] += w * s_h;", "H12[12 * a + c] += w * w * s_h;"),
    "H_block_rows_and_columns_mixed": ("s_h += J[r][a] * om[r] * J[r][c];", "s_h += J[r][a] * om[r] * J[r][11 - c];"),
    "half_rounding_truncates": ("double r = ldexp(nearbyint(ldexp(v, -q)), q);", "double r = ldexp(trunc(ldexp(v, -q)), q);"),
    "half_ten_significant_bits": ("int q = e - 11;", "int q = e - 10;"),
    "half_subnormal_spacing": ("if (q < -24) q = -24;", "if (q < -25) q = -25;"),
    "half_texels_ignored": ("return (prm->texel_f16 && ci != 1) ? o_half(I[ci]) : (double)I[ci];",
                            "return (double)I[ci];"),
    "half_texel_depth_rounded": ("return (prm->texel_f16 && ci != 1) ? o_half(I[ci]) : (double)I[ci];",
                                 "return prm->texel_f16 ? o_half(I[ci]) : (double)I[ci];"),
    "range_cue_horizontal_only": ("zd = sqrt(pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2]);",
                                  "zd = sqrt(pb[0] * pb[0] + pb[1] * pb[1]);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, oracle_lib, room3, street3):
    before, after = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "pba_oracle_mutated.c"
    mutated.write_text(src.replace(before, after))
    lib = oracle_lib.load(oracle_lib.build(force=True, src=str(mutated), out=str(tmp_path / "libmut.so")))
    failed = []
    for pin, fn in [("projection_golden", lambda: P.pin_projection_golden(oracle_lib, lib)),
                    ("roundtrip", lambda: P.pin_roundtrip(oracle_lib, lib)),
                    ("proj_jacobian_fd", lambda: P.pin_proj_jacobian_fd(oracle_lib, lib)),
                    ("boxplus", lambda: P.pin_boxplus(oracle_lib, lib)),
                    ("jacobian_fd_pinhole", lambda: P.pin_jacobian_fd(oracle_lib, lib, room3)),
                    ("jacobian_fd_spherical", lambda: P.pin_jacobian_fd(oracle_lib, lib, street3)),
                    ("ramp_grad_mode0", lambda: P.pin_ramp_grad_mode0(oracle_lib, lib)),
                    ("gauge", lambda: max(P.pin_gauge(oracle_lib, lib, room3), P.pin_gauge(oracle_lib, lib, street3))),
                    ("cost_gradient", lambda: P.pin_cost_gradient(oracle_lib, lib, room3)),
                    ("plane_shift", lambda: P.pin_plane_shift(oracle_lib, lib)),
                    ("single_channel", lambda: P.pin_single_channel(oracle_lib, lib)),
                    ("cholesky", lambda: P.pin_cholesky(oracle_lib, lib)),
                    ("extrinsic_equivalence", lambda: P.pin_extrinsic_equivalence(oracle_lib, lib, room3)),
                    ("jacobian_fd_extrinsic", lambda: P.pin_jacobian_fd_extrinsic(oracle_lib, lib, room3)),
                    ("offset_jacobian_fd", lambda: P.pin_offset_jacobian_fd(oracle_lib, lib, room3)),
                    ("offset_gradient_fd", lambda: P.pin_offset_gradient_fd(oracle_lib, lib, room3)),
                    ("residual_brute_force", lambda: P.pin_residual_brute_force(oracle_lib, lib, room3, street3)),
                    ("relative_jacobian", lambda: max(P.pin_relative_jacobian(oracle_lib, lib, room3),
                                                      P.pin_relative_jacobian(oracle_lib, lib, street3))),
                    ("hessian_zero_residual", lambda: P.pin_hessian_zero_residual(oracle_lib, lib)),
                    ("half_rounding", lambda: P.pin_half_rounding(oracle_lib, lib)),
                    ("huber_hessian", lambda: max(P.pin_huber_hessian(oracle_lib, lib, room3),
                                                  P.pin_huber_hessian(oracle_lib, lib, street3)))]:
        try:
            err = fn()
        except (AssertionError, ValueError, ArithmeticError, Exception):
            failed.append(pin)
            continue
        if not err < P.PIN_TOL[pin]:
            failed.append(pin)
        if failed:
            break
    assert failed, f"no pin caught the planted mistake {name}"


# Planted mistakes in the oracle's normal estimation (Python, Sec. IV-A).
PY_SRC = os.path.join(os.path.dirname(SRC), "__init__.py")

NORMAL_MUTATIONS = {
    "mean_not_subtracted": ("cov = S2 / Nn[..., None] - mean[..., :, None] * mean[..., None, :]",
                            "cov = S2 / Nn[..., None]"),
    "largest_eigenvector": ("n = evec[:, :, 0].reshape(H, W, 3)", "n = evec[:, :, 2].reshape(H, W, 3)"),
    "oriented_away_from_observer": ("n = np.where((nP > 0)[..., None], -n, n)",
                                    "n = np.where((nP < 0)[..., None], -n, n)"),
    "columns_not_wrapped": ("cols = cols % W", "cols = cols"),
    "radius_grows_with_range": ("np.clip(scale / np.where(valid, d, 1.0)", "np.clip(scale * np.where(valid, d, 1.0)"),
    "radius_inclusive": ("(dd2 < rad * rad) & valid[rr, cc]", "(dd2 <= rad * rad) & valid[rr, cc]"),
    "invalid_neighbours_used": ("(dd2 < rad * rad) & valid[rr, cc]", "(dd2 < rad * rad)"),
    "collinear_points_kept": ("(ev[..., 1] > collinear * ev[..., 2])", "(ev[..., 2] > 0)"),
    "min_count_ignored": ("ok = valid & (N >= min_count)", "ok = valid & (N >= 1)"),
}


@pytest.mark.parametrize("name", sorted(NORMAL_MUTATIONS))
def test_planted_normal_mistake_is_caught(name, oracle_lib, room3, street3):
    import types
    before, after = NORMAL_MUTATIONS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle_mutated")
    mod.__file__ = PY_SRC
    exec(compile(src.replace(before, after), PY_SRC, "exec"), mod.__dict__)
    lib = oracle_lib.load()
    failed = []
    for pin, fn in [("normals_plane", lambda: P.pin_normals_plane(mod, lib)),
                    ("normals_counts", lambda: P.pin_normals_counts(mod, lib)),
                    ("normals_degenerate", lambda: P.pin_normals_degenerate(mod, lib)),
                    ("normals_brute_force", lambda: max(P.pin_normals_brute_force(mod, lib, room3),
                                                        P.pin_normals_brute_force(mod, lib, street3)))]:
        try:
            err = fn()
        except Exception:
            failed.append(pin)
            break
        if not err < P.PIN_TOL[pin]:
            failed.append(pin)
            break
    assert failed, f"no pin caught the planted mistake {name}"


PYRAMID_MUTATIONS = {
    "principal_point_halved": ("cx=(float(g(\"cx\")) + 0.5) / 2.0 - 0.5", "cx=float(g(\"cx\")) / 2.0"),
    "block_sum_not_averaged": ("out[..., 0] = s[..., 0] * 0.25", "out[..., 0] = s[..., 0] * 0.5"),
    "depth_sum_not_averaged": ("out[..., 1] = s[..., 1] * 0.25", "out[..., 1] = s[..., 1] * 0.3"),
    "normals_not_normalised": ("out[..., 2 + k] = s[..., 2 + k] / np.where(norm > 0, norm, 1.0)",
                               "out[..., 2 + k] = s[..., 2 + k] * 0.25"),
    "any_valid_instead_of_all": ("vb = valid.reshape(H, 2, W, 2).all(axis=(1, 3))",
                                 "vb = valid.reshape(H, 2, W, 2).any(axis=(1, 3))"),
    "fine_to_coarse_order": ("for li in range(n_levels - 1, -1, -1):", "for li in range(n_levels):"),
}


@pytest.mark.parametrize("name", sorted(PYRAMID_MUTATIONS))
def test_planted_pyramid_mistake_is_caught(name, oracle_lib):
    import types
    before, after = PYRAMID_MUTATIONS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle_mutated")
    mod.__file__ = PY_SRC
    exec(compile(src.replace(before, after), PY_SRC, "exec"), mod.__dict__)
    lib = oracle_lib.load()
    failed = []
    for pin, fn in [("pyramid_projection", lambda: P.pin_pyramid_projection(mod, lib)),
                    ("downsample_closed_forms", lambda: P.pin_downsample_closed_forms(mod, lib)),
                    ("coarse_to_fine", lambda: P.pin_coarse_to_fine(mod, lib))]:
        try:
            err = fn()
        except Exception:
            failed.append(pin)
            break
        if not err < P.PIN_TOL[pin]:
            failed.append(pin)
            break
    assert failed, f"no pin caught the planted mistake {name}"


VARIABLE_MUTATIONS = {
    "first_variable_dropped": ("        if v >= 0:\n            S[6 * k", "        if v > 0:\n            S[6 * k"),
    "reduced_gradient_halved": ("    br = S.T @ np.asarray(b, dtype=np.float64)\n", "    br = 0.5 * S.T @ np.asarray(b, dtype=np.float64)\n"),
    "reduced_matrix_not_projected": ("    Hr = S.T @ np.asarray(H, dtype=np.float64) @ S\n    br",
                                     "    Hr = S.T @ np.asarray(H, dtype=np.float64) @ S * 2.0\n    br"),
}


@pytest.mark.parametrize("name", sorted(VARIABLE_MUTATIONS))
def test_planted_variable_mistake_is_caught(name, oracle_lib, room3, fusion):
    import types
    before, after = VARIABLE_MUTATIONS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle_mutated")
    mod.__file__ = PY_SRC
    exec(compile(src.replace(before, after), PY_SRC, "exec"), mod.__dict__)
    lib = oracle_lib.load()
    failed = []
    for pin, fn in [("variables_reduce_to_gauge", lambda: P.pin_variables_reduce_to_gauge(mod, lib, room3)),
                    ("tied_gradient", lambda: P.pin_tied_gradient(mod, lib, fusion))]:
        try:
            err = fn()
        except Exception:
            failed.append(pin)
            break
        if not err < P.PIN_TOL[pin]:
            failed.append(pin)
            break
    assert failed, f"no pin caught the planted mistake {name}"


GRAPH_MUTATIONS = {
    "angle_uses_R_i_R_j": ("np.trace(Ri.T @ Rj)", "np.trace(Ri @ Rj)"),
    "distance_from_a_rotation_column": ("np.linalg.norm(poses[i][:, 3] - poses[j][:, 3])",
                                        "np.linalg.norm(poses[i][:, 2] - poses[j][:, 2])"),
    "criteria_joined_by_or": ("(ang < max_angle and dist < max_dist) or is_seq",
                              "(ang < max_angle or dist < max_dist) or is_seq"),
    "ratio_over_pixels_not_points": ('ratio = r["count"] / r["n_points"] if r["n_points"] else 0.0',
                                     'ratio = r["count"] / channels[i][..., 0].size if r["n_points"] else 0.0'),
    "sequential_edges_ignored": ("is_seq = sequential and j == i + 1", "is_seq = False"),
}


@pytest.mark.parametrize("name", sorted(GRAPH_MUTATIONS))
def test_planted_graph_mistake_is_caught(name, oracle_lib, room8):
    import types
    before, after = GRAPH_MUTATIONS[name]
    src = open(PY_SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle_mutated")
    mod.__file__ = PY_SRC
    exec(compile(src.replace(before, after), PY_SRC, "exec"), mod.__dict__)
    try:
        err = P.pin_build_pairs(mod, oracle_lib.load(), room8)
    except Exception:
        return
    assert not err < P.PIN_TOL["build_pairs"], f"no pin caught the planted mistake {name}"
