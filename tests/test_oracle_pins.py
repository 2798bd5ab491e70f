"""The FP64 oracle against closed forms, library routines, finite differences
and invariants of the formulation (CPU only)."""
import numpy as np
import pytest

import oracle_pins as P


def test_projection_closed_form(oracle_lib):
    assert P.pin_projection_golden(oracle_lib, oracle_lib.load()) < P.PIN_TOL["projection_golden"]


def test_unproject_project_roundtrip(oracle_lib):
    assert P.pin_roundtrip(oracle_lib, oracle_lib.load()) < P.PIN_TOL["roundtrip"]


def test_projection_jacobian_fd(oracle_lib):
    assert P.pin_proj_jacobian_fd(oracle_lib, oracle_lib.load()) < P.PIN_TOL["proj_jacobian_fd"]


def test_boxplus_is_right_multiplication_by_exp(oracle_lib):
    assert P.pin_boxplus(oracle_lib, oracle_lib.load()) < P.PIN_TOL["boxplus"]


def test_point_jacobians_fd_pinhole(oracle_lib, room3):
    assert P.pin_jacobian_fd(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["jacobian_fd_pinhole"]


def test_point_jacobians_fd_spherical(oracle_lib, street3):
    assert P.pin_jacobian_fd(oracle_lib, oracle_lib.load(), street3) < P.PIN_TOL["jacobian_fd_spherical"]


def test_paper_image_jacobians_exact_on_ramps(oracle_lib):
    assert P.pin_ramp_grad_mode0(oracle_lib, oracle_lib.load()) < P.PIN_TOL["ramp_grad_mode0"]


@pytest.mark.parametrize("which", ["room3", "street3"])
def test_gauge_null_space(oracle_lib, which, request):
    w = request.getfixturevalue(which)
    assert P.pin_gauge(oracle_lib, oracle_lib.load(), w) < P.PIN_TOL["gauge"]


def test_cost_gradient_is_twice_b(oracle_lib, room3):
    assert P.pin_cost_gradient(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["cost_gradient"]


def test_integer_shift_of_plane_gives_zero_error(oracle_lib):
    assert P.pin_plane_shift(oracle_lib, oracle_lib.load()) < P.PIN_TOL["plane_shift"]


def test_single_channel_reduces_to_classic_photometric_error(oracle_lib):
    assert P.pin_single_channel(oracle_lib, oracle_lib.load()) < P.PIN_TOL["single_channel"]


def test_extrinsic_offset_equals_composed_sensor_poses(oracle_lib, room3):
    assert P.pin_extrinsic_equivalence(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["extrinsic_equivalence"]


def test_point_jacobians_fd_with_extrinsic_offset(oracle_lib, room3):
    assert P.pin_jacobian_fd_extrinsic(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["jacobian_fd_extrinsic"]


def test_gauge_null_space_with_extrinsic_offset(oracle_lib, room3):
    from paper_2303_16878_gb300 import synth
    wx = synth.with_extrinsic(room3, synth.offset_transform(0.3, 20.0, seed=9))
    assert P.pin_gauge(oracle_lib, oracle_lib.load(), wx) < P.PIN_TOL["gauge"]


def test_pose_angle_is_the_rotation_magnitude(oracle_lib):
    """Graph construction's first criterion (Sec. IV-B): the angle between two
    poses, against scipy's rotation-vector magnitude of R_i^T R_j."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(21)
    for _ in range(50):
        Xi, Xj = np.zeros((3, 4)), np.zeros((3, 4))
        Xi[:, :3] = Rotation.from_rotvec(rng.normal(0, 1, 3)).as_matrix()
        Xj[:, :3] = Rotation.from_rotvec(rng.normal(0, 1, 3)).as_matrix()
        ref = Rotation.from_matrix(Xi[:, :3].T @ Xj[:, :3]).magnitude()
        assert abs(oracle_lib.pose_angle(Xi, Xj) - ref) < 1e-7


def test_build_pairs_keeps_ratio_above_threshold(oracle_lib, room8):
    """The pair criterion uses the count of valid residuals (pinned above)
    over the source's points; sequential edges are kept regardless."""
    r = oracle_lib.build_pairs(room8.sensors, room8.frame_sensor, room8.channels, room8.poses_init, room8.params,
                               np.radians(60), 2.0, 0.5, sequential=True)
    kept = {tuple(p) for p in r["pairs"].tolist()}
    for (i, j), c in r["candidates"].items():
        assert ((i, j) in kept) == (c["ratio"] > 0.5 or c["sequential"])
        assert c["count"] <= c["n_points"]
    assert all((i, i + 1) in kept for i in range(room8.n_frames - 1))


def test_cholesky_matches_numpy_solve(oracle_lib):
    assert P.pin_cholesky(oracle_lib, oracle_lib.load()) < P.PIN_TOL["cholesky"]


def test_system_symmetric_psd_rank(oracle_lib, room8):
    r = oracle_lib.linearize(room8.sensors, room8.frame_sensor, room8.channels, room8.poses_init,
                             room8.pairs, room8.params)
    H = r["H"]
    assert np.array_equal(H, H.T)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] >= -1e-12 * ev[-1]
    assert np.count_nonzero(ev > 1e-9 * ev[-1]) == H.shape[0] - 6


def test_self_pair_has_zero_error(oracle_lib, room3):
    """Frame i against itself at the same pose: pbar = p_u and u' = u."""
    s = room3.sensors[0]
    pr = oracle_lib.linearize_pair(s, room3.params, room3.channels[0], room3.channels[0],
                                   room3.poses_gt[0], room3.poses_gt[0])
    assert pr["count"] > 0.9 * pr["n_points"]
    assert pr["cost"] < 1e-18
    assert np.abs(pr["b"]).max() < 1e-9


def test_solve_step_fixes_gauge_and_solves_damped_system(oracle_lib, room8):
    r = oracle_lib.linearize(room8.sensors, room8.frame_sensor, room8.channels, room8.poses_init,
                             room8.pairs, room8.params)
    lam = oracle_lib.initial_lambda(r["H"])
    dx, ok = oracle_lib.solve_step(r["H"], r["b"], lam)
    assert ok
    assert np.all(dx[:6] == 0)
    A = r["H"][6:, 6:] + lam * np.eye(r["H"].shape[0] - 6)
    np.testing.assert_allclose(A @ dx[6:], -r["b"][6:], rtol=0, atol=1e-9 * np.abs(r["b"]).max())


def test_lm_converges_towards_ground_truth(oracle_lib):
    """RGB-D room at 80x60, 4 frames, 2 cm / 1 deg init noise: every accepted
    step lowers F, and the poses approach ground truth to the accuracy that
    bilinear interpolation of the renders allows."""
    from conftest import workload
    w = workload("room", n_frames=4, width=80, height=60, f=60.0)
    poses, lam = w.poses_init.copy(), None
    costs = []
    for _ in range(12):
        o = oracle_lib.lm_iteration(w, poses, lam)
        if o["accepted"]:
            assert o["new_cost"] < o["cost"]
        poses, lam = o["poses"], o["lam"]
        costs.append(o["cost"])
    t_err0 = max(np.linalg.norm(w.poses_init[k][:, 3] - w.poses_gt[k][:, 3]) for k in range(4))
    r_err0 = max(np.linalg.norm(w.poses_init[k][:, :3].T @ w.poses_gt[k][:, :3] - np.eye(3)) for k in range(4))
    t_err = max(np.linalg.norm(poses[k][:, 3] - w.poses_gt[k][:, 3]) for k in range(4))
    r_err = max(np.linalg.norm(poses[k][:, :3].T @ w.poses_gt[k][:, :3] - np.eye(3)) for k in range(4))
    assert costs[-1] < 0.1 * costs[0]
    # at 80x60 (1 deg pixels) interpolation bias keeps the minimum ~1 cm / ~0.3 deg off ground truth
    assert t_err < 0.25 * t_err0 and t_err < 0.012
    assert r_err < 0.15 * r_err0


def test_normals_of_a_plane_are_its_normal(oracle_lib):
    assert P.pin_normals_plane(oracle_lib, oracle_lib.load()) < P.PIN_TOL["normals_plane"]


def test_normal_neighbourhood_sizes_match_lattice_counts(oracle_lib):
    assert P.pin_normals_counts(oracle_lib, oracle_lib.load()) < P.PIN_TOL["normals_counts"]


@pytest.mark.parametrize("which", ["room3", "street3"])
def test_normals_match_brute_force_plane_fit(oracle_lib, which, request):
    w = request.getfixturevalue(which)
    assert P.pin_normals_brute_force(oracle_lib, oracle_lib.load(), w) < P.PIN_TOL["normals_brute_force"]


def test_no_normal_where_the_plane_is_undetermined(oracle_lib):
    assert P.pin_normals_degenerate(oracle_lib, oracle_lib.load()) < P.PIN_TOL["normals_degenerate"]


def test_coarse_level_projection_is_the_halved_pixel_grid(oracle_lib):
    assert P.pin_pyramid_projection(oracle_lib, oracle_lib.load()) < P.PIN_TOL["pyramid_projection"]


def test_downsample_closed_forms(oracle_lib):
    assert P.pin_downsample_closed_forms(oracle_lib, oracle_lib.load()) < P.PIN_TOL["downsample_closed_forms"]


def test_coarse_to_fine_converges_on_a_tiny_room(oracle_lib):
    assert P.pin_coarse_to_fine(oracle_lib, oracle_lib.load()) < P.PIN_TOL["coarse_to_fine"]


def test_tied_frames_gradient_matches_finite_differences(oracle_lib, fusion):
    assert P.pin_tied_gradient(oracle_lib, oracle_lib.load(), fusion) < P.PIN_TOL["tied_gradient"]


def test_default_variables_reduce_to_the_gauge_fixed_step(oracle_lib, room3):
    assert P.pin_variables_reduce_to_gauge(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["variables_reduce_to_gauge"]


def test_other_branch_only_touches_flagged_rejections(oracle_lib, street3):
    """The other-branch evaluation (used to account for points a float32
    implementation decides the other way) leaves every valid point unchanged
    and validates only points whose decision lies within its margin."""
    w = street3
    s = w.sensors[0]
    lib = oracle_lib.load()
    forced = 0
    for i, j in ((0, 1), (0, 2), (1, 2)):
        pts, _ = oracle_lib.frame_points(s, w.params, w.channels[i], lib=lib)
        for k in range(len(pts)):
            a = oracle_lib.point_residual(s, w.params, w.channels[j], w.poses_init[i], w.poses_init[j], pts[k],
                                          lib=lib)
            b = oracle_lib.point_residual(s, w.params, w.channels[j], w.poses_init[i], w.poses_init[j], pts[k],
                                          lib=lib, other_branch=True)
            if a["valid"]:
                assert b["valid"] and np.array_equal(a["e"], b["e"]) and np.array_equal(a["Ji"], b["Ji"])
            elif b["valid"]:
                assert a["flag"]
                forced += 1
    assert forced > 0


def test_offset_jacobian_matches_finite_differences(oracle_lib, room3):
    assert P.pin_offset_jacobian_fd(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["offset_jacobian_fd"]


def test_offset_gradient_is_twice_b_o(oracle_lib, room3):
    assert P.pin_offset_gradient_fd(oracle_lib, oracle_lib.load(), room3) < P.PIN_TOL["offset_gradient_fd"]


def test_residuals_match_brute_force(oracle_lib, room3, street3):
    """Validity, e and rho of every rule (depth limit, window, usable taps,
    occlusion, target normal, both Huber branches) against a vectorised
    evaluation from the definitions."""
    assert P.pin_residual_brute_force(oracle_lib, oracle_lib.load(), room3, street3) < P.PIN_TOL["residual_brute_force"]


def test_build_pairs_matches_an_independent_graph(oracle_lib, room8):
    """Candidates by scipy's rotation magnitude and the translation distance,
    ratios by the brute-force residual evaluation, kept pairs by the ratio
    threshold or sequence (Sec. IV-B)."""
    assert P.pin_build_pairs(oracle_lib, oracle_lib.load(), room8) < P.PIN_TOL["build_pairs"]


@pytest.mark.parametrize("which", ["room3", "street3", "room3_offset"])
def test_target_jacobian_is_the_source_jacobian_mapped_by_the_relative_pose(oracle_lib, which, request):
    """J_j = J_i T (the residual depends on the poses only through X_j^-1 X_i),
    on the oracle's separately computed J_i and J_j."""
    w = request.getfixturevalue(which.replace("_offset", ""))
    if which.endswith("_offset"):
        w = P._with_offset(w)
    assert P.pin_relative_jacobian(oracle_lib, oracle_lib.load(), w) < P.PIN_TOL["relative_jacobian"]


def test_hessian_equals_gauss_newton_matrix_at_zero_residual(oracle_lib):
    """d b / d dx = H where every residual vanishes (Sec. IV-C normal equations;
    pins the Omega weighting of H)."""
    assert P.pin_hessian_zero_residual(oracle_lib, oracle_lib.load()) < P.PIN_TOL["hessian_zero_residual"]


@pytest.mark.parametrize("which", ["room3", "street3"])
def test_huber_weight_of_the_normal_equations(oracle_lib, which, request):
    """Single-point pair blocks equal w J^T Omega J from finite-difference
    Jacobians and the brute-force chi, on both sides of delta."""
    w = request.getfixturevalue(which)
    assert P.pin_huber_hessian(oracle_lib, oracle_lib.load(), w) < P.PIN_TOL["huber_hessian"]


def test_binary16_rounding_of_texel_values(oracle_lib):
    """R25's rounding against numpy's IEEE float16 conversion (ties to even, subnormals, overflow)."""
    assert P.pin_half_rounding(oracle_lib, oracle_lib.load()) < P.PIN_TOL["half_rounding"]
