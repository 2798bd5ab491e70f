"""Multi-sensor bundle adjustment (Sec. V, fusion) on the GPU: an RGB-D camera
and a LiDAR on one platform, their frames of one platform pose tied to one
pose variable (pba_set_variables), against the FP64 oracle; and the coupled /
consecutive convergence-basin sweep on a platform frame aligned to itself.

Bars: the damped step's poses to 1e-4 of the step and the new cost to 1e-5;
LM-converged poses within 1e-4 m / 1e-5 rad of the oracle's; tied frames
bit-identical poses, fixed frames unchanged.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_COST = 1e-5


def make(w, **kw):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    return pba.problem_from_workload(w, **kw)


@pytest.mark.parametrize("solver", [0, 1])
def test_tied_damped_step_matches_oracle(oracle_lib, fusion, solver):
    w = fusion
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, w.params)
    S = oracle_lib.selection(w.frame_var, w.n_vars)
    lam = 10.0 * float(np.diag(S.T @ ref["H"] @ S).max())
    dx, ok = oracle_lib.solve_step_vars(ref["H"], ref["b"], lam, w.frame_var, w.n_vars)
    cand = oracle_lib.apply_update(w.poses_init, dx)
    new = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, cand, w.pairs, w.params, want_system=False)
    assert ok and new["cost"] < ref["cost"]
    p = make(w, texel=0, solver=solver)
    p.linearize()
    st = p.solve_step(lam)
    assert st["accepted"] and st["status"] == 0
    assert abs(st["new_cost"] - new["cost"]) <= TOL_COST * new["cost"]
    got = p.get_poses()
    step_ref = np.abs(cand - w.poses_init).max()
    assert np.abs(got - cand).max() <= 1e-4 * step_ref + 1e-12


@pytest.mark.parametrize("solver", [0, 1])
def test_coupled_lm_converges_to_oracle_poses(oracle_lib, fusion, solver):
    w = fusion
    poses, lam = w.poses_init.copy(), None
    for _ in range(8):
        o = oracle_lib.lm_iteration(w, poses, lam)
        poses, lam = o["poses"], o["lam"]
    p = make(w, texel=0, solver=solver)
    for _ in range(8):
        p.iterate()
    got = p.get_poses()
    n = w.n_frames // 2
    for k in range(w.n_frames):
        assert np.linalg.norm(got[k][:, 3] - poses[k][:, 3]) <= 1e-4
        R = got[k][:, :3].T @ poses[k][:, :3]
        assert np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)) <= 1e-5
    for k in range(n):  # camera and LiDAR frames of one platform pose move together
        assert np.array_equal(got[k], got[n + k])
    assert np.array_equal(got[0], w.poses_init[0]) and np.array_equal(got[n], w.poses_init[n])


def test_set_variables_rejects_bad_mappings(fusion):
    import paper_2303_16878_gb300 as pba
    p = make(fusion)
    n = fusion.n_frames
    for fv, nv in ((np.zeros(n), 1),                      # nothing held fixed
                   (np.r_[-1, np.zeros(n - 1)], 0),        # n_vars < 1
                   (np.r_[-1, np.full(n - 1, 3)], 3),      # entry outside [-1, n_vars)
                   (np.r_[-1, np.zeros(n - 1)], 2),        # variable 1 moves nothing
                   (np.r_[-1, np.arange(n - 1)], n)):      # n_vars > n_frames - 1
        with pytest.raises(pba.PbaError):
            p.set_variables(fv, nv)
    with pytest.raises(ValueError):
        p.set_variables(np.zeros(3), 1)
    p.set_variables(None)
    p.iterate()


# ------------------------------------------------------------------ convergence basin (Sec. V, fusion)

def _self_alignment(w, mode, k, motion):
    """Platform frame k aligned to a copy of itself: frame A at the true pose
    (fixed), frame B at X * motion (a 3x4 rigid motion); the optimum is B = A.
    mode: 'rgbd', 'lidar' or 'coupled' (both sensors, B's camera and LiDAR
    frames tied)."""
    from paper_2303_16878_gb300 import synth
    n = w.n_frames // 2
    cam, lid = w.channels[k], w.channels[n + k]
    X = w.poses_gt[k]
    XB = synth.compose(X, motion)
    if mode == "rgbd":
        ch, fs, sens = [cam, cam], [0, 0], [w.sensors[0]]
    elif mode == "lidar":
        ch, fs, sens = [lid, lid], [0, 0], [w.sensors[1]]
    else:
        ch, fs, sens = [cam, cam, lid, lid], [0, 0, 1, 1], list(w.sensors)
    m = len(ch)
    poses = np.stack([X, XB] * (m // 2))
    pairs = np.array([[0, 1]] if m == 2 else [[0, 1], [2, 3]], dtype=np.int32)
    fv = np.array([-1, 0] * (m // 2), dtype=np.int32)
    return synth.Workload(f"self-{mode}", sens, np.array(fs, dtype=np.int32), ch, poses, poses, pairs,
                          dict(w.params), fv, 1)


def _run(sw, poses=None, levels=(10, 5, 5)):
    import paper_2303_16878_gb300 as pba
    p = pba.problem_from_workload(sw, poses=poses, texel=0)
    p.build_pyramid(len(levels))
    p.optimize(list(levels), rel_tol=1e-6)
    out = p.get_poses()
    p.close()
    return out


def _error(XB, XA):
    D = np.linalg.inv(np.vstack([XA, [0, 0, 0, 1]])) @ np.vstack([XB, [0, 0, 0, 1]])
    return float(np.linalg.norm(D[:3, 3])), float(np.degrees(np.arccos(np.clip((np.trace(D[:3, :3]) - 1) / 2, -1, 1))))


def basin_sweep(w, magnitudes=(0.025, 0.05, 0.1, 0.2, 0.4), n_dirs=4, seed=11):
    """Success counts per mode and initial error: translation `m` metres along a
    random direction and rotation 20 m degrees about a random axis (so 0.1 m
    goes with 2 deg); success = final error below 1 cm and 0.2 deg."""
    rng = np.random.default_rng(seed)
    table = {mode: [] for mode in ("rgbd", "lidar", "coupled", "consecutive")}
    for mag in magnitudes:
        wins = {mode: 0 for mode in table}
        for _ in range(n_dirs):
            from paper_2303_16878_gb300 import synth
            t = rng.normal(size=3)
            r = rng.normal(size=3)
            motion = np.zeros((3, 4))
            motion[:, :3] = synth.rot_vec(math.radians(20.0 * mag) * r / np.linalg.norm(r))
            motion[:, 3] = mag * t / np.linalg.norm(t)
            for mode in ("rgbd", "lidar", "coupled"):
                sw = _self_alignment(w, mode, 0, motion)
                got = _run(sw)
                et, er = _error(got[1], got[0])
                wins[mode] += int(et < 0.01 and er < 0.2)
            # consecutive: LiDAR alone, then the camera from the LiDAR's result
            sl = _self_alignment(w, "lidar", 0, motion)
            gl = _run(sl)
            sr = _self_alignment(w, "rgbd", 0, motion)
            gr = _run(sr, poses=np.stack([sr.poses_init[0], gl[1]]))
            et, er = _error(gr[1], gr[0])
            wins["consecutive"] += int(et < 0.01 and er < 0.2)
        for mode in table:
            table[mode].append(wins[mode])
    return dict(magnitudes=list(magnitudes), n_dirs=n_dirs, success=table)


def test_convergence_basin_coupled_and_consecutive(fusion):
    """Coupled and consecutive refinement converge from at least as many initial
    errors as the camera alone, every mode converges from the smallest one."""
    make(fusion).close()  # skips without a GPU
    res = basin_sweep(fusion)
    s = res["success"]
    print("basin sweep", res)
    for mode in s:
        assert s[mode][0] == res["n_dirs"], (mode, res)
    assert sum(s["coupled"]) >= sum(s["rgbd"]), res
    assert sum(s["consecutive"]) >= sum(s["rgbd"]), res


# ------------------------------------------------------------------ the camera offset as an LM variable (R23)

def _offset_workload():
    import dataclasses
    from paper_2303_16878_gb300 import synth
    w = synth.make_fusion_room(tilt_deg=12.0)
    true = np.asarray(w.sensors[0].extrinsic)
    err = np.zeros((3, 4))
    err[:, :3] = synth.rot_vec(np.radians(0.5) * np.array([0.6, -0.64, 0.48]))
    err[:, 3] = 0.02 * np.array([-0.48, 0.8, 0.36])
    bad = dataclasses.replace(w.sensors[0], extrinsic=synth.compose(true, err))
    return dataclasses.replace(w, sensors=[bad, w.sensors[1]]), true


def _rot_angle(A, B):
    return float(np.arccos(np.clip((np.trace(A[:, :3].T @ B[:, :3]) - 1) / 2, -1, 1)))


@pytest.mark.parametrize("solver", [0, 1])
def test_free_offset_damped_step_matches_oracle(oracle_lib, solver):
    """A strongly damped step with the camera offset free: poses and offset as
    the oracle's (offset blocks per point, R23) to 1e-4 of the step."""
    w, _ = _offset_workload()
    lin = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, w.params)
    H, b = oracle_lib.offset_system(w, w.sensors, w.poses_init, lin, [0])
    blocks_var = np.concatenate([w.frame_var, [w.n_vars]])
    S = oracle_lib.selection(blocks_var, w.n_vars + 1)
    lam = 10.0 * float(np.diag(S.T @ H @ S).max())
    ref = oracle_lib.lm_iteration_offsets(w, w.poses_init, w.sensors, lam, [0])
    assert ref["accepted"]
    p = make(w, texel=0, solver=solver)
    p.set_offset_free(0)
    p.linearize()
    st = p.solve_step(lam)
    assert st["accepted"] and abs(st["new_cost"] - ref["new_cost"]) <= TOL_COST * ref["new_cost"]
    step = np.abs(ref["candidate"] - w.poses_init).max()
    assert np.abs(p.get_poses() - ref["candidate"]).max() <= 1e-4 * step + 1e-12
    Xo_ref = oracle_lib._extrinsic_of(ref["candidate_sensors"][0])
    ostep = np.abs(Xo_ref - np.asarray(w.sensors[0].extrinsic)).max()
    assert np.abs(p.get_extrinsic(0) - Xo_ref).max() <= 1e-4 * ostep + 1e-12
    assert np.array_equal(p.get_extrinsic(1), np.asarray(w.sensors[1].extrinsic))


@pytest.mark.parametrize("solver", [0, 1])
def test_free_offset_lm_matches_oracle_and_recovers_the_offset(oracle_lib, solver):
    """Eight LM iterations with poses and the camera offset free (camera and
    LiDAR frames of one platform pose tied): poses and offset within 1e-4 m /
    1e-5 rad of the oracle's, and the offset within 1 cm / 0.1 deg of the true
    one from 2 cm / 0.5 deg (the platform tilts by up to 12 deg, so the
    offset's translation is observable)."""
    from paper_2303_16878_gb300 import synth
    w, true = _offset_workload()
    P, sens, lam = w.poses_init.copy(), list(w.sensors), None
    for _ in range(8):
        r = oracle_lib.lm_iteration_offsets(w, P, sens, lam, [0])
        P, sens, lam = r["poses"], r["sensors"], r["lam"]
    p = make(w, texel=0, solver=solver)
    p.set_offset_free(0)
    for _ in range(8):
        p.iterate()
    got = p.get_poses()
    for k in range(w.n_frames):
        assert np.linalg.norm(got[k][:, 3] - P[k][:, 3]) <= 1e-4 and _rot_angle(got[k], P[k]) <= 1e-5
    Xo, Xo_ref = p.get_extrinsic(0), oracle_lib._extrinsic_of(sens[0])
    assert np.linalg.norm(Xo[:, 3] - Xo_ref[:, 3]) <= 1e-4 and _rot_angle(Xo, Xo_ref) <= 1e-5
    t1, r1 = synth.offset_error(true, Xo)
    assert t1 < 0.01 and r1 < 0.1, (t1, r1)


def test_refine_extrinsic_recovers_the_camera_offset():
    """At the true poses of the tilted platform, a camera offset off by 2 cm /
    0.5 deg is refined by BFGS with the adjoint gradient to within 1 cm /
    0.1 deg of the true one, the LiDAR's offset untouched."""
    from paper_2303_16878_gb300 import synth
    w, true = _offset_workload()
    p = make(w, poses=w.poses_gt, texel=0)
    t0, r0 = synth.offset_error(true, p.get_extrinsic(0))
    out = p.refine_extrinsic(0, max_iters=40, rel_tol=1e-9)
    t1, r1 = synth.offset_error(true, p.get_extrinsic(0))
    assert out["cost_after"] < out["cost_before"]
    assert t0 > 0.019 and r0 > 0.49 and t1 < 0.01 and r1 < 0.1, (t0, r0, t1, r1, out)
    assert np.array_equal(p.get_extrinsic(1), np.asarray(w.sensors[1].extrinsic))
