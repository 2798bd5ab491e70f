"""The joint configuration at full size: 300 LiDAR frames of 128 x 1024 and
600 RGB-D frames of 640 x 480 on one platform in the hall, the camera's
offset given with a seeded 2 cm / 0.5 deg error; poses (camera and LiDAR
frames of one instant tied, Sec. V) and the camera offset refined jointly;
then a batch of 16 independent LiDAR problems of 50-400 frames linearised in
one launch.

Bars: 50 seeded pairs of each configuration against the oracle as in
test_gpu_large.py (masks outside the decision margin; the sampled
sub-system's H, b 1e-4 and cost 1e-5, each pair's H12 / b12 1e-3 and cost
1e-4, with the points decided the other way accounted for; at most 1e-5 of
the residuals (+2) decided the other way); the joint
refinement lowers the cost and brings the offset to within 1 cm / 0.25 deg
of the true one; batch problems share no block of H.
"""
import numpy as np
import pytest

from parity_helpers import check_sampled_pairs

pytestmark = pytest.mark.gpu

_CACHE = {}


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _host(ch):
    return ch.detach().cpu().numpy()


def _check_sampled_pairs(oracle_lib, w, p, n_sample, seed):
    """50 seeded pairs against the oracle (FP16 texels: R25), see parity_helpers."""
    n, res, flipped = check_sampled_pairs(oracle_lib, w, p, n_sample, seed, dict(w.params, texel_f16=1), _host, rel)
    assert n == min(n_sample, len(w.pairs)) and res > 0


def test_joint_hall_parity_and_refinement(oracle_lib):
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    gpu()
    w = synth.make_joint_hall()
    n_cam = int(np.sum(w.frame_sensor == 0))
    assert n_cam == 600 and w.n_frames == 900
    p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_MIXED)
    p.autotune(1)
    cam_pairs = [q for q, (i, j) in enumerate(w.pairs.tolist()) if i < n_cam]
    assert 0 < len(cam_pairs) < len(w.pairs)
    _check_sampled_pairs(oracle_lib, w, p, 50, 9)
    t0, r0 = synth.offset_error(w.extrinsic_gt[0], p.get_extrinsic(0))
    c0, _ = p.linearize()
    # poses and the camera offset jointly, coarse to fine (the offset as an LM variable)
    p.set_offset_free(0)
    p.build_pyramid(3)
    log = p.optimize([10, 5, 5], rel_tol=1e-7)
    c1 = log[-1]["cost_last"]
    t1, r1 = synth.offset_error(w.extrinsic_gt[0], p.get_extrinsic(0))
    got = p.get_poses()
    assert c1 < c0
    assert t1 < 0.01 and r1 < 0.25, (t0, r0, t1, r1, log)
    for k in range(300):  # tied frames share their pose exactly
        assert np.array_equal(got[2 * k], got[n_cam + k])
    assert np.array_equal(p.get_extrinsic(1), np.eye(3, 4))
    p.close()


def test_batch_of_sixteen_problems_in_one_launch(oracle_lib):
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    gpu()
    w, spans = synth.make_street_batch()
    sizes = [n for _, n in spans]
    assert len(spans) == 16 and min(sizes) >= 50 and max(sizes) <= 400 and len(set(sizes)) > 8
    p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_MIXED)
    _check_sampled_pairs(oracle_lib, w, p, 50, 10)
    H, b = p.get_system()
    owner = np.repeat(np.arange(16), sizes)
    blk = owner[np.arange(6 * w.n_frames) // 6]
    assert not np.any(H[blk[:, None] != blk[None, :]])  # no coupling between problems
    st = p.iterate()
    assert st["status"] == 0 and st["new_cost"] < st["cost"]
    p.close()
