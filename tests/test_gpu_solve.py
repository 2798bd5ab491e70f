"""The damped solve of the LM step (Sec. IV-C) in its forms on the same
systems: the one-launch cluster solve (PBA_SOLVE_MIXED where the FP32 factor
fits the cluster's shared memory), the block-sparse envelope solve
(PBA_SOLVE_SPARSE, and PBA_SOLVE_MIXED above the cluster's size), the
per-tile-step launches of the same mixed-precision arithmetic
(PBA_SOLVE_MIXED_STEPS) and the FP64 Cholesky.

Bars: after one iteration the poses of the mixed solves agree with the FP64
Cholesky to max(1e-8, 1e-10 kappa) of the step, kappa the condition number of
the Jacobi-scaled damped system (after its three fixed passes the refinement
requires |r| <= 1e-10 |b'|, else the step is rejected),
accept/reject decisions are identical, and a singular damped system is
rejected by all three.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _room(n_frames):
    from paper_2303_16878_gb300 import synth
    return synth.make_rgbd_room(n_frames=n_frames, width=48, height=36, f=36.0, seed=7)


# systems whose FP32 factor fits the shared memory of a 16-CTA cluster (227 KB
# per CTA, tile rows i -> CTA i mod 16): up to 130 frames (774 unknowns); 150
# and 160 frames take the block-sparse solve
CLUSTER_FRAMES = {3, 12, 40, 100, 130}


@pytest.mark.parametrize("n_frames", [3, 12, 40, 100, 130, 150, 160])
def test_cluster_solve_matches_per_step_and_f64(n_frames):
    """Sizes from one tile (a single-CTA cluster) through 16 CTAs with two tile
    rows each, to systems too large for the cluster (per-step launches)."""
    gpu()
    import paper_2303_16878_gb300 as pba
    w = _room(n_frames)
    solvers = (pba.PBA_SOLVE_MIXED, pba.PBA_SOLVE_MIXED_STEPS, pba.PBA_SOLVE_CHOLESKY_F64)
    ps = [pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16, solver=s) for s in solvers]
    try:
        launches = [p.iteration_launches() for p in ps]
        assert launches[0] < launches[1], launches  # one cluster launch, or the sparse solve's six
        for lam in (None, 1e-3, 1e-6):
            stats = []
            for p in ps:
                p.set_poses(w.poses_init)
                p.set_lambda(lam)
            ps[2].linearize()
            H, _ = ps[2].get_system()
            for p in ps:
                stats.append(p.iterate())
            assert all(s["status"] == 0 for s in stats)
            assert len({s["accepted"] for s in stats}) == 1
            # the refined solution satisfies |r| <= 1e-10 |b'| for the Jacobi-scaled system
            # A' = D (H_ff + lambda I) D, so its step is within kappa(A') 1e-10 of the exact one
            A = H[6:, 6:] + stats[2]["lambda_used"] * np.eye(H.shape[0] - 6)
            d = 1.0 / np.sqrt(np.diag(A))
            kappa = np.linalg.cond(d[:, None] * A * d[None, :])
            poses = [p.get_poses() for p in ps]
            step = max(np.abs(poses[2] - w.poses_init).max(), 1e-6)
            bar = max(1e-8, 1e-10 * kappa) * max(step, 1e-3)
            for q in poses[:2]:
                assert np.abs(q - poses[2]).max() <= bar
            # the cost after the step is the same function of the same poses
            for s in stats[:2]:
                assert s["new_cost"] == pytest.approx(stats[2]["new_cost"], rel=1e-6)
    finally:
        for p in ps:
            p.close()


def test_singular_system_is_rejected_by_every_solver():
    """A frame without pairs leaves a zero block in H_ff; with lambda = 0 the
    first pivot of that block is 0, the factorisation fails (PBA_ENOTPD) and
    the step is rejected with the poses kept."""
    gpu()
    import paper_2303_16878_gb300 as pba
    w = _room(12)
    last = w.poses_init.shape[0] - 1
    pairs = np.array([pq for pq in np.asarray(w.pairs) if last not in pq])
    w = dataclasses.replace(w, pairs=pairs)
    for solver in (pba.PBA_SOLVE_MIXED, pba.PBA_SOLVE_MIXED_STEPS, pba.PBA_SOLVE_CHOLESKY_F64,
                   pba.PBA_SOLVE_SPARSE):
        p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16, solver=solver)
        try:
            p.set_lambda(0.0)
            s = p.iterate()
            assert s["status"] == pba._lib.PBA_ENOTPD and s["accepted"] == 0
            np.testing.assert_array_equal(p.get_poses(), w.poses_init)
            # with damping the same system solves and the step is taken
            p.set_lambda(1e-3)
            s = p.iterate()
            assert s["status"] == 0 and s["accepted"] == 1
        finally:
            p.close()


def _compare_with_f64(w, lams=(None, 1e-3, 1e-6), frame_var=None, n_vars=None):
    """One LM iteration with PBA_SOLVE_SPARSE and with the FP64 Cholesky from the
    same poses and lambda: the same accept decision and poses within
    max(1e-8, 1e-10 kappa) of the step (kappa of the Jacobi-scaled damped
    system in pose variables)."""
    import paper_2303_16878_gb300 as pba
    ps = [pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F32, solver=s)
          for s in (pba.PBA_SOLVE_SPARSE, pba.PBA_SOLVE_CHOLESKY_F64)]
    try:
        if frame_var is not None:
            for p in ps:
                p.set_variables(frame_var, n_vars)
        for lam in lams:
            for p in ps:
                p.set_poses(w.poses_init)
                p.set_lambda(lam)
            ps[1].linearize()
            H, _ = ps[1].get_system()
            stats = [p.iterate() for p in ps]
            assert all(s["status"] == 0 for s in stats), stats
            assert stats[0]["accepted"] == stats[1]["accepted"]
            fv = np.arange(w.n_frames) - 1 if frame_var is None else np.asarray(frame_var)
            nv = w.n_frames - 1 if frame_var is None else n_vars
            S = np.zeros((6 * w.n_frames, 6 * nv))
            for k, v in enumerate(fv):
                if v >= 0:
                    S[6 * k:6 * k + 6, 6 * v:6 * v + 6] = np.eye(6)
            A = S.T @ H @ S + stats[1]["lambda_used"] * np.eye(6 * nv)
            d = 1.0 / np.sqrt(np.diag(A))
            kappa = np.linalg.cond(d[:, None] * A * d[None, :])
            poses = [p.get_poses() for p in ps]
            step = max(np.abs(poses[1] - w.poses_init).max(), 1e-6)
            assert np.abs(poses[0] - poses[1]).max() <= max(1e-8, 1e-10 * kappa) * max(step, 1e-3)
            assert stats[0]["new_cost"] == pytest.approx(stats[1]["new_cost"], rel=1e-6)
    finally:
        for p in ps:
            p.close()


def test_sparse_solve_on_a_chain():
    """A chain of 60 frames (pairs j - i <= 3): one component, banded."""
    gpu()
    _compare_with_f64(_room(60))


def test_sparse_solve_on_a_loop():
    """40 frames around the room's circle with the pairs closing the loop
    (j - i <= 3 modulo 40): the envelope of the natural order spans the whole
    matrix, reverse Cuthill-McKee orders it as a narrow band."""
    gpu()
    w = _room(40)
    n = w.n_frames
    pairs = sorted({(min(i, (i + d) % n), max(i, (i + d) % n)) for i in range(n) for d in (1, 2, 3)})
    _compare_with_f64(dataclasses.replace(w, pairs=np.array(pairs, dtype=np.int32)))


def test_sparse_solve_on_independent_components():
    """Three independent chains (12, 30 and 5 frames; the first frame of each
    held fixed): three components, three clusters in one launch."""
    gpu()
    from paper_2303_16878_gb300 import synth
    parts = [_room(12), synth.make_rgbd_room(n_frames=30, width=48, height=36, f=36.0, seed=8),
             synth.make_rgbd_room(n_frames=5, width=48, height=36, f=36.0, seed=9)]
    chans, gt, init, pairs, fv, base, nvar = [], [], [], [], [], 0, 0
    for w in parts:
        chans += list(w.channels)
        gt.append(w.poses_gt)
        init.append(w.poses_init)
        pairs += [(base + i, base + j) for i, j in w.pairs.tolist()]
        fv += [-1] + list(range(nvar, nvar + w.n_frames - 1))
        nvar += w.n_frames - 1
        base += w.n_frames
    w = synth.Workload("three", parts[0].sensors, np.zeros(base, dtype=np.int32), chans, np.concatenate(gt),
                       np.concatenate(init), np.array(pairs, dtype=np.int32), parts[0].params)
    _compare_with_f64(w, frame_var=np.array(fv, dtype=np.int32), n_vars=nvar)


def test_sparse_solve_with_tied_frames(fusion):
    """Camera and LiDAR frames of one platform pose share a variable (Sec. V):
    pairs whose frames map to one variable add H_ij + H_ji to its diagonal block."""
    gpu()
    _compare_with_f64(fusion, frame_var=fusion.frame_var, n_vars=fusion.n_vars)
