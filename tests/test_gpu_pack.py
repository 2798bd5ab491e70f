"""Pixel validity at its thresholds (Sec. IV-A): the packing kernels decide
range_min <= d <= range_max and |n|^2 > 0.25 in float32 with exact fallbacks;
the decisions must equal the oracle's double evaluation of the same float32
inputs on every pixel, including depths one ulp around range limits that are
not float32 numbers and normals whose squared length lies within rounding of
0.25.  Checked through the per-frame point counts and, for the usable flags
(a pixel and its four neighbours valid), through H and b of a linearisation.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RANGE_MIN, RANGE_MAX = 0.7, 4.3   # not float32 numbers


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _adversarial(w, seed=11, depths_too=True):
    """Every third pixel of every frame gets a depth one ulp around a range limit
    (depths_too) or its normal shortened to |n| = 0.5 and walked by a few ulps, so
    that |n|^2 straddles 0.25 within rounding."""
    rng = np.random.default_rng(seed)
    chans = []
    f32 = np.float32
    lo, hi = f32(RANGE_MIN), f32(RANGE_MAX)
    depths = np.array([np.nextafter(lo, f32(0)), lo, np.nextafter(lo, f32(10)),
                       np.nextafter(hi, f32(0)), hi, np.nextafter(hi, f32(10))], dtype=np.float32)
    for c in w.channels:
        c = c.copy()
        flat = c.reshape(-1, 5)
        idx = np.arange(0, flat.shape[0], 3)
        kind = rng.integers(0, 2, size=idx.size)
        for k, i in zip(kind, idx):
            if flat[i, 1] <= 0:
                continue
            if k == 0 and depths_too:
                flat[i, 1] = depths[rng.integers(0, depths.size)]
            else:
                v = flat[i, 2:5].astype(np.float64)
                if not np.linalg.norm(v) > 0:
                    continue
                n = (0.5 * v / np.linalg.norm(v)).astype(np.float32)
                # walk the components by a few ulps so |n|^2 (in double) straddles 0.25
                for _ in range(int(rng.integers(0, 4))):
                    j = int(rng.integers(0, 3))
                    n[j] = np.nextafter(n[j], np.float32(np.sign(n[j]) * (1 if rng.random() < 0.5 else -1) * 10))
                flat[i, 2:5] = n
        chans.append(c)
    return dataclasses.replace(w, channels=chans)


def test_point_counts_match_the_oracle_at_the_thresholds(oracle_lib):
    gpu()
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    w = synth.make_rgbd_room(n_frames=4, width=96, height=72, f=72.0, seed=5)
    w = _adversarial(w)
    params = dict(w.params, range_min=RANGE_MIN, range_max=RANGE_MAX)
    near = 0
    for c in w.channels:
        n2 = (c[..., 2].astype(np.float64) ** 2 + c[..., 3].astype(np.float64) ** 2
              + c[..., 4].astype(np.float64) ** 2)
        near += int((np.abs(n2 - 0.25) < 1e-6).sum())
    assert near > 100  # the inputs do exercise the near-threshold branch
    p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16, params=params)
    try:
        for k in range(w.n_frames):
            pts, _ = oracle_lib.frame_points(w.sensors[w.frame_sensor[k]], params, w.channels[k])
            assert p.frame_points(k) == len(pts)
    finally:
        p.close()


def test_usable_flags_match_the_oracle_at_the_thresholds(oracle_lib):
    gpu()
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    w = synth.make_rgbd_room(n_frames=4, width=96, height=72, f=72.0, seed=5)
    w = _adversarial(w, seed=12, depths_too=False)
    params = dict(w.params, range_min=RANGE_MIN, range_max=RANGE_MAX)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params)
    p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F32, params=params)
    try:
        cost, count = p.linearize()
        H, b = p.get_system()
        rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))
        assert abs(count - ref["count"]) <= 2
        assert rel(H, ref["H"]) <= 1e-4 and rel(b, ref["b"]) <= 1e-4
        assert abs(cost - ref["cost"]) <= 1e-5 * ref["cost"]
    finally:
        p.close()
