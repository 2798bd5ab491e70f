"""Normal estimation on the GPU (Sec. IV-A) against the FP64 oracle.

Bar: the set of pixels that get a normal is bit-exact outside the oracle's
decision margin, intensity and depth stay untouched, and every normal lies
within tol = 1e-5 + 64 u D sqrt(ev2) / (ev1 - ev0) of the oracle's (max-norm
of the difference; u = 2^-24; ev the oracle's covariance eigenvalues; D the
largest depth among the points used).  The second term is the first-order
perturbation bound of the plane's eigenvector: the GPU forms the points in
float32, so each point relative to the centre carries an absolute error of a
few u D, which perturbs the covariance by a few u D sqrt(ev2) and the
eigenvector by that over the gap ev1 - ev0 of the two smallest eigenvalues;
the Jacobi eigen-solver adds an error of a few u ev2 / (ev1 - ev0), smaller
since sqrt(ev2) <= 2 D.  Where tol exceeds 0.05 the plane is not determined
to float32 accuracy (nearly collinear points): there only the orientation
(n . p <= 0) and unit length are checked, and such pixels must stay rare
(at most 5%).
"""
import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def estimate_on_gpu(w, frames, scale, max_radius):
    import paper_2303_16878_gb300 as pba
    gpu()
    p = pba.problem_from_workload(w)
    p.estimate_normals(frames[0], len(frames), scale=scale, max_radius=max_radius)
    return p, p.get_channels(frames[0], len(frames))


def compare_frame(oracle_lib, w, k, got, scale, max_radius):
    s = w.sensors[int(w.frame_sensor[k])]
    ref = oracle_lib.estimate_normals(s, w.channels[k], scale, max_radius, params=w.params)
    raw = w.channels[k]
    assert np.array_equal(got[..., :2], raw[..., :2]), "intensity / depth changed"
    has_ref = np.linalg.norm(ref["normals"], axis=-1) > 0
    has_got = np.linalg.norm(got[..., 2:5], axis=-1) > 0
    free = ~ref["margin"]
    assert np.array_equal(has_ref & free, has_got & free), \
        f"{int(np.count_nonzero((has_ref != has_got) & free))} pixels decide differently"
    both = has_ref & has_got
    ev = ref["eig"]
    d = raw[..., 1].astype(np.float64)
    tol = 1e-5 + 64 * U32 * ref["dmax"] * np.sqrt(np.maximum(ev[..., 2], 0)) / np.maximum(ev[..., 1] - ev[..., 0],
                                                                                          1e-300)
    loose = both & (tol > 0.05)
    tight = both & ~loose
    err = np.abs(got[..., 2:5].astype(np.float64) - ref["normals"]).max(axis=-1)
    worst = float((err / tol)[tight].max()) if tight.any() else 0.0
    assert worst <= 1.0, f"normal error {worst:.3g} x tolerance (max abs {float(err[tight].max()):.3g})"
    # about 2% on the LiDAR street (near-collinear neighbourhoods: thin poles, sparse rows)
    assert loose.sum() <= 0.05 * max(both.sum(), 1), f"{int(loose.sum())} of {int(both.sum())} ill-determined planes"
    from paper_2303_16878_gb300 import synth
    n_got = got[..., 2:5].astype(np.float64)
    assert np.abs(np.linalg.norm(n_got[both], axis=-1) - 1).max() < 1e-5
    rays, _ = synth._pixel_rays(s)  # the viewing ray of each pixel: p = depth x ray
    assert np.all(np.sum(n_got * rays, axis=-1)[both] <= 1e-6), "a normal faces away from the sensor"
    # pixels with a unit normal: the ones the pixel-point builder keeps
    return int(np.count_nonzero(has_got & (d > 0)))


@pytest.mark.parametrize("which,scale,max_radius", [("room3", 6.0, 4), ("street3", 8.0, 4), ("street3", 20.0, 7)])
def test_normals_match_oracle(oracle_lib, which, scale, max_radius, request):
    w = request.getfixturevalue(which)
    p, got = estimate_on_gpu(w, list(range(w.n_frames)), scale, max_radius)
    for k in range(w.n_frames):
        n_pts = compare_frame(oracle_lib, w, k, got[k], scale, max_radius)
        assert p.frame_points(k) == n_pts


def test_full_size_lidar_frame_normals(oracle_lib):
    """One 64 x 1024 frame of the 50-frame street, estimated with the other 49."""
    w = workload("street")
    p, got = estimate_on_gpu(w, list(range(w.n_frames)), 8.0, 5)
    for k in (0, 37):
        compare_frame(oracle_lib, w, k, got[k], 8.0, 5)


def test_linearisation_after_estimation_equals_upload_of_the_same_channels(room3):
    """estimate_normals rebuilds texels, points and the pair plan: the system
    equals that of a problem given the resulting channels directly."""
    import paper_2303_16878_gb300 as pba
    p, got = estimate_on_gpu(room3, list(range(room3.n_frames)), 6.0, 4)
    c1, n1 = p.linearize()
    H1, b1 = p.get_system()
    q = pba.problem_from_workload(room3)
    q.upload_frames(0, np.ascontiguousarray(got))
    c2, n2 = q.linearize()
    H2, b2 = q.get_system()
    assert n1 == n2 and c1 == c2
    assert np.array_equal(H1, H2) and np.array_equal(b1, b2)


def test_frames_without_depth_get_no_normals(room3):
    import paper_2303_16878_gb300 as pba
    gpu()
    w = room3
    p = pba.problem_from_workload(w)
    empty = np.zeros_like(w.channels[1])
    empty[..., 0] = w.channels[1][..., 0]
    p.upload_frames(1, empty[None])
    p.estimate_normals(0, w.n_frames, scale=6.0, max_radius=4)
    got = p.get_channels(1, 1)[0]
    assert not np.any(got[..., 2:5]) and p.frame_points(1) == 0
    p.linearize()  # pairs with an empty frame contribute nothing but still run


def test_estimate_normals_rejects_bad_arguments(room3):
    import paper_2303_16878_gb300 as pba
    gpu()
    p = pba.problem_from_workload(room3)
    for kw in (dict(max_radius=1), dict(max_radius=pba._lib.PBA_NORMALS_MAX_RADIUS + 1), dict(scale=float("nan")),
               dict(scale=-1.0)):
        with pytest.raises(pba.PbaError):
            p.estimate_normals(0, 1, **kw)
    with pytest.raises(pba.PbaError):
        p.estimate_normals(2, 2)
    q = pba.Problem(room3.sensors, 2, room3.params)
    with pytest.raises(pba.PbaError) as e:
        q.estimate_normals(0, 1)
    assert e.value.code == pba._lib.PBA_ENOTREADY


@pytest.mark.parametrize("which,scale,max_radius", [("room3", 6.0, 4), ("street3", 8.0, 4)])
def test_linearisation_of_estimated_normals_matches_oracle(oracle_lib, which, scale, max_radius, request):
    """Normal estimation feeding the hot path (Sec. IV-A then Sec. IV-C): the
    GPU estimates normals from depth, rebuilds FP16 texels and points and
    linearises; the oracle estimates its own normals in FP64, samples the
    target's intensity and normals as binary16 values (R25) and linearises.
    H, b to 1e-4 and the cost to 1e-5 (relative), the count within the
    pixels whose normal decision lies inside the oracle's margin + 2.  Pixels
    whose plane is not determined to float32 accuracy (tol > 0.05 in
    compare_frame) keep different normals on the two sides; their share of
    the residuals is what separates the two sums."""
    import paper_2303_16878_gb300 as pba
    w = request.getfixturevalue(which)
    p, got = estimate_on_gpu(w, list(range(w.n_frames)), scale, max_radius)
    cost, count = p.linearize()
    H, b = p.get_system()
    chans, near = [], 0
    for k in range(w.n_frames):
        s = w.sensors[int(w.frame_sensor[k])]
        ref = oracle_lib.estimate_normals(s, w.channels[k], scale, max_radius, params=w.params)
        c = w.channels[k].copy()
        c[..., 2:5] = ref["normals"].astype(np.float32)
        chans.append(c)
        near += int(np.count_nonzero(ref["margin"]))
    o = oracle_lib.linearize(w.sensors, w.frame_sensor, chans, w.poses_init, w.pairs,
                             dict(w.params, texel_f16=1))
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))
    assert abs(count - o["count"]) <= near + 2, (count, o["count"], near)
    assert rel(H, o["H"]) <= 1e-4, rel(H, o["H"])
    assert rel(b, o["b"]) <= 1e-4, rel(b, o["b"])
    assert abs(cost - o["cost"]) <= 1e-5 * o["cost"], (cost, o["cost"])
    p.close()
