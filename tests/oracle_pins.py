"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each pin returns an error measure; `PIN_TOL` holds the bar.  The pins are used
twice: by test_oracle_pins.py on the oracle as committed, and by
test_oracle_mutations.py on copies with a planted mistake, where at least one
pin must fail.  Sources of truth:
  - hand-derived closed forms of Eq. pinhole-projection / Eq. spherical-projection (tests/golden/projection_closed_form.json);
  - scipy's rotation and bilinear-interpolation routines and numpy's linear solver;
  - central finite differences of the oracle's own residual and cost;
  - invariants of the formulation: the 6-dim gauge null space of H (the
    residual depends on X_i, X_j only through X_j^-1 X_i, Eq. uprime), exact zero
    error for integer-pixel shifts of a fronto-parallel plane.
"""
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

PIN_TOL = {
    "projection_golden": 1e-9,
    "roundtrip": 1e-9,
    "proj_jacobian_fd": 1e-6,
    "boxplus": 1e-12,
    "jacobian_fd_pinhole": 1e-6,
    "jacobian_fd_spherical": 1e-6,
    "ramp_grad_mode0": 1e-6,
    "gauge": 1e-10,
    "cost_gradient": 1e-5,
    "plane_shift": 1e-9,
    "single_channel": 1e-9,
    "cholesky": 1e-10,
    "extrinsic_equivalence": 1e-9,
    "jacobian_fd_extrinsic": 1e-6,
    "normals_plane": 1e-9,
    "normals_counts": 0.5,
    "normals_brute_force": 1e-8,
    "normals_degenerate": 0.5,
    "pyramid_projection": 1e-9,
    "downsample_closed_forms": 1e-12,
    "coarse_to_fine": 0.5,
    "tied_gradient": 1e-4,  # central differences of F ~ 900 at h = 2e-8: roundoff eps F / h ~ 1e-5 absolute
    "variables_reduce_to_gauge": 1e-12,
    "offset_jacobian_fd": 1e-6,
    "offset_gradient_fd": 1e-4,  # central differences of F at h = 2e-8 (roundoff eps F / h)
    "residual_brute_force": 1e-9,
    "build_pairs": 0.5,
    "relative_jacobian": 1e-12,
    "hessian_zero_residual": 1e-6,
    "huber_hessian": 1e-5,
    "half_rounding": 0.5,
}


def _sensor_from(d):
    from paper_2303_16878_gb300 import synth
    if d["model"] == 0:
        return synth.Sensor(0, d["width"], d["height"], d["fx"], d["fy"], d["cx"], d["cy"])
    return synth.spherical_sensor(d["width"], d["height"], d["vfov_up_deg"], d["vfov_down_deg"])


def pin_projection_golden(O, lib):
    g = json.load(open(os.path.join(HERE, "golden", "projection_closed_form.json")))
    err = 0.0
    for key in ("pinhole", "spherical"):
        s = _sensor_from(g[key]["sensor"])
        for c in g[key]["cases"]:
            uv = O.project(s, c["p"], lib=lib)
            err = max(err, float(np.abs(uv - np.array(c["uv"])).max()))
    return err


def pin_roundtrip(O, lib):
    """pi(pi^-1(u, d)) = u and the depth / range of pi^-1(u, d) is d."""
    from paper_2303_16878_gb300 import synth
    rng = np.random.default_rng(11)
    err = 0.0
    for s in (synth.pinhole_sensor(160, 120, 120.0, 80.0, 60.0), synth.spherical_sensor(1024, 64, 16.6, -16.6)):
        for _ in range(200):
            u = rng.uniform(0, s.width - 1)
            v = rng.uniform(0, s.height - 1)
            d = rng.uniform(0.5, 80.0)
            p = O.unproject(s, u, v, d, lib=lib)
            uv = O.project(s, p, lib=lib)
            du = abs(uv[0] - u)
            if s.model == 1:
                du = min(du, abs(du - s.width))
            dist = p[2] if s.model == 0 else float(np.linalg.norm(p))
            err = max(err, du, abs(uv[1] - v), abs(dist - d) / d)
    return err


def pin_proj_jacobian_fd(O, lib):
    from paper_2303_16878_gb300 import synth
    rng = np.random.default_rng(12)
    err = 0.0
    for s in (synth.pinhole_sensor(160, 120, 120.0, 80.0, 60.0), synth.spherical_sensor(1024, 64, 16.6, -16.6)):
        for _ in range(50):
            p = rng.normal(0, 3, 3)
            p[2] = abs(p[2]) + 1.0 if s.model == 0 else p[2] * 0.2
            J = O.proj_jacobian(s, p, lib=lib)
            h = 1e-6
            Jf = np.zeros((2, 3))
            for a in range(3):
                d = np.zeros(3)
                d[a] = h
                Jf[:, a] = (O.project(s, p + d, lib=lib) - O.project(s, p - d, lib=lib)) / (2 * h)
            err = max(err, float(np.abs(J - Jf).max() / np.abs(Jf).max()))
    return err


def pin_boxplus(O, lib):
    """X [+] dx = X exp(dx): the 4x4 product of X with [R(dq) dt; 0 1], R(dq)
    the rotation of the unit quaternion with imaginary part dq (scipy)."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(13)
    err = 0.0
    for _ in range(50):
        X = np.zeros((3, 4))
        X[:, :3] = Rotation.from_rotvec(rng.normal(0, 1, 3)).as_matrix()
        X[:, 3] = rng.normal(0, 2, 3)
        dx = np.concatenate([rng.normal(0, 0.5, 3), rng.normal(0, 0.2, 3)])
        q = dx[3:]
        qw = math.sqrt(1.0 - float(q @ q))
        dR = Rotation.from_quat([q[0], q[1], q[2], qw]).as_matrix()
        E = np.eye(4)
        E[:3, :3] = dR
        E[:3, 3] = dx[:3]
        X4 = np.eye(4)
        X4[:3] = X
        ref = (X4 @ E)[:3]
        err = max(err, float(np.abs(O.boxplus(X, dx, lib=lib) - ref).max()))
    # |dq| >= 1 has no unit quaternion with imaginary part dq: the reading
    # normalises (1, dq), the quaternion scipy builds from (dq, 1)
    for _ in range(20):
        X = np.zeros((3, 4))
        X[:, :3] = Rotation.from_rotvec(rng.normal(0, 1, 3)).as_matrix()
        X[:, 3] = rng.normal(0, 2, 3)
        q = rng.normal(0, 1, 3)
        q *= rng.uniform(1.0, 3.0) / np.linalg.norm(q)
        dx = np.concatenate([rng.normal(0, 0.5, 3), q])
        E = np.eye(4)
        E[:3, :3] = Rotation.from_quat([q[0], q[1], q[2], 1.0]).as_matrix()
        E[:3, 3] = dx[:3]
        X4 = np.eye(4)
        X4[:3] = X
        err = max(err, float(np.abs(O.boxplus(X, dx, lib=lib) - (X4 @ E)[:3]).max()))
    # X [+] 0 = X
    err = max(err, float(np.abs(O.boxplus(X, np.zeros(6), lib=lib) - X).max()))
    return err


def _fd_point_jacobians(O, lib, w, params, n_points=300, h=1e-6, seed=0, pairs=((0, 1), (1, 2))):
    rng = np.random.default_rng(seed)
    s = w.sensors[0]
    worst, used = 0.0, 0
    for i, j in pairs:
        pts, _ = O.frame_points(s, params, w.channels[i], lib=lib)
        Xi, Xj = w.poses_init[i], w.poses_init[j]
        for k in rng.permutation(len(pts))[:n_points]:
            r = O.point_residual(s, params, w.channels[j], Xi, Xj, pts[k], lib=lib)
            if not r["valid"] or r["flag"]:
                continue
            Jfi, Jfj, ok = np.zeros((5, 6)), np.zeros((5, 6)), True
            for a in range(6):
                d = np.zeros(6)
                d[a] = h
                ev = [O.point_residual(s, params, w.channels[j], O.boxplus(Xi, sg * d, lib=lib), Xj, pts[k], lib=lib)
                      for sg in (1, -1)]
                ev += [O.point_residual(s, params, w.channels[j], Xi, O.boxplus(Xj, sg * d, lib=lib), pts[k], lib=lib)
                       for sg in (1, -1)]
                if not all(e["valid"] for e in ev):
                    ok = False
                    break
                Jfi[:, a] = (ev[0]["e"] - ev[1]["e"]) / (2 * h)
                Jfj[:, a] = (ev[2]["e"] - ev[3]["e"]) / (2 * h)
            if not ok:
                continue
            used += 1
            scale = max(np.abs(Jfi).max(), np.abs(Jfj).max(), 1e-12)
            worst = max(worst, float(np.abs(Jfi - r["Ji"]).max() / scale),
                        float(np.abs(Jfj - r["Jj"]).max() / scale))
    assert used >= 20, "too few usable points for the finite-difference check"
    return worst


def pin_jacobian_fd(O, lib, w):
    """J_i, J_j (Supp.) against central differences of e under X [+] dx,
    with the exact derivative of the bilinear interpolant (grad_mode 1)."""
    params = dict(w.params, grad_mode=1)
    return _fd_point_jacobians(O, lib, w, params)


def ramp_workload(model=0):
    """Two frames whose target channels are affine in the pixel coordinates
    (intensity and depth ramps, constant unit normal): central differences
    equal the exact gradient and bilinear interpolation is exact, so the
    paper's image Jacobians (grad_mode 0) are the true derivatives."""
    from paper_2303_16878_gb300 import synth
    if model == 0:
        s = synth.pinhole_sensor(64, 48, 50.0, 32.0, 24.0)
    else:
        s = synth.spherical_sensor(256, 32, 15.0, -15.0)
    H, W = s.height, s.width
    cols = np.arange(W)[None, :].astype(np.float64)
    rows = np.arange(H)[:, None].astype(np.float64)
    def img(g0, gc, gr, d0, dc, dr, n):
        c = np.zeros((H, W, 5), dtype=np.float32)
        c[..., 0] = g0 + gc * cols + gr * rows
        c[..., 1] = d0 + dc * cols + dr * rows
        c[..., 2:] = np.asarray(n, dtype=np.float32)
        return c
    # dyadic slopes and offsets keep every texel exactly affine in float32
    if model == 0:
        src = img(0.25, 2.0 ** -8, -2.0 ** -9, 2.0, 0.0, 0.0, (0.0, 0.0, -1.0))
        tgt = img(0.3125, 2.0 ** -7, 2.0 ** -8, 2.125, 2.0 ** -9, 2.0 ** -10, (0.0, 0.0, -1.0))
    else:
        # columns wrap at the seam, where no ramp is affine: keep only the
        # middle half of the azimuth range valid, far from the seam
        src = img(0.25, 2.0 ** -10, 2.0 ** -7, 10.0, 2.0 ** -9, 2.0 ** -5, (-1.0, 0.0, 0.0))
        tgt = img(0.3125, 2.0 ** -9, 2.0 ** -6, 10.25, 2.0 ** -8, 2.0 ** -4, (-1.0, 0.0, 0.0))
        for c in (src, tgt):
            c[:, : W // 4] = 0.0
            c[:, 3 * W // 4:] = 0.0
    X0 = synth.IDENTITY_3x4.copy()
    X1 = synth.IDENTITY_3x4.copy()
    X1[:, :3] = synth.rot_vec(np.array([0.01, -0.02, 0.015]))
    X1[:, 3] = (0.03, -0.02, 0.04)
    poses = np.stack([X0, X1])
    params = synth.default_params(occ_abs=10.0, occ_rel=1.0, huber_delta=1e9, grad_mode=0)
    return synth.Workload("ramp", [s], np.zeros(2, dtype=np.int32), [src, tgt], poses, poses.copy(),
                          np.array([[0, 1]], dtype=np.int32), params)


def pin_ramp_grad_mode0(O, lib):
    worst = 0.0
    for model in (0, 1):
        w = ramp_workload(model)
        worst = max(worst, _fd_point_jacobians(O, lib, w, w.params, n_points=200, pairs=((0, 1),)))
    return worst


def gauge_directions(poses):
    """The six infinitesimal global motions G = exp(eps xi) applied as
    X_k -> G X_k, written in each frame's [dt, dq] coordinates:
    dt_k = R_k^T (rho + phi x t_k), dq_k = R_k^T phi / 2 (R(dq) ~ I + 2 [dq]x)."""
    V = []
    for xi in np.eye(6):
        rho, phi = xi[:3], xi[3:]
        v = []
        for X in poses:
            R, t = X[:, :3], X[:, 3]
            v.append(np.concatenate([R.T @ (rho + np.cross(phi, t)), 0.5 * R.T @ phi]))
        V.append(np.concatenate(v))
    return np.stack(V, axis=1)


def pin_gauge(O, lib, w):
    """H V = 0 and b^T V = 0 for the gauge directions V (either grad mode)."""
    worst = 0.0
    for gm in (0, 1):
        params = dict(w.params, grad_mode=gm)
        r = O.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params, lib=lib)
        V = gauge_directions(w.poses_init)
        H, b = r["H"], r["b"]
        worst = max(worst, float(np.linalg.norm(H @ V) / (np.linalg.norm(H) * np.linalg.norm(V))),
                    float(np.linalg.norm(b @ V) / (np.linalg.norm(b) * np.linalg.norm(V))))
    return worst


def pin_cost_gradient(O, lib, w):
    """dF / d dx_k (central differences of Eq. total-error-multicue under X_k [+] dx) equals 2 b_k
    (grad_mode 1, non-unit Omega, a Huber delta that some residuals exceed)."""
    params = dict(w.params, grad_mode=1, w_depth=0.5, w_normal=0.3, huber_delta=0.05)
    s = w.sensors[0]
    r = O.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params, lib=lib)
    b = r["b"]
    worst = 0.0
    for k in range(1, w.n_frames):
        for a in range(6):
            done = False
            # small steps: the bilinear interpolant has kinks at cell edges, and
            # a point crossing one within +-h biases the difference by O(h)
            for h in (2e-8, 1e-8, 5e-9):
                Fs, masks = [], []
                for sg in (1, -1):
                    d = np.zeros(6)
                    d[a] = sg * h
                    poses = w.poses_init.copy()
                    poses[k] = O.boxplus(poses[k], d, lib=lib)
                    F, mk = 0.0, []
                    for (i, j) in w.pairs.tolist():
                        if k not in (i, j):
                            continue
                        pr = O.linearize_pair(s, params, w.channels[i], w.channels[j], poses[i], poses[j], lib=lib)
                        F += pr["cost"]
                        mk.append(pr["mask"])
                    Fs.append(F)
                    masks.append(mk)
                if all(np.array_equal(x, y) for x, y in zip(masks[0], masks[1])):
                    g = (Fs[0] - Fs[1]) / (2 * h)
                    worst = max(worst, abs(g - 2 * b[6 * k + a]) / (np.abs(2 * b[6 * k:6 * k + 6]).max() + 1e-30))
                    done = True
                    break
            assert done, "mask changed under every finite-difference step"
    return worst


def pin_plane_shift(O, lib):
    """Integer-pixel shift of a fronto-parallel plane: every residual is 0."""
    from paper_2303_16878_gb300 import synth
    w = synth.make_plane_shift()
    s = w.sensors[0]
    pts, _ = O.frame_points(s, w.params, w.channels[0], lib=lib)
    worst, used = 0.0, 0
    for k in range(0, len(pts), 3):
        r = O.point_residual(s, w.params, w.channels[1], w.poses_gt[0], w.poses_gt[1], pts[k], lib=lib)
        if r["valid"]:
            used += 1
            worst = max(worst, float(np.abs(r["e"]).max()))
    assert used > 100
    return worst


def pin_single_channel(O, lib):
    """With Omega = diag(1, 0, 0, 0, 0), rho = identity and no occlusion test,
    F equals the classic photometric error of Eq. total-error summed by brute force:
    u' from Eq. uprime composed as X_j^-1 X_i, I_j^g(u') by scipy's order-1 spline
    (bilinear), over the source pixels whose samples are usable."""
    from scipy.ndimage import map_coordinates
    from paper_2303_16878_gb300 import synth
    w = synth.make_plane_shift(shift_px=(0, 0))
    X1 = synth.IDENTITY_3x4.copy()
    X1[:, :3] = synth.rot_vec(np.array([0.004, -0.006, 0.01]))
    X1[:, 3] = (0.0731, -0.0417, 0.05)
    poses = np.stack([synth.IDENTITY_3x4, X1])
    s = w.sensors[0]
    params = dict(w.params, w_depth=0.0, w_normal=0.0, huber_delta=1e12, occ_abs=1e6, occ_rel=0.0)
    r = O.linearize(w.sensors, w.frame_sensor, w.channels, poses, w.pairs, params, want_system=False, lib=lib)
    src, tgt = w.channels[0].astype(np.float64), w.channels[1].astype(np.float64)
    A = np.eye(4)
    A[:3] = poses[1]
    Bm = np.eye(4)
    Bm[:3] = poses[0]
    Xji = np.linalg.inv(A) @ Bm
    total, n = 0.0, 0
    for row in range(s.height):
        for col in range(s.width):
            d = src[row, col, 1]
            if d <= 0:
                continue
            p = np.array([(col - s.cx) / s.fx * d, (row - s.cy) / s.fy * d, d, 1.0])
            q = Xji @ p
            u, v = s.fx * q[0] / q[2] + s.cx, s.fy * q[1] / q[2] + s.cy
            if not (1 <= u < s.width - 2 and 1 <= v < s.height - 2):
                continue
            gj = map_coordinates(tgt[..., 0], [[v], [u]], order=1)[0]
            total += (src[row, col, 0] - gj) ** 2
            n += 1
    assert n == r["count"], (n, r["count"])
    return abs(total - r["cost"]) / max(total, 1e-30)


def pin_extrinsic_equivalence(O, lib, w):
    """Supp. offset form: with extrinsic X_o and platform poses X_k the error
    equals the error with no offset and sensor poses X_k X_o (composed here
    with numpy), point by point; compare cost and count of every pair."""
    from paper_2303_16878_gb300 import synth
    Xo = synth.offset_transform(0.3, 20.0, seed=9)  # a large offset, so mistakes are visible
    wx = synth.with_extrinsic(w, Xo)
    a = O.linearize(wx.sensors, wx.frame_sensor, wx.channels, wx.poses_init, wx.pairs, wx.params,
                    want_system=False, want_pairs=True, lib=lib)
    sensor_poses = np.stack([synth.compose(X, Xo) for X in wx.poses_init])
    b = O.linearize(w.sensors, w.frame_sensor, w.channels, sensor_poses, w.pairs, w.params,
                    want_system=False, want_pairs=True, lib=lib)
    assert b["count"] > 0
    if not np.array_equal(a["pair_count"], b["pair_count"]):
        return float(np.abs(a["pair_count"] - b["pair_count"]).max())
    return float(np.abs(a["pair_cost"] - b["pair_cost"]).max() / max(np.abs(b["pair_cost"]).max(), 1e-30))


def pin_jacobian_fd_extrinsic(O, lib, w):
    """J_i, J_j against central differences with a non-identity offset X_o."""
    from paper_2303_16878_gb300 import synth
    wx = synth.with_extrinsic(w, synth.offset_transform(0.3, 20.0, seed=9))
    return _fd_point_jacobians(O, lib, wx, dict(wx.params, grad_mode=1))


def pin_cholesky(O, lib):
    rng = np.random.default_rng(14)
    worst = 0.0
    for n in (1, 5, 42, 120):
        B = rng.normal(size=(n, n))
        A = B @ B.T + n * np.eye(n)
        rhs = rng.normal(size=n)
        x = O.cholesky_solve(A, rhs, lib=lib)
        ref = np.linalg.solve(A, rhs)
        worst = max(worst, float(np.abs(x - ref).max() / np.abs(ref).max()))
    return worst


# ---------------------------------------------------------------- normals (Sec. IV-A)

def _plane_depth(s, n, c):
    """Depth image of the plane n . p = c seen by sensor s (closed form: the
    ray p = z r (pinhole, r = K^-1 [u v 1]) or p = rho r (spherical, r the unit
    ray), so z = c / (n . r)); 0 where the plane lies behind."""
    H, W = s.height, s.width
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    if s.model == 0:
        r = np.stack([(u - s.cx) / s.fx, (v - s.cy) / s.fy, np.ones_like(u)], -1)
    else:
        az, el = (u - s.cx) / s.fx, (v - s.cy) / s.fy
        r = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1)
    den = r @ np.asarray(n, dtype=np.float64)
    z = np.where(np.abs(den) > 1e-9, c / np.where(np.abs(den) > 1e-9, den, 1.0), -1.0)
    ch = np.zeros((H, W, 5))
    ch[..., 1] = np.where((z > 0) & (z < 50.0), z, 0.0)
    return ch


def pin_normals_plane(O, lib=None):
    """Points of one plane: every pixel gets exactly the plane's normal, turned
    towards the sensor (n . p < 0), for a pinhole and a spherical sensor and
    radii varying with the depth.  Returns the largest |n - n_true| (inf if a
    valid pixel with at least 5 neighbours got no normal, or another one did)."""
    from paper_2303_16878_gb300 import synth
    cases = [(synth.pinhole_sensor(48, 40, 40.0, 23.5, 19.5), np.array([0.3, -0.2, 0.93]), 2.5, 6.0, 4),
             (synth.spherical_sensor(96, 16, 10.0, -25.0), np.array([0.1, 0.05, 1.0]), -1.7, 12.0, 5)]
    worst = 0.0
    for s, n, c, scale, rmax in cases:
        n = n / np.linalg.norm(n)
        ch = _plane_depth(s, n, c * np.linalg.norm(n))
        out = O.estimate_normals(s, ch, scale, rmax, lib=lib)
        valid = (ch[..., 1] > 0) & (out["count"] >= 5)
        has = np.linalg.norm(out["normals"], axis=-1) > 0
        if not np.array_equal(valid, has) or valid.sum() < 100:
            return float("inf")
        toward = -n if c > 0 else n  # the sensor sits on the side n . p < c
        worst = max(worst, float(np.abs(out["normals"][valid] - toward).max()))
    return worst


# Lattice points (a, b) with a^2 + b^2 < r^2, counted by hand: 9 for r = 1.5
# (the 3 x 3 block), 21 for r = 2.5, 69 for r = 5 (81 points with a^2 + b^2 <= 25
# minus the 12 on the circle).  The half disc b >= 0 holds 6, 13 and 39 of
# them (rows b = 0..4 of r = 5: 9 + 9 + 9 + 7 + 5); the quarter disc a, b >= 0
# of r = 2.5 holds 8.
LATTICE_DISC = {1.5: 9, 2.5: 21, 5.0: 69}
LATTICE_HALF = {1.5: 6, 2.5: 13, 5.0: 39}
LATTICE_QUARTER_2_5 = 8


def pin_normals_counts(O, lib=None):
    """Neighbourhood sizes |U| on constant-depth images: interior pixels use the
    full disc of radius clamp(scale / d, 1.5, max_radius); a pinhole corner
    uses a quarter disc; a spherical image wraps its columns, so column 0 of
    an interior row uses the full disc.  Returns the number of mismatches."""
    from paper_2303_16878_gb300 import synth
    bad = 0
    for model in (0, 1):
        s = (synth.pinhole_sensor(24, 20, 20.0, 11.5, 9.5) if model == 0
             else synth.spherical_sensor(64, 20, 15.0, -15.0))
        for d, scale, rmax, r in ((4.0, 4.0, 4, 1.5), (2.0, 5.0, 4, 2.5), (1.0, 10.0, 5, 5.0), (0.5, 10.0, 5, 5.0)):
            ch = np.zeros((s.height, s.width, 5))
            ch[..., 1] = d
            N = O.estimate_normals(s, ch, scale, rmax, lib=lib)["count"]
            bad += int(N[10, 12] != LATTICE_DISC[r])
            edge = LATTICE_DISC[r] if model == 1 else LATTICE_HALF[r]
            bad += int(N[10, 0] != edge) + int(N[10, s.width - 1] != edge)
            if r == 2.5 and model == 0:
                bad += int(N[0, 0] != LATTICE_QUARTER_2_5)
    return float(bad)


def pin_normals_brute_force(O, lib, w, stride=5):
    """Every stride-th pixel of frame 0 of w: the neighbour set enumerated pixel
    by pixel, the points unprojected with the closed forms of Sec. III, and the
    best-fitting plane taken from numpy's SVD of the centred points (the
    singular vector of the smallest singular value).  Compared where the two
    smallest singular values are well apart; returns the largest |n - n_bf|."""
    s = w.sensors[0]
    ch = w.channels[0]
    scale, rmax = (6.0, 4) if s.model == 0 else (8.0, 4)
    out = O.estimate_normals(s, ch, scale, rmax, params=w.params, lib=lib)
    H, W = s.height, s.width
    d = ch[..., 1].astype(np.float64)
    valid = (d > 0) & (d >= w.params["range_min"]) & (d <= w.params["range_max"])

    def point(r, c):
        if s.model == 0:
            return d[r, c] * np.array([(c - s.cx) / s.fx, (r - s.cy) / s.fy, 1.0])
        az, el = (c - s.cx) / s.fx, (r - s.cy) / s.fy
        return d[r, c] * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])

    worst, used = 0.0, 0
    for k in range(0, H * W, stride):
        r0, c0 = divmod(k, W)
        if not valid[r0, c0]:
            continue
        rad = min(max(scale / d[r0, c0], 1.5), float(rmax))
        pts = []
        for r in range(max(0, r0 - rmax), min(H, r0 + rmax + 1)):
            for c in (range(W) if s.model == 1 else range(max(0, c0 - rmax), min(W, c0 + rmax + 1))):
                dc = c - c0
                if s.model == 1:
                    dc = min(abs(dc), W - abs(dc))
                if (r - r0) ** 2 + dc ** 2 < rad * rad and valid[r, c]:
                    pts.append(point(r, c))
        if len(pts) != out["count"][r0, c0]:
            return float("inf")
        if len(pts) < 5:
            continue
        X = np.array(pts)
        X -= X.mean(axis=0)
        _, sv, vt = np.linalg.svd(X)
        if sv[1] - sv[2] < 1e-3 * sv[0]:
            continue
        nb = vt[2] if np.dot(vt[2], point(r0, c0)) <= 0 else -vt[2]
        worst = max(worst, float(np.abs(out["normals"][r0, c0] - nb).max()))
        used += 1
    return worst if used > 200 else float("inf")


def pin_normals_degenerate(O, lib=None):
    """No normal where the plane is undetermined: a single valid row of a
    pinhole image (collinear points), and valid pixels isolated on a grid of
    pitch 3 (a neighbourhood of radius below 3 holds only the pixel itself).  Returns
    the number of pixels that got a normal."""
    from paper_2303_16878_gb300 import synth
    s = synth.pinhole_sensor(32, 24, 30.0, 15.5, 11.5)
    n_bad = 0
    ch = _plane_depth(s, np.array([0.0, 0.0, 1.0]), 2.0)
    ch[np.arange(24) != 12, :, 1] = 0.0
    n_bad += int(np.count_nonzero(np.linalg.norm(O.estimate_normals(s, ch, 5.0, 4, lib=lib)["normals"], axis=-1)))
    ch = _plane_depth(s, np.array([0.2, 0.1, 1.0]) / np.linalg.norm([0.2, 0.1, 1.0]), 2.0)
    keep = np.zeros((24, 32), dtype=bool)
    keep[::3, ::3] = True
    ch[~keep, 1] = 0.0
    out = O.estimate_normals(s, ch, 5.0, 4, lib=lib)  # r = clamp(5 / d, ...) is about 2.5
    n_bad += int(np.count_nonzero(np.linalg.norm(out["normals"], axis=-1)))
    return float(n_bad)


# ---------------------------------------------------------------- pyramid (Sec. IV-A) and coarse to fine (Sec. IV-C)

def pin_pyramid_projection(O, lib=None):
    """Coarse pixel k covers fine pixels 2k, 2k + 1 and is centred on fine
    coordinate 2k + 1/2, so any point projects to u_c = (u_f + 1/2) / 2 - 1/2
    (and v alike) at the next level, for both models.  Returns the largest
    deviation in coarse pixels over seeded points."""
    from paper_2303_16878_gb300 import synth
    rng = np.random.default_rng(11)
    worst = 0.0
    for s in (synth.pinhole_sensor(160, 120, 120.0, 80.0, 60.0), synth.spherical_sensor(1024, 64, 16.6, -16.6)):
        c = O.downsample_sensor(s)
        if (c["width"], c["height"]) != (s.width // 2, s.height // 2):
            return float("inf")
        for _ in range(200):
            p = rng.normal(size=3) * 3.0
            p[2] = abs(p[2]) + 0.5 if s.model == 0 else p[2]
            uf = O.project(s, p, lib=lib)
            uc = O.project(c, p, lib=lib)
            du = abs(uc[0] - ((uf[0] + 0.5) / 2 - 0.5))
            if s.model == 1:  # the azimuth wraps with period W / 2 at the coarse level
                du = min(du, abs(du - c["width"]))
            worst = max(worst, du, abs(uc[1] - ((uf[1] + 0.5) / 2 - 0.5)))
    return worst


def pin_downsample_closed_forms(O, lib=None):
    """Closed forms of the 2 x 2 summary: a constant image stays constant; an
    affine intensity ramp g = a + b c + e r (dyadic, exact in float32) gives
    the ramp at the block centre (2r + 1/2, 2c + 1/2); four normals placed
    symmetrically about -z average to exactly -z; one invalid fine pixel
    invalidates its block only; odd sizes drop the last row and column.
    Returns the largest error (inf on a validity mismatch)."""
    prm = dict(range_min=0.0, range_max=100.0)
    H, W = 7, 9
    x = np.zeros((H, W, 5), dtype=np.float32)
    r, c = np.mgrid[0:H, 0:W]
    x[..., 0] = 0.25 + 0.0625 * c + 0.03125 * r
    x[..., 1] = 2.5
    x[..., 4] = -1.0
    y = O.downsample(x, prm)
    if y.shape != (3, 4, 5):
        return float("inf")
    rc, cc = np.mgrid[0:3, 0:4]
    err = float(np.abs(y[..., 0] - (0.25 + 0.0625 * (2 * cc + 0.5) + 0.03125 * (2 * rc + 0.5))).max())
    err = max(err, float(np.abs(y[..., 1] - 2.5).max()), float(np.abs(y[..., 2:] - [0, 0, -1]).max()))
    a = 0.6
    b = math.sqrt(1 - a * a)
    x[0:2, 0:2, 2:5] = np.array([[[a, 0, -b], [-a, 0, -b]], [[0, a, -b], [0, -a, -b]]], dtype=np.float32)
    x[3, 5, 1] = 0.0  # block (1, 2) loses one pixel
    y = O.downsample(x, prm)
    err = max(err, float(np.abs(y[0, 0, 2:] - [0, 0, -1]).max()))
    valid = y[..., 1] > 0
    expect = np.ones((3, 4), dtype=bool)
    expect[1, 2] = False
    if not np.array_equal(valid, expect) or np.any(y[1, 2] != 0):
        return float("inf")
    return err


def _pose_error(P, G):
    """Largest translation [m] and rotation [rad] error of the poses relative
    to frame 0 (the gauge) against ground truth."""
    P = np.asarray(P).reshape(-1, 3, 4)
    G = np.asarray(G).reshape(-1, 3, 4)

    def h(X):
        return np.vstack([X, [0, 0, 0, 1]])
    et = er = 0.0
    for k in range(1, len(P)):
        D = np.linalg.inv(np.linalg.inv(h(G[0])) @ h(G[k])) @ (np.linalg.inv(h(P[0])) @ h(P[k]))
        et = max(et, float(np.linalg.norm(D[:3, 3])))
        er = max(er, float(np.arccos(np.clip((np.trace(D[:3, :3]) - 1) / 2, -1, 1))))
    return et, er


def pin_coarse_to_fine(O, lib=None):
    """Brute-force convergence on a tiny problem: from 4.7 cm / 2.9 deg
    initial errors, three levels of 10 / 5 / 2 iterations reach the ground
    truth within 1 cm and 0.3 deg (the interpolation-limited optimum of
    rendered images), and F never increases within a level.  Returns the
    number of violated conditions."""
    from paper_2303_16878_gb300 import synth
    w = synth.make_rgbd_room(n_frames=4, width=160, height=120, f=120.0)
    r = O.coarse_to_fine(w, w.poses_init, 3, [10, 5, 2], 1e-4, lib=lib)
    et, er = _pose_error(r["poses"], w.poses_gt)
    bad = int(et > 0.01) + int(er > math.radians(0.3))
    bad += sum(int(lv["cost_last"] > lv["cost_first"]) for lv in r["log"])
    bad += int([lv["level"] for lv in r["log"]] != [2, 1, 0])
    return float(bad)


# ---------------------------------------------------------------- pose variables (frames sharing a pose)

def pin_tied_gradient(O, lib, w):
    """Frames of several sensors captured at one platform pose move together
    (w.frame_var): the derivative of F under the common perturbation
    X_f [+] dx for every frame f of variable v (central differences) equals
    2 (S^T b)_v.  Returns the largest relative deviation."""
    params = dict(w.params, grad_mode=1)
    r = O.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params, lib=lib)
    S = O.selection(w.frame_var, w.n_vars)
    br = S.T @ r["b"]
    worst = 0.0
    for v in range(w.n_vars):
        frames = [k for k in range(w.n_frames) if w.frame_var[k] == v]
        for a in range(6):
            done = False
            for h in (2e-8, 1e-8, 5e-9):
                Fs, masks = [], []
                for sg in (1, -1):
                    d = np.zeros(6)
                    d[a] = sg * h
                    poses = w.poses_init.copy()
                    for k in frames:
                        poses[k] = O.boxplus(poses[k], d, lib=lib)
                    F, mk = 0.0, []
                    for (i, j) in w.pairs.tolist():
                        if i not in frames and j not in frames:
                            continue
                        s = w.sensors[int(w.frame_sensor[i])]
                        pr = O.linearize_pair(s, params, w.channels[i], w.channels[j], poses[i], poses[j], lib=lib)
                        F += pr["cost"]
                        mk.append(pr["mask"])
                    Fs.append(F)
                    masks.append(mk)
                if all(np.array_equal(x, y) for x, y in zip(masks[0], masks[1])):
                    g = (Fs[0] - Fs[1]) / (2 * h)
                    worst = max(worst, abs(g - 2 * br[6 * v + a]) / (np.abs(2 * br[6 * v:6 * v + 6]).max() + 1e-30))
                    done = True
                    break
            assert done, "mask changed under every finite-difference step"
    return worst


def pin_variables_reduce_to_gauge(O, lib, w):
    """With frame_var = (-1, 0, 1, ..., N - 2) the variable-space step is the
    gauge-fixed step (frame 0 removed from H, Sec. IV-C).  Returns the
    largest difference of the two dx."""
    r = O.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, w.params, lib=lib)
    lam = O.initial_lambda(r["H"])
    fv = np.arange(-1, w.n_frames - 1)
    if abs(O.initial_lambda_vars(r["H"], fv, w.n_frames - 1) - lam) > 1e-15 * lam:
        return float("inf")
    a, ok_a = O.solve_step(r["H"], r["b"], lam, lib=lib)
    b, ok_b = O.solve_step_vars(r["H"], r["b"], lam, fv, w.n_frames - 1, lib=lib)
    if not (ok_a and ok_b):
        return float("inf")
    return float(np.abs(a - b).max() / np.abs(a).max())


# ---------------------------------------------------------------- the sensor offset as a variable (R23)

def _with_offset(w):
    from paper_2303_16878_gb300 import synth
    return synth.with_extrinsic(w, synth.offset_transform(0.3, 20.0, seed=9))


def _sensor_with(s, X):
    import dataclasses
    return dataclasses.replace(s, extrinsic=np.asarray(X, dtype=np.float64).reshape(3, 4))


def pin_offset_jacobian_fd(O, lib, w, n_points=200, h=1e-6, seed=3):
    """J_o = (J_i + J_j) A_o against central differences of e under X_o [+] d
    (points rebuilt from the same pixels with the perturbed offset), grad_mode 1."""
    wx = _with_offset(w)
    params = dict(wx.params, grad_mode=1)
    s = wx.sensors[0]
    Xo = np.asarray(s.extrinsic)
    rng = np.random.default_rng(seed)
    worst, used = 0.0, 0
    i, j = 0, 1
    pts, _ = O.frame_points(s, params, wx.channels[i], lib=lib)
    Xi, Xj = wx.poses_init[i], wx.poses_init[j]
    shifted = {}
    for a in range(6):
        for sg in (1, -1):
            d = np.zeros(6)
            d[a] = sg * h
            sp = _sensor_with(s, O.boxplus(Xo, d, lib=lib))
            shifted[(a, sg)] = (sp, O.frame_points(sp, params, wx.channels[i], lib=lib)[0])
    for k in rng.permutation(len(pts))[:n_points]:
        r = O.point_residual(s, params, wx.channels[j], Xi, Xj, pts[k], lib=lib)
        if not r["valid"] or r["flag"]:
            continue
        Jo = O.offset_jacobian(Xo, r["Ji"], r["Jj"])
        Jf, ok = np.zeros((5, 6)), True
        for a in range(6):
            ev = []
            for sg in (1, -1):
                sp, pp = shifted[(a, sg)]
                ev.append(O.point_residual(sp, params, wx.channels[j], Xi, Xj, pp[k], lib=lib))
            if not all(e["valid"] for e in ev):
                ok = False
                break
            Jf[:, a] = (ev[0]["e"] - ev[1]["e"]) / (2 * h)
        if not ok:
            continue
        used += 1
        worst = max(worst, float(np.abs(Jf - Jo).max() / max(np.abs(Jf).max(), 1e-12)))
    assert used >= 20, "too few usable points for the finite-difference check"
    return worst


def pin_offset_gradient_fd(O, lib, w):
    """dF / d d_o (central differences of F over all pairs under X_o [+] d)
    equals 2 sum_pairs b_o (pair_offset_blocks), grad_mode 1."""
    wx = _with_offset(w)
    params = dict(wx.params, grad_mode=1)
    s = wx.sensors[0]
    Xo = np.asarray(s.extrinsic)
    bo = sum(O.pair_offset_blocks(s, params, wx.channels[i], wx.channels[j], wx.poses_init[i], wx.poses_init[j],
                                  lib=lib)["b_o"] for i, j in wx.pairs.tolist())
    worst = 0.0
    for a in range(6):
        done = False
        for h in (2e-8, 1e-8, 5e-9):
            Fs, cnt = [], []
            for sg in (1, -1):
                d = np.zeros(6)
                d[a] = sg * h
                sp = _sensor_with(s, O.boxplus(Xo, d, lib=lib))
                r = O.linearize([sp], wx.frame_sensor, wx.channels, wx.poses_init, wx.pairs, params,
                                want_system=False, want_pairs=True, lib=lib)
                Fs.append(r["cost"])
                cnt.append(r["pair_count"])
            if np.array_equal(cnt[0], cnt[1]):
                g = (Fs[0] - Fs[1]) / (2 * h)
                worst = max(worst, abs(g - 2 * bo[a]) / (np.abs(2 * bo).max() + 1e-30))
                done = True
                break
        assert done, "validity changed under every finite-difference step"
    return worst


# ------------------------------------------------- the residual by brute force

def _h44(X):
    M = np.eye(4)
    M[:3] = np.asarray(X, dtype=np.float64).reshape(3, 4)
    return M


def _bf_residuals(s, params, src, tgt, Xi, Xj, pix):
    """Residuals of the source pixels `pix` (row * W + col) of image `src`
    against `tgt`, evaluated from the definitions with homogeneous 4 x 4
    matrices and scipy's order-1 spline, vectorised over the points:
    p_u = X_o pi^-1(u, d) (Sec. III), pbar = X_o^-1 X_j^-1 X_i p_u (Eq. uprime),
    u' = pi(pbar), a pixel valid iff range_min <= d <= range_max, d > 0 and
    |n| > 0.5 (Sec. IV-A), a texel usable iff it and its four neighbours are
    valid, the four bilinear taps usable (pinhole window 1 <= u' < W - 2, every
    model 1 <= v' < H - 2, spherical columns wrapping), zeta = (g_u, depth or
    range of pbar, rotated n_u) (Supp.), the occlusion and target-normal tests,
    chi^2 = e^T Omega e and the Huber rho of Eq. total-error-multicue.
    Returns (valid, e, rho, reason) with reason 0 valid, 1 depth limit,
    2 window, 3 not usable, 4 occlusion, 5 target normal."""
    from scipy.ndimage import map_coordinates
    H, W = s.height, s.width
    src = src.astype(np.float64)
    tgt64 = tgt.astype(np.float64)
    rows, cols = pix // W, pix % W
    d = src[rows, cols, 1]
    u0, v0 = cols.astype(np.float64), rows.astype(np.float64)
    if s.model == 0:
        p = np.stack([(u0 - s.cx) / s.fx * d, (v0 - s.cy) / s.fy * d, d], axis=1)
    else:
        az, el = (u0 - s.cx) / s.fx, (v0 - s.cy) / s.fy
        p = d[:, None] * np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=1)
    Xo = _h44(s.extrinsic)
    A = np.linalg.inv(Xo) @ np.linalg.inv(_h44(Xj)) @ _h44(Xi) @ Xo
    pb = p @ A[:3, :3].T + A[:3, 3]
    nb = src[rows, cols, 2:5] @ A[:3, :3].T
    if s.model == 0:
        zeta_d = pb[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = s.fx * pb[:, 0] / pb[:, 2] + s.cx
            v = s.fy * pb[:, 1] / pb[:, 2] + s.cy
    else:
        zeta_d = np.linalg.norm(pb, axis=1)
        u = s.fx * np.arctan2(pb[:, 1], pb[:, 0]) + s.cx
        v = s.fy * np.arctan2(pb[:, 2], np.hypot(pb[:, 0], pb[:, 1])) + s.cy
    n2 = (tgt64[..., 2:5] ** 2).sum(-1)
    dt = tgt64[..., 1]
    valid_px = (dt > 0) & (dt >= params["range_min"]) & (dt <= params["range_max"]) & (n2 > 0.25)
    img = tgt64
    if params.get("texel_f16", 0):
        # R25: sampled intensity and normals are the binary16 values (numpy's IEEE conversion);
        # validity stays with the float32 channels
        img = tgt64.copy()
        for c in (0, 2, 3, 4):
            img[..., c] = tgt[..., c].astype(np.float16).astype(np.float64)
    if s.model == 1:  # wrap columns: three copies side by side, u shifted into the middle one
        valid_px = np.concatenate([valid_px] * 3, axis=1)
        img = np.concatenate([img] * 3, axis=1)
    usable = np.zeros_like(valid_px)
    usable[1:-1, 1:-1] = (valid_px[1:-1, 1:-1] & valid_px[:-2, 1:-1] & valid_px[2:, 1:-1]
                          & valid_px[1:-1, :-2] & valid_px[1:-1, 2:])
    reason = np.zeros(len(pix), dtype=np.int64)
    reason[~(zeta_d > params["z_min"])] = 1
    in_win = (v >= 1.0) & (v < H - 2)
    if s.model == 0:
        in_win &= (u >= 1.0) & (u < W - 2)
    reason[(reason == 0) & ~in_win] = 2
    live = reason == 0
    uu = np.where(live, u + (W if s.model == 1 else 0), 1.0)
    vv = np.where(live, v, 1.0)
    c0, r0 = np.floor(uu).astype(np.int64), np.floor(vv).astype(np.int64)
    taps_ok = usable[r0, c0] & usable[r0, c0 + 1] & usable[r0 + 1, c0] & usable[r0 + 1, c0 + 1]
    reason[live & ~taps_ok] = 3
    I = np.stack([map_coordinates(img[..., c], [vv, uu], order=1) for c in range(5)], axis=1)
    occ = np.abs(zeta_d - I[:, 1]) > params["occ_abs"] + params["occ_rel"] * zeta_d
    reason[(reason == 0) & occ] = 4
    reason[(reason == 0) & (np.linalg.norm(I[:, 2:5], axis=1) < 0.5)] = 5
    e = np.column_stack([src[rows, cols, 0], zeta_d, nb]) - I
    om = np.array([params["w_int"], params["w_depth"]] + [params["w_normal"]] * 3)
    chi = np.sqrt((om * e * e).sum(1))
    delta = params["huber_delta"]
    rho = np.where(chi <= delta, chi * chi, 2 * delta * chi - delta * delta)
    return reason == 0, e, rho, reason, p @ Xo[:3, :3].T + Xo[:3, 3]


def _residual_case(O, lib, w, params, reasons, stride):
    s = w.sensors[0]
    Ro = np.asarray(s.extrinsic, dtype=np.float64).reshape(3, 4)[:, :3]
    om = np.array([params["w_int"], params["w_depth"]] + [params["w_normal"]] * 3)
    worst = 0.0
    for i, j in np.asarray(w.pairs)[:4]:
        pts, pix = O.frame_points(s, params, w.channels[i], lib=lib)
        pix = np.asarray(pix, dtype=np.int64)
        ok, e, rho, reason, pu = _bf_residuals(s, params, w.channels[i], w.channels[j],
                                               w.poses_init[i], w.poses_init[j], pix)
        src = w.channels[i].reshape(-1, 5).astype(np.float64)
        worst = max(worst, float(np.abs(pts[:, :3] - pu).max()),
                    float(np.abs(pts[:, 3] - src[pix, 0]).max()),
                    float(np.abs(pts[:, 4:7] - src[pix, 2:5] @ Ro.T).max()))
        for k in range(0, len(pix), stride):
            r = O.point_residual(s, params, w.channels[j], w.poses_init[i], w.poses_init[j], pts[k], lib=lib)
            if r["flag"]:
                continue
            reasons[reason[k]] += 1
            if r["valid"] != bool(ok[k]):
                return 1.0
            if r["valid"]:
                reasons[6] += int(rho[k] < e[k] @ (om * e[k]) - 1e-12)   # on the linear branch of Huber
                worst = max(worst, float(np.abs(r["e"] - e[k]).max()),
                            abs(r["rho"] - rho[k]) / max(1.0, abs(rho[k])))
    return worst


def _flipped_normal_columns(w, every=7):
    """Every `every`-th column of each image with its normal negated: bilinear
    samples between such a column and its neighbour have |n| < 0.5."""
    import dataclasses
    chans = []
    for c in w.channels:
        c = c.copy()
        c[:, ::every, 2:5] *= -1.0
        chans.append(c)
    return dataclasses.replace(w, channels=chans)


def pin_residual_brute_force(O, lib, room, street, stride=3):
    """Per-point validity, e and rho of the oracle against `_bf_residuals`, on
    the RGB-D room (with and without a sensor offset), the LiDAR street, and the
    room with flipped normal columns and z_min = 2 m, at thresholds that make
    every rejection rule and the Huber branch fire (tight occlusion bounds,
    delta below typical chi).  Points whose decision the oracle flags as within
    its margin are skipped; every other point must agree in validity, and valid
    points in e and rho.  The source points themselves (p_u, g_u, n_u^o) are
    checked against the same unprojection."""
    base = dict(w_depth=0.5, w_normal=0.3, huber_delta=0.05, occ_abs=0.02, occ_rel=0.01)
    reasons = np.zeros(7, dtype=np.int64)
    worst = 0.0
    for w, over in ((room, {}), (street, {}), (_with_offset(room), {}),
                    (_flipped_normal_columns(room), dict(z_min=2.0)), (room, dict(texel_f16=1)),
                    (street, dict(texel_f16=1))):
        worst = max(worst, _residual_case(O, lib, w, dict(w.params, **base, **over), reasons, stride))
    # valid, depth limit, window, not usable, occlusion, target normal, Huber's linear branch
    assert reasons[0] > 100 and np.all(reasons[1:] > 0), reasons
    return worst


# ------------------------------------------ J_j from J_i (relative-pose invariance)

def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def pin_relative_jacobian(O, lib, w, stride=7):
    """The residual depends on X_i, X_j only through A = X_j^-1 X_i (Eq.
    uprime), so a perturbation of X_j acts as a perturbation of X_i mapped by
    the adjoint of A^-1: J_j = J_i T with R = R_j^T R_i, t = R_j^T (t_i - t_j)
    and T = [[-R^T, 2 R^T [t]x], [0, -R^T]] in the box-plus chart (dq the
    quaternion's imaginary part, so rotations enter doubled).  Checked on the
    oracle's separately computed J_i and J_j over three pairs; returns the
    largest |J_j - J_i T| relative to max |J_j| of the point."""
    s = w.sensors[0]
    worst, used = 0.0, 0
    for i, j in ((0, 1), (1, 2), (2, 0)):
        Xi, Xj = w.poses_init[i], w.poses_init[j]
        R = Xj[:, :3].T @ Xi[:, :3]
        t = Xj[:, :3].T @ (Xi[:, 3] - Xj[:, 3])
        T = np.zeros((6, 6))
        T[:3, :3] = -R.T
        T[:3, 3:] = 2.0 * R.T @ _skew(t)
        T[3:, 3:] = -R.T
        pts, _ = O.frame_points(s, w.params, w.channels[i], lib=lib)
        for k in range(0, len(pts), stride):
            r = O.point_residual(s, w.params, w.channels[j], Xi, Xj, pts[k], lib=lib)
            if not r["valid"]:
                continue
            used += 1
            worst = max(worst, float(np.abs(r["Jj"] - r["Ji"] @ T).max() / max(np.abs(r["Jj"]).max(), 1e-30)))
    assert used > 100
    return worst


# ------------------------------------------- binary16 texel values (R25)

def pin_half_rounding(O, lib, n=20000, seed=9):
    """The oracle's binary16 rounding against numpy's IEEE conversion to
    float16 (round to nearest, ties to even): random values over the normal
    and subnormal ranges, exact midpoints between neighbouring binary16
    numbers (ties), values around the largest finite number and the overflow
    threshold, signed zeros.  Returns the number of mismatches."""
    rng = np.random.default_rng(seed)
    normal = rng.uniform(-2.0, 2.0, n).astype(np.float32)
    tiny = (rng.uniform(-1.0, 1.0, n) * 2.0 ** rng.integers(-26, -12, n)).astype(np.float32)
    h = rng.uniform(-1000.0, 1000.0, n).astype(np.float16)
    up = np.nextafter(h, np.float16(np.inf))
    ties = ((h.astype(np.float64) + up.astype(np.float64)) / 2).astype(np.float32)  # exact in float32
    edge = np.array([65504.0, 65519.0, 65520.0, 65535.0, -65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                     2.0 ** -14, 0.0, -0.0, 1.0, 0.5, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11], dtype=np.float32)
    x = np.concatenate([normal, tiny, ties, edge])
    assert np.count_nonzero(ties.astype(np.float16) == h) > n // 4  # half of the ties go down, to the even one
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    got = O.half_round(x, lib=lib)
    bad = ~((got == ref) | (np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref))))
    return int(np.count_nonzero(bad))


# ---------------------------------------------- the weights of H (Sec. IV-C)

def affine_plane_workload(shift_px=(2.75, 1.5), depth=2.0, f=40.0):
    """Two pinhole frames facing a fronto-parallel plane at constant depth,
    the second translated so that the image moves by a fractional number of
    pixels.  The intensity is affine in the pixel coordinates (dyadic slope,
    exact in binary16), so bilinear interpolation is exact at every sub-pixel
    position and the residual is zero at the true poses: pixel u of frame 0
    sees the plane point that frame 1 sees at u - shift."""
    from paper_2303_16878_gb300 import synth
    W, H = 48, 40
    s = synth.pinhole_sensor(W, H, f, W / 2.0, H / 2.0)
    cols = np.arange(W)[None, :].astype(np.float64)
    rows = np.arange(H)[:, None].astype(np.float64)

    def img(dc, dr):
        c = np.zeros((H, W, 5), dtype=np.float32)
        c[..., 0] = 0.25 + 2.0 ** -8 * (cols + dc) + 2.0 ** -9 * (rows + dr)
        c[..., 1] = depth
        c[..., 4] = -1.0
        return c
    X0 = synth.IDENTITY_3x4.copy()
    X1 = synth.IDENTITY_3x4.copy()
    X1[0, 3] = shift_px[0] * depth / f
    X1[1, 3] = shift_px[1] * depth / f
    poses = np.stack([X0, X1])
    params = synth.default_params(w_int=1.0, w_depth=0.5, w_normal=0.3, huber_delta=1e9, occ_abs=0.1,
                                  occ_rel=0.05)
    return synth.Workload("affine-plane", [s], np.zeros(2, dtype=np.int32), [img(0.0, 0.0), img(*shift_px)],
                          poses, poses.copy(), np.array([[0, 1]], dtype=np.int32), params)


def pin_hessian_zero_residual(O, lib, h=1e-5):
    """Where every residual is zero, the Gauss-Newton matrix of the LM normal
    equations (Sec. IV-C) is the exact Hessian of F / 2: d b / d dx = H, since
    b = sum w J^T Omega e and the terms with the derivative of J are
    multiplied by e = 0.  Central differences of the oracle's b under
    X_k [+] (+-h e_a) on the affine plane (non-unit Omega, both gradient
    modes; b itself is pinned as dF / d dx / 2 by the cost-gradient pin)
    must equal column 6 k + a of the oracle's H, for both frames; a weight
    left out of H or put into it twice (Omega, Huber), or a transposed block,
    moves H away from them.  Returns the largest difference relative to
    max |H|."""
    w = affine_plane_workload()
    s = w.sensors[0]
    worst = 0.0
    for gm in (0, 1):
        params = dict(w.params, grad_mode=gm)
        r0 = O.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_gt, w.pairs, params, lib=lib)
        assert r0["count"] > 800, r0["count"]
        assert np.abs(r0["b"]).max() < 1e-9 * np.abs(r0["H"]).max()
        H = r0["H"]
        for k in (0, 1):
            for a in range(6):
                bs, counts = [], []
                for sg in (1, -1):
                    d = np.zeros(6)
                    d[a] = sg * h
                    poses = w.poses_gt.copy()
                    poses[k] = O.boxplus(poses[k], d, lib=lib)
                    r = O.linearize(w.sensors, w.frame_sensor, w.channels, poses, w.pairs, params, lib=lib)
                    bs.append(r["b"])
                    counts.append(r["count"])
                assert counts[0] == counts[1] == r0["count"], "a point changed validity under the step"
                fd = (bs[0] - bs[1]) / (2 * h)
                worst = max(worst, float(np.abs(fd - H[:, 6 * k + a]).max() / np.abs(H).max()))
    return worst


def pin_huber_hessian(O, lib, w, n_each=12, h=1e-6, seed=5):
    """The Huber weight of the LM normal equations (Sec. IV-C; reading R1:
    w = 1 when chi <= delta, else delta / chi, chi = sqrt(e^T Omega e)): the
    12 x 12 block of a pair whose source image holds a single valid pixel
    equals w J^T Omega J, with J = [J_i J_j] from central differences of e
    under X [+] dx (grad_mode 1) and chi, hence w, from the brute-force
    residual `_bf_residuals`; neither comes from the oracle's accumulation.
    Points on both sides of delta are taken (n_each of each).  Returns the
    largest difference relative to max |H| of the point."""
    params = dict(w.params, grad_mode=1, w_depth=0.5, w_normal=0.3, huber_delta=0.05)
    om = np.array([params["w_int"], params["w_depth"]] + [params["w_normal"]] * 3)
    s = w.sensors[0]
    rng = np.random.default_rng(seed)
    worst, used = 0.0, [0, 0]
    i, j = 0, 1
    Xi, Xj = w.poses_init[i], w.poses_init[j]
    pts, pix = O.frame_points(s, params, w.channels[i], lib=lib)
    for k in rng.permutation(len(pts)):
        if min(used) >= n_each:
            break
        ok, e_bf, _, _, _ = _bf_residuals(s, params, w.channels[i], w.channels[j], Xi, Xj,
                                          np.array([pix[k]], dtype=np.int64))
        r = O.point_residual(s, params, w.channels[j], Xi, Xj, pts[k], lib=lib)
        if not ok[0] or not r["valid"] or r["flag"]:
            continue
        chi = float(np.sqrt(om @ (e_bf[0] * e_bf[0])))
        branch = int(chi > params["huber_delta"])
        if used[branch] >= n_each:
            continue
        J = np.zeros((5, 12))
        good = True
        for a in range(6):
            d = np.zeros(6)
            d[a] = h
            ev = [O.point_residual(s, params, w.channels[j], O.boxplus(Xi, sg * d, lib=lib), Xj, pts[k], lib=lib)
                  for sg in (1, -1)]
            ev += [O.point_residual(s, params, w.channels[j], Xi, O.boxplus(Xj, sg * d, lib=lib), pts[k], lib=lib)
                   for sg in (1, -1)]
            if not all(x["valid"] for x in ev):
                good = False
                break
            J[:, a] = (ev[0]["e"] - ev[1]["e"]) / (2 * h)
            J[:, 6 + a] = (ev[2]["e"] - ev[3]["e"]) / (2 * h)
        if not good:
            continue
        wt = 1.0 if chi <= params["huber_delta"] else params["huber_delta"] / chi
        ref = wt * (J.T * om) @ J
        src1 = np.zeros_like(w.channels[i])
        row, col = divmod(int(pix[k]), s.width)
        src1[row, col] = w.channels[i][row, col]
        pr = O.linearize_pair(s, params, src1, w.channels[j], Xi, Xj, lib=lib)
        assert pr["count"] == 1
        worst = max(worst, float(np.abs(pr["H"] - ref).max() / np.abs(ref).max()))
        used[branch] += 1
    assert min(used) >= n_each, f"too few points on one side of delta: {used}"
    return worst


# ------------------------------------------------------- graph construction

def pin_build_pairs(O, lib, w):
    """Graph construction (Sec. IV-B) against an independent evaluation: the
    candidate set from scipy's rotation magnitude of R_i^T R_j and numpy's
    translation distance (thresholds at the medians, so that each criterion
    removes pairs), every candidate's ratio against the valid fraction of
    `_bf_residuals` over all points of i (up to the oracle's margin-flagged
    points), and the kept set (ratio above the median ratio, or sequential).
    Returns 0 when all agree, else 1."""
    from scipy.spatial.transform import Rotation
    poses = np.asarray(w.poses_init, dtype=np.float64).reshape(-1, 3, 4)
    n = poses.shape[0]
    ang, dist = {}, {}
    for i in range(n):
        for j in range(i + 1, n):
            if w.frame_sensor[i] == w.frame_sensor[j]:
                ang[(i, j)] = Rotation.from_matrix(poses[i][:, :3].T @ poses[j][:, :3]).magnitude()
                dist[(i, j)] = float(np.linalg.norm(poses[i][:, 3] - poses[j][:, 3]))
    max_angle, max_dist = float(np.median(list(ang.values()))), float(np.median(list(dist.values())))
    expect = {ij for ij in ang if (ang[ij] < max_angle and dist[ij] < max_dist) or ij[1] == ij[0] + 1}
    assert any(ang[ij] >= max_angle and dist[ij] < max_dist for ij in ang)
    assert any(dist[ij] >= max_dist and ang[ij] < max_angle for ij in ang)
    # ratios of every candidate by brute force
    bf = {}
    for (i, j) in expect:
        s = w.sensors[w.frame_sensor[i]]
        _, pix = O.frame_points(s, w.params, w.channels[i], lib=lib)
        ok = _bf_residuals(s, w.params, w.channels[i], w.channels[j], poses[i], poses[j],
                           np.asarray(pix, dtype=np.int64))[0]
        bf[(i, j)] = (float(ok.mean()) if len(ok) else 0.0, len(ok))
    min_ratio = float(np.median([v[0] for v in bf.values()]))
    r = O.build_pairs(w.sensors, w.frame_sensor, w.channels, poses, w.params, max_angle, max_dist, min_ratio,
                      sequential=True, lib=lib)
    if set(r["candidates"]) != expect:
        return 1.0
    kept = {tuple(p) for p in r["pairs"].tolist()}
    for ij, c in r["candidates"].items():
        ratio, npts = bf[ij]
        slack = c["flagged"] / max(npts, 1) + 1e-12
        if c["n_points"] != npts or abs(c["ratio"] - ratio) > slack:
            return 1.0
        if abs(ratio - min_ratio) > slack and (ij in kept) != (ratio > min_ratio or ij[1] == ij[0] + 1):
            return 1.0
    return 0.0


def all_pins(O, lib, room, street):
    """Every pin's error on library `lib` (room: 3-frame RGB-D, street: 3-frame LiDAR)."""
    return {
        "projection_golden": pin_projection_golden(O, lib),
        "roundtrip": pin_roundtrip(O, lib),
        "proj_jacobian_fd": pin_proj_jacobian_fd(O, lib),
        "boxplus": pin_boxplus(O, lib),
        "jacobian_fd_pinhole": pin_jacobian_fd(O, lib, room),
        "jacobian_fd_spherical": pin_jacobian_fd(O, lib, street),
        "ramp_grad_mode0": pin_ramp_grad_mode0(O, lib),
        "gauge": max(pin_gauge(O, lib, room), pin_gauge(O, lib, street)),
        "cost_gradient": pin_cost_gradient(O, lib, room),
        "plane_shift": pin_plane_shift(O, lib),
        "single_channel": pin_single_channel(O, lib),
        "cholesky": pin_cholesky(O, lib),
        "extrinsic_equivalence": pin_extrinsic_equivalence(O, lib, room),
        "jacobian_fd_extrinsic": pin_jacobian_fd_extrinsic(O, lib, room),
        "normals_plane": pin_normals_plane(O, lib),
        "normals_counts": pin_normals_counts(O, lib),
        "normals_brute_force": max(pin_normals_brute_force(O, lib, room), pin_normals_brute_force(O, lib, street)),
        "normals_degenerate": pin_normals_degenerate(O, lib),
        "pyramid_projection": pin_pyramid_projection(O, lib),
        "downsample_closed_forms": pin_downsample_closed_forms(O, lib),
        "coarse_to_fine": pin_coarse_to_fine(O, lib),
        "offset_jacobian_fd": pin_offset_jacobian_fd(O, lib, room),
        "offset_gradient_fd": pin_offset_gradient_fd(O, lib, room),
        "residual_brute_force": pin_residual_brute_force(O, lib, room, street),
        "relative_jacobian": max(pin_relative_jacobian(O, lib, room), pin_relative_jacobian(O, lib, street),
                                 pin_relative_jacobian(O, lib, _with_offset(room))),
        "hessian_zero_residual": pin_hessian_zero_residual(O, lib),
        "half_rounding": pin_half_rounding(O, lib),
        "huber_hessian": max(pin_huber_hessian(O, lib, room), pin_huber_hessian(O, lib, street)),
    }


def graph_pins(O, lib, room8):
    return {"build_pairs": pin_build_pairs(O, lib, room8)}
