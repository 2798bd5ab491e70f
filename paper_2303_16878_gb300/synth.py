"""Seeded synthetic scenes, sensor renders, trajectories and pair lists.

This module produces the inputs of the photometric bundle-adjustment path
(Sec. IV, Eq. uprime to Eq. total-error-multicue and the supplementary error terms): per-frame five-channel
cue images (intensity g, depth or range d, normal n_x n_y n_z, Sec. IV-A),
ground-truth and perturbed sensor poses, and a directed pair list (Sec. IV-B).

It ray-casts analytic scenes (axis-aligned boxes seen from outside, rooms seen
from inside) along each pixel's viewing ray, as any renderer must.  It contains
none of the bundle-adjustment arithmetic: no residuals, no Jacobians, no robust
weights, no normal equations and no pose updates.  Both the CPU oracle and the
CUDA path consume what it returns, and neither imports the other.

Everything is a pure function of the integer seeds, so every test and benchmark
input can be regenerated bit for bit on any machine.

Pose convention: a pose is a 3x4 row-major matrix [R | t] mapping points of the
sensor (platform) frame into the world frame, p_w = R p + t (Eq. 1).
Pinhole sensor frame: x right, y down, z forward; depth is the z coordinate.
Spherical (LiDAR) sensor frame: x forward, y left, z up; d is the range.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

PINHOLE = 0
SPHERICAL = 1

IDENTITY_3x4 = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0]])


# --------------------------------------------------------------------------
# sensors
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Sensor:
    """Intrinsics of one sensor (Eq. camera-matrix-p pinhole K, Eq. spherical-projection K_[1,2])."""

    model: int
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    extrinsic: np.ndarray = dataclasses.field(default_factory=lambda: IDENTITY_3x4.copy())

    def as_dict(self) -> Dict:
        return dict(model=self.model, width=self.width, height=self.height,
                    fx=self.fx, fy=self.fy, cx=self.cx, cy=self.cy,
                    extrinsic=np.asarray(self.extrinsic, dtype=np.float64).reshape(12))


def pinhole_sensor(width: int, height: int, f: float, cx: float, cy: float) -> Sensor:
    return Sensor(PINHOLE, width, height, f, f, cx, cy)


def spherical_sensor(width: int, height: int, vfov_up_deg: float, vfov_down_deg: float) -> Sensor:
    """Spherical sensor with azimuth decreasing left to right over 360 degrees
    and row 0 at the top elevation (the reading of the spherical K taken for
    the paper's "resolution and offset" wording of Eq. spherical-projection)."""
    up = math.radians(vfov_up_deg)
    down = math.radians(vfov_down_deg)
    vfov = up - down
    fx = -width / (2.0 * math.pi)
    cx = width / 2.0
    fy = -(height - 1) / vfov
    cy = (height - 1) * up / vfov
    return Sensor(SPHERICAL, width, height, fx, fy, cx, cy)


def _pixel_rays(s: Sensor) -> Tuple[np.ndarray, bool]:
    """Viewing ray of every pixel centre in the sensor frame, shape (H, W, 3).

    Pinhole rays have unit z so the hit distance along them is the depth;
    spherical rays have unit length so the hit distance is the range.
    """
    cols = np.arange(s.width, dtype=np.float64)[None, :]
    rows = np.arange(s.height, dtype=np.float64)[:, None]
    if s.model == PINHOLE:
        x = np.broadcast_to((cols - s.cx) / s.fx, (s.height, s.width))
        y = np.broadcast_to((rows - s.cy) / s.fy, (s.height, s.width))
        return np.stack([x, y, np.ones_like(x)], axis=-1), True
    az = np.broadcast_to((cols - s.cx) / s.fx, (s.height, s.width))
    el = np.broadcast_to((rows - s.cy) / s.fy, (s.height, s.width))
    ce = np.cos(el)
    return np.stack([ce * np.cos(az), ce * np.sin(az), np.sin(el)], axis=-1), False


# --------------------------------------------------------------------------
# rotations (for building trajectories; plain matrix algebra)
# --------------------------------------------------------------------------

def rot_axis_angle(axis: Sequence[float], angle: float) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def rot_vec(v: np.ndarray) -> np.ndarray:
    th = float(np.linalg.norm(v))
    if th < 1e-15:
        return np.eye(3)
    return rot_axis_angle(v / th, th)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """3x4 pose of a pinhole camera (x right, y down, z forward) at `eye`."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, dtype=np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    out = np.zeros((3, 4))
    out[:, 0], out[:, 1], out[:, 2], out[:, 3] = x, y, z, eye
    return out


def compose(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a * b for 3x4 rigid transforms."""
    out = np.zeros((3, 4))
    out[:, :3] = a[:, :3] @ b[:, :3]
    out[:, 3] = a[:, :3] @ b[:, 3] + a[:, 3]
    return out


def perturb_poses(poses: np.ndarray, sigma_t: float, sigma_r: float, seed: int,
                  keep_first: bool = True) -> np.ndarray:
    """Right-multiply each pose by a random rigid motion: translation
    N(0, sigma_t) per axis, rotation vector N(0, sigma_r) per axis [rad]."""
    rng = np.random.default_rng(seed)
    out = poses.copy()
    for k in range(poses.shape[0]):
        dt = rng.normal(0.0, sigma_t, 3)
        dr = rng.normal(0.0, sigma_r, 3)
        if keep_first and k == 0:
            continue
        d = np.zeros((3, 4))
        d[:, :3] = rot_vec(dr)
        d[:, 3] = dt
        out[k] = compose(poses[k], d)
    return out


# --------------------------------------------------------------------------
# procedural texture
# --------------------------------------------------------------------------

def _hash2(i: np.ndarray, j: np.ndarray, seed: int) -> np.ndarray:
    """Lattice hash to [0, 1) (integer mixing, 32-bit)."""
    m = np.uint64(0xFFFFFFFF)
    x = (i.astype(np.int64).astype(np.uint64) * np.uint64(0x8DA6B343)) & m
    x ^= (j.astype(np.int64).astype(np.uint64) * np.uint64(0xD8163841)) & m
    x ^= np.uint64((seed * 0xCB1AB31F) & 0xFFFFFFFF)
    x = (x ^ (x >> np.uint64(16))) * np.uint64(0x7FEB352D) & m
    x = (x ^ (x >> np.uint64(15))) * np.uint64(0x846CA68B) & m
    x = x ^ (x >> np.uint64(16))
    return x.astype(np.float64) / 4294967296.0


def value_noise(s: np.ndarray, t: np.ndarray, seed: int, octaves: int = 4) -> np.ndarray:
    """Fractal value noise in [0, 1] with C1 (smoothstep) interpolation."""
    total = np.zeros_like(s)
    amp, freq, norm = 0.5, 1.0, 0.0
    for o in range(octaves):
        ss, tt = s * freq, t * freq
        i0, j0 = np.floor(ss), np.floor(tt)
        fs, ft = ss - i0, tt - j0
        fs = fs * fs * (3 - 2 * fs)
        ft = ft * ft * (3 - 2 * ft)
        sd = seed * 7919 + o * 104729
        h00 = _hash2(i0, j0, sd)
        h10 = _hash2(i0 + 1, j0, sd)
        h01 = _hash2(i0, j0 + 1, sd)
        h11 = _hash2(i0 + 1, j0 + 1, sd)
        v = (h00 * (1 - fs) + h10 * fs) * (1 - ft) + (h01 * (1 - fs) + h11 * fs) * ft
        total += amp * v
        norm += amp
        amp *= 0.5
        freq *= 2.0
    return total / norm


# --------------------------------------------------------------------------
# scenes and ray casting
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Box:
    lo: np.ndarray
    hi: np.ndarray
    inside: bool = False        # True: viewed from inside (a room), hit the exit face
    albedo: float = 0.8
    tex_freq: float = 2.0       # texture base frequency [cycles / m]
    tex_seed: int = 0
    tex_contrast: float = 0.8   # intensity = albedo * (1 - c + c * noise)


@dataclasses.dataclass
class Scene:
    boxes: List[Box]
    lambertian: bool = False    # intensity *= |n . ray| (LiDAR reflectance)


def _cast(scene: Scene, origin: np.ndarray, dirs: np.ndarray, d_max: float = np.inf):
    """Nearest hit of rays origin + t * dirs (dirs: (K, 3)) against the scene.
    Returns (t, normal_world, intensity); t = inf where nothing is hit.
    Boxes farther than d_max from the origin are skipped."""
    k = dirs.shape[0]
    best_t = np.full(k, np.inf)
    best_axis = np.zeros(k, dtype=np.int64)
    best_box = np.full(k, -1, dtype=np.int64)
    d = [np.ascontiguousarray(dirs[:, a]) for a in range(3)]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = [1.0 / d[a] for a in range(3)]
    for bi, b in enumerate(scene.boxes):
        if not b.inside:
            nearest = np.clip(origin, b.lo, b.hi)
            if np.linalg.norm(nearest - origin) > d_max * 1.01:
                continue
        tmin, tmax = [], []
        with np.errstate(invalid="ignore"):
            for a in range(3):
                t1 = (b.lo[a] - origin[a]) * inv[a]
                t2 = (b.hi[a] - origin[a]) * inv[a]
                if origin[a] == b.lo[a] or origin[a] == b.hi[a]:  # 0 * inf on the slab plane
                    t1 = np.where(np.isnan(t1), -np.inf, t1)
                    t2 = np.where(np.isnan(t2), np.inf, t2)
                tmin.append(np.minimum(t1, t2))
                tmax.append(np.maximum(t1, t2))
        if b.inside:
            t_hit = np.minimum(np.minimum(tmax[0], tmax[1]), tmax[2])
            axis = np.where(tmax[0] == t_hit, 0, np.where(tmax[1] == t_hit, 1, 2))
            ok = t_hit > 1e-9
        else:
            t_near = np.maximum(np.maximum(tmin[0], tmin[1]), tmin[2])
            t_far = np.minimum(np.minimum(tmax[0], tmax[1]), tmax[2])
            axis = np.where(tmin[0] == t_near, 0, np.where(tmin[1] == t_near, 1, 2))
            ok = (t_near <= t_far) & (t_near > 1e-9)
            t_hit = t_near
        upd = ok & (t_hit < best_t)
        best_t = np.where(upd, t_hit, best_t)
        best_axis = np.where(upd, axis, best_axis)
        best_box = np.where(upd, bi, best_box)
    hit = np.isfinite(best_t)
    rows_all = np.arange(k)
    # the face normal points against the ray (outside boxes: outward normal of
    # the entry face; rooms: inward normal of the exit face)
    sign = -np.sign(dirs[rows_all, best_axis])
    normal = np.zeros((k, 3))
    normal[rows_all, best_axis] = np.where(hit, sign, 0.0)
    point = origin[None, :] + np.where(hit, best_t, 0.0)[:, None] * dirs
    inten = np.zeros(k)
    for bi, b in enumerate(scene.boxes):
        sel = hit & (best_box == bi)
        if not np.any(sel):
            continue
        ax = best_axis[sel]
        p = point[sel]
        # texture coordinates: the two world axes spanning the face
        s_idx = np.where(ax == 0, 1, 0)
        t_idx = np.where(ax == 2, 1, 2)
        rows = np.arange(p.shape[0])
        s = p[rows, s_idx] * b.tex_freq
        t = p[rows, t_idx] * b.tex_freq
        nz = value_noise(s, t, b.tex_seed * 31 + ax)
        inten[sel] = b.albedo * (1.0 - b.tex_contrast + b.tex_contrast * nz)
    if scene.lambertian:
        dn = np.linalg.norm(dirs, axis=1)
        cosang = np.abs(np.sum(normal * dirs, axis=1)) / np.maximum(dn, 1e-30)
        inten = inten * cosang
    return best_t, normal, inten


def render(scene: Scene, sensor: Sensor, sensor_pose: np.ndarray,
           d_min: float, d_max: float) -> np.ndarray:
    """Five-channel image (H, W, 5) float32: g, d, n_x, n_y, n_z (Sec. IV-A).

    d is the depth (pinhole) or range (spherical) of the nearest surface, 0
    where no surface lies within [d_min, d_max] (an invalid pixel).  Normals
    are the analytic surface normals in the sensor frame, oriented towards the
    sensor, and zero at invalid pixels.
    """
    rays, _ = _pixel_rays(sensor)
    r = sensor_pose[:, :3]
    o = sensor_pose[:, 3]
    d_world = rays.reshape(-1, 3) @ r.T
    t, n_world, inten = _cast(scene, o, d_world, d_max)
    valid = np.isfinite(t) & (t >= d_min) & (t <= d_max)
    n_sensor = n_world @ r  # R^T n for each row
    out = np.zeros((sensor.height * sensor.width, 5), dtype=np.float64)
    out[:, 0] = np.where(valid, inten, 0.0)
    out[:, 1] = np.where(valid, t, 0.0)
    out[:, 2:5] = np.where(valid[:, None], n_sensor, 0.0)
    return out.reshape(sensor.height, sensor.width, 5).astype(np.float32)


def quantize_fp16(channels: np.ndarray) -> np.ndarray:
    """Round the intensity and normal channels to the nearest binary16 value
    (like a sensor with a 10-bit mantissa), leaving depth in float32."""
    out = channels.copy()
    for c in (0, 2, 3, 4):
        out[..., c] = out[..., c].astype(np.float16).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """One bundle-adjustment problem instance."""

    name: str
    sensors: List[Sensor]
    frame_sensor: np.ndarray     # (N,) int32
    channels: List[np.ndarray]   # N arrays (H, W, 5) float32
    poses_gt: np.ndarray         # (N, 3, 4) float64
    poses_init: np.ndarray       # (N, 3, 4) float64
    pairs: np.ndarray            # (M, 2) int32, directed (source i, target j)
    params: Dict                 # method configuration (weights, Huber delta, thresholds)
    frame_var: Optional[np.ndarray] = None  # pose variable per frame (-1 fixed); None: frame 0 fixed
    n_vars: int = 0
    extrinsic_gt: Optional[List[np.ndarray]] = None  # true sensor offsets when the sensors carry perturbed ones

    @property
    def n_frames(self) -> int:
        return len(self.channels)

    def channels_array(self) -> np.ndarray:
        """All frames stacked (N, H, W, 5); valid only when sizes agree."""
        return np.stack(self.channels, axis=0)

    def subset(self, frames: Sequence[int]) -> "Workload":
        frames = list(frames)
        remap = {f: k for k, f in enumerate(frames)}
        keep = [p for p in self.pairs.tolist() if p[0] in remap and p[1] in remap]
        pairs = np.array([[remap[a], remap[b]] for a, b in keep], dtype=np.int32).reshape(-1, 2)
        return Workload(self.name + "-subset", self.sensors, self.frame_sensor[frames].copy(),
                        [self.channels[f] for f in frames], self.poses_gt[frames].copy(),
                        self.poses_init[frames].copy(), pairs, dict(self.params))


def default_params(**over) -> Dict:
    """Method configuration; values the paper leaves open take these defaults."""
    p = dict(w_int=1.0, w_depth=1.0, w_normal=1.0, huber_delta=0.1,
             occ_abs=0.1, occ_rel=0.05, z_min=0.05, range_min=0.0, range_max=1e30,
             grad_mode=0)
    p.update(over)
    return p


def _room_scene(seed: int) -> Scene:
    rng = np.random.default_rng(seed)
    room = Box(np.array([-2.5, -2.5, 0.0]), np.array([2.5, 2.5, 3.0]), inside=True,
               albedo=1.0, tex_freq=float(rng.uniform(2.5, 3.5)), tex_seed=int(rng.integers(1, 1 << 20)),
               tex_contrast=0.85)
    return Scene([room])


def make_rgbd_room(n_frames: int = 8, width: int = 160, height: int = 120, f: float = 120.0,
                   cx: Optional[float] = None, cy: Optional[float] = None,
                   seed: int = 1, sigma_t: float = 0.02, sigma_r_deg: float = 1.0,
                   pair_window: int = 3, fp16_exact: bool = False,
                   depth_noise: float = 0.0, intensity_noise: float = 0.0,
                   params: Optional[Dict] = None) -> Workload:
    """RGB-D pinhole sequence in a 5 x 5 x 3 m room of six textured planes.

    Cameras sit on a 1 m circle at 1.5 m height and look at a common point on
    the +y wall, so all pairs within `pair_window` frames overlap.  Depth is
    clipped to 0.5-5 m.  Seeds: scene 1000+seed, trajectory 2000+seed,
    perturbation 3000+seed.
    """
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    scene = _room_scene(1000 + seed)
    sensor = pinhole_sensor(width, height, f, cx, cy)
    rng = np.random.default_rng(2000 + seed)
    poses = np.zeros((n_frames, 3, 4))
    for k in range(n_frames):
        th = 2 * math.pi * k / n_frames + rng.uniform(-0.05, 0.05)
        eye = np.array([math.cos(th), math.sin(th), 1.5 + rng.uniform(-0.05, 0.05)])
        target = np.array([rng.uniform(-0.3, 0.3), 2.5, 1.3 + rng.uniform(-0.2, 0.2)])
        poses[k] = look_at(eye, target)
    chans = []
    for k in range(n_frames):
        c = render(scene, sensor, poses[k], 0.5, 5.0)
        if depth_noise > 0 or intensity_noise > 0:
            nrng = np.random.default_rng(5000 + seed * 977 + k)
            valid = c[..., 1] > 0
            z = c[..., 1].astype(np.float64)
            c[..., 1] = np.where(valid, z + nrng.normal(0, 1, z.shape) * depth_noise * z * z, 0).astype(np.float32)
            c[..., 0] = np.where(valid, c[..., 0] + nrng.normal(0, intensity_noise, z.shape), 0).astype(np.float32)
        if fp16_exact:
            c = quantize_fp16(c)
        chans.append(c)
    init = perturb_poses(poses, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    pairs = [(i, j) for i in range(n_frames) for j in range(i + 1, n_frames) if j - i <= pair_window]
    prm = default_params()
    if params:
        prm.update(params)
    return Workload(f"rgbd-room-{n_frames}x{width}x{height}", [sensor],
                    np.zeros(n_frames, dtype=np.int32), chans, poses, init,
                    np.array(pairs, dtype=np.int32).reshape(-1, 2), prm)


def _street_scene(seed: int, x_lo: float, x_hi: float) -> Scene:
    rng = np.random.default_rng(seed)
    boxes = [Box(np.array([x_lo - 150, -150.0, -1.0]), np.array([x_hi + 150, 150.0, 0.0]),
                 albedo=0.35, tex_freq=1.5, tex_seed=int(rng.integers(1, 1 << 20)), tex_contrast=0.7)]
    for side in (+1, -1):
        x = x_lo - 60.0
        while x < x_hi + 60.0:
            length = rng.uniform(8, 20)
            depth = rng.uniform(6, 15)
            height = rng.uniform(4, 15)
            y0 = 7.0 + rng.uniform(0, 1.5)
            lo = np.array([x, y0 if side > 0 else -y0 - depth, 0.0])
            hi = np.array([x + length, y0 + depth if side > 0 else -y0, height])
            boxes.append(Box(lo, hi, albedo=float(rng.uniform(0.3, 0.95)),
                             tex_freq=float(rng.uniform(0.8, 2.0)),
                             tex_seed=int(rng.integers(1, 1 << 20)), tex_contrast=0.75))
            x += length + rng.uniform(0.0, 4.0)
        x = x_lo - 40.0 + rng.uniform(0, 4)
        while x < x_hi + 40.0:
            y = side * rng.uniform(4.5, 5.5)
            boxes.append(Box(np.array([x - 0.15, y - 0.15, 0.0]), np.array([x + 0.15, y + 0.15, 5.0]),
                             albedo=0.9, tex_freq=3.0, tex_seed=int(rng.integers(1, 1 << 20)),
                             tex_contrast=0.3))
            x += rng.uniform(6, 10)
        x = x_lo - 30.0 + rng.uniform(0, 10)
        while x < x_hi + 30.0:
            y = side * rng.uniform(2.8, 3.6)
            boxes.append(Box(np.array([x, y - 0.9, 0.0]), np.array([x + 4.2, y + 0.9, 1.5]),
                             albedo=float(rng.uniform(0.2, 0.9)), tex_freq=2.5,
                             tex_seed=int(rng.integers(1, 1 << 20)), tex_contrast=0.6))
            x += rng.uniform(7, 16)
    return Scene(boxes, lambertian=True)


def _street_trajectory(n_frames: int, spacing: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0, 2 * math.pi)
    poses = np.zeros((n_frames, 3, 4))
    for k in range(n_frames):
        x = k * spacing
        y = 0.6 * math.sin(x / 9.0 + phase)
        dy = 0.6 / 9.0 * math.cos(x / 9.0 + phase)
        yaw = math.atan2(dy, 1.0) + rng.uniform(-0.02, 0.02)
        r = rot_axis_angle((0, 0, 1), yaw) @ rot_axis_angle((0, 1, 0), rng.uniform(-0.01, 0.01))
        poses[k, :, :3] = r
        poses[k, :, 3] = (x, y, 1.8 + rng.uniform(-0.03, 0.03))
    return poses


def overlap_ratio(src: np.ndarray, tgt: np.ndarray, sensor: Sensor, pose_src: np.ndarray,
                  pose_tgt: np.ndarray, rel_tol: float = 0.05, stride: int = 1) -> float:
    """Fraction of frame src's valid pixels that are seen by frame tgt at the
    same distance (visibility test for building the pair list, Sec. IV-B
    criterion 3).  Uses the renderer's own ray geometry and nearest pixels;
    `stride` > 1 estimates the ratio on every stride-th pixel (raster order)."""
    rays, is_pin = _pixel_rays(sensor)
    d = src[..., 1].astype(np.float64)
    valid = d > 0
    if stride > 1:
        sub = np.zeros(valid.size, dtype=bool)
        sub[::stride] = True
        valid &= sub.reshape(valid.shape)
    if not np.any(valid):
        return 0.0
    pts = rays[valid] * d[valid][:, None]
    pw = pts @ pose_src[:, :3].T + pose_src[:, 3]
    pt = (pw - pose_tgt[:, 3]) @ pose_tgt[:, :3]
    if is_pin:
        z = pt[:, 2]
        ok = z > 1e-3
        zz = np.where(ok, z, 1.0)
        col = np.rint(sensor.fx * pt[:, 0] / zz + sensor.cx)
        row = np.rint(sensor.fy * pt[:, 1] / zz + sensor.cy)
        dist = z
    else:
        rxy = np.hypot(pt[:, 0], pt[:, 1])
        col = np.rint(sensor.fx * np.arctan2(pt[:, 1], pt[:, 0]) + sensor.cx) % sensor.width
        row = np.rint(sensor.fy * np.arctan2(pt[:, 2], rxy) + sensor.cy)
        dist = np.linalg.norm(pt, axis=1)
        ok = np.ones(pt.shape[0], dtype=bool)
    ok &= (col >= 0) & (col < sensor.width) & (row >= 0) & (row < sensor.height)
    ci = np.where(ok, col, 0).astype(np.int64)
    ri = np.where(ok, row, 0).astype(np.int64)
    dt = tgt[..., 1].astype(np.float64)[ri, ci]
    ok &= (dt > 0) & (np.abs(dt - dist) <= rel_tol * dist + 0.05)
    return float(np.count_nonzero(ok)) / float(pts.shape[0])


def make_lidar_street(n_frames: int = 50, width: int = 1024, height: int = 64,
                      vfov_up_deg: float = 16.6, vfov_down_deg: float = -16.6,
                      spacing: float = 1.0, seed: int = 2, sigma_t: float = 0.10,
                      sigma_r_deg: float = 0.5, drop: float = 0.05, min_overlap: float = 0.3,
                      max_pair_distance: float = 40.0, fp16_exact: bool = False,
                      params: Optional[Dict] = None) -> Workload:
    """LiDAR spherical-projection sequence along a synthetic street.

    Ground plane, two rows of textured box buildings, poles and parked cars;
    range 1-80 m; intensity = Lambertian |n . ray| x textured albedo; a
    fraction `drop` of returns is removed (Bernoulli); 50 poses along a 50 m
    path.  Pairs (i < j) are kept when the overlap ratio exceeds `min_overlap`.
    Seeds: scene 1000+seed, trajectory 2000+seed, perturbation 3000+seed,
    dropped returns 4000+seed.
    """
    poses = _street_trajectory(n_frames, spacing, 2000 + seed)
    scene = _street_scene(1000 + seed, 0.0, (n_frames - 1) * spacing)
    sensor = spherical_sensor(width, height, vfov_up_deg, vfov_down_deg)
    drng = np.random.default_rng(4000 + seed)
    chans = []
    for k in range(n_frames):
        c = render(scene, sensor, poses[k], 1.0, 80.0)
        keep = drng.random((height, width)) >= drop
        c = np.where(keep[..., None], c, 0.0).astype(np.float32)
        if fp16_exact:
            c = quantize_fp16(c)
        chans.append(c)
    pairs = []
    for i in range(n_frames):
        for j in range(i + 1, n_frames):
            if np.linalg.norm(poses[i, :, 3] - poses[j, :, 3]) > max_pair_distance:
                continue
            if overlap_ratio(chans[i], chans[j], sensor, poses[i], poses[j], stride=7) > min_overlap:
                pairs.append((i, j))
    init = perturb_poses(poses, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    prm = default_params(w_depth=0.1, huber_delta=0.2, occ_abs=0.3, occ_rel=0.05, z_min=0.5,
                         range_min=1.0, range_max=80.0)
    if params:
        prm.update(params)
    return Workload(f"lidar-street-{n_frames}x{height}x{width}", [sensor],
                    np.zeros(n_frames, dtype=np.int32), chans, poses, init,
                    np.array(pairs, dtype=np.int32).reshape(-1, 2), prm)


def with_extrinsic(w: Workload, Xo: np.ndarray) -> Workload:
    """The same renders described with a sensor mounted at offset Xo on the
    platform: every sensor gets extrinsic Xo and the platform poses become
    X_sensor Xo^-1, so that platform pose times offset is the render pose."""
    Xo = np.asarray(Xo, dtype=np.float64).reshape(3, 4)
    inv = np.zeros((3, 4))
    inv[:, :3] = Xo[:, :3].T
    inv[:, 3] = -Xo[:, :3].T @ Xo[:, 3]
    sensors = [dataclasses.replace(s, extrinsic=Xo.copy()) for s in w.sensors]
    gt = np.stack([compose(X, inv) for X in w.poses_gt])
    init = np.stack([compose(X, inv) for X in w.poses_init])
    return Workload(w.name + "-offset", sensors, w.frame_sensor.copy(), w.channels, gt, init, w.pairs.copy(),
                    dict(w.params))


def offset_transform(t_m: float = 0.02, r_deg: float = 0.5, seed: int = 5) -> np.ndarray:
    """A seeded sensor offset: translation of norm t_m, rotation of r_deg degrees."""
    rng = np.random.default_rng(seed)
    t = rng.normal(size=3)
    a = rng.normal(size=3)
    X = np.zeros((3, 4))
    X[:, :3] = rot_vec(a / np.linalg.norm(a) * math.radians(r_deg))
    X[:, 3] = t / np.linalg.norm(t) * t_m
    return X


def make_plane_shift(width: int = 48, height: int = 40, f: float = 40.0, depth: float = 2.0,
                     shift_px: Tuple[int, int] = (3, 2), seed: int = 7) -> Workload:
    """Two pinhole frames facing a fronto-parallel textured plane at constant
    depth, the second translated so that the image moves by an integer number
    of pixels: every pixel of frame 0 lands exactly on a pixel centre of
    frame 1 with the same intensity, depth and normal."""
    sensor = pinhole_sensor(width, height, f, width / 2.0, height / 2.0)
    wall = Box(np.array([-50.0, -50.0, depth]), np.array([50.0, 50.0, depth + 1.0]),
               albedo=1.0, tex_freq=4.0, tex_seed=seed, tex_contrast=0.9)
    scene = Scene([wall])
    poses = np.zeros((2, 3, 4))
    poses[0] = IDENTITY_3x4
    poses[1] = IDENTITY_3x4
    poses[1, 0, 3] = shift_px[0] * depth / f
    poses[1, 1, 3] = shift_px[1] * depth / f
    chans = [render(scene, sensor, poses[k], 0.1, 100.0) for k in range(2)]
    return Workload("plane-shift", [sensor], np.zeros(2, dtype=np.int32), chans, poses,
                    poses.copy(), np.array([[0, 1]], dtype=np.int32), default_params())


def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


# camera axes (x right, y down, z forward) in the platform frame (x forward, y left, z up)
CAMERA_ON_PLATFORM = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


def make_fusion_room(n_poses: int = 4, cam_width: int = 160, cam_height: int = 120, f: float = 120.0,
                     lidar_width: int = 512, lidar_height: int = 32, vfov_up_deg: float = 16.6,
                     vfov_down_deg: float = -16.6, cam_offset=(0.10, 0.0, 0.10), seed: int = 7,
                     sigma_t: float = 0.02, sigma_r_deg: float = 1.0, coupled: bool = True,
                     tilt_deg: float = 0.0, fp16_exact: bool = False,
                     params: Optional[Dict] = None) -> Workload:
    """A platform carrying an RGB-D camera and a 3D LiDAR (Sec. V, fusion) in
    the textured room of make_rgbd_room.

    Platform frame: x forward, y left, z up.  The LiDAR sits at the platform
    origin (identity offset); the camera `cam_offset` from it, looking along
    the platform x axis.  Platform poses: n_poses points near the room centre
    at 1.2-1.3 m height, heading towards the +y wall +- 15 deg, pitched by up
    to 3 deg, plus (tilt_deg > 0) roll and pitch of up to +-tilt_deg (the
    rotational diversity under which an offset's translation is observable:
    with rotations about one axis only, its component along that axis is not).  Frames 0..n-1
    are the camera's, n..2n-1 the LiDAR's; frames k and n + k were captured at
    platform pose k.  Pairs: camera (i, j), j - i <= 3; LiDAR (n + i, n + j)
    for all i < j.  With `coupled`, frame_var ties frames k and n + k to one
    variable and holds platform pose 0 fixed.  Seeds: scene 1000 + seed,
    trajectory 2000 + seed, perturbation 3000 + seed (the same perturbation
    for the two frames of a platform pose)."""
    scene = _room_scene(1000 + seed)
    cam = pinhole_sensor(cam_width, cam_height, f, cam_width / 2.0, cam_height / 2.0)
    Xc = np.zeros((3, 4))
    Xc[:, :3] = CAMERA_ON_PLATFORM
    Xc[:, 3] = cam_offset
    cam.extrinsic = Xc
    lidar = spherical_sensor(lidar_width, lidar_height, vfov_up_deg, vfov_down_deg)
    rng = np.random.default_rng(2000 + seed)
    plat = np.zeros((n_poses, 3, 4))
    for k in range(n_poses):
        th = 2 * math.pi * k / max(n_poses, 1)
        yaw = math.pi / 2 + rng.uniform(-0.26, 0.26)
        plat[k, :, :3] = rot_z(yaw) @ rot_y(rng.uniform(-0.05, 0.05))
        if tilt_deg > 0:
            tr = np.random.default_rng(2500 + seed + 31 * k).uniform(-1.0, 1.0, 2) * math.radians(tilt_deg)
            plat[k, :, :3] = plat[k, :, :3] @ rot_y(tr[0]) @ rot_axis_angle((1, 0, 0), tr[1])
        plat[k, :, 3] = [0.4 * math.cos(th), 0.4 * math.sin(th) - 0.3, 1.2 + rng.uniform(0.0, 0.1)]
    chans = []
    for k in range(n_poses):
        chans.append(render(scene, cam, compose(plat[k], Xc), 0.5, 5.0))
    for k in range(n_poses):
        chans.append(render(scene, lidar, plat[k], 0.5, 8.0))
    if fp16_exact:
        chans = [quantize_fp16(c) for c in chans]
    init_plat = perturb_poses(plat, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    poses = np.concatenate([plat, plat])
    init = np.concatenate([init_plat, init_plat])
    pairs = [(i, j) for i in range(n_poses) for j in range(i + 1, n_poses) if j - i <= 3]
    pairs += [(n_poses + i, n_poses + j) for i in range(n_poses) for j in range(i + 1, n_poses)]
    prm = default_params(range_min=0.5, range_max=8.0)
    if params:
        prm.update(params)
    fv = None
    if coupled:
        fv = np.array([k - 1 for k in range(n_poses)] * 2, dtype=np.int32)
    return Workload(f"fusion-room-{n_poses}", [cam, lidar],
                    np.array([0] * n_poses + [1] * n_poses, dtype=np.int32), chans, poses, init,
                    np.array(pairs, dtype=np.int32).reshape(-1, 2), prm, fv, n_poses - 1 if coupled else 0)


# --------------------------------------------------------------------------
# the same renderer on torch tensors (CPU or CUDA), for the large workloads
# --------------------------------------------------------------------------

def _mulmod32_t(a, c: int):
    """(a * c) mod 2^32 for int64 tensors 0 <= a < 2^32 without overflowing int64."""
    lo = a & 0xFFFF
    hi = a >> 16
    return ((lo * c) + (((hi * c) & 0xFFFF) << 16)) & 0xFFFFFFFF


def _hash2_t(i, j, seed: int):
    """_hash2 on int64 tensors, bit for bit."""
    m = 0xFFFFFFFF
    x = _mulmod32_t(i & m, 0x8DA6B343)
    x = x ^ _mulmod32_t(j & m, 0xD8163841)
    x = x ^ ((seed * 0xCB1AB31F) & m)
    x = _mulmod32_t(x ^ (x >> 16), 0x7FEB352D)
    x = _mulmod32_t(x ^ (x >> 15), 0x846CA68B)
    x = x ^ (x >> 16)
    return x.double() / 4294967296.0


def value_noise_t(s, t, seed, octaves: int = 4):
    """value_noise on float64 tensors; `seed` an int or an int64 tensor of
    per-element seeds (the same integer arithmetic, so the same values)."""
    import torch
    total = torch.zeros_like(s)
    amp, freq, norm = 0.5, 1.0, 0.0
    for o in range(octaves):
        ss, tt = s * freq, t * freq
        i0, j0 = torch.floor(ss), torch.floor(tt)
        fs, ft = ss - i0, tt - j0
        fs = fs * fs * (3 - 2 * fs)
        ft = ft * ft * (3 - 2 * ft)
        sd = seed * 7919 + o * 104729
        ii, jj = i0.long(), j0.long()
        h00 = _hash2_t(ii, jj, sd)
        h10 = _hash2_t(ii + 1, jj, sd)
        h01 = _hash2_t(ii, jj + 1, sd)
        h11 = _hash2_t(ii + 1, jj + 1, sd)
        v = (h00 * (1 - fs) + h10 * fs) * (1 - ft) + (h01 * (1 - fs) + h11 * fs) * ft
        total = total + amp * v
        norm += amp
        amp *= 0.5
        freq *= 2.0
    return total / norm


def _scene_tensors(scene: Scene, device):
    import torch
    lo = torch.as_tensor(np.array([b.lo for b in scene.boxes], dtype=np.float64), device=device)
    hi = torch.as_tensor(np.array([b.hi for b in scene.boxes], dtype=np.float64), device=device)
    inside = torch.as_tensor([b.inside for b in scene.boxes], device=device)
    albedo = torch.as_tensor([b.albedo for b in scene.boxes], dtype=torch.float64, device=device)
    freq = torch.as_tensor([b.tex_freq for b in scene.boxes], dtype=torch.float64, device=device)
    seed = torch.as_tensor([b.tex_seed for b in scene.boxes], dtype=torch.int64, device=device)
    contrast = torch.as_tensor([b.tex_contrast for b in scene.boxes], dtype=torch.float64, device=device)
    return dict(lo=lo, hi=hi, inside=inside, albedo=albedo, freq=freq, seed=seed, contrast=contrast)


def _cast_t(scene: Scene, origin: np.ndarray, dirs, d_max: float = math.inf, st=None):
    """_cast on a (K, 3) float64 tensor of ray directions, all boxes at once
    (the first box of the smallest hit distance wins, as in the loop of _cast;
    boxes that _cast skips lie beyond d_max and change no valid pixel)."""
    import torch
    dev = dirs.device
    st = st or _scene_tensors(scene, dev)
    k = dirs.shape[0]
    keep = [bi for bi, b in enumerate(scene.boxes)
            if b.inside or np.linalg.norm(np.clip(origin, b.lo, b.hi) - origin) <= d_max * 1.01]
    sel = torch.as_tensor(keep, dtype=torch.long, device=dev)
    lo, hi, inside = st["lo"][sel], st["hi"][sel], st["inside"][sel]
    o = torch.as_tensor(origin, dtype=torch.float64, device=dev)
    inv = 1.0 / dirs                                   # (K, 3)
    t1 = (lo[None, :, :] - o) * inv[:, None, :]        # (K, B, 3)
    t2 = (hi[None, :, :] - o) * inv[:, None, :]
    on_lo = (lo == o)[None, :, :]
    on_hi = (hi == o)[None, :, :]
    on = on_lo | on_hi                                 # the 0 * inf case on a slab plane
    t1 = torch.where(on & torch.isnan(t1), torch.full_like(t1, -math.inf), t1)
    t2 = torch.where(on & torch.isnan(t2), torch.full_like(t2, math.inf), t2)
    tmin = torch.minimum(t1, t2)
    tmax = torch.maximum(t1, t2)
    t_exit = torch.minimum(torch.minimum(tmax[..., 0], tmax[..., 1]), tmax[..., 2])
    t_near = torch.maximum(torch.maximum(tmin[..., 0], tmin[..., 1]), tmin[..., 2])
    ax_in = torch.where(tmax[..., 0] == t_exit, 0, torch.where(tmax[..., 1] == t_exit, 1, 2))
    ax_out = torch.where(tmin[..., 0] == t_near, 0, torch.where(tmin[..., 1] == t_near, 1, 2))
    t_hit = torch.where(inside[None, :], t_exit, t_near)
    axis = torch.where(inside[None, :], ax_in, ax_out)
    ok = torch.where(inside[None, :], t_exit > 1e-9, (t_near <= t_exit) & (t_near > 1e-9))
    t_hit = torch.where(ok, t_hit, torch.full_like(t_hit, math.inf))
    best_t, arg = torch.min(t_hit, dim=1)              # first minimum: the lowest box index
    hit = torch.isfinite(best_t)
    best_axis = torch.gather(axis, 1, arg[:, None])[:, 0]
    best_box = sel[arg]
    rows_all = torch.arange(k, device=dev)
    sign = -torch.sign(dirs[rows_all, best_axis])
    normal = torch.zeros((k, 3), dtype=torch.float64, device=dev)
    normal[rows_all, best_axis] = torch.where(hit, sign, torch.zeros_like(sign))
    point = o[None, :] + torch.where(hit, best_t, torch.zeros_like(best_t))[:, None] * dirs
    s_idx = torch.where(best_axis == 0, 1, 0)
    t_idx = torch.where(best_axis == 2, 1, 2)
    fq = st["freq"][best_box]
    s = point[rows_all, s_idx] * fq
    t = point[rows_all, t_idx] * fq
    nz = value_noise_t(s, t, st["seed"][best_box] * 31 + best_axis)
    inten = st["albedo"][best_box] * (1.0 - st["contrast"][best_box] + st["contrast"][best_box] * nz)
    inten = torch.where(hit, inten, torch.zeros_like(inten))
    if scene.lambertian:
        dn = torch.linalg.norm(dirs, dim=1)
        cosang = torch.abs(torch.sum(normal * dirs, dim=1)) / torch.clamp(dn, min=1e-30)
        inten = inten * cosang
    return best_t, normal, inten


def render_t(scene: Scene, sensor: Sensor, sensor_pose: np.ndarray, d_min: float, d_max: float, device="cpu",
             rays=None, st=None):
    """render() on torch: a (H, W, 5) float32 tensor on `device`."""
    import torch
    if rays is None:
        rays = torch.as_tensor(_pixel_rays(sensor)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    r = torch.as_tensor(sensor_pose[:, :3], dtype=torch.float64, device=device)
    o = np.asarray(sensor_pose[:, 3], dtype=np.float64)
    d_world = rays @ r.T
    t, n_world, inten = _cast_t(scene, o, d_world, d_max, st)
    valid = torch.isfinite(t) & (t >= d_min) & (t <= d_max)
    n_sensor = n_world @ r
    out = torch.zeros((sensor.height * sensor.width, 5), dtype=torch.float64, device=device)
    zero = torch.zeros_like(t)
    out[:, 0] = torch.where(valid, inten, zero)
    out[:, 1] = torch.where(valid, t, zero)
    out[:, 2:5] = torch.where(valid[:, None], n_sensor, torch.zeros_like(n_sensor))
    return out.reshape(sensor.height, sensor.width, 5).float()


def quantize_fp16_t(ch):
    out = ch.clone()
    for c in (0, 2, 3, 4):
        out[..., c] = out[..., c].half().float()
    return out


def _hall_scene(seed: int) -> Scene:
    """Multi-room indoor scene: a 20 x 12 x 3 m hall seen from inside, split
    into four rooms by 0.12 m partition walls with 1.2 m doorways, plus
    furniture boxes along the outer walls.  Every surface is textured."""
    rng = np.random.default_rng(seed)

    def tex():
        return dict(albedo=float(rng.uniform(0.5, 1.0)), tex_freq=float(rng.uniform(2.0, 4.0)),
                    tex_seed=int(rng.integers(1, 1 << 20)), tex_contrast=0.8)
    boxes = [Box(np.array([-10.0, -6.0, 0.0]), np.array([10.0, 6.0, 3.0]), inside=True, **tex())]
    th = 0.06

    def wall_x(y, x0, x1):  # a partition along x at height 0..3
        boxes.append(Box(np.array([x0, y - th, 0.0]), np.array([x1, y + th, 3.0]), **tex()))

    def wall_y(x, y0, y1):
        boxes.append(Box(np.array([x - th, y0, 0.0]), np.array([x + th, y1, 3.0]), **tex()))
    # y = 0 partition with doorways at x in [-6.0, -4.8], [6.0, 7.2]
    wall_x(0.0, -10.0, -6.0)
    wall_x(0.0, -4.8, 6.0)
    wall_x(0.0, 7.2, 10.0)
    # x = -3 (south half) doorway y in [-3.5, -2.3]; x = 4 (north half) doorway y in [2.0, 3.2]
    wall_y(-3.0, -6.0, -3.5)
    wall_y(-3.0, -2.3, 0.0)
    wall_y(4.0, 0.0, 2.0)
    wall_y(4.0, 3.2, 6.0)
    # furniture along the outer walls (the path stays at least 1.5 m away from them)
    for _ in range(18):
        side = int(rng.integers(0, 4))
        w, d, h = rng.uniform(0.6, 1.8), rng.uniform(0.4, 0.8), rng.uniform(0.5, 2.0)
        if side < 2:
            x = rng.uniform(-9.5, 9.5 - w)
            y0 = -6.0 if side == 0 else 6.0 - d
            lo, hi = [x, y0, 0.0], [x + w, y0 + d, h]
        else:
            y = rng.uniform(-5.5, 5.5 - w)
            x0 = -10.0 if side == 2 else 10.0 - d
            lo, hi = [x0, y, 0.0], [x0 + d, y + w, h]
        boxes.append(Box(np.array(lo), np.array(hi), **tex()))
    return Scene(boxes)


def _hall_path(n: int, seed: int, height: float = 1.4, tilt_deg: float = 0.0) -> np.ndarray:
    """Platform poses (x forward, y left, z up) along a closed Catmull-Rom
    spline through the hall's four rooms and its doorways, resampled to n
    poses equally spaced in arc length; heading along the path with smooth
    yaw (+-15 deg) and pitch (-8..+4 deg) wobble, height +- 0.1 m; with
    tilt_deg > 0 a further smooth roll and pitch of amplitude tilt_deg (a
    hand-held platform)."""
    rng = np.random.default_rng(seed)
    way = np.array([[-7.0, -3.0], [-5.4, -1.2], [-5.4, 1.5], [-4.0, 3.2], [0.5, 3.5], [3.0, 2.6], [5.0, 2.6],
                    [6.6, 1.5], [6.6, -1.3], [5.0, -3.0], [0.0, -3.2], [-2.0, -2.9], [-4.5, -2.9]])
    way = way + rng.uniform(-0.15, 0.15, way.shape)
    m = len(way)
    dense = []
    for i in range(m):
        p0, p1, p2, p3 = way[(i - 1) % m], way[i], way[(i + 1) % m], way[(i + 2) % m]
        for u in np.linspace(0.0, 1.0, 200, endpoint=False):
            u2, u3 = u * u, u * u * u
            dense.append(0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u2 +
                                (-p0 + 3 * p1 - 3 * p2 + p3) * u3))
    dense = np.array(dense)
    seg = np.linalg.norm(np.diff(np.vstack([dense, dense[:1]]), axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    targets = np.linspace(0.0, s[-1], n, endpoint=False)
    loop = np.vstack([dense, dense[:1]])
    xy = np.stack([np.interp(targets, s, loop[:, 0]), np.interp(targets, s, loop[:, 1])], axis=1)
    tang = np.roll(xy, -1, axis=0) - np.roll(xy, 1, axis=0)
    ph = rng.uniform(0, 2 * math.pi, 3)
    poses = np.zeros((n, 3, 4))
    for k in range(n):
        a = 2 * math.pi * k / n
        yaw = math.atan2(tang[k, 1], tang[k, 0]) + math.radians(15.0) * math.sin(3 * a + ph[0])
        pitch = math.radians(-2.0 + 6.0 * math.sin(5 * a + ph[1]))
        poses[k, :, :3] = rot_z(yaw) @ rot_y(-pitch)
        if tilt_deg > 0:
            tilt = math.radians(tilt_deg)
            poses[k, :, :3] = poses[k, :, :3] @ rot_y(tilt * math.sin(7 * a + ph[0])) @ \
                rot_axis_angle((1, 0, 0), tilt * math.sin(11 * a + ph[1]))
        poses[k, :, 3] = [xy[k, 0], xy[k, 1], height + 0.1 * math.sin(4 * a + ph[2])]
    return poses


def _pose_angle_deg(A: np.ndarray, B: np.ndarray) -> float:
    c = (np.trace(A[:, :3].T @ B[:, :3]) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def overlap_ratios_t(src, tgts, sensor: Sensor, pose_src: np.ndarray, poses_tgt: np.ndarray, rays,
                     rel_tol: float = 0.05, stride: int = 7) -> np.ndarray:
    """overlap_ratio of frame src against each of the frames tgts (a list of
    (H, W, 5) tensors on src's device; poses_tgt (C, 3, 4)), on torch, all
    candidates at once; rays: the sensor's (H * W, 3) float64 pixel rays."""
    import torch
    dev = src.device
    C = len(tgts)
    if C == 0:
        return np.zeros(0)
    d = src[..., 1].reshape(-1).double()
    idx = torch.arange(0, d.numel(), stride, device=dev)
    dv = d[idx]
    keep = dv > 0
    n = int(keep.sum())
    if n == 0:
        return np.zeros(C)
    pts = rays[idx][keep] * dv[keep][:, None]
    Rs = torch.as_tensor(pose_src[:, :3], dtype=torch.float64, device=dev)
    ts = torch.as_tensor(pose_src[:, 3], dtype=torch.float64, device=dev)
    pw = pts @ Rs.T + ts                                                  # (P, 3)
    Rt = torch.as_tensor(np.asarray(poses_tgt)[:, :, :3], dtype=torch.float64, device=dev)   # (C, 3, 3)
    tt = torch.as_tensor(np.asarray(poses_tgt)[:, :, 3], dtype=torch.float64, device=dev)    # (C, 3)
    pt = torch.einsum("cpi,cij->cpj", pw[None, :, :] - tt[:, None, :], Rt)                   # (C, P, 3)
    if sensor.model == PINHOLE:
        z = pt[..., 2]
        ok = z > 1e-3
        zz = torch.where(ok, z, torch.ones_like(z))
        col = torch.round(sensor.fx * pt[..., 0] / zz + sensor.cx)
        row = torch.round(sensor.fy * pt[..., 1] / zz + sensor.cy)
        dist = z
    else:
        rxy = torch.hypot(pt[..., 0], pt[..., 1])
        col = torch.remainder(torch.round(sensor.fx * torch.atan2(pt[..., 1], pt[..., 0]) + sensor.cx), sensor.width)
        row = torch.round(sensor.fy * torch.atan2(pt[..., 2], rxy) + sensor.cy)
        dist = torch.linalg.norm(pt, dim=-1)
        ok = torch.ones_like(dist, dtype=torch.bool)
    ok = ok & (col >= 0) & (col < sensor.width) & (row >= 0) & (row < sensor.height)
    ci = torch.where(ok, col, torch.zeros_like(col)).long()
    ri = torch.where(ok, row, torch.zeros_like(row)).long()
    dep = torch.stack([t[..., 1] for t in tgts]).double()                 # (C, H, W)
    cidx = torch.arange(C, device=dev)[:, None].expand_as(ci)
    dt = dep[cidx, ri, ci]
    ok = ok & (dt > 0) & (torch.abs(dt - dist) <= rel_tol * dist + 0.05)
    return (ok.sum(dim=1).double() / float(n)).cpu().numpy()


def _noisy(ch, seed: int, depth_noise: float, intensity_noise: float):
    """Depth noise sigma = depth_noise * z^2 and intensity noise (seeded, on the channels' device)."""
    import torch
    g = torch.Generator(device=ch.device)
    g.manual_seed(seed)
    valid = ch[..., 1] > 0
    z = ch[..., 1].double()
    nz = torch.randn(z.shape, generator=g, device=ch.device, dtype=torch.float64)
    ni = torch.randn(z.shape, generator=g, device=ch.device, dtype=torch.float64)
    out = ch.clone()
    out[..., 1] = torch.where(valid, z + nz * depth_noise * z * z, torch.zeros_like(z)).float()
    out[..., 0] = torch.where(valid, ch[..., 0].double() + ni * intensity_noise, torch.zeros_like(z)).float()
    return out


def make_rgbd_hall(n_frames: int = 200, width: int = 640, height: int = 480, f: float = 525.0, seed: int = 3,
                   sigma_t: float = 0.02, sigma_r_deg: float = 1.0, depth_noise: float = 1e-3,
                   intensity_noise: float = 0.01, max_angle_deg: float = 30.0, max_dist: float = 1.0,
                   min_ratio: float = 1.0 / 3.0, device="cuda", fp16_exact: bool = False,
                   params: Optional[Dict] = None) -> Workload:
    """RGB-D 640 x 480 sequence of n_frames along a smooth closed spline
    through the four rooms of _hall_scene; depth noise sigma = 1 mm z^2,
    intensity noise sigma = 0.01 (with fp16_exact, intensity and normals
    rounded to binary16 afterwards).  Pairs by the Sec. IV-B rule on the initial poses: rotation
    angle < 30 deg, translation < 1 m, overlap ratio (renderer geometry) >
    1/3, plus consecutive frames (a sequential acquisition, closing the
    loop).  Channels are torch tensors on `device`.  Seeds: scene 1000 + seed,
    trajectory 2000 + seed, perturbation 3000 + seed, noise 5000 + seed."""
    import torch
    scene = _hall_scene(1000 + seed)
    cam = pinhole_sensor(width, height, f, (width - 1) / 2.0, (height - 1) / 2.0)
    Xc = np.zeros((3, 4))
    Xc[:, :3] = CAMERA_ON_PLATFORM
    cam.extrinsic = Xc
    plat = _hall_path(n_frames, 2000 + seed)
    rays = torch.as_tensor(_pixel_rays(cam)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    st = _scene_tensors(scene, device)
    chans = []
    for k in range(n_frames):
        c = render_t(scene, cam, compose(plat[k], Xc), 0.5, 5.0, device=device, rays=rays, st=st)
        c = _noisy(c, 5000 + seed * 977 + k, depth_noise, intensity_noise)
        chans.append(quantize_fp16_t(c) if fp16_exact else c)
    init = perturb_poses(plat, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    pairs = []
    for i in range(n_frames):
        cand = [j for j in range(i + 1, n_frames) if np.linalg.norm(init[i, :, 3] - init[j, :, 3]) < max_dist and
                _pose_angle_deg(init[i], init[j]) < max_angle_deg]
        ratios = overlap_ratios_t(chans[i], [chans[j] for j in cand], cam, compose(plat[i], Xc),
                                  np.array([compose(plat[j], Xc) for j in cand]).reshape(-1, 3, 4), rays)
        pairs += [(i, j) for j, r in zip(cand, ratios) if r > min_ratio]
    # a sequential acquisition: consecutive frames are paired as well (Sec. IV-B)
    have = set(pairs)
    for i in range(n_frames):
        j = (i + 1) % n_frames
        if (min(i, j), max(i, j)) not in have:
            pairs.append((min(i, j), max(i, j)))
    pairs.sort()
    prm = default_params(range_min=0.5, range_max=5.0)
    if params:
        prm.update(params)
    return Workload(f"rgbd-hall-{n_frames}x{width}x{height}", [cam], np.zeros(n_frames, dtype=np.int32), chans,
                    plat, init, np.array(pairs, dtype=np.int32).reshape(-1, 2), prm)


def make_lidar_street_graph(n_frames: int = 500, width: int = 2048, height: int = 128, vfov_up_deg: float = 22.5,
                            vfov_down_deg: float = -22.5, spacing: float = 1.0, seed: int = 4,
                            sigma_t: float = 0.10, sigma_r_deg: float = 0.5, drop: float = 0.05,
                            degree=(2, 20), window: int = 40, min_overlap: float = 0.3, device="cuda",
                            fp16_exact: bool = False, params: Optional[Dict] = None) -> Workload:
    """LiDAR 128 x 2048 sequence of n_frames along the synthetic street with an
    uneven overlap graph: frame i is the source of d_i pairs, d_i uniform in
    [2, 20], towards frames j != i within `window` frames whose overlap ratio
    exceeds `min_overlap`, drawn at random (seeded) among them.  Channels are
    torch tensors on `device`.  Seeds: scene 1000 + seed, trajectory 2000 +
    seed, perturbation 3000 + seed, dropped returns 4000 + seed, graph
    6000 + seed."""
    import torch
    poses = _street_trajectory(n_frames, spacing, 2000 + seed)
    scene = _street_scene(1000 + seed, 0.0, (n_frames - 1) * spacing)
    sensor = spherical_sensor(width, height, vfov_up_deg, vfov_down_deg)
    rays = torch.as_tensor(_pixel_rays(sensor)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(4000 + seed)
    st = _scene_tensors(scene, device)
    chans = []
    for k in range(n_frames):
        c = render_t(scene, sensor, poses[k], 1.0, 80.0, device=device, rays=rays, st=st)
        keep = torch.rand((height, width), generator=g, device=device) >= drop
        c = torch.where(keep[..., None], c, torch.zeros_like(c))
        chans.append(quantize_fp16_t(c) if fp16_exact else c)
    rng = np.random.default_rng(6000 + seed)
    pairs = []
    for i in range(n_frames):
        near = [j for j in range(max(0, i - window), min(n_frames, i + window + 1)) if j != i]
        ratios = overlap_ratios_t(chans[i], [chans[j] for j in near], sensor, poses[i], poses[near], rays)
        cand = [j for j, r in zip(near, ratios) if r > min_overlap]
        d = int(rng.integers(degree[0], degree[1] + 1))
        for j in sorted(rng.permutation(cand)[:d].tolist()):
            pairs.append((i, j))
    init = perturb_poses(poses, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    prm = default_params(w_depth=0.1, huber_delta=0.2, occ_abs=0.3, occ_rel=0.05, z_min=0.5,
                         range_min=1.0, range_max=80.0)
    if params:
        prm.update(params)
    return Workload(f"lidar-street-graph-{n_frames}x{height}x{width}", [sensor],
                    np.zeros(n_frames, dtype=np.int32), chans, poses, init,
                    np.array(pairs, dtype=np.int32).reshape(-1, 2), prm)


def offset_error(Xa: np.ndarray, Xb: np.ndarray) -> Tuple[float, float]:
    """Translation [m] and rotation [deg] of Xa^-1 Xb (3x4 rigid transforms)."""
    R = Xa[:, :3].T @ Xb[:, :3]
    t = Xa[:, :3].T @ (Xb[:, 3] - Xa[:, 3])
    return float(np.linalg.norm(t)), math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))))


def make_joint_hall(n_lidar: int = 300, lidar_width: int = 1024, lidar_height: int = 128,
                    vfov_up_deg: float = 45.0, vfov_down_deg: float = -45.0, cam_width: int = 640,
                    cam_height: int = 480, f: float = 525.0, rate: int = 2, cam_offset=(0.10, 0.0, 0.10),
                    offset_error_m: float = 0.02, offset_error_deg: float = 0.5, seed: int = 5,
                    sigma_t: float = 0.02, sigma_r_deg: float = 1.0, tilt_deg: float = 10.0, device="cuda",
                    fp16_exact: bool = False, params: Optional[Dict] = None) -> Workload:
    """Joint LiDAR + RGB-D platform in the hall (Sec. V, fusion): n_lidar LiDAR
    frames (128 x 1024, vfov +-45 deg, the platform origin) and rate x n_lidar
    camera frames (640 x 480, `cam_offset` ahead / above, looking forward)
    along the hall's spline path, hand-held (roll and pitch of up to tilt_deg,
    so that the offset's translation is observable); camera frame rate k and
    LiDAR frame k share a platform pose.  The camera's offset given to the problem (the sensor's
    extrinsic) is the true one composed with a seeded error of
    offset_error_m / offset_error_deg; extrinsic_gt holds the true offsets.
    Frames: cameras first, then LiDARs; frame_var ties camera rate k and
    LiDAR k and holds the first platform pose fixed.  Pairs: camera (i, j)
    by the Sec. IV-B rule (30 deg, 1 m, overlap > 1/3) plus consecutive
    frames; LiDAR (i, j), j - i <= 4, overlap > 0.3.  Channels are torch
    tensors on `device`.  Seeds: scene 1000 + seed, path 2000 + seed,
    perturbation 3000 + seed, offset error 4000 + seed."""
    import torch
    n_cam = rate * n_lidar
    scene = _hall_scene(1000 + seed)
    st = _scene_tensors(scene, device)
    cam = pinhole_sensor(cam_width, cam_height, f, (cam_width - 1) / 2.0, (cam_height - 1) / 2.0)
    Xc = np.zeros((3, 4))
    Xc[:, :3] = CAMERA_ON_PLATFORM
    Xc[:, 3] = cam_offset
    lidar = spherical_sensor(lidar_width, lidar_height, vfov_up_deg, vfov_down_deg)
    plat = _hall_path(n_cam, 2000 + seed, height=1.5, tilt_deg=tilt_deg)
    rays_c = torch.as_tensor(_pixel_rays(cam)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    rays_l = torch.as_tensor(_pixel_rays(lidar)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    chans = [render_t(scene, cam, compose(plat[k], Xc), 0.5, 5.0, device, rays_c, st) for k in range(n_cam)]
    chans += [render_t(scene, lidar, plat[rate * k], 0.5, 12.0, device, rays_l, st) for k in range(n_lidar)]
    if fp16_exact:
        chans = [quantize_fp16_t(c) for c in chans]
    rng = np.random.default_rng(4000 + seed)
    ax = rng.normal(size=3)
    d = rng.normal(size=3)
    err = np.zeros((3, 4))
    err[:, :3] = rot_vec(math.radians(offset_error_deg) * ax / np.linalg.norm(ax))
    err[:, 3] = offset_error_m * d / np.linalg.norm(d)
    cam.extrinsic = compose(Xc, err)
    init_plat = perturb_poses(plat, sigma_t, math.radians(sigma_r_deg), 3000 + seed)
    poses = np.concatenate([plat, plat[::rate]])
    init = np.concatenate([init_plat, init_plat[::rate]])
    pairs = []
    for i in range(n_cam):
        cand = [j for j in range(i + 1, n_cam) if np.linalg.norm(init[i, :, 3] - init[j, :, 3]) < 1.0 and
                _pose_angle_deg(init[i], init[j]) < 30.0]
        ratios = overlap_ratios_t(chans[i], [chans[j] for j in cand], cam, compose(plat[i], Xc),
                                  np.array([compose(plat[j], Xc) for j in cand]).reshape(-1, 3, 4), rays_c)
        pairs += [(i, j) for j, r in zip(cand, ratios) if r > 1.0 / 3.0]
        if i + 1 < n_cam and (i, i + 1) not in pairs:
            pairs.append((i, i + 1))
    for i in range(n_lidar):
        near = list(range(i + 1, min(n_lidar, i + 5)))
        ratios = overlap_ratios_t(chans[n_cam + i], [chans[n_cam + j] for j in near], lidar, plat[rate * i],
                                  plat[[rate * j for j in near]].reshape(-1, 3, 4), rays_l)
        pairs += [(n_cam + i, n_cam + j) for j, r in zip(near, ratios) if r > 0.3]
    fv = np.array([k - 1 for k in range(n_cam)] + [rate * k - 1 for k in range(n_lidar)], dtype=np.int32)
    prm = default_params(range_min=0.5, range_max=12.0)
    if params:
        prm.update(params)
    ident = IDENTITY_3x4.copy()
    return Workload(f"joint-hall-{n_lidar}x{lidar_height}x{lidar_width}+{n_cam}x{cam_width}x{cam_height}",
                    [cam, lidar], np.array([0] * n_cam + [1] * n_lidar, dtype=np.int32), chans, poses, init,
                    np.array(sorted(pairs), dtype=np.int32).reshape(-1, 2), prm, fv, n_cam - 1, [Xc, ident])


def make_street_batch(n_problems: int = 16, sizes=(50, 400), width: int = 1024, height: int = 64, seed: int = 6,
                      device="cuda", fp16_exact: bool = False, params: Optional[Dict] = None):
    """n_problems independent LiDAR street problems (sizes drawn uniformly in
    `sizes`, seed 3005 + seed) concatenated into one workload: frames of
    problem k follow those of problem k - 1, pairs stay within a problem
    ((i, j), j - i <= 3, overlap > 0.3), and the first frame of every problem
    is held fixed (frame_var), so the problems share nothing but the launch.
    Returns (workload, list of (first frame, n_frames) per problem)."""
    import torch
    rng = np.random.default_rng(3005 + seed)
    ns = [int(x) for x in rng.integers(sizes[0], sizes[1] + 1, n_problems)]
    sensor = spherical_sensor(width, height, 16.6, -16.6)
    rays = torch.as_tensor(_pixel_rays(sensor)[0].reshape(-1, 3), dtype=torch.float64, device=device)
    chans, poses, init, pairs, fv, spans = [], [], [], [], [], []
    g = torch.Generator(device=device)
    g.manual_seed(4000 + seed)
    n_var = 0
    for k, n in enumerate(ns):
        base = len(chans)
        P = _street_trajectory(n, 1.0, 2000 + 100 * seed + k)
        scene = _street_scene(1000 + 100 * seed + k, 0.0, (n - 1) * 1.0)
        st = _scene_tensors(scene, device)
        for f in range(n):
            c = render_t(scene, sensor, P[f], 1.0, 80.0, device, rays, st)
            keep = torch.rand((height, width), generator=g, device=device) >= 0.05
            c = torch.where(keep[..., None], c, torch.zeros_like(c))
            chans.append(quantize_fp16_t(c) if fp16_exact else c)
        for i in range(n):
            near = list(range(i + 1, min(n, i + 4)))
            ratios = overlap_ratios_t(chans[base + i], [chans[base + j] for j in near], sensor, P[i], P[near], rays)
            pairs += [(base + i, base + j) for j, r in zip(near, ratios) if r > 0.3]
        poses.append(P)
        init.append(perturb_poses(P, 0.10, math.radians(0.5), 3000 + 100 * seed + k))
        fv += [-1] + list(range(n_var, n_var + n - 1))
        n_var += n - 1
        spans.append((base, n))
    prm = default_params(w_depth=0.1, huber_delta=0.2, occ_abs=0.3, occ_rel=0.05, z_min=0.5,
                         range_min=1.0, range_max=80.0)
    if params:
        prm.update(params)
    w = Workload(f"street-batch-{n_problems}x{height}x{width}", [sensor], np.zeros(len(chans), dtype=np.int32),
                 chans, np.concatenate(poses), np.concatenate(init), np.array(pairs, dtype=np.int32).reshape(-1, 2),
                 prm, np.array(fv, dtype=np.int32), n_var)
    return w, spans
