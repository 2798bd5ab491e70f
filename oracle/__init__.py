"""FP64 CPU oracle of the photometric bundle-adjustment step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package entry's smoke
check and by the benchmark's CPU-baseline leg, never by the product path.
The arithmetic lives in `pba_oracle.c` (plain C, double precision, one point at
a time, following the paper's equations); this module compiles it with gcc and
marshals numpy arrays.  It shares no code with the CUDA library.

The Levenberg-Marquardt driver (`lm_iteration`) is written out here in Python:
linearise, damp and solve (Sec. IV-C), apply X [+] dx (Supp.), re-evaluate the
cost, accept when it decreased (lambda / 10) or reject (lambda x 10).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pba_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

PINHOLE = 0
SPHERICAL = 1


class OSensor(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("pad_", ctypes.c_int), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("Xo", ctypes.c_double * 12)]


class OParams(ctypes.Structure):
    _fields_ = [("w_int", ctypes.c_double), ("w_depth", ctypes.c_double), ("w_normal", ctypes.c_double),
                ("huber_delta", ctypes.c_double), ("occ_abs", ctypes.c_double), ("occ_rel", ctypes.c_double),
                ("z_min", ctypes.c_double), ("range_min", ctypes.c_double), ("range_max", ctypes.c_double),
                ("margin_px", ctypes.c_double), ("margin_rel", ctypes.c_double),
                ("grad_mode", ctypes.c_int), ("other_branch", ctypes.c_int), ("texel_f16", ctypes.c_int)]


def build(force: bool = False, src: Optional[str] = None, out: Optional[str] = None) -> str:
    """Compile pba_oracle.c into a shared library (gcc, -ffp-contract=off so
    x86 and Arm builds round identically).  `src` / `out` compile another copy
    of the source (tests plant a mistake in a private copy this way)."""
    src = src or _SRC
    out = out or _LIB_PATH
    if not force and src == _SRC and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_lib = None


def load(path: Optional[str] = None):
    """The oracle library; `path` loads another build (a planted-mistake copy)."""
    return _load(path)


def _load(path: Optional[str] = None):
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(lib):
    P = ctypes.POINTER
    d, i32, i64, u32 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    S, Pr = P(OSensor), P(OParams)
    lib.o_half.argtypes = [ctypes.c_float]
    lib.o_half.restype = d
    lib.o_project.argtypes = [S, P(d), P(d)]
    lib.o_unproject.argtypes = [S, d, d, d, P(d)]
    lib.o_proj_jacobian.argtypes = [S, P(d), P(d)]
    lib.o_boxplus.argtypes = [P(d), P(d), P(d)]
    lib.o_frame_points.argtypes = [S, Pr, P(ctypes.c_float), P(d), P(i32), ctypes.c_int]
    lib.o_frame_points.restype = ctypes.c_int
    lib.o_point_residual.argtypes = [S, Pr, P(ctypes.c_float), P(d), P(d), P(d), P(d), P(d), P(d),
                                     P(d), P(d), P(ctypes.c_int)]
    lib.o_point_residual.restype = ctypes.c_int
    lib.o_linearize_pair.argtypes = [S, Pr, P(ctypes.c_float), P(ctypes.c_float), P(d), P(d), P(d), P(d),
                                     P(d), P(i64), P(u32), P(u32)]
    lib.o_linearize_pair.restype = ctypes.c_int
    lib.o_linearize.argtypes = [ctypes.c_int, S, P(i32), P(P(ctypes.c_float)), P(d), ctypes.c_int, P(i32), Pr,
                                P(d), P(d), P(d), P(i64), P(d), P(d), P(d), P(i64)]
    lib.o_linearize.restype = ctypes.c_int
    lib.o_cholesky_solve.argtypes = [ctypes.c_int, P(d), P(d), P(d)]
    lib.o_cholesky_solve.restype = ctypes.c_int
    lib.o_solve_step.argtypes = [ctypes.c_int, P(d), P(d), d, P(d)]
    lib.o_solve_step.restype = ctypes.c_int
    lib.o_apply_update.argtypes = [ctypes.c_int, P(d), P(d), P(d)]
    lib.o_offset_map.argtypes = [P(d), P(d)]
    lib.o_offset_jacobian.argtypes = [P(d), P(d), P(d), P(d)]
    lib.o_pair_offset_blocks.argtypes = [S, Pr, P(ctypes.c_float), P(ctypes.c_float), P(d), P(d), P(d)]
    lib.o_pair_offset_blocks.restype = ctypes.c_int
    return lib


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _sensor(s) -> OSensor:
    """Accepts a synth.Sensor-like object or a dict with the same fields."""
    g = (lambda k: s[k]) if isinstance(s, dict) else (lambda k: getattr(s, k))
    o = OSensor()
    o.model, o.width, o.height = int(g("model")), int(g("width")), int(g("height"))
    o.fx, o.fy, o.cx, o.cy = float(g("fx")), float(g("fy")), float(g("cx")), float(g("cy"))
    xo = np.asarray(g("extrinsic"), dtype=np.float64).reshape(12)
    for k in range(12):
        o.Xo[k] = xo[k]
    return o


def _params(p: Dict, margin_px: float = 1e-3, margin_rel: float = 1e-4) -> OParams:
    o = OParams()
    for k in ("w_int", "w_depth", "w_normal", "huber_delta", "occ_abs", "occ_rel", "z_min",
              "range_min", "range_max"):
        setattr(o, k, float(p[k]))
    o.margin_px = float(p.get("margin_px", margin_px))
    o.margin_rel = float(p.get("margin_rel", margin_rel))
    o.grad_mode = int(p.get("grad_mode", 0))
    o.other_branch = int(p.get("other_branch", 0))
    # R25: the target's intensity and normals sampled as binary16 values (FP16 texels)
    o.texel_f16 = int(p.get("texel_f16", 0))
    return o


# ---------------------------------------------------------------- primitives

def half_round(x, lib=None) -> np.ndarray:
    """Each float32 value rounded to the nearest binary16 number (R25), as float64."""
    lib = lib or _load()
    x = np.asarray(x, dtype=np.float32)
    return np.array([lib.o_half(float(v)) for v in x.reshape(-1)]).reshape(x.shape)


def project(sensor, p, lib=None) -> np.ndarray:
    lib, p = lib or _load(), _f64(p)
    uv = np.zeros(2)
    lib.o_project(ctypes.byref(_sensor(sensor)), _ptr(p, ctypes.c_double), _ptr(uv, ctypes.c_double))
    return uv


def unproject(sensor, u: float, v: float, d: float, lib=None) -> np.ndarray:
    lib = lib or _load()
    p = np.zeros(3)
    lib.o_unproject(ctypes.byref(_sensor(sensor)), u, v, d, _ptr(p, ctypes.c_double))
    return p


def proj_jacobian(sensor, p, lib=None) -> np.ndarray:
    lib, p = lib or _load(), _f64(p)
    J = np.zeros(6)
    lib.o_proj_jacobian(ctypes.byref(_sensor(sensor)), _ptr(p, ctypes.c_double), _ptr(J, ctypes.c_double))
    return J.reshape(2, 3)


def boxplus(X, dx, lib=None) -> np.ndarray:
    lib, X, dx = lib or _load(), _f64(X).reshape(12), _f64(dx).reshape(6)
    out = np.zeros(12)
    lib.o_boxplus(_ptr(X, ctypes.c_double), _ptr(dx, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out.reshape(3, 4)


def frame_points(sensor, params: Dict, channels: np.ndarray, lib=None):
    """(points (P, 7) = p_u, g_u, n_u^o ; pixel indices (P,)) in raster order."""
    lib = lib or _load()
    ch = np.ascontiguousarray(channels, dtype=np.float32)
    s = _sensor(sensor)
    cap = s.width * s.height
    out = np.zeros((cap, 7))
    pix = np.zeros(cap, dtype=np.int32)
    n = lib.o_frame_points(ctypes.byref(s), ctypes.byref(_params(params)), _ptr(ch, ctypes.c_float),
                           _ptr(out, ctypes.c_double), _ptr(pix, ctypes.c_int32), cap)
    return out[:n].copy(), pix[:n].copy()


def point_residual(sensor, params: Dict, tgt_channels: np.ndarray, Xi, Xj, pt, lib=None,
                   other_branch: bool = False) -> Dict:
    """One pixel-point's residual, Jacobians, rho, weight and margin flag.
    other_branch: overrule rejections whose decision lies within its margin
    (the contribution a float32 implementation may count)."""
    lib = lib or _load()
    if other_branch:
        params = dict(params, other_branch=1)
    tgt = np.ascontiguousarray(tgt_channels, dtype=np.float32)
    Xi, Xj, pt = _f64(Xi).reshape(12), _f64(Xj).reshape(12), _f64(pt).reshape(7)
    e, Ji, Jj = np.zeros(5), np.zeros(30), np.zeros(30)
    rho, w, flag = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    ok = lib.o_point_residual(ctypes.byref(_sensor(sensor)), ctypes.byref(_params(params)),
                              _ptr(tgt, ctypes.c_float), _ptr(Xi, ctypes.c_double), _ptr(Xj, ctypes.c_double),
                              _ptr(pt, ctypes.c_double), _ptr(e, ctypes.c_double), _ptr(Ji, ctypes.c_double),
                              _ptr(Jj, ctypes.c_double), ctypes.byref(rho), ctypes.byref(w), ctypes.byref(flag))
    return dict(valid=bool(ok), e=e, Ji=Ji.reshape(5, 6), Jj=Jj.reshape(5, 6), rho=rho.value, w=w.value,
                flag=bool(flag.value))


def point_contribution(sensor, params: Dict, tgt_channels: np.ndarray, Xi, Xj, pt, lib=None,
                       other_branch: bool = False):
    """(H12, b12, rho) of one pixel-point, w J^T Omega J and w J^T Omega e with
    J = [J_i J_j] (the terms o_linearize_pair sums), or None when rejected."""
    r = point_residual(sensor, params, tgt_channels, Xi, Xj, pt, lib=lib, other_branch=other_branch)
    if not r["valid"]:
        return None
    J = np.hstack([r["Ji"], r["Jj"]])
    om = np.array([params["w_int"], params["w_depth"]] + [params["w_normal"]] * 3)
    return r["w"] * (J.T * om) @ J, r["w"] * (J.T * om) @ r["e"], r["rho"]


def linearize_pair(sensor, params: Dict, src: np.ndarray, tgt: np.ndarray, Xi, Xj, lib=None) -> Dict:
    """H12 (12x12), b12, cost, count, mask and margin-flag bit words of one pair."""
    lib = lib or _load()
    src = np.ascontiguousarray(src, dtype=np.float32)
    tgt = np.ascontiguousarray(tgt, dtype=np.float32)
    Xi, Xj = _f64(Xi).reshape(12), _f64(Xj).reshape(12)
    s = _sensor(sensor)
    cap_words = (s.width * s.height + 31) // 32 + 1
    H, b = np.zeros(144), np.zeros(12)
    cost, count = ctypes.c_double(0.0), ctypes.c_int64(0)
    mask = np.zeros(cap_words, dtype=np.uint32)
    flags = np.zeros(cap_words, dtype=np.uint32)
    n = lib.o_linearize_pair(ctypes.byref(s), ctypes.byref(_params(params)), _ptr(src, ctypes.c_float),
                             _ptr(tgt, ctypes.c_float), _ptr(Xi, ctypes.c_double), _ptr(Xj, ctypes.c_double),
                             _ptr(H, ctypes.c_double), _ptr(b, ctypes.c_double), ctypes.byref(cost),
                             ctypes.byref(count), _ptr(mask, ctypes.c_uint32), _ptr(flags, ctypes.c_uint32))
    if n < 0:
        raise MemoryError("oracle: allocation failed")
    nw = (n + 31) // 32
    return dict(H=H.reshape(12, 12), b=b, cost=cost.value, count=count.value, n_points=n,
                mask=mask[:nw].copy(), flags=flags[:nw].copy())


def accounted_pair(s, params, src, tgt, Xi, Xj, other_mask, r, lib=None):
    """The oracle's sums of one pair (r = linearize_pair's result) with every
    point that another implementation decided the other way (other_mask: its
    valid-point bit words) moved to that side: the point's contribution (from
    the oracle, or from the oracle's other-branch evaluation when the oracle
    rejected it) is removed or added.  Returns (H, b, cost, count, n_flipped,
    n_unexplained); n_unexplained counts points decided the other way with no
    other-branch evaluation (outside every decision margin)."""
    H, b, cost, count = r["H"].copy(), r["b"].copy(), r["cost"], r["count"]
    n = r["n_points"]
    diff = np.unpackbits((other_mask ^ r["mask"]).view(np.uint8), bitorder="little")[:n]
    ok_o = np.unpackbits(r["mask"].view(np.uint8), bitorder="little")[:n]
    idx = np.nonzero(diff)[0]
    unexplained = 0
    if idx.size:
        pts, _ = frame_points(s, params, src, lib=lib)
        for k in idx.tolist():
            c = point_contribution(s, params, tgt, Xi, Xj, pts[k], lib=lib, other_branch=not ok_o[k])
            if c is None:
                unexplained += 1
                continue
            sign = -1.0 if ok_o[k] else 1.0
            H += sign * c[0]
            b += sign * c[1]
            cost += sign * c[2]
            count += int(sign)
    return H, b, cost, count, int(idx.size), unexplained


def offset_map(extrinsic) -> np.ndarray:
    """A_o (6 x 6): the offset perturbation d acts like A_o d on both poses (R23)."""
    lib = _load()
    A = np.zeros(36)
    lib.o_offset_map(_ptr(_f64(extrinsic).reshape(12), ctypes.c_double), _ptr(A, ctypes.c_double))
    return A.reshape(6, 6)


def pair_offset_blocks(sensor, params: Dict, src: np.ndarray, tgt: np.ndarray, Xi, Xj, lib=None) -> Dict:
    """Offset blocks of one pair (R23): H_io, H_jo, H_oo (6x6 each) and b_o."""
    lib = lib or _load()
    src = np.ascontiguousarray(src, dtype=np.float32)
    tgt = np.ascontiguousarray(tgt, dtype=np.float32)
    out = np.zeros(114)
    n = lib.o_pair_offset_blocks(ctypes.byref(_sensor(sensor)), ctypes.byref(_params(params)),
                                 _ptr(src, ctypes.c_float), _ptr(tgt, ctypes.c_float),
                                 _ptr(_f64(Xi).reshape(12), ctypes.c_double),
                                 _ptr(_f64(Xj).reshape(12), ctypes.c_double), _ptr(out, ctypes.c_double))
    if n < 0:
        raise MemoryError("oracle: allocation failed")
    return dict(H_io=out[:36].reshape(6, 6), H_jo=out[36:72].reshape(6, 6), H_oo=out[72:108].reshape(6, 6),
                b_o=out[108:].copy())


def offset_jacobian(extrinsic, Ji, Jj) -> np.ndarray:
    """J_o = (J_i + J_j) A_o (5 x 6, R23)."""
    lib = _load()
    Jo = np.zeros(30)
    lib.o_offset_jacobian(_ptr(_f64(extrinsic).reshape(12), ctypes.c_double), _ptr(_f64(Ji).reshape(30), ctypes.c_double),
                          _ptr(_f64(Jj).reshape(30), ctypes.c_double), _ptr(Jo, ctypes.c_double))
    return Jo.reshape(5, 6)


def linearize(sensors: Sequence, frame_sensor, channels: Sequence[np.ndarray], poses, pairs, params: Dict,
              want_system: bool = True, want_pairs: bool = False, lib=None) -> Dict:
    """Dense H (6N x 6N, gauge not fixed), b, total cost F (Eq. total-error-multicue), count."""
    lib = lib or _load()
    n = len(channels)
    chans = [np.ascontiguousarray(c, dtype=np.float32) for c in channels]
    cptrs = (ctypes.POINTER(ctypes.c_float) * n)(*[_ptr(c, ctypes.c_float) for c in chans])
    sarr = (OSensor * len(sensors))(*[_sensor(s) for s in sensors])
    fs = np.ascontiguousarray(frame_sensor, dtype=np.int32)
    poses = _f64(poses).reshape(n, 12)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    m = pairs.shape[0]
    H = np.zeros((6 * n, 6 * n)) if want_system else None
    b = np.zeros(6 * n) if want_system else None
    pH = np.zeros((m, 12, 12)) if want_pairs else None
    pb = np.zeros((m, 12)) if want_pairs else None
    pc = np.zeros(m)
    pn = np.zeros(m, dtype=np.int64)
    cost, count = ctypes.c_double(0.0), ctypes.c_int64(0)
    st = lib.o_linearize(n, sarr, _ptr(fs, ctypes.c_int32), cptrs, _ptr(poses, ctypes.c_double), m,
                         _ptr(pairs, ctypes.c_int32), ctypes.byref(_params(params)), _ptr(H, ctypes.c_double),
                         _ptr(b, ctypes.c_double), ctypes.byref(cost), ctypes.byref(count),
                         _ptr(pH, ctypes.c_double), _ptr(pb, ctypes.c_double), _ptr(pc, ctypes.c_double),
                         _ptr(pn, ctypes.c_int64))
    if st != 0:
        raise ValueError(f"oracle: malformed pair list (status {st})")
    return dict(H=H, b=b, cost=cost.value, count=count.value, pair_H=pH, pair_b=pb, pair_cost=pc,
                pair_count=pn)


def cholesky_solve(A, rhs, lib=None) -> np.ndarray:
    lib, A, rhs = lib or _load(), _f64(A), _f64(rhs)
    x = np.zeros(rhs.shape[0])
    st = lib.o_cholesky_solve(rhs.shape[0], _ptr(A, ctypes.c_double), _ptr(rhs, ctypes.c_double),
                              _ptr(x, ctypes.c_double))
    if st != 0:
        raise np.linalg.LinAlgError("oracle: matrix not positive definite")
    return x


def solve_step(H, b, lam: float, lib=None):
    """dx (6N) with dx_0 = 0; returns (dx, ok)."""
    lib, H, b = lib or _load(), _f64(H), _f64(b)
    n = b.shape[0] // 6
    dx = np.zeros(6 * n)
    st = lib.o_solve_step(n, _ptr(H, ctypes.c_double), _ptr(b, ctypes.c_double), float(lam),
                          _ptr(dx, ctypes.c_double))
    return dx, st == 0


def apply_update(poses, dx, lib=None) -> np.ndarray:
    lib, poses, dx = lib or _load(), _f64(poses), _f64(dx)
    n = poses.reshape(-1, 12).shape[0]
    out = np.zeros((n, 12))
    lib.o_apply_update(n, _ptr(poses.reshape(n, 12), ctypes.c_double), _ptr(dx, ctypes.c_double),
                       _ptr(out, ctypes.c_double))
    return out.reshape(n, 3, 4)


def initial_lambda(H) -> float:
    """lambda_0 = 1e-4 * max diag(H_ff) (frame 0 excluded)."""
    d = np.diag(np.asarray(H))[6:]
    return 1e-4 * float(d.max()) if d.size else 0.0


def selection(frame_var, n_vars: int) -> np.ndarray:
    """S (6N x 6 n_vars) with S[6k + a, 6 v + a] = 1 when frame k's pose moves
    with variable v (frame_var[k] = v); rows of frames with frame_var[k] = -1
    (held fixed) are zero.  The pose perturbations are dx_frames = S dx_vars."""
    fv = np.asarray(frame_var, dtype=np.int64)
    S = np.zeros((6 * fv.size, 6 * n_vars))
    for k, v in enumerate(fv):
        if v >= 0:
            S[6 * k:6 * k + 6, 6 * v:6 * v + 6] = np.eye(6)
    return S


def solve_step_vars(H, b, lam: float, frame_var, n_vars: int, lib=None):
    """Damped Gauss-Newton step when frames share pose variables or are held
    fixed: F(X [+] S dx_v) has gradient S^T b and Gauss-Newton matrix S^T H S,
    so dx_v = -(S^T H S + lam I)^-1 S^T b (the oracle's Cholesky) and the
    frames move by S dx_v.  Returns (dx_frames (6N), ok)."""
    S = selection(frame_var, n_vars)
    Hr = S.T @ np.asarray(H, dtype=np.float64) @ S
    br = S.T @ np.asarray(b, dtype=np.float64)
    try:
        x = cholesky_solve(Hr + lam * np.eye(Hr.shape[0]), -br, lib=lib)
    except np.linalg.LinAlgError:
        return np.zeros(S.shape[0]), False
    return S @ x, True


def initial_lambda_vars(H, frame_var, n_vars: int) -> float:
    """lambda_0 = 1e-4 * max diag(S^T H S)."""
    S = selection(frame_var, n_vars)
    d = np.diag(S.T @ np.asarray(H, dtype=np.float64) @ S)
    return 1e-4 * float(d.max()) if d.size else 0.0


def offset_system(w, sensors, poses, lin: Dict, free: Sequence[int], lib=None):
    """H and b over the blocks [frames..., free offsets...]: the frames' system
    of `lin` plus, per pair of a sensor with a free offset, its offset blocks
    from pair_offset_blocks (R23) at rows/columns of that offset."""
    n = len(w.channels)
    nb = n + len(free)
    H = np.zeros((6 * nb, 6 * nb))
    b = np.zeros(6 * nb)
    H[:6 * n, :6 * n] = lin["H"]
    b[:6 * n] = lin["b"]
    for i, j in np.asarray(w.pairs).reshape(-1, 2).tolist():
        s = int(w.frame_sensor[i])
        if s not in free:
            continue
        o = 6 * (n + list(free).index(s))
        blk = pair_offset_blocks(sensors[s], w.params, w.channels[i], w.channels[j], poses[i], poses[j], lib=lib)
        for f, Hfo in ((i, blk["H_io"]), (j, blk["H_jo"])):
            H[6 * f:6 * f + 6, o:o + 6] += Hfo
            H[o:o + 6, 6 * f:6 * f + 6] += Hfo.T
        H[o:o + 6, o:o + 6] += blk["H_oo"]
        b[o:o + 6] += blk["b_o"]
    return H, b


def _with_offsets(sensors, offsets: Dict):
    out = []
    for k, s in enumerate(sensors):
        if k in offsets:
            d = s.as_dict() if hasattr(s, "as_dict") else dict(s)
            d["extrinsic"] = np.asarray(offsets[k], dtype=np.float64).reshape(12)
            out.append(d)
        else:
            out.append(s)
    return out


def _extrinsic_of(s) -> np.ndarray:
    g = s["extrinsic"] if isinstance(s, dict) else s.extrinsic
    return np.asarray(g, dtype=np.float64).reshape(3, 4)


def lm_iteration_offsets(w, poses, sensors, lam: Optional[float], free: Sequence[int], lib=None) -> Dict:
    """One Levenberg-Marquardt iteration whose variables are the frames' (as in
    lm_iteration) and the offsets of the sensors in `free` (R23), at `poses`
    with `sensors` carrying the current offsets.  Returns the accepted poses
    and sensors, the new lambda and both costs."""
    lin = linearize(sensors, w.frame_sensor, w.channels, poses, w.pairs, w.params, lib=lib)
    H, b = offset_system(w, sensors, poses, lin, free, lib=lib)
    n = len(w.channels)
    fv = getattr(w, "frame_var", None)
    if fv is None:
        fv, nf = np.arange(-1, n - 1), n - 1
    else:
        nf = w.n_vars
    blocks_var = np.concatenate([np.asarray(fv), nf + np.arange(len(free))])
    S = selection(blocks_var, nf + len(free))
    Hr, br = S.T @ H @ S, S.T @ b
    if lam is None:
        lam = 1e-4 * float(np.diag(Hr).max())
    try:
        x = cholesky_solve(Hr + lam * np.eye(Hr.shape[0]), -br, lib=lib)
        ok = True
    except np.linalg.LinAlgError:
        x, ok = np.zeros(Hr.shape[0]), False
    dx = S @ x
    cand = apply_update(poses, dx[:6 * n], lib=lib)
    offs = {s: boxplus(_extrinsic_of(sensors[s]), dx[6 * (n + k):6 * (n + k) + 6], lib=lib).reshape(3, 4)
            for k, s in enumerate(free)}
    cand_sensors = _with_offsets(sensors, offs)
    new = linearize(cand_sensors, w.frame_sensor, w.channels, cand, w.pairs, w.params, want_system=False, lib=lib)
    accepted = ok and new["cost"] < lin["cost"]
    return dict(poses=cand if accepted else np.asarray(poses).copy(),
                sensors=cand_sensors if accepted else list(sensors), accepted=accepted,
                lam=lam / 10.0 if accepted else lam * 10.0, lam_used=lam, cost=lin["cost"], new_cost=new["cost"],
                candidate=cand, candidate_sensors=cand_sensors, solve_ok=ok)


def lm_iteration(w, poses, lam: Optional[float], lib=None) -> Dict:
    """One Levenberg-Marquardt iteration on workload-like `w` (sensors,
    frame_sensor, channels, pairs, params; optionally frame_var / n_vars, the
    pose variables of the frames, else frame 0 fixed and every other frame
    free) at `poses`.  lam=None takes the initial damping.  Returns the
    accepted poses, the new lambda, both costs."""
    lin = linearize(w.sensors, w.frame_sensor, w.channels, poses, w.pairs, w.params, lib=lib)
    fv = getattr(w, "frame_var", None)
    if fv is not None:
        if lam is None:
            lam = initial_lambda_vars(lin["H"], fv, w.n_vars)
        dx, ok = solve_step_vars(lin["H"], lin["b"], lam, fv, w.n_vars, lib=lib)
    else:
        if lam is None:
            lam = initial_lambda(lin["H"])
        dx, ok = solve_step(lin["H"], lin["b"], lam, lib=lib)
    cand = apply_update(poses, dx, lib=lib)
    new = linearize(w.sensors, w.frame_sensor, w.channels, cand, w.pairs, w.params, want_system=False, lib=lib)
    accepted = ok and new["cost"] < lin["cost"]
    return dict(poses=cand if accepted else np.asarray(poses).copy(), accepted=accepted,
                lam=lam / 10.0 if accepted else lam * 10.0, lam_used=lam, cost=lin["cost"],
                new_cost=new["cost"], count=lin["count"], H=lin["H"], b=lin["b"], dx=dx,
                candidate=cand, solve_ok=ok)


def pose_angle(Xi, Xj) -> float:
    """Rotation angle between two poses: acos((trace(R_i^T R_j) - 1) / 2)."""
    Ri, Rj = np.asarray(Xi)[:, :3], np.asarray(Xj)[:, :3]
    return float(np.arccos(np.clip(0.5 * (np.trace(Ri.T @ Rj) - 1.0), -1.0, 1.0)))


def build_pairs(sensors, frame_sensor, channels, poses, params: Dict, max_angle: float, max_dist: float,
                min_ratio: float, sequential: bool = False, lib=None) -> Dict:
    """Graph construction (Sec. IV-B): directed pairs (i, j), i < j, same
    sensor, with rotation angle < max_angle and translation < max_dist,
    kept when (valid residuals of i against j) / (points of i) > min_ratio;
    with `sequential`, (i, i + 1) is always kept.  Also returns each
    candidate's ratio and how many of its points lie within the float32
    decision margin (their validity may differ in a float32 implementation)."""
    lib = lib or _load()
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 3, 4)
    n = poses.shape[0]
    out, info = [], {}
    for i in range(n):
        for j in range(i + 1, n):
            if frame_sensor[i] != frame_sensor[j]:
                continue
            ang = pose_angle(poses[i], poses[j])
            dist = float(np.linalg.norm(poses[i][:, 3] - poses[j][:, 3]))
            is_seq = sequential and j == i + 1
            if not ((ang < max_angle and dist < max_dist) or is_seq):
                continue
            r = linearize_pair(sensors[frame_sensor[i]], params, channels[i], channels[j], poses[i], poses[j],
                               lib=lib)
            ratio = r["count"] / r["n_points"] if r["n_points"] else 0.0
            flagged = int(sum(bin(int(x)).count("1") for x in r["flags"]))
            info[(i, j)] = dict(ratio=ratio, n_points=r["n_points"], count=r["count"], flagged=flagged,
                                sequential=is_seq)
            if ratio > min_ratio or is_seq:
                out.append((i, j))
    return dict(pairs=np.array(out, dtype=np.int32).reshape(-1, 2), candidates=info)


# ------------------------------------------------------------------ Sec. IV-A: normals

def estimate_normals(sensor, channels: np.ndarray, scale: float, max_radius: int, params: Dict = None,
                     min_count: int = 5, collinear: float = 1e-6, lib=None) -> Dict:
    """Normal image of one frame (Sec. IV-A): for every pixel u with valid
    depth, unproject the valid pixels u' with |u - u'| < r(u) (pixel
    distance; columns wrap for the spherical model), r(u) = clamp(scale /
    d(u), 1.5, max_radius) (a radius inversely proportional to the range, at
    least the 3 x 3 block), fit the least-squares plane (normal = eigenvector
    of the smallest eigenvalue of the points' covariance, numpy.linalg.eigh)
    and orient it towards the observer (n . p_u < 0).  A pixel gets a normal
    when at least min_count points are used and the points are not collinear
    (middle eigenvalue > collinear * largest); other pixels get 0.
    Returns normals (H, W, 3), eig (H, W, 3, ascending), count (H, W),
    radius (H, W), depth_valid (H, W), dmax (H, W: the largest depth among
    the points used) and margin (H, W): pixels where a
    decision lies close to its threshold (an integer squared offset within
    1e-4 relative of r^2, the collinearity ratio within 1e-4 of its bound, or
    |n . p| < 1e-4 |p|), so that float32 arithmetic may decide otherwise."""
    s = sensor
    g = (lambda k: s[k]) if isinstance(s, dict) else (lambda k: getattr(s, k))
    H, W, model = int(g("height")), int(g("width")), int(g("model"))
    d = np.asarray(channels)[..., 1].astype(np.float64)
    rmin = (params or {}).get("range_min", 0.0)
    rmax = (params or {}).get("range_max", 1e30)
    valid = (d > 0) & (d >= rmin) & (d <= rmax)
    # unprojected points of every pixel, through the oracle's own pi^-1
    P = np.zeros((H, W, 3))
    for r in range(H):
        for c in range(W):
            if valid[r, c]:
                P[r, c] = unproject(s, float(c), float(r), d[r, c], lib=lib)
    rad = np.where(valid, np.clip(scale / np.where(valid, d, 1.0), 1.5, float(max_radius)), 0.0)
    S1 = np.zeros((H, W, 3))
    S2 = np.zeros((H, W, 3, 3))
    N = np.zeros((H, W), dtype=np.int64)
    dmax = np.where(valid, d, 0.0)
    near = np.zeros((H, W), dtype=bool)
    for dr in range(-max_radius, max_radius + 1):
        for dc in range(-max_radius, max_radius + 1):
            dd2 = dr * dr + dc * dc
            near |= valid & (np.abs(dd2 - rad * rad) <= 1e-4 * rad * rad) & (rad > 1.5) & (rad < max_radius)
            rows = np.arange(H)[:, None] + dr
            cols = np.arange(W)[None, :] + dc
            if model == 1:
                cols = cols % W
            inside = (rows >= 0) & (rows < H) & (cols >= 0) & (cols < W)
            rr = np.clip(rows, 0, H - 1)
            cc = np.clip(cols, 0, W - 1)
            take = inside & valid & (dd2 < rad * rad) & valid[rr, cc]
            q = P[rr, cc] - P  # relative to the centre pixel's point
            q = np.where(take[..., None], q, 0.0)
            S1 += q
            S2 += q[..., :, None] * q[..., None, :]
            N += take
            dmax = np.maximum(dmax, np.where(take, d[rr, cc], 0.0))
    Nn = np.maximum(N, 1)[..., None]
    mean = S1 / Nn
    cov = S2 / Nn[..., None] - mean[..., :, None] * mean[..., None, :]
    ev, evec = np.linalg.eigh(cov.reshape(-1, 3, 3))
    ev = ev.reshape(H, W, 3)
    n = evec[:, :, 0].reshape(H, W, 3)
    nP = np.sum(n * P, axis=-1)
    n = np.where((nP > 0)[..., None], -n, n)
    ok = valid & (N >= min_count) & (ev[..., 1] > collinear * ev[..., 2])
    near |= valid & (N >= min_count) & (np.abs(ev[..., 1] - collinear * ev[..., 2]) <= 1e-4 * ev[..., 2])
    near |= ok & (np.abs(nP) < 1e-4 * np.linalg.norm(P, axis=-1))
    n = np.where(ok[..., None], n, 0.0)
    return dict(normals=n, eig=ev, count=N, radius=rad, depth_valid=valid, margin=near, dmax=dmax)


# ------------------------------------------------------------------ Sec. IV-A: pyramids, Sec. IV-C: coarse to fine

def downsample_sensor(sensor):
    """Intrinsics of the level with half the resolution (Sec. IV-A, each level
    half the previous one).  Coarse pixel k covers fine pixels 2k and 2k + 1,
    so its centre is fine coordinate 2k + 1/2: u_coarse = (u_fine + 1/2) / 2 -
    1/2 for every projected point, i.e. f' = f / 2 and c' = (c + 1/2) / 2 - 1/2
    for both models (Eq. pinhole-projection, Eq. spherical-projection are
    affine in K).  Sizes are halved (rounded down)."""
    s = sensor
    g = (lambda k: s[k]) if isinstance(s, dict) else (lambda k: getattr(s, k))
    out = dict(model=int(g("model")), width=int(g("width")) // 2, height=int(g("height")) // 2,
               fx=float(g("fx")) / 2.0, fy=float(g("fy")) / 2.0,
               cx=(float(g("cx")) + 0.5) / 2.0 - 0.5, cy=(float(g("cy")) + 0.5) / 2.0 - 0.5)
    ext = g("extrinsic") if (isinstance(s, dict) and "extrinsic" in s) or hasattr(s, "extrinsic") else None
    out["extrinsic"] = np.asarray(ext if ext is not None else np.eye(3, 4), dtype=np.float64).reshape(12)
    return out


def downsample(channels: np.ndarray, params: Dict) -> np.ndarray:
    """Five-channel image of the next pyramid level (Sec. IV-A): coarse pixel
    (r, c) summarises the 2 x 2 block of fine pixels (2r..2r+1, 2c..2c+1).  It
    is valid when all four are valid pixels (d > 0, range_min <= d <=
    range_max, |n| > 0.5); then g and d are the block means and n the
    normalised sum of the four normals, each computed in float64 from the
    float32 inputs ((a + b) + (c + d) summed exactly, one rounding to float32
    at the end; |s| = sqrt((s_x^2 + s_y^2) + s_z^2)).  Invalid coarse pixels are
    all zero."""
    x = np.asarray(channels, dtype=np.float32)
    H, W = x.shape[0] // 2, x.shape[1] // 2
    x = x[:2 * H, :2 * W].astype(np.float64)
    d = x[..., 1]
    n2 = x[..., 2] * x[..., 2] + x[..., 3] * x[..., 3] + x[..., 4] * x[..., 4]
    valid = (d > 0) & (d >= params["range_min"]) & (d <= params["range_max"]) & (n2 > 0.25)
    blocks = x.reshape(H, 2, W, 2, 5)
    vb = valid.reshape(H, 2, W, 2).all(axis=(1, 3))
    s = (blocks[:, 0, :, 0] + blocks[:, 0, :, 1]) + (blocks[:, 1, :, 0] + blocks[:, 1, :, 1])
    out = np.zeros((H, W, 5))
    out[..., 0] = s[..., 0] * 0.25
    out[..., 1] = s[..., 1] * 0.25
    norm = np.sqrt((s[..., 2] * s[..., 2] + s[..., 3] * s[..., 3]) + s[..., 4] * s[..., 4])
    for k in range(3):
        out[..., 2 + k] = s[..., 2 + k] / np.where(norm > 0, norm, 1.0)
    out = np.where((vb & (norm > 0))[..., None], out, 0.0)
    return out.astype(np.float32)


def pyramid(w, n_levels: int):
    """Levels 0 (the input) .. n_levels - 1 of a workload-like `w`: a list of
    (sensors, channels) with every frame downsampled level by level."""
    levels = [([s.as_dict() if hasattr(s, "as_dict") else dict(s) for s in w.sensors], list(w.channels))]
    for _ in range(1, n_levels):
        sens, chans = levels[-1]
        levels.append(([downsample_sensor(s) for s in sens], [downsample(c, w.params) for c in chans]))
    return levels


class _Level:
    def __init__(self, w, sensors, channels):
        self.sensors, self.channels = sensors, channels
        self.frame_sensor, self.pairs, self.params = w.frame_sensor, w.pairs, w.params
        self.frame_var, self.n_vars = getattr(w, "frame_var", None), getattr(w, "n_vars", 0)


def coarse_to_fine(w, poses, n_levels: int, max_iters: Sequence[int], rel_tol: float, lib=None) -> Dict:
    """The hierarchical optimisation of Sec. IV-C: Levenberg-Marquardt from
    the coarsest level to the finest, each level starting from the poses of
    the previous one with a fresh damping (initial_lambda).  A level ends
    after max_iters[level] iterations (coarsest first) or at the first
    accepted step whose relative decrease of F, (F - F_new) / F, is below
    rel_tol (the error-variation criterion); rejected steps count as
    iterations.  Returns the final poses and one log entry per level."""
    levels = pyramid(w, n_levels)
    poses = np.asarray(poses, dtype=np.float64).reshape(-1, 3, 4).copy()
    log = []
    for li in range(n_levels - 1, -1, -1):
        lw = _Level(w, *levels[li])
        lam, its, acc, first, last = None, 0, 0, None, None
        for _ in range(int(max_iters[n_levels - 1 - li])):
            r = lm_iteration(lw, poses, lam, lib=lib)
            its += 1
            first = r["cost"] if first is None else first
            lam = r["lam"]
            poses = r["poses"]
            last = r["new_cost"] if r["accepted"] else r["cost"]
            if r["accepted"]:
                acc += 1
                if (r["cost"] - r["new_cost"]) < rel_tol * r["cost"]:
                    break
        log.append(dict(level=li, iterations=its, accepted=acc, cost_first=first, cost_last=last))
    return dict(poses=poses, log=log)
