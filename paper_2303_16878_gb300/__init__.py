"""GB300-native photometric LiDAR and RGB-D bundle adjustment.

The compute path is libpba (CUDA for sm_103a, C ABI in include/pba.h); this
package is a thin binding over it.  `Problem` mirrors the C calls one to one:
it converts numpy arrays and torch tensors into pointers and sizes and raises
`PbaError` on a non-zero status.  PyTorch is used only for device memory and
streams.  `synth` generates seeded synthetic workloads.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (PBA_PATH_BATCHED, PBA_PATH_PLAIN, PBA_PINHOLE, PBA_SOLVE_CHOLESKY_F64, PBA_SOLVE_MIXED,
                   PBA_SOLVE_MIXED_STEPS, PBA_SOLVE_SPARSE, PBA_SPHERICAL, PBA_TEXEL_F16, PBA_TEXEL_F32,
                   PbaError)

__all__ = ["Problem", "PbaError", "PBA_PATH_BATCHED", "PBA_PATH_PLAIN", "PBA_TEXEL_F16", "PBA_TEXEL_F32",
           "PBA_PINHOLE", "PBA_SPHERICAL", "PBA_SOLVE_CHOLESKY_F64", "PBA_SOLVE_MIXED", "PBA_SOLVE_MIXED_STEPS",
           "PBA_SOLVE_SPARSE",
           "problem_from_workload"]


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stats(s: _lib.PbaIterStats) -> Dict:
    return dict(cost=s.cost, new_cost=s.new_cost, lambda_used=s.lambda_used, lambda_next=s.lambda_next,
                n_valid=int(s.n_valid), accepted=bool(s.accepted), status=int(s.status),
                n_nonfinite=int(s.n_nonfinite), nonfinite_pairs=int(s.nonfinite_pairs))


class Problem:
    """One bundle-adjustment problem on the current CUDA device (C: pba_problem)."""

    def __init__(self, sensors: Sequence, n_frames: int, params: Dict, frame_sensor=None,
                 path: int = PBA_PATH_BATCHED, texel: int = PBA_TEXEL_F16, stream=None,
                 solver: int = PBA_SOLVE_CHOLESKY_F64):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        self.n_frames = int(n_frames)
        sens = (_lib.PbaSensor * len(sensors))()
        self._sizes = []
        for k, s in enumerate(sensors):
            g = (lambda key: s[key]) if isinstance(s, dict) else (lambda key: getattr(s, key))
            sens[k].model, sens[k].width, sens[k].height = int(g("model")), int(g("width")), int(g("height"))
            sens[k].fx, sens[k].fy, sens[k].cx, sens[k].cy = (float(g("fx")), float(g("fy")), float(g("cx")),
                                                              float(g("cy")))
            xo = np.asarray(g("extrinsic"), dtype=np.float64).reshape(12)
            for e in range(12):
                sens[k].extrinsic[e] = xo[e]
            self._sizes.append((sens[k].height, sens[k].width))
        self._sens = sens
        fs = None
        if frame_sensor is not None:
            self._fs = np.ascontiguousarray(frame_sensor, dtype=np.int32)
            fs = self._fs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        else:
            self._fs = np.zeros(self.n_frames, dtype=np.int32)
        cfg = _lib.PbaConfig()
        cfg.n_frames, cfg.n_sensors = self.n_frames, len(sensors)
        cfg.sensors = ctypes.cast(sens, ctypes.POINTER(_lib.PbaSensor))
        cfg.frame_sensor = fs
        for key in ("w_int", "w_depth", "w_normal", "huber_delta", "occ_abs", "occ_rel", "z_min", "range_min",
                    "range_max"):
            setattr(cfg, key, float(params[key]))
        cfg.grad_mode = int(params.get("grad_mode", 0))
        cfg.texel_precision = int(texel)
        cfg.path = int(path)
        cfg.solver = int(solver)
        self.path, self.texel, self.solver = int(path), int(texel), int(solver)
        st = self._lib.pba_create(ctypes.byref(cfg), ctypes.c_void_p(self._stream_handle(stream)),
                                  ctypes.byref(self._h))
        if st != 0:
            msg = self._lib.pba_last_error(None)
            raise PbaError(st, msg.decode() if msg else "pba_create failed")

    @staticmethod
    def _stream_handle(stream) -> int:
        if stream is None:
            return 0
        if isinstance(stream, int):
            return stream
        return int(stream.cuda_stream)

    def _check(self, st: int, what: str):
        if st != 0:
            msg = self._lib.pba_last_error(self._h)
            raise PbaError(st, f"{what}: {msg.decode() if msg else ''}")

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if self._h and not getattr(self, "_owner", None):
            self._lib.pba_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        self._check(self._lib.pba_set_stream(self._h, ctypes.c_void_p(self._stream_handle(stream))), "set_stream")

    # -------------------------------------------------------------- inputs
    def _check_shape(self, first: int, shape):
        shape = tuple(shape)
        if len(shape) == 3:
            shape = (1,) + shape
        count = shape[0]
        if len(shape) != 4 or shape[3] != 5 or count < 1 or first < 0 or first + count > self.n_frames:
            raise ValueError(f"channels must be (count, H, W, 5) within the frame range, got {shape}")
        for k in range(first, first + count):
            if shape[1:3] != self._sizes[int(self._fs[k])]:
                raise ValueError(f"frame {k}: image {shape[1:3]} does not match its sensor {self._sizes[int(self._fs[k])]}")
        return count

    def upload_frames(self, first: int, channels):
        """channels: (count, H, W, 5) float32 numpy array or CUDA torch tensor."""
        if _is_torch(channels):
            if str(channels.dtype) != "torch.float32" or not channels.is_contiguous():
                raise ValueError("channels must be a contiguous float32 tensor")
            count = self._check_shape(first, channels.shape)
            self._check(self._lib.pba_upload_frames(self._h, first, count, ctypes.c_void_p(channels.data_ptr()),
                                                    1 if channels.is_cuda else 0), "upload_frames")
            return
        arr = np.ascontiguousarray(channels, dtype=np.float32)
        if arr.ndim == 3:
            arr = arr[None]
        self._check_shape(first, arr.shape)
        self._check(self._lib.pba_upload_frames(self._h, first, arr.shape[0], arr.ctypes.data_as(ctypes.c_void_p), 0),
                    "upload_frames")

    def set_extrinsic(self, sensor: int, X):
        """Replace a sensor's offset X_o (3x4); its frames' points are rebuilt."""
        if _is_torch(X):
            X = X.detach().cpu().numpy()
        arr = np.ascontiguousarray(X, dtype=np.float64).reshape(12)
        self._check(self._lib.pba_set_extrinsic(self._h, int(sensor), arr.ctypes.data_as(ctypes.c_void_p)),
                    "set_extrinsic")

    def estimate_normals(self, first: int = 0, count: Optional[int] = None, scale: float = 10.0,
                         max_radius: int = 5):
        """Sec. IV-A: recompute the normal channels of uploaded frames from their
        depth (plane fit over a radius clamp(scale / d, 1.5, max_radius) pixels,
        oriented towards the observer) and rebuild their pixel-points."""
        count = self.n_frames - first if count is None else int(count)
        self._check(self._lib.pba_estimate_normals(self._h, int(first), count, float(scale), int(max_radius)),
                    "estimate_normals")

    def get_channels(self, first: int = 0, count: int = 1, out=None):
        """The (count, H, W, 5) float32 cue images of uploaded frames as stored on
        the device (after estimate_normals: with the estimated normals)."""
        H, W = self._sizes[int(self._fs[first])]
        for k in range(first, first + count):
            if self._sizes[int(self._fs[k])] != (H, W):
                raise ValueError("get_channels: frames of one call must share the image size")
        if out is not None and _is_torch(out) and out.is_cuda:
            if not out.is_contiguous() or out.numel() != count * H * W * 5 or str(out.dtype) != "torch.float32":
                raise ValueError(f"get_channels: out must be a contiguous float32 tensor of {count * H * W * 5} values")
            self._check(self._lib.pba_get_channels(self._h, int(first), int(count), ctypes.c_void_p(out.data_ptr()), 1),
                        "get_channels")
            return out
        arr = np.empty((count, H, W, 5), dtype=np.float32)
        self._check(self._lib.pba_get_channels(self._h, int(first), int(count),
                                               arr.ctypes.data_as(ctypes.c_void_p), 0), "get_channels")
        return arr

    def set_variables(self, frame_var=None, n_vars: int = 0):
        """Pose variables of the solve: frame k moves with variable frame_var[k]
        (-1: held fixed); None restores frame 0 fixed, every other frame free."""
        if frame_var is None:
            self._check(self._lib.pba_set_variables(self._h, None, 0), "set_variables")
            return
        fv = np.ascontiguousarray(frame_var, dtype=np.int32).reshape(-1)
        if fv.size != self.n_frames:
            raise ValueError(f"frame_var needs {self.n_frames} entries, got {fv.size}")
        self._check(self._lib.pba_set_variables(self._h, fv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                int(n_vars)), "set_variables")

    # -------------------------------------------------------------- pyramid (Sec. IV-A, IV-C)
    def build_pyramid(self, n_levels: int = 3):
        """Levels 1..n_levels-1, each half the resolution of the previous one,
        downsampled on the device from the uploaded frames."""
        self._check(self._lib.pba_build_pyramid(self._h, int(n_levels)), "build_pyramid")
        self._n_levels = int(n_levels)

    def level(self, level: int) -> "Problem":
        """The problem of one pyramid level (borrowed from this one; level 0 is self)."""
        if level == 0:
            return self
        h = ctypes.c_void_p()
        self._check(self._lib.pba_pyramid_level(self._h, int(level), ctypes.byref(h)), "pyramid_level")
        q = Problem.__new__(Problem)
        q._lib, q._h, q._owner = self._lib, h, self
        q.n_frames, q._fs = self.n_frames, self._fs
        q._sizes = list(self._sizes)
        for _ in range(int(level)):
            q._sizes = [(hh // 2, ww // 2) for hh, ww in q._sizes]
        q.path, q.texel, q.solver = self.path, self.texel, self.solver
        q.n_pairs = getattr(self, "n_pairs", 0)
        return q

    def optimize(self, max_iters=(10, 5, 2), rel_tol: float = 1e-4):
        """Coarse-to-fine Levenberg-Marquardt over the first len(max_iters)
        levels (max_iters coarsest first); returns one dict per level."""
        n = len(max_iters)
        its = (ctypes.c_int32 * n)(*[int(x) for x in max_iters])
        st = (_lib.PbaLevelStats * n)()
        self._check(self._lib.pba_optimize(self._h, n, its, float(rel_tol), st), "optimize")
        return [dict(level=s.level, iterations=s.iterations, accepted=s.accepted, status=s.status,
                     cost_first=s.cost_first, cost_last=s.cost_last) for s in st]

    def refine_extrinsic(self, sensor: int, max_iters: int = 20, rel_tol: float = 1e-7) -> Dict:
        """BFGS on one sensor's offset with the adjoint gradient (pba_refine_extrinsic)."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        self._check(self._lib.pba_refine_extrinsic(self._h, int(sensor), int(max_iters), float(rel_tol),
                                                   ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
                    "refine_extrinsic")
        return dict(cost_before=a.value, cost_after=b.value, iterations=n.value)

    def set_offset_free(self, sensor: int, free: bool = True):
        """Make one sensor's offset X_o a variable of the LM steps (or fix it again)."""
        self._check(self._lib.pba_set_offset_free(self._h, int(sensor), 1 if free else 0), "set_offset_free")

    def get_extrinsic(self, sensor: int) -> np.ndarray:
        """The sensor's current offset X_o (3x4), as last set or refined."""
        out = np.zeros(12)
        self._check(self._lib.pba_get_extrinsic(self._h, int(sensor), out.ctypes.data_as(ctypes.c_void_p)),
                    "get_extrinsic")
        return out.reshape(3, 4)

    def frame_points(self, frame: int) -> int:
        n = ctypes.c_int32()
        self._check(self._lib.pba_frame_points(self._h, frame, ctypes.byref(n)), "frame_points")
        return n.value

    def set_poses(self, poses):
        """All N poses, (N, 3, 4) or (N, 12): a numpy array, or a torch tensor on
        the host or a CUDA device.  A contiguous float64 CUDA tensor is read on
        the device (keep it unchanged until the problem's stream has passed
        this call); anything else goes through a float64 host copy."""
        if _is_torch(poses):
            t = poses.detach()
            if t.numel() != 12 * self.n_frames:
                raise ValueError(f"poses must hold {self.n_frames} x 12 values, got shape {tuple(poses.shape)}")
            if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()):
                poses = t.cpu().double().numpy()
            else:
                self._check(self._lib.pba_set_poses(self._h, ctypes.c_void_p(t.data_ptr()), 1), "set_poses")
                return
        arr = np.ascontiguousarray(poses, dtype=np.float64)
        if arr.size != 12 * self.n_frames:
            raise ValueError(f"poses must hold {self.n_frames} x 12 values, got shape {arr.shape}")
        self._check(self._lib.pba_set_poses(self._h, arr.ctypes.data_as(ctypes.c_void_p), 0), "set_poses")

    def get_poses(self) -> np.ndarray:
        out = np.zeros((self.n_frames, 12))
        self._check(self._lib.pba_get_poses(self._h, out.ctypes.data_as(ctypes.c_void_p)), "get_poses")
        return out.reshape(self.n_frames, 3, 4)

    def set_pairs(self, pairs):
        arr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self.n_pairs = arr.shape[0]
        self._check(self._lib.pba_set_pairs(self._h, arr.ctypes.data_as(ctypes.c_void_p), arr.shape[0]), "set_pairs")

    def build_pairs(self, max_angle: float, max_dist: float, min_ratio: float, sequential: bool = False):
        """Graph construction (Sec. IV-B) at the current poses: (pairs (m, 2) int32, ratios (m,))."""
        n = ctypes.c_int32()
        cap = self.n_frames * (self.n_frames - 1) // 2 + 1
        pairs = np.zeros((cap, 2), dtype=np.int32)
        ratios = np.zeros(cap, dtype=np.float32)
        self._check(self._lib.pba_build_pairs(self._h, float(max_angle), float(max_dist), float(min_ratio),
                                              1 if sequential else 0, pairs.ctypes.data_as(ctypes.c_void_p),
                                              ratios.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)),
                    "build_pairs")
        return pairs[: n.value].copy(), ratios[: n.value].copy()

    # -------------------------------------------------------------- linearise / solve
    def linearize(self):
        cost, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self._lib.pba_linearize(self._h, ctypes.byref(cost), ctypes.byref(n)), "linearize")
        return cost.value, n.value

    def cost_gradient(self, poses: bool = True, extrinsics: bool = True, images: bool = False, device=None):
        """Total cost F and its gradient (pba_cost_gradient): returns
        (cost, n_valid, dF/dposes (N, 3, 4) or None, dF/dX_o (S, 3, 4) or None,
        dF/dchannels (total pixels * 5,) float32 or None) as CUDA tensors."""
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        n_s = len(self._sizes)
        total_px = int(sum(self._sizes[int(k)][0] * self._sizes[int(k)][1] for k in self._fs))
        dP = torch.zeros((self.n_frames, 3, 4), dtype=torch.float64, device=dev) if poses else None
        dE = torch.zeros((n_s, 3, 4), dtype=torch.float64, device=dev) if extrinsics else None
        dI = torch.zeros(total_px * 5, dtype=torch.float32, device=dev) if images else None
        cost, n = ctypes.c_double(), ctypes.c_int64()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._lib.pba_cost_gradient(self._h, ctypes.byref(cost), ctypes.byref(n), ptr(dP), ptr(dE),
                                                ptr(dI)), "cost_gradient")
        return cost.value, n.value, dP, dE, dI

    def tangent_gradient(self, X, G):
        """dF/d dx in the box-plus chart (pba_tangent_gradient) from matrix
        gradients G = dF/dX at the 3x4 transforms X: CUDA tensors (..., 3, 4)
        -> float64 CUDA tensor (..., 6)."""
        import torch
        Xc = torch.as_tensor(X, dtype=torch.float64).contiguous()
        Gc = torch.as_tensor(G, dtype=torch.float64, device=Xc.device).contiguous()
        if Xc.shape != Gc.shape or Xc.shape[-2:] != (3, 4) or not Xc.is_cuda:
            raise ValueError("tangent_gradient: X and G must be CUDA tensors of equal shape (..., 3, 4)")
        n = Xc.numel() // 12
        g = torch.empty(Xc.shape[:-2] + (6,), dtype=torch.float64, device=Xc.device)
        torch.cuda.current_stream(Xc.device).synchronize()  # X, G written on torch's stream; the library uses its own
        self._check(self._lib.pba_tangent_gradient(self._h, ctypes.c_void_p(Xc.data_ptr()),
                                                   ctypes.c_void_p(Gc.data_ptr()), int(n),
                                                   ctypes.c_void_p(g.data_ptr())), "tangent_gradient")
        return g

    def get_system(self):
        n6 = 6 * self.n_frames
        H, b = np.zeros((n6, n6)), np.zeros(n6)
        self._check(self._lib.pba_get_system(self._h, H.ctypes.data_as(ctypes.c_void_p),
                                             b.ctypes.data_as(ctypes.c_void_p)), "get_system")
        return H, b

    def get_pair_system(self):
        m = self.n_pairs
        H, b, c, n = np.zeros((m, 12, 12)), np.zeros((m, 12)), np.zeros(m), np.zeros(m, dtype=np.int64)
        self._check(self._lib.pba_get_pair_system(self._h, *(x.ctypes.data_as(ctypes.c_void_p) for x in (H, b, c, n))),
                    "get_pair_system")
        return dict(H=H, b=b, cost=c, count=n)

    def set_mask_export(self, enable: bool):
        self._check(self._lib.pba_set_mask_export(self._h, 1 if enable else 0), "set_mask_export")

    def get_mask(self, pair: int, n_points: int) -> np.ndarray:
        nw = max(1, (n_points + 31) // 32)
        out = np.zeros(nw, dtype=np.uint32)
        self._check(self._lib.pba_get_mask(self._h, pair, out.ctypes.data_as(ctypes.c_void_p), nw), "get_mask")
        return out[: (n_points + 31) // 32]

    def solve_step(self, lam: float) -> Dict:
        s = _lib.PbaIterStats()
        self._check(self._lib.pba_solve_step(self._h, float(lam), ctypes.byref(s)), "solve_step")
        return _stats(s)

    def set_lambda(self, lam: Optional[float]):
        self._check(self._lib.pba_set_lambda(self._h, -1.0 if lam is None else float(lam)), "set_lambda")

    def iterate(self) -> Dict:
        s = _lib.PbaIterStats()
        self._check(self._lib.pba_iterate(self._h, ctypes.byref(s)), "iterate")
        return _stats(s)

    def iterate_frames(self, channels, poses=None) -> Dict:
        """pba_iterate_frames: one LM iteration on new images of every frame.
        channels: host float32 holding all frames back to back in frame order
        (each H x W x 5 of its sensor), a numpy array or a CPU torch tensor
        (page-locked, e.g. .pin_memory(), for the copies to overlap the
        linearisation); poses: (N, 3, 4) / (N, 12) host values or None."""
        total = 5 * sum(self._sizes[int(self._fs[k])][0] * self._sizes[int(self._fs[k])][1]
                        for k in range(self.n_frames))
        if _is_torch(channels):
            if channels.is_cuda or str(channels.dtype) != "torch.float32" or not channels.is_contiguous():
                raise ValueError("channels must be a contiguous float32 host tensor")
            n, ptr, keep = channels.numel(), channels.data_ptr(), channels
        else:
            keep = np.ascontiguousarray(channels, dtype=np.float32)
            n, ptr = keep.size, keep.ctypes.data
        if n != total:
            raise ValueError(f"channels must hold {total} floats (every frame, H x W x 5), got {n}")
        pp = None
        if poses is not None:
            if _is_torch(poses):
                poses = poses.detach().cpu().numpy()
            pp = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1)
            if pp.size != 12 * self.n_frames:
                raise ValueError(f"poses must hold {self.n_frames} x 12 values")
        s = _lib.PbaIterStats()
        self._check(self._lib.pba_iterate_frames(self._h, ctypes.c_void_p(ptr),
                                                 None if pp is None else pp.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.byref(s)), "iterate_frames")
        del keep
        return _stats(s)

    def iterate_async(self, n: int = 1):
        self._check(self._lib.pba_iterate_async(self._h, int(n)), "iterate_async")

    def get_stats(self) -> Dict:
        s = _lib.PbaIterStats()
        self._check(self._lib.pba_get_stats(self._h, ctypes.byref(s)), "get_stats")
        return _stats(s)

    def iterate_timed(self):
        """One iteration launched kernel by kernel with CUDA events between its
        phases; returns (stats, {phase name: device ms})."""
        ms = (ctypes.c_float * _lib.PBA_N_PHASES)()
        s = _lib.PbaIterStats()
        self._check(self._lib.pba_iterate_timed(self._h, ms, _lib.PBA_N_PHASES, ctypes.byref(s)), "iterate_timed")
        return _stats(s), dict(zip(_lib.PHASE_NAMES, list(ms)))

    def autotune(self, repeats: int = 2):
        """Time the occupancy variants of the linearisation kernel on this
        problem and keep the fastest; returns (variant_full, variant_cost)."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.pba_autotune(self._h, int(repeats), ctypes.byref(a), ctypes.byref(b)), "autotune")
        return a.value, b.value

    def tuning(self) -> Dict:
        """The settings of the linearisation (pba_get_tuning): variants (occupancy
        budget, staged taps from 4 on), work-item sizes, the reduction scheme of
        the work items' sums (0 shared-memory table, 1 shuffle butterfly), whether they came from
        the process's tuning cache, the tuned pass times in ms and the staged
        tiles' timeout flag."""
        t = _lib.PbaTuning()
        self._check(self._lib.pba_get_tuning(self._h, ctypes.byref(t)), "get_tuning")
        return dict(variant_full=t.variant_full, variant_cost=t.variant_cost, chunk=t.chunk,
                    chunk_tail=t.chunk_tail, reduction=t.reduction, from_cache=bool(t.from_cache), ms_full=t.ms_full, ms_cost=t.ms_cost,
                    tile_err=int(t.tile_err))

    def set_tuning(self, tuning: Dict):
        """Apply a tuning as tuning() reports it (variant_full, variant_cost,
        chunk, chunk_tail, reduction (0 when absent); other keys ignored)
        without timing anything."""
        t = _lib.PbaTuning()
        t.variant_full, t.variant_cost = int(tuning["variant_full"]), int(tuning["variant_cost"])
        t.chunk, t.chunk_tail = int(tuning["chunk"]), int(tuning["chunk_tail"])
        t.reduction = int(tuning.get("reduction", 0))
        self._check(self._lib.pba_set_tuning(self._h, ctypes.byref(t)), "set_tuning")

    def set_variants(self, variant_full: int, variant_cost: int):
        """Occupancy variants of the linearisation kernel (0 .. PBA_N_VARIANTS - 1)."""
        self._check(self._lib.pba_set_variants(self._h, int(variant_full), int(variant_cost)), "set_variants")

    def iteration_launches(self) -> int:
        n = ctypes.c_int32()
        self._check(self._lib.pba_iteration_launches(self._h, ctypes.byref(n)), "iteration_launches")
        return n.value


def problem_from_workload(w, path: int = PBA_PATH_BATCHED, texel: int = PBA_TEXEL_F16, params: Optional[Dict] = None,
                          poses=None, stream=None, solver: int = PBA_SOLVE_CHOLESKY_F64) -> Problem:
    """Create a Problem from a synth.Workload: upload every frame (grouped by
    image size), set the initial poses and the pair list."""
    prm = dict(w.params)
    if params:
        prm.update(params)
    p = Problem(w.sensors, w.n_frames, prm, frame_sensor=w.frame_sensor, path=path, texel=texel, stream=stream,
                solver=solver)
    k = 0
    while k < w.n_frames:
        j = k
        while j + 1 < w.n_frames and w.channels[j + 1].shape == w.channels[k].shape:
            j += 1
        if _is_torch(w.channels[k]):  # device tensors (the large generators): upload from the device
            import torch
            block = torch.stack(w.channels[k:j + 1]).contiguous()
            torch.cuda.synchronize()  # the library copies on its own stream
            p.upload_frames(k, block)
        else:
            p.upload_frames(k, np.stack(w.channels[k:j + 1]))
        k = j + 1
    p.set_poses(w.poses_init if poses is None else poses)
    p.set_pairs(w.pairs)
    if getattr(w, "frame_var", None) is not None:
        p.set_variables(w.frame_var, w.n_vars)
    return p
