"""Coefficients of the arctangent polynomial used by pba_device.cuh.

atan(t) for t in [0, 1] is approximated by t + t s Q(s), s = t^2, Q of
degree DEG - 1 (the leading coefficient held at 1, so the kernel's last
operation adds a short term to t and rounds once), fitted here in float64 for
a small maximum absolute error: weighted
least squares on Chebyshev nodes, the weights raised where the error is
largest (Lawson's iteration towards the minimax polynomial).  The kernel
reduces atan2(y, x) to this interval with t = min(|x|, |y|) / max(|x|, |y|)
and writes the angle as sgn(y) (B + sigma r), B in {0, pi/2, pi}, so that the
projection's column is an exact offset plus a short term (see
spherical_project).  Run to print the coefficients and the float32 error of
the kernel's evaluation of r (Horner in float32 with fused multiply-adds,
the ratio from a reciprocal refined by one Newton step).
"""
import numpy as np

DEG = 8


def fit(deg=DEG, nodes=8000, iters=40):
    """Coefficients of Q (degree deg - 1) with atan(t) ~ t + t s Q(s)."""
    k = np.arange(nodes)
    t = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / nodes))  # Chebyshev nodes on [0, 1]
    s = t * t
    V = np.stack([s ** i for i in range(deg)], axis=1)
    target = np.arctan(t) - t
    w = np.ones_like(t)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * (t * s * w)[:, None], target * w, rcond=None)
        err = np.abs(t * s * (V @ c) - target)
        w = w * np.sqrt(err / err.max() + 1e-3)
        w /= w.max()
    return c


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def eval_r_f32(c, y, x):
    """r = atan(min / max) as the kernel forms it, in float32."""
    c32 = c.astype(np.float32)
    ax, ay = np.abs(x).astype(np.float32), np.abs(y).astype(np.float32)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    rc = (np.float32(1) / mx).astype(np.float32)
    t0 = (mn * rc).astype(np.float32)
    e = _fma32(-t0, mx, mn)
    t = _fma32(e, rc, t0)
    s = (t * t).astype(np.float32)
    q = np.full_like(s, c32[-1])
    for ci in c32[-2::-1]:
        q = _fma32(q, s, np.full_like(s, ci))
    return _fma32((t * s).astype(np.float32), q, t), mn.astype(np.float64) / mx.astype(np.float64)


if __name__ == "__main__":
    c = fit()
    for i, ci in enumerate(c):
        print(f"    {float(np.float32(ci))!r}f,  // Q: s^{i}")
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 2_000_000)
    rad = rng.uniform(0.1, 100, ang.size)
    x, y = (rad * np.cos(ang)).astype(np.float32), (rad * np.sin(ang)).astype(np.float32)
    r, ratio = eval_r_f32(c, y, x)
    err = np.abs(r.astype(np.float64) - np.arctan(ratio))
    print("max abs error of r (float32 evaluation):", err.max())
