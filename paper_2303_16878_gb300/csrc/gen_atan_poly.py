"""Coefficients of the arctangent polynomial used by pba_linearize.cu.

atan(t) for t in [0, 1] is approximated by t * P(t^2), P of degree DEG,
fitted here by weighted least squares (relative to t) on Chebyshev nodes, in
float64; the kernel reduces atan2(y, x) to this interval with
t = min(|x|, |y|) / max(|x|, |y|) and the usual octant reflections.
Run to print the coefficients and the float32 error of the kernel's
evaluation order (Horner in float32 with fused multiply-adds).
"""
import numpy as np

DEG = 8


def fit(deg=DEG, nodes=4000):
    k = np.arange(nodes)
    t = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / nodes))  # Chebyshev nodes on [0, 1]
    s = t * t
    V = np.stack([s ** i for i in range(deg + 1)], axis=1)
    # minimise the error of t * P(s) against atan(t), weighted by 1 / t
    target = np.where(t > 0, np.arctan(t) / np.where(t > 0, t, 1.0), 1.0)
    c, *_ = np.linalg.lstsq(V, target, rcond=None)
    return c


def eval_f32(c, y, x):
    c32 = c.astype(np.float32)
    ax, ay = np.abs(x).astype(np.float32), np.abs(y).astype(np.float32)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    t = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.full_like(s, c32[-1])
    for ci in c32[-2::-1]:
        p = (p * s + ci).astype(np.float32)
    r = (t * p).astype(np.float32)
    r = np.where(ay > ax, np.float32(np.pi / 2) - r, r).astype(np.float32)
    r = np.where(x < 0, np.float32(np.pi) - r, r).astype(np.float32)
    return np.where(y < 0, -r, r).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    for i, ci in enumerate(c):
        print(f"    {float(np.float32(ci))!r}f,  // s^{i}")
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 2_000_000)
    rad = rng.uniform(0.1, 100, ang.size)
    x, y = (rad * np.cos(ang)).astype(np.float32), (rad * np.sin(ang)).astype(np.float32)
    err = np.abs(eval_f32(c, y, x).astype(np.float64) - np.arctan2(y.astype(np.float64), x.astype(np.float64)))
    print("max abs error (float32 evaluation):", err.max())
