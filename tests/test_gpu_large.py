"""The large configurations at full size, in the benchmark's launch
configuration (batched path, FP16 texels, autotuned variants, graph
iteration), against the FP64 oracle on seeded samples of pairs:

  - RGB-D 640 x 480, 200 frames along a spline through a multi-room hall,
    depth noise 1 mm z^2, intensity noise 0.01, pairs by the Sec. IV-B rule;
  - LiDAR 128 x 2048, 500 frames along the street, an uneven overlap graph
    (each frame the source of 2-20 pairs with more than 30 % overlap).

Bars on 50 seeded pairs per configuration, against the oracle's sums with
the points decided the other way inside the margin accounted for
(parity_helpers.check_sampled_pairs): the valid masks agree outside the
oracle's decision margin; the sampled sub-system's H and b to 1e-4 and its
cost to 1e-5 (relative Frobenius), each pair's H12 and b12 to 1e-3 and cost
to 1e-4 (float32 pixel-points at depth discontinuities; see the helper); at
most 1e-5 of the sample's residuals (+2) decided the other way; for the
whole system: exact symmetry and the gauge null space; one LM iteration
runs.  The TMA-staged kernel variant gives the unstaged variant's per-pair
systems bit for bit at full size.  The
generators render on the GPU (torch), so these tests need one; the inputs
are the same seeded scenes on any device.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_CACHE = {}


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def big(name):
    gpu()
    from paper_2303_16878_gb300 import synth
    if name not in _CACHE:
        _CACHE[name] = synth.make_rgbd_hall() if name == "hall" else synth.make_lidar_street_graph()
    return _CACHE[name]


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _host(ch):
    return ch.detach().cpu().numpy()


from parity_helpers import check_sampled_pairs  # noqa: E402


@pytest.mark.parametrize("name", ["hall", "street_graph"])
def test_large_config_sampled_pairs_match_oracle(oracle_lib, name):
    """50 seeded pairs: the valid masks agree on every point outside the
    oracle's decision margin, and the GPU's blocks, costs and counts meet the
    bars of check_sampled_pairs against the oracle's sums with the points
    decided the other way (inside the margin) accounted for by their own
    contributions; over the sample at most 1e-5 of the residuals (+2) are
    decided the other way.  FP16 texels: the oracle samples the target's
    intensity and normals as binary16 values (R25)."""
    import paper_2303_16878_gb300 as pba
    w = big(name)
    p = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_MIXED)
    p.autotune(1)
    n, res, flipped = check_sampled_pairs(oracle_lib, w, p, 50, 8, dict(w.params, texel_f16=1), _host, rel)
    assert n == min(50, len(w.pairs)) and res > 0
    H, b = p.get_system()
    assert np.array_equal(H, H.T)
    # gauge: H annihilates a common motion of all frames (6 directions of the global frame)
    from oracle_pins import gauge_directions
    V = gauge_directions(w.poses_init)
    assert np.linalg.norm(H @ V) <= 1e-4 * np.linalg.norm(H) * np.linalg.norm(V)
    p.set_mask_export(False)
    st = p.iterate()
    assert st["status"] == 0
    p.close()


def test_hall_adjoint_on_a_four_frame_subset(oracle_lib):
    """The adjoint's tangent pose gradient on four consecutive full-size frames
    equals twice the oracle's b with exact Jacobians (grad_mode 1: the
    derivative of the bilinear interpolant, which the adjoint differentiates;
    Eq. total-error-multicue, Huber with the decisions held fixed)."""
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import autograd
    torch = gpu()
    w = big("hall").subset(range(4))
    host = [_host(c) for c in w.channels]
    # the problem samples FP16 texels: the oracle samples binary16 target values too (R25)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, host, w.poses_init, w.pairs,
                               dict(w.params, grad_mode=1, texel_f16=1))
    p = pba.problem_from_workload(w, texel=pba.PBA_TEXEL_F16)
    cost, _, dposes, _, _ = p.cost_gradient(poses=True, extrinsics=False, images=False, device="cuda")
    X = torch.as_tensor(w.poses_init, dtype=torch.float64, device="cuda")
    gt = autograd.tangent_gradient(p, X, dposes.reshape(-1, 3, 4)).reshape(-1).cpu().numpy()
    assert rel(gt, 2.0 * ref["b"]) <= 1e-4
    assert abs(cost - ref["cost"]) <= 1e-5 * ref["cost"]
    p.close()


@pytest.mark.parametrize("name", ["hall", "street_graph"])
def test_staged_tiles_at_full_size(name):
    """The TMA-staged variant of the kernel (taps of each 32-point step from a
    shared-memory tile) on the full-size configurations, whose steps straddle
    tile edges, image borders and (LiDAR 128 x 2048) the wrap seam: the per-pair
    systems, costs and counts equal the unstaged variant's bit for bit, and no
    tile wait ran out."""
    import paper_2303_16878_gb300 as pba
    w = big(name)
    p = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_MIXED)
    out = []
    for v in (1, 1 + pba._lib.PBA_N_VARIANTS // 2):
        p.set_variants(v, v)
        cost, count = p.linearize()
        out.append((cost, count, p.get_pair_system()))
    (c0, n0, s0), (c1, n1, s1) = out
    assert c0 == c1 and n0 == n1
    for key in ("H", "b", "cost", "count"):
        assert np.array_equal(s0[key], s1[key]), key
    assert p.tuning()["tile_err"] == 0
    p.close()
