"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars (relative Frobenius norms unless stated): H and b <= 1e-4, total cost
<= 1e-5, converged poses <= 1e-4 m and <= 1e-5 rad; valid-residual masks
bit-exact on every point whose validity decisions are not within the oracle's
float32 decision margin (flagged points), with at most 1e-5 of the residuals
(+2) disagreeing at all.
"""
import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu

TOL_H = 1e-4
TOL_B = 1e-4
TOL_COST = 1e-5


def oprm(params, texel):
    """The oracle's parameters for a GPU run with texel precision `texel`:
    FP16 texels sample the target's intensity and normals as binary16 values
    (reading R25), which the oracle evaluates exactly when asked."""
    return dict(params, texel_f16=int(texel == 1))


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make(w, path, texel, params=None, poses=None, solver=0):
    import paper_2303_16878_gb300 as pba
    gpu()
    return pba.problem_from_workload(w, path=path, texel=texel, params=params, poses=poses, solver=solver)


CASES = [
    ("batched", 1, 0), ("batched", 0, 0), ("batched", 1, 1), ("batched", 0, 1),
    ("plain", 0, 0), ("plain", 0, 1),
]


def _path(name):
    import paper_2303_16878_gb300 as pba
    return pba.PBA_PATH_BATCHED if name == "batched" else pba.PBA_PATH_PLAIN


@pytest.mark.parametrize("path,texel,grad_mode", CASES)
@pytest.mark.parametrize("which", ["room8", "street3", "room8x"])
def test_system_matches_oracle(oracle_lib, which, path, texel, grad_mode, request):
    w = request.getfixturevalue(which)
    params = oprm(dict(w.params, grad_mode=grad_mode), texel if path == "batched" else 0)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params,
                               want_pairs=True)
    p = make(w, _path(path), texel, params={"grad_mode": grad_mode})
    cost, count = p.linearize()
    H, b = p.get_system()
    ps = p.get_pair_system()
    assert abs(count - ref["count"]) <= 1e-5 * ref["count"] + 2
    assert abs(cost - ref["cost"]) <= TOL_COST * ref["cost"]
    assert rel(H, ref["H"]) <= TOL_H
    assert rel(b, ref["b"]) <= TOL_B
    assert rel(ps["H"], ref["pair_H"]) <= TOL_H
    assert rel(ps["b"], ref["pair_b"]) <= TOL_B
    assert np.abs(ps["count"] - ref["pair_count"]).max() <= 2
    p.close()


@pytest.mark.parametrize("texel", [0, 1])
@pytest.mark.parametrize("which", ["room8", "street3"])
def test_valid_mask_bit_exact_outside_decision_margin(oracle_lib, which, texel, request):
    import paper_2303_16878_gb300 as pba
    w = request.getfixturevalue(which)
    p = make(w, pba.PBA_PATH_BATCHED, texel)
    p.set_mask_export(True)
    p.linearize()
    total, disagree = 0, 0
    for q, (i, j) in enumerate(w.pairs.tolist()):
        r = oracle_lib.linearize_pair(w.sensors[0], oprm(w.params, texel), w.channels[i], w.channels[j],
                                      w.poses_init[i], w.poses_init[j])
        assert p.frame_points(i) == r["n_points"]
        m = p.get_mask(q, r["n_points"])
        diff = m ^ r["mask"]
        assert not np.any(diff & ~r["flags"]), f"pair {q}: mask differs on unflagged points"
        disagree += int(sum(bin(int(x)).count("1") for x in diff))
        total += r["count"]
    assert disagree <= 1e-5 * total + 2
    p.close()


def test_full_size_lidar_street_sampled_pairs(oracle_lib):
    """50 frames of 64 x 1024 with every overlapping pair in one persistent
    launch (the benchmark's configuration); the oracle recomputes a seeded
    sample of pairs one by one, and the whole system is checked for the
    properties that hold at any size."""
    import paper_2303_16878_gb300 as pba
    import oracle_pins
    w = workload("street")
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    cost, count = p.linearize()
    H, b = p.get_system()
    ps = p.get_pair_system()
    rng = np.random.default_rng(5)
    sample = rng.choice(len(w.pairs), size=8, replace=False)
    for q in sample:
        i, j = w.pairs[q]
        r = oracle_lib.linearize_pair(w.sensors[0], oprm(w.params, 1), w.channels[i], w.channels[j],
                                      w.poses_init[i], w.poses_init[j])
        assert abs(ps["count"][q] - r["count"]) <= 2
        assert abs(ps["cost"][q] - r["cost"]) <= 1e-4 * r["cost"] + 1e-9
        assert rel(ps["H"][q], r["H"]) <= TOL_H
        assert rel(ps["b"][q], r["b"]) <= TOL_B
    assert count == int(ps["count"].sum())
    assert abs(cost - ps["cost"].sum()) <= 1e-9 * cost
    np.testing.assert_array_equal(H, H.T)
    V = oracle_pins.gauge_directions(w.poses_init)
    assert np.linalg.norm(H @ V) <= 1e-6 * np.linalg.norm(H) * np.linalg.norm(V)
    p.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_damped_step_matches_oracle(oracle_lib, room8, solver):
    """A strongly damped step is well conditioned, so its dx is fixed to the
    accuracy of H and b; compare the updated poses (FP64 Cholesky and the
    FP32-factorisation + FP64-refinement solver)."""
    import paper_2303_16878_gb300 as pba
    w = room8
    prm = oprm(w.params, 1)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, prm)
    lam = 10.0 * float(np.diag(ref["H"])[6:].max())
    dx, ok = oracle_lib.solve_step(ref["H"], ref["b"], lam)
    cand = oracle_lib.apply_update(w.poses_init, dx)
    new = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, cand, w.pairs, prm, want_system=False)
    assert ok and new["cost"] < ref["cost"]
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16, solver=solver)
    p.linearize()
    st = p.solve_step(lam)
    assert st["accepted"] and st["status"] == 0
    assert abs(st["new_cost"] - new["cost"]) <= TOL_COST * new["cost"]
    got = p.get_poses()
    step_ref = np.abs(cand - w.poses_init).max()
    assert np.abs(got - cand).max() <= 1e-4 * step_ref + 1e-12
    p.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_lm_converges_to_oracle_poses(oracle_lib, solver):
    """Ten LM iterations from the same start: GPU (device-side lambda schedule,
    captured graph) and oracle reach the same poses within 1e-4 m / 1e-5 rad."""
    import paper_2303_16878_gb300 as pba
    w = workload("room", n_frames=4, width=80, height=60, f=60.0)
    poses, lam = w.poses_init.copy(), None
    for _ in range(10):
        o = oracle_lib.lm_iteration(w, poses, lam)
        poses, lam = o["poses"], o["lam"]
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F32, solver=solver)
    for _ in range(10):
        p.iterate()
    got = p.get_poses()
    for k in range(w.n_frames):
        assert np.linalg.norm(got[k][:, 3] - poses[k][:, 3]) <= 1e-4
        R = got[k][:, :3].T @ poses[k][:, :3]
        ang = np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1))
        assert ang <= 1e-5
    p.close()


def test_graph_iteration_equals_explicit_calls(room8):
    """pba_iterate (captured graph, device lambda, full linearisation at the
    candidate) and pba_linearize + pba_solve_step (cost-only pass at the
    candidate) with the same lambda take the same step; after an accepted
    iteration the current system equals a fresh linearisation at the new poses."""
    import paper_2303_16878_gb300 as pba
    a = make(room8, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    b = make(room8, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    sa = a.iterate()
    cost, _ = b.linearize()
    sb = b.solve_step(sa["lambda_used"])
    assert sa["cost"] == cost and sa["accepted"] == sb["accepted"]
    assert abs(sa["new_cost"] - sb["new_cost"]) <= 1e-12 * sb["new_cost"]
    np.testing.assert_array_equal(a.get_poses(), b.get_poses())
    Ha, ba = a.get_system()
    b.linearize()
    Hb, bb = b.get_system()
    assert rel(Ha, Hb) <= 1e-12 and rel(ba, bb) <= 1e-12
    a.close()
    b.close()


def test_autotuned_variants_agree(oracle_lib, street3):
    """Whatever occupancy variant the autotuner keeps, the system is the same
    (within float32 reordering) and matches the oracle."""
    import paper_2303_16878_gb300 as pba
    w = street3
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, oprm(w.params, 1))
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    p.linearize()
    H0, b0 = p.get_system()
    vf, vc = p.autotune(1)
    assert vf in range(pba._lib.PBA_N_VARIANTS) and vc in range(pba._lib.PBA_N_VARIANTS)
    for v in [None] + list(range(pba._lib.PBA_N_VARIANTS)):
        if v is not None:
            p.set_variants(v, v)
        cost, _ = p.linearize()
        H1, b1 = p.get_system()
        assert rel(H1, H0) <= 1e-6 and rel(b1, b0) <= 1e-6
        assert rel(H1, ref["H"]) <= TOL_H and abs(cost - ref["cost"]) <= TOL_COST * ref["cost"]
        p.iterate()  # the graph is rebuilt for the variant
        p.set_poses(w.poses_init)
    with pytest.raises(pba.PbaError):
        p.set_variants(pba._lib.PBA_N_VARIANTS, 0)
    p.close()


@pytest.mark.parametrize("which", ["room8", "street3"])
def test_staged_tiles_give_the_same_system(oracle_lib, which, request):
    """Variants 4 .. 7 read each step's bilinear taps from a TMA-staged tile of
    the target's FP16 texels (steps whose taps do not fit the tile, or straddle
    the spherical wrap seam, read them directly): the same texel values, so the
    system, cost and count equal those of variants 0 .. 3 bit for bit, for the
    full and the cost-only pass, and match the oracle; no tile wait runs out."""
    import paper_2303_16878_gb300 as pba
    w = request.getfixturevalue(which)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, oprm(w.params, 1))
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    for v in range(pba._lib.PBA_N_VARIANTS // 2):
        out = []
        for vv in (v, v + pba._lib.PBA_N_VARIANTS // 2):
            p.set_variants(vv, vv)
            assert p.tuning()["variant_full"] == vv
            cost, count = p.linearize()
            H, b = p.get_system()
            sys_ = p.get_pair_system()
            st = p.solve_step(1e-3)  # the cost-only pass at the candidate
            p.set_poses(w.poses_init)
            p.set_lambda(None)
            it = p.iterate()  # the graph's speculative full pass at the candidate
            p.set_poses(w.poses_init)
            out.append((cost, count, H, b, sys_["H"], st["new_cost"], it["n_valid"], it["new_cost"]))
        a, c = out
        assert a[0] == c[0] and a[1] == c[1] and a[5] == c[5] and a[6] == c[6] and a[7] == c[7]
        assert np.array_equal(a[2], c[2]) and np.array_equal(a[3], c[3]) and np.array_equal(a[4], c[4])
        assert rel(c[2], ref["H"]) <= TOL_H and abs(c[0] - ref["cost"]) <= TOL_COST * ref["cost"]
    assert p.tuning()["tile_err"] == 0
    p.close()


def test_staged_variants_fall_back_without_tiles(room8):
    """FP32 texels have no staged tiles: variants 4 .. 7 run (and are reported)
    as 0 .. 3."""
    import paper_2303_16878_gb300 as pba
    p = make(room8, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F32)
    p.set_variants(6, 5)
    t = p.tuning()
    assert (t["variant_full"], t["variant_cost"]) == (2, 1)
    p.linearize()
    p.close()


def test_autotuner_reports_its_tuple_and_caches_it(oracle_lib, street3):
    """pba_autotune searches work-item size x tail size x occupancy variant;
    the chosen tuple is reported, the system with it matches the oracle, and
    an identical configuration in the same process takes the cached tuple
    without timing."""
    import paper_2303_16878_gb300 as pba
    w = street3
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, oprm(w.params, 1))
    a = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    a.autotune(1)
    ta = a.tuning()
    assert ta["chunk"] in (512, 1024, 2048) and ta["chunk_tail"] in (128, 256) and ta["ms_full"] > 0
    assert ta["reduction"] in (0, 1)
    cost, _ = a.linearize()
    H, _ = a.get_system()
    assert rel(H, ref["H"]) <= TOL_H and abs(cost - ref["cost"]) <= TOL_COST * ref["cost"]
    b = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    b.autotune(1)
    tb = b.tuning()
    assert tb["from_cache"] and (tb["chunk"], tb["chunk_tail"], tb["variant_full"], tb["reduction"]) == \
        (ta["chunk"], ta["chunk_tail"], ta["variant_full"], ta["reduction"])
    a.close()
    b.close()


def test_given_tuning_is_applied_without_timing(oracle_lib, street3):
    """pba_set_tuning applies a tuple as pba_get_tuning reports it (here one
    the autotuner never tries: 640-point items, 96-point tail) without timing;
    the system with it matches the oracle; tuples outside the documented
    ranges are refused and leave the tuning as it was."""
    import paper_2303_16878_gb300 as pba
    w = street3
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, oprm(w.params, 1))
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    given = dict(variant_full=pba._lib.PBA_N_VARIANTS - 1, variant_cost=1, chunk=640, chunk_tail=96, reduction=1)
    p.set_tuning(given)
    t = p.tuning()
    assert {k: t[k] for k in given} == given and not t["from_cache"] and t["ms_full"] == 0
    cost, _ = p.linearize()
    H, b = p.get_system()
    assert rel(H, ref["H"]) <= TOL_H and abs(cost - ref["cost"]) <= TOL_COST * ref["cost"]
    for bad in (dict(given, chunk=650), dict(given, chunk_tail=1024), dict(given, chunk_tail=0),
                dict(given, chunk=16384), dict(given, variant_cost=pba._lib.PBA_N_VARIANTS),
                dict(given, reduction=2), dict(given, reduction=-1)):
        with pytest.raises(pba.PbaError):
            p.set_tuning(bad)
        assert {k: p.tuning()[k] for k in given} == given
    assert p.iterate()["status"] == 0
    p.close()


@pytest.mark.parametrize("texel", [1, 0])
@pytest.mark.parametrize("which", ["room8", "street3"])
def test_reduction_schemes_agree(oracle_lib, which, texel, request):
    """The two reductions of a work item's 30 sums (0: transposed table in
    shared memory, 1: shuffle butterfly) give the same counts exactly and the
    same system and cost up to float32 summation order, both within the
    oracle's bars, at every occupancy variant and at short work items (many
    partial sums per pair); the iteration graph follows a changed scheme."""
    import paper_2303_16878_gb300 as pba
    w = request.getfixturevalue(which)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, oprm(w.params, texel))
    p = make(w, pba.PBA_PATH_BATCHED, texel)
    for v in range(pba._lib.PBA_N_VARIANTS // 2):
        out = []
        for red in (0, 1):
            p.set_tuning(dict(variant_full=v, variant_cost=v, chunk=256, chunk_tail=64, reduction=red))
            assert p.tuning()["reduction"] == red
            cost, count = p.linearize()
            H, b = p.get_system()
            p.set_lambda(None)
            it = p.iterate()
            p.set_poses(w.poses_init)
            out.append((cost, count, H, b, it["n_valid"]))
        (c0, n0, H0, b0, i0), (c1, n1, H1, b1, i1) = out
        assert n0 == n1 and i0 == i1 and abs(n0 - ref["count"]) <= 1e-5 * ref["count"] + 2
        assert abs(c0 - c1) <= 1e-6 * abs(c0) and rel(H1, H0) <= 1e-5 and rel(b1, b0) <= 1e-5
        for H, b, c in ((H0, b0, c0), (H1, b1, c1)):
            assert rel(H, ref["H"]) <= TOL_H and rel(b, ref["b"]) <= TOL_B
            assert abs(c - ref["cost"]) <= TOL_COST * ref["cost"]
    p.close()


def test_mixed_and_f64_solvers_agree_on_the_lidar_street():
    """One LM iteration on the full 50-frame street: the mixed solver's step
    equals the FP64 Cholesky step to the refinement tolerance."""
    import paper_2303_16878_gb300 as pba
    w = workload("street")
    a = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_CHOLESKY_F64)
    b = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16, solver=pba.PBA_SOLVE_MIXED)
    for lam in (None, 1e-3):
        for p in (a, b):
            p.set_poses(w.poses_init)
            p.set_lambda(lam)
        sa, sb = a.iterate(), b.iterate()
        assert sa["status"] == 0 and sb["status"] == 0 and sa["accepted"] == sb["accepted"]
        step = np.abs(a.get_poses() - w.poses_init).max()
        assert np.abs(a.get_poses() - b.get_poses()).max() <= 1e-8 * max(step, 1e-3)
    a.close()
    b.close()


def test_linearize_is_deterministic(room8):
    import paper_2303_16878_gb300 as pba
    p = make(room8, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    p.linearize()
    H1, b1 = p.get_system()
    p.linearize()
    H2, b2 = p.get_system()
    np.testing.assert_array_equal(H1, H2)
    np.testing.assert_array_equal(b1, b2)
    p.close()


def test_plain_and_batched_agree(room8):
    import paper_2303_16878_gb300 as pba
    a = make(room8, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F32)
    b = make(room8, pba.PBA_PATH_PLAIN, pba.PBA_TEXEL_F32)
    ca, na = a.linearize()
    cb, nb = b.linearize()
    Ha, ba = a.get_system()
    Hb, bb = b.get_system()
    assert abs(na - nb) <= 2
    assert rel(Ha, Hb) <= TOL_H and rel(ba, bb) <= TOL_B
    a.close()
    b.close()


# ------------------------------------------------------------------ edge cases

def test_self_pair_and_empty_frames(oracle_lib):
    """A self pair (i, i) at equal poses gives zero error (with FP16 texels the
    error of sampling the binary16 target values, R25: the oracle's cost); a
    frame without a single valid pixel yields no residuals and zero blocks; a
    pair that sees nothing of its target contributes nothing.  In the self
    pair every point lands exactly on a pixel centre, i.e. on a floor() tie,
    so its valid set may differ from the oracle's on points the oracle
    flags."""
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    base = workload("room", n_frames=3)
    chans = [c.copy() for c in base.channels]
    chans[2][..., 1] = 0.0  # frame 2: no valid pixel
    far = base.poses_init.copy()
    far[1][:, 3] += np.array([0.0, 0.0, -50.0])  # frame 1 far away: nothing projects into frame 0
    pairs = np.array([[0, 0], [2, 0], [0, 2], [1, 0], [0, 1]], dtype=np.int32)
    w = synth.Workload("edge", base.sensors, base.frame_sensor, chans, base.poses_gt, far, pairs, base.params)
    for texel in (0, 1):
        refs = [oracle_lib.linearize_pair(w.sensors[0], oprm(w.params, texel), w.channels[i], w.channels[j],
                                          far[i], far[j]) for i, j in pairs.tolist()]
        p = make(w, pba.PBA_PATH_BATCHED, texel)
        assert p.frame_points(2) == 0
        cost, count = p.linearize()
        ps = p.get_pair_system()
        for q, r in enumerate(refs):
            flagged = int(sum(bin(int(x)).count("1") for x in r["flags"]))
            assert abs(ps["count"][q] - r["count"]) <= flagged + 2, q
        assert ps["count"][0] > 0.9 * p.frame_points(0)
        if texel == 0:
            assert ps["cost"][0] < 1e-6
        else:
            # e = g - binary16(g), n - binary16(n) at the pixel itself; every point sits on a
            # floor() tie, so the two valid sets differ near invalid pixels: compare the
            # mean cost per residual (the same population of rounding errors)
            mo, mg = refs[0]["cost"] / refs[0]["count"], ps["cost"][0] / ps["count"][0]
            assert 0 < refs[0]["cost"] < 1e-2 and abs(mg - mo) <= 0.02 * mo, (mg, mo)
        assert np.abs(ps["b"][0]).max() < 1e-3 * np.abs(ps["H"][0]).max() ** 0.5
        assert ps["count"][1] == 0 and ps["count"][2] == 0 and np.all(ps["H"][1] == 0) and np.all(ps["H"][2] == 0)
        for q in (3, 4):
            assert ps["count"][q] == refs[q]["count"]
            if refs[q]["count"]:
                assert rel(ps["H"][q], refs[q]["H"]) <= TOL_H
        p.close()


def test_single_frame_problem():
    """N = 1: the gauge-fixed system is empty; the step keeps the pose."""
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    base = workload("room", n_frames=3)
    w = synth.Workload("one", base.sensors, base.frame_sensor[:1], base.channels[:1], base.poses_gt[:1],
                       base.poses_init[:1], np.array([[0, 0]], dtype=np.int32), base.params)
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F16)
    st = p.iterate()
    assert st["status"] == 0
    np.testing.assert_array_equal(p.get_poses(), w.poses_init)
    p.close()


def test_invalid_arguments_fail_loudly():
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    gpu()
    base = workload("room", n_frames=3)
    s2 = synth.pinhole_sensor(80, 60, 60.0, 40.0, 30.0)
    p = pba.Problem([base.sensors[0], s2], 3, base.params, frame_sensor=[0, 0, 1])
    with pytest.raises(pba.PbaError) as e:
        p.linearize()
    assert e.value.code == pba._lib.PBA_ENOTREADY
    p.upload_frames(0, np.stack(base.channels[:2]))
    with pytest.raises(ValueError):
        p.upload_frames(2, base.channels[2])  # 160 x 120 image for an 80 x 60 sensor
    p.upload_frames(2, np.zeros((60, 80, 5), dtype=np.float32))
    p.set_poses(base.poses_init)
    with pytest.raises(pba.PbaError) as e:
        p.set_pairs([[0, 2]])  # different sensors
    assert e.value.code == pba._lib.PBA_EINVAL
    with pytest.raises(pba.PbaError) as e:
        p.set_pairs([[0, 7]])
    assert e.value.code == pba._lib.PBA_EINVAL
    p.close()


def test_nonfinite_inputs_are_counted_in_the_status_word(oracle_lib):
    """The status word of a linearisation.  A NaN pose: every pair that
    touches the frame has a non-finite relative pose, yields no residual and
    is counted; the other pairs equal the oracle's.  NaN intensities at valid
    pixels of a source frame: those residuals are left out of H, b and F and
    counted; the rest of the system equals the oracle's with those pixels
    removed (frame 0 is the target of no pair, so only its points change)."""
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    w = workload("room", n_frames=4, width=80, height=60, f=60.0)
    # a NaN pose
    poses = w.poses_init.copy()
    poses[3, 0, 3] = np.nan
    p = make(w, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F32)
    p.set_poses(poses)
    p.linearize()
    ps = p.get_pair_system()
    st = p.solve_step(1.0)
    touching = [q for q, (i, j) in enumerate(w.pairs.tolist()) if 3 in (i, j)]
    assert st["nonfinite_pairs"] == len(touching) > 0 and st["n_nonfinite"] == 0 and st["status"] == 0
    assert np.all(ps["count"][touching] == 0)
    for q, (i, j) in enumerate(w.pairs.tolist()):
        if q in touching:
            continue
        r = oracle_lib.linearize_pair(w.sensors[0], w.params, w.channels[i], w.channels[j], poses[i], poses[j])
        assert abs(ps["count"][q] - r["count"]) <= 2 and rel(ps["H"][q], r["H"]) <= TOL_H
    p.close()
    # NaN intensities at 60 valid pixels of frame 0
    rng = np.random.default_rng(4)
    chans = [c.copy() for c in w.channels]
    valid = np.flatnonzero(chans[0][..., 1].reshape(-1) > 0)
    bad = rng.choice(valid, size=60, replace=False)
    chans[0].reshape(-1, 5)[bad, 0] = np.nan
    wn = synth.Workload("nan", w.sensors, w.frame_sensor, chans, w.poses_gt, w.poses_init, w.pairs, w.params)
    removed = [c.copy() for c in w.channels]
    removed[0].reshape(-1, 5)[bad, 1] = 0.0
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, removed, w.poses_init, w.pairs, w.params)
    # the points of the NaN pixels that the oracle takes as residuals (with their finite intensity)
    pts, pix = oracle_lib.frame_points(w.sensors[0], w.params, w.channels[0])
    at = {int(x): k for k, x in enumerate(pix)}
    expect, flagged = 0, 0
    for i, j in w.pairs.tolist():
        if i != 0:
            continue
        for x in bad.tolist():
            r = oracle_lib.point_residual(w.sensors[0], w.params, w.channels[j], w.poses_init[0], w.poses_init[j],
                                          pts[at[x]])
            expect += int(r["valid"])
            flagged += int(r["flag"])
    assert expect > 20
    p = make(wn, pba.PBA_PATH_BATCHED, pba.PBA_TEXEL_F32)
    cost, count = p.linearize()
    H, b = p.get_system()
    st = p.solve_step(1.0)
    assert abs(st["n_nonfinite"] - expect) <= flagged and st["nonfinite_pairs"] == 0
    assert np.all(np.isfinite(H)) and np.all(np.isfinite(b)) and np.isfinite(cost)
    assert abs(count - ref["count"]) <= 1e-5 * ref["count"] + 2
    assert rel(H, ref["H"]) <= TOL_H and rel(b, ref["b"]) <= TOL_B
    assert abs(cost - ref["cost"]) <= TOL_COST * ref["cost"]
    p.close()
