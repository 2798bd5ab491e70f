"""Host-side logic of bench.py that needs no GPU: the clock-sample summary and
the JSON line built from a measurement."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _line(t, sm, power, pcap="Not Active", hw="Not Active"):
    return f"2026/01/02 03:04:{t:06.3f}, 0, {sm}, 2070, {power}, 0x0, {hw}, Not Active, Not Active, {pcap}\n"


def test_clock_summary_keeps_the_timed_region():
    import bench
    lines = [_line(1.0, 1200, 150), _line(2.0, 2032, 900), _line(2.1, 2040, 950, pcap="Active"),
             _line(2.2, 2025, 940), _line(3.5, 1100, 140, hw="Active")]
    rows = bench.parse_clock_lines(lines)
    assert len(rows) == 5
    t0, t1 = rows[1]["ts"], rows[3]["ts"]
    s = bench.summarise_clocks(rows, (t0, t1))
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2032 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the region


def test_clock_summary_widens_a_short_region():
    import bench
    rows = bench.parse_clock_lines([_line(1.0, 2000, 800), _line(1.3, 2010, 820), _line(1.45, 2020, 810)])
    s = bench.summarise_clocks(rows, (rows[2]["ts"] - 0.01, rows[2]["ts"] + 0.01), slack=0.5)
    assert s["samples"] == 3 and s["window"].startswith("timed region +-")
    assert bench.summarise_clocks([], (0.0, 1.0)) is None


def test_json_line_carries_the_contract_keys_and_its_arithmetic():
    """The GPU arm's line from a fake measurement: contract keys, the roofline
    arithmetic (algorithmic FLOPs by camera model over the kernel's event time
    against the nominal ALU peak; DRAM traffic from the ncu table of the kept
    variant, null without an entry) and JSON serialisability."""
    import argparse
    import json
    import bench
    args = argparse.Namespace(steps=100, warmup=3, workload="street")
    out = dict(value=1.7e10, ms_per_step=1.3, n_valid=22_000_000, n_valid_mean=21_500_000.0, n_points=68_000_000,
               n_pairs=1170, launches=10, variants=(1, 2),
               clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 6, "window": "timed region"},
               phase_ms={"solve": 0.17, "update": 0.02, "linearize": 1.08, "reduce_assemble": 0.05, "accept": 0.01},
               solve_update_f64_ms=0.78, plain_ms_per_step=29.0,
               e2e={"value": 6.8e9, "unit": bench.UNIT, "h2d_bytes_per_step": 65540800, "d2h_bytes_per_step": 4848})
    line = bench.make_line(args, 1, out, 50, 152, 6693.8)
    json.dumps(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches"):
        assert k in line, k
    assert line["gpu_launches"] == 1000 and line["scalar_residuals_per_s"] == 5 * 1.7e10
    r = line["roofline"]
    flops = 21_500_000.0 * bench.FLOP_PER_RESIDUAL_FULL + 68_000_000 * bench.FLOP_PER_POINT_SPHERICAL
    assert abs(r["achieved"] - flops / 1.08e-3 / 1e12) < 1e-9 * r["achieved"]
    assert abs(r["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12 and 0 < r["frac"] < 1
    assert abs(line["speedup_vs_plain"] - 29.0 / 1.3) < 1e-12
    # traffic: null without a capture of the kept variant, the capture's bytes with one
    assert r["traffic"] is None and r["hbm"]["frac"] is None
    bench.LINEARIZE_NCU[("street", 1, 1024, 256, 0)] = {"dram_bytes": 4.0e8, "units": {"sm_issue": 0.7}}
    try:
        r = bench.make_line(args, 1, out, 50, 152, 6693.8)["roofline"]
    finally:
        bench.LINEARIZE_NCU.pop(("street", 1, 1024, 256, 0))
    assert r["traffic"] == 4.0e8 and abs(r["hbm"]["frac"] - 4.0e8 / 1.08e-3 / 1e9 / 6693.8) < 1e-12
    # a mixed pinhole / spherical workload counts each model's points and residuals
    out2 = dict(out, points_by_model={0: 10_000_000, 1: 5_000_000}, residual_share_by_model={0: 0.75, 1: 0.25})
    r2 = bench.make_line(args, 1, out2, 50, 152, 6693.8)["roofline"]
    f2 = (21_500_000.0 * (0.75 * bench.FLOP_PER_RESIDUAL[0] + 0.25 * bench.FLOP_PER_RESIDUAL[1])
          + 10_000_000 * bench.FLOP_PER_POINT[0] + 5_000_000 * bench.FLOP_PER_POINT[1])
    assert abs(r2["achieved"] - f2 / 1.08e-3 / 1e12) < 1e-9 * r2["achieved"]


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference: one line with impl, the metric and unit of the GPU arm,
    a cpu_baseline describing the run and an e2e object with zero copies; the
    per-step sample budget keeps 100 + 3 steps near 150 s of oracle work."""
    import argparse
    import json
    import bench
    calls = []

    def fake_sample(w, seconds, seed=0):
        calls.append(seconds)
        return dict(value=5.0e5 + seed, unit=bench.UNIT, cores=1, kind="oracle", sample="fake", seconds=seconds,
                    pairs=3)

    class FakePool:
        def __init__(self, name, workers=None):
            self.n = 4

        def sample(self, seconds, seed=0):
            return fake_sample(None, seconds, seed)

        def close(self):
            calls.append("closed")

    monkeypatch.setattr(bench, "OraclePool", FakePool)
    args = argparse.Namespace(workload="street", steps=100, warmup=3, cpu_seconds=12.0, gpus=1)
    bench.run_reference(args)
    assert calls.pop() == "closed"
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 100 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 4
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert len(calls) == 103 and 0.5 <= calls[0] <= 12.0 and 103 * calls[0] <= 160.0
    assert abs(line["value"] - (5.0e5 + sum(range(3, 103)) / 100)) < 1e-6


def test_hbm_peak_comes_from_the_measured_file_or_says_fallback(tmp_path):
    import json
    import bench
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6693.8, "bf16_tflops": 1900.0}))
    assert bench.measured_hbm(str(f)) == (6693.8, "measured: MEASURED_PEAKS.json hbm_gbs")
    gbs, src = bench.measured_hbm(str(tmp_path / "absent.json"))
    assert gbs == 6800.0 and src.startswith("fallback")
    f.write_text("{}")
    assert bench.measured_hbm(str(f))[1].startswith("fallback")


def test_main_wires_the_measurement_into_one_line(monkeypatch, capsys):
    """main() on a faked single-GPU run: the measurement of run_ours, the SM
    count, the HBM peak and the CPU baseline end up in one JSON line."""
    import json
    import sys
    import types
    import torch
    import bench
    out = dict(value=1.7e10, ms_per_step=1.3, n_valid=22_000_000, n_valid_mean=21_500_000.0, n_points=68_000_000,
               n_pairs=1170, launches=10, variants=(1, 2), clocks=None,
               phase_ms={"solve": 0.17, "update": 0.02, "linearize": 1.08, "reduce_assemble": 0.05, "accept": 0.01},
               solve_update_f64_ms=0.78, build_pairs={}, normals={}, adjoint={})
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(bench, "run_ours", lambda args, rank, world, device: (out, types.SimpleNamespace(n_frames=50)))
    monkeypatch.setattr(bench, "oracle_sample", lambda w, seconds, seed=0: dict(
        value=5.3e5, unit=bench.UNIT, cores=1, kind="oracle", sample="fake", seconds=seconds, pairs=3))

    class FakePool:
        def __init__(self, name, workers=None):
            self.n = 16

        def sample(self, seconds, seed=0, want_blocks=False):
            return dict(value=8.0e6, unit=bench.UNIT, cores=16, kind="oracle", sample="fake16", seconds=seconds)

        def close(self):
            pass

    monkeypatch.setattr(bench, "OraclePool", FakePool)
    monkeypatch.setattr(bench, "sample_slices", lambda w, n, k, masks=None: [])
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "7", "--warmup", "3", "--workload", "street"])
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.main()
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["steps"] == 7 and line["gpu_launches"] == 70 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["value"] == 8.0e6 and line["cpu_baseline"]["cores"] == 16
    assert line["cpu_baseline_one_core"]["value"] == 5.3e5 and line["roofline"]["peak"] > 80.0
    assert line["roofline"]["hbm"]["peak_source"].startswith(("measured", "fallback"))


def test_oracle_pool_times_disjoint_slices_concurrently():
    """Two spawn-started oracle processes on the small RGB-D room: one sample
    covers more pairs than either slice alone, reports 2 cores, and its rate
    is the residuals of both over the slower one's time; the processes end on
    close()."""
    import bench
    pool = bench.OraclePool("room", workers=2)
    try:
        r = pool.sample(0.3, seed=1)
    finally:
        pool.close()
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["pairs"] >= 2
    assert abs(r["value"] - r["residuals"] / r["seconds"]) < 1e-6 * r["value"]
    assert all(not p.is_alive() for p in pool.procs)


def test_oracle_pool_reports_a_dead_worker_quickly():
    """A worker that cannot build its workload ends at once; the pool raises
    within seconds instead of waiting for its timeout."""
    import time
    import pytest
    import bench
    t0 = time.time()
    with pytest.raises(RuntimeError):
        bench.OraclePool("no-such-workload", workers=2, ready_timeout=120.0)
    assert time.time() - t0 < 60.0


def test_stated_error_is_the_sampled_subsystem_error():
    """stated_error: the stacked blocks' relative Frobenius errors, each pair's
    largest, the count difference and the share decided the other way."""
    import numpy as np
    import bench
    rng = np.random.default_rng(3)
    H = rng.normal(size=(3, 12, 12))
    b = rng.normal(size=(3, 12))
    ps = {"H": H + 1e-6 * rng.normal(size=H.shape), "b": b.copy(), "cost": np.array([1.0, 2.0, 3.0]),
          "count": np.array([10, 20, 31])}
    blocks = {0: (H[0], b[0], 1.0, 10, 0), 1: (H[1], b[1], 2.0, 20, 1), 2: (H[2], b[2], 3.3, 30, 2)}
    e = bench.stated_error(ps, blocks)
    dH = np.sqrt(sum(np.sum((ps["H"][q] - H[q]) ** 2) for q in range(3)) / np.sum(H ** 2))
    assert abs(e["H_rel"] - dH) < 1e-15 and e["b_rel"] == 0.0
    assert abs(e["cost_rel"] - 0.3 / 6.3) < 1e-12 and e["per_pair_max"]["count_diff"] == 1
    assert e["decided_other_way"] == 3 / 60 and e["pairs"] == 3


def test_sample_slices_keep_only_their_frames():
    """The CPU legs' slices: disjoint seeded pairs, each slice's frames
    renumbered, the same channels and poses as the full workload."""
    import numpy as np
    import bench
    from conftest import workload
    w = workload("room")
    sl = bench.sample_slices(w, 3, 9, masks={q: np.array([q], dtype=np.uint32) for q in range(len(w.pairs))})
    ids = [q for _, qs, _ in sl for q in qs]
    assert len(ids) == 9 and len(set(ids)) == 9
    for sub, qs, masks in sl:
        assert sorted(masks) == list(range(len(qs)))
        for n, q in enumerate(qs):
            i, j = w.pairs[q]
            si, sj = sub.pairs[n]
            assert np.array_equal(sub.channels[si], w.channels[i]) and np.array_equal(sub.channels[sj], w.channels[j])
            assert np.array_equal(sub.poses_init[si], w.poses_init[i]) and masks[n][0] == q


def test_pyramid_leg_reports_every_level_and_the_schedule(monkeypatch):
    """The per-level timing leg on a stand-in for the problem: one entry per
    level with its pixel count (sensor sizes halved per level), points,
    residuals and times, coarse levels tuned, and the schedule's per-level
    outcome."""
    import types
    import bench

    calls = []

    class Level:
        def __init__(self, lv):
            self.lv = lv
            self._sizes = [(480 >> lv, 640 >> lv), (128 >> lv, 1024 >> lv)]
            self._fs = [0, 0, 1]

        def autotune(self, repeats):
            calls.append(("autotune", self.lv))

        def frame_points(self, i):
            return 1000 >> (2 * self.lv)

    class Prob:
        def __init__(self):
            self.levels = {lv: Level(lv) for lv in range(3)}

        def build_pyramid(self, n):
            calls.append(("build", n))

        def level(self, lv):
            return self.levels[lv]

        def set_poses(self, p):
            pass

        def set_lambda(self, x):
            pass

        def optimize(self, schedule):
            return [dict(level=2 - k, iterations=n, accepted=n - 1, status=0, cost_first=10.0 - k, cost_last=9.0 - k)
                    for k, n in enumerate(schedule)]

    def fake_time(q, init, stream, flush, steps, warmup):
        return [2.0 / (1 + q.lv)] * steps, [100.0 / (1 + q.lv)] * steps

    monkeypatch.setattr(bench, "time_iterations", fake_time)
    torch_stub = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setitem(__import__("sys").modules, "torch", torch_stub)
    import numpy as np
    w = types.SimpleNamespace(pairs=np.array([[0, 1], [1, 2], [2, 0]]))
    out = bench.pyramid_leg(Prob(), w, None, None, None, 4, 1)
    assert calls[0] == ("build", 3) and ("autotune", 1) in calls and ("autotune", 2) in calls
    assert ("autotune", 0) not in calls
    px = [lv["pixels"] for lv in out["levels"]]
    assert px == [2 * 480 * 640 + 128 * 1024, 2 * 240 * 320 + 64 * 512, 2 * 120 * 160 + 32 * 256]
    assert [lv["points_per_iteration"] for lv in out["levels"]] == [3000, 3 * 250, 3 * 62]
    assert out["levels"][1]["ms_per_iteration"] == 1.0 and out["levels"][1]["residuals_per_iteration"] == 50.0
    assert abs(out["levels"][0]["residuals_per_s"] - 100.0 / 2e-3) < 1e-6
    assert out["schedule"] == [10, 5, 2] and [x["level"] for x in out["optimize_levels"]] == [2, 1, 0]
    assert out["optimize_levels"][0]["iterations"] == 10 and out["optimize_ms"] >= 0.0


def test_solve_roof_is_the_dense_cholesky_work_at_the_measured_rate():
    """The solve's roof object: n = 6 x pose variables unknowns, n^3 / 3 FLOP of a
    dense Cholesky, its time at the measured FP64 rate, and null without a rate."""
    import bench
    r = bench.solve_roof(2.85, 599, 1.1)
    n = 6 * 599
    assert r["unknowns"] == n and r["solve_ms"] == 2.85 and r["fp64_dgemm_tflops_measured"] == 1.1
    assert abs(r["dense_cholesky_gflop"] - n ** 3 / 3e9) < 1e-9
    assert abs(r["dense_cholesky_ms_at_measured_fp64"] - n ** 3 / 3e9 / 1.1) < 1e-9
    assert "latency" in r["bound"]
    assert bench.solve_roof(2.85, 599, None) is None and bench.solve_roof(None, 599, 1.1) is None
