"""Graph construction on the GPU (Sec. IV-B) against the oracle: the same
pair list, except candidates whose ratio lies within the oracle's float32
decision margin of the threshold."""
import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu


def _compare(oracle_lib, w, max_angle, max_dist, min_ratio, sequential):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    ref = oracle_lib.build_pairs(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.params, max_angle,
                                 max_dist, min_ratio, sequential)
    p = pba.problem_from_workload(w)
    pairs_before = p.n_pairs
    got, ratios = p.build_pairs(max_angle, max_dist, min_ratio, sequential)
    got_set = {tuple(x) for x in got.tolist()}
    ref_set = {tuple(x) for x in ref["pairs"].tolist()}
    for key in got_set ^ ref_set:
        c = ref["candidates"][key]
        margin = (c["flagged"] + 2) / max(c["n_points"], 1)
        assert abs(c["ratio"] - min_ratio) <= margin, (key, c)
    for k, key in enumerate(got.tolist()):
        c = ref["candidates"][tuple(key)]
        assert abs(ratios[k] - c["ratio"]) <= (c["flagged"] + 2) / max(c["n_points"], 1) + 1e-6
    # the problem's own pairs are untouched and still linearise
    assert p.n_pairs == pairs_before
    cost, count = p.linearize()
    assert count > 0
    p.close()
    return got


def test_build_pairs_room(oracle_lib, room8):
    got = _compare(oracle_lib, room8, np.radians(30.0), 1.5, 1.0 / 3.0, False)
    assert len(got) > 0


def test_build_pairs_street_sequential(oracle_lib):
    w = workload("street", n_frames=12)
    got = _compare(oracle_lib, w, np.radians(30.0), 6.0, 0.3, True)
    assert all((i, i + 1) in {tuple(x) for x in got.tolist()} for i in range(11))
