"""pba_iterate_frames: one LM iteration on new images of every frame, with the
upload overlapped by the linearisation of the pairs whose frames have arrived.

The overlapped pass takes the plan's work items in another order (by the lane
in which their frames arrive), but every item still writes its own partial-sum
slot and the per-pair reduction sums the slots in the plan's order, so the
system is the one pba_linearize forms, bit for bit.  The tests compare the
iteration with a problem that takes the same frames through pba_upload_frames
and pba_iterate: the cost at the start, the outcome and the poses after the
step must agree to rounding (the candidate's cost comes from the cost-only
pass here and from the full pass there: the same per-point arithmetic).
"""
import ctypes

import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu


def _flat(w, channels=None):
    import torch
    ch = w.channels if channels is None else channels
    host = [c.detach().cpu().numpy() if hasattr(c, "detach") else np.asarray(c) for c in ch]
    return torch.from_numpy(np.concatenate([h.astype(np.float32).reshape(-1) for h in host])).pin_memory()


def _same_step(st, ref, n_valid, poses, poses_ref, cost_rel=1e-12, pose_abs=1e-12):
    """st: pba_iterate_frames; ref: pba_iterate on the same system; n_valid: the
    residual count of that system's linearisation (pba_iterate reports the
    candidate's, pba_iterate_frames the count at the poses it linearised at).
    The batched path's sums are deterministic (bit for bit, hence the 1e-12
    defaults); the plain path adds its per-pair sums with float atomics."""
    assert st["status"] == 0 and ref["status"] == 0
    assert st["accepted"] == ref["accepted"]
    assert st["cost"] == pytest.approx(ref["cost"], rel=cost_rel)
    assert st["new_cost"] == pytest.approx(ref["new_cost"], rel=1e-6)
    assert st["n_valid"] == n_valid
    assert np.abs(poses - poses_ref).max() <= pose_abs


def _cases():
    return {"room16": lambda: workload("room", n_frames=16),
            "street": lambda: workload("street"),
            "fusion": lambda: workload("fusion")}


@pytest.mark.parametrize("which", ["room16", "street", "fusion"])
def test_iterate_frames_equals_upload_and_iterate(which):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    w = _cases()[which]()
    init = np.ascontiguousarray(w.poses_init.reshape(-1, 12))
    flat = _flat(w)
    a = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16,
                                  solver=pba.PBA_SOLVE_MIXED)
    ref = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16,
                                    solver=pba.PBA_SOLVE_MIXED)
    a.set_lambda(None)
    st = a.iterate_frames(flat, init)
    ref.set_poses(init)
    ref.set_lambda(None)
    _, n0 = ref.linearize()
    r = ref.iterate()
    _same_step(st, r, n0, a.get_poses(), ref.get_poses())
    # the next call: new frames (the same values) at the poses reached; pba_iterate
    # continues from the system it formed at its candidate
    st = a.iterate_frames(flat)
    r2 = ref.iterate()
    _same_step(st, r2, r["n_valid"] if r["accepted"] else n0, a.get_poses(), ref.get_poses())
    a.close()
    ref.close()


def test_iterate_frames_with_changed_point_counts():
    """New images whose valid pixel counts differ from the uploaded ones: the
    pass started on the previous plan is redone on the rebuilt one, and the
    result equals a problem built from the new images; the following call
    (counts unchanged since) overlaps again with the new plan."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import dataclasses
    import paper_2303_16878_gb300 as pba
    w = workload("room", n_frames=16)
    chans = [np.array(c, dtype=np.float32, copy=True) for c in w.channels]
    for k, (r, c) in ((3, (20, 30)), (10, (60, 90)), (15, (5, 5))):
        chans[k][r:r + 24, c:c + 24, 1] = 0.0  # no depth: these pixels are no longer points
    w2 = dataclasses.replace(w, channels=chans)
    init = np.ascontiguousarray(w.poses_init.reshape(-1, 12))
    a = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16,
                                  solver=pba.PBA_SOLVE_MIXED)
    before = [a.frame_points(k) for k in range(w.n_frames)]
    ref = pba.problem_from_workload(w2, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16,
                                    solver=pba.PBA_SOLVE_MIXED)
    flat = _flat(w2)
    for _ in range(2):
        a.set_lambda(None)
        st = a.iterate_frames(flat, init)
        ref.set_poses(init)
        ref.set_lambda(None)
        _, n0 = ref.linearize()
        r = ref.iterate()
        _same_step(st, r, n0, a.get_poses(), ref.get_poses())
    after = [a.frame_points(k) for k in range(w.n_frames)]
    assert [k for k in range(w.n_frames) if after[k] != before[k]] == [3, 10, 15]
    a.close()
    ref.close()


def test_iterate_frames_on_the_plain_path_and_bad_arguments():
    """The plain per-pair path takes the sequential route (uploads, then the
    iteration) with the same outcome; a NULL channels pointer or a buffer of
    the wrong size is refused."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    w = workload("room", n_frames=4)
    init = np.ascontiguousarray(w.poses_init.reshape(-1, 12))
    flat = _flat(w)
    a = pba.problem_from_workload(w, path=pba.PBA_PATH_PLAIN, texel=pba.PBA_TEXEL_F32)
    ref = pba.problem_from_workload(w, path=pba.PBA_PATH_PLAIN, texel=pba.PBA_TEXEL_F32)
    a.set_lambda(None)
    st = a.iterate_frames(flat, init)
    ref.set_poses(init)
    ref.set_lambda(None)
    _, n0 = ref.linearize()
    r = ref.iterate()
    # float atomics: the sums agree to float32 rounding, the step to its effect
    _same_step(st, r, n0, a.get_poses(), ref.get_poses(), cost_rel=1e-6, pose_abs=1e-6)
    assert a._lib.pba_iterate_frames(a._h, None, None, None) == pba._lib.PBA_EINVAL
    with pytest.raises(ValueError):
        a.iterate_frames(flat[:-5])
    a.close()
    ref.close()
