"""pba_linearize_pairs_noalloc, the linearisation entry point that allocates
nothing.

It serves callers that cannot allocate device memory: code handed its buffers
by a host framework that owns the memory pool, or loops whose memory budget is
fixed at start-up.  They pass inputs and outputs; the working memory is a
static array inside the library.  The test calls it through the C ABI on
buffers the test allocates, twice in a row (the second call in a different
pair order, so stale scratch contents would show), and compares each output
with pba_get_pair_system of a problem on the same inputs, within the parity
tolerances of the other GPU tests; on depths and normals at the validity
thresholds it is compared with the oracle directly.  Kept in a file collected
last.
"""
import ctypes

import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _structs(w):
    from paper_2303_16878_gb300 import _lib
    s = w.sensors[0]
    sen = _lib.PbaSensor()
    sen.model, sen.width, sen.height = s.model, s.width, s.height
    sen.fx, sen.fy, sen.cx, sen.cy = s.fx, s.fy, s.cx, s.cy
    for e, v in enumerate(np.asarray(s.extrinsic, dtype=np.float64).reshape(12)):
        sen.extrinsic[e] = v
    cfg = _lib.PbaConfig()
    for key in ("w_int", "w_depth", "w_normal", "huber_delta", "occ_abs", "occ_rel", "z_min", "range_min",
                "range_max"):
        setattr(cfg, key, float(w.params[key]))
    cfg.grad_mode = int(w.params.get("grad_mode", 0))
    return sen, cfg


@pytest.mark.parametrize("which", ["room8", "street3"])
def test_noalloc_matches_problem_on_two_calls(which, request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import _lib
    w = request.getfixturevalue(which)
    lib = _lib.load()
    p = pba.problem_from_workload(w, path=pba.PBA_PATH_PLAIN, texel=pba.PBA_TEXEL_F32)
    p.linearize()
    ref = p.get_pair_system()
    p.close()

    sen, cfg = _structs(w)
    dev = torch.device("cuda", torch.cuda.current_device())
    chans = torch.from_numpy(np.stack(w.channels).astype(np.float32)).to(dev).contiguous()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses_init.reshape(-1, 12))).to(dev)
    m = len(w.pairs)
    out = torch.empty((m, _lib.PBA_NOALLOC_PAIR_STRIDE), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for order in (np.arange(m), np.arange(m)[::-1].copy()):
        pairs = torch.from_numpy(np.ascontiguousarray(w.pairs[order], dtype=np.int32)).to(dev)
        out.fill_(float("nan"))
        st = lib.pba_linearize_pairs_noalloc(ctypes.byref(sen), ctypes.byref(cfg), chans.data_ptr(), w.n_frames,
                                             poses.data_ptr(), pairs.data_ptr(), m, out.data_ptr(),
                                             stream.cuda_stream)
        assert st == _lib.PBA_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        H = got[:, :144].reshape(m, 12, 12)
        b = got[:, 144:156]
        assert rel(H, ref["H"][order]) <= TOL
        assert rel(b, ref["b"][order]) <= TOL
        assert rel(got[:, 156], ref["cost"][order]) <= 1e-5
        assert np.abs(got[:, 157] - ref["count"][order]).max() <= 2


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_16878_gb300 import _lib
    w = workload("room", n_frames=3)
    lib = _lib.load()
    sen, cfg = _structs(w)
    dev = torch.device("cuda", torch.cuda.current_device())
    chans = torch.zeros((3, 120, 160, 5), dtype=torch.float32, device=dev)
    poses = torch.zeros((3, 12), dtype=torch.float64, device=dev)
    m = _lib.PBA_NOALLOC_MAX_PAIRS + 1
    pairs = torch.zeros((m, 2), dtype=torch.int32, device=dev)
    out = torch.zeros((m, _lib.PBA_NOALLOC_PAIR_STRIDE), dtype=torch.float64, device=dev)
    st = lib.pba_linearize_pairs_noalloc(ctypes.byref(sen), ctypes.byref(cfg), chans.data_ptr(), 3, poses.data_ptr(),
                                         pairs.data_ptr(), m, out.data_ptr(), None)
    assert st == _lib.PBA_ETOOBIG
    assert torch.count_nonzero(out).item() == 0


def test_noalloc_decides_range_limits_like_the_oracle(oracle_lib):
    """Depths one float32 ulp around range limits that are not float32 numbers
    (0.7 and 4.3 m), and normals with |n|^2 within rounding of 0.25: the
    entry point keeps exactly the points the oracle keeps (its limits are the
    float images rounded inwards; near 0.25 the double sum decides), and its
    blocks meet the parity bars against the oracle's."""
    import dataclasses
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_16878_gb300 import _lib, synth
    from test_gpu_pack import RANGE_MAX, RANGE_MIN, _adversarial
    w = synth.make_rgbd_room(n_frames=4, width=96, height=72, f=72.0, seed=5)
    w = _adversarial(w)
    w = dataclasses.replace(w, params=dict(w.params, range_min=RANGE_MIN, range_max=RANGE_MAX))
    lib = _lib.load()
    sen, cfg = _structs(w)
    dev = torch.device("cuda", torch.cuda.current_device())
    chans = torch.from_numpy(np.stack(w.channels).astype(np.float32)).to(dev).contiguous()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses_init.reshape(-1, 12))).to(dev)
    m = len(w.pairs)
    pairs = torch.from_numpy(np.ascontiguousarray(w.pairs, dtype=np.int32)).to(dev)
    out = torch.empty((m, _lib.PBA_NOALLOC_PAIR_STRIDE), dtype=torch.float64, device=dev)
    st = lib.pba_linearize_pairs_noalloc(ctypes.byref(sen), ctypes.byref(cfg), chans.data_ptr(), w.n_frames,
                                         poses.data_ptr(), pairs.data_ptr(), m, out.data_ptr(), None)
    assert st == _lib.PBA_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for q, (i, j) in enumerate(w.pairs.tolist()):
        r = oracle_lib.linearize_pair(w.sensors[0], w.params, w.channels[i], w.channels[j], w.poses_init[i],
                                      w.poses_init[j])
        flagged = int(sum(bin(int(x)).count("1") for x in r["flags"]))
        assert abs(got[q, 157] - r["count"]) <= flagged + 2, q
        assert rel(got[q, :144].reshape(12, 12), r["H"]) <= TOL and rel(got[q, 144:156], r["b"]) <= TOL
        assert abs(got[q, 156] - r["cost"]) <= 1e-5 * r["cost"]
