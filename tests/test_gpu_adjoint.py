"""The adjoint (pba_cost_gradient and its autograd wrapper) against central
finite differences of the FP64 oracle's total cost, and the pose gradient in
the box-plus chart against the oracle's 2 b (grad_mode 1, exact Jacobians).
Bar: 1e-4 relative (norm of the difference over the norm of the reference)."""
import numpy as np
import pytest

from conftest import workload

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _problem(w):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_16878_gb300 as pba
    return pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F32)


def _oracle_cost(O, w, poses, channels=None, sensors=None):
    r = O.linearize(sensors or w.sensors, w.frame_sensor, channels or w.channels, poses, w.pairs, w.params,
                    want_system=False)
    return r["cost"], r["count"]


def _fd(O, w, f_poses=None, f_sens=None, f_chan=None, h=1e-6):
    """Central difference of the oracle's F along a perturbation built by the callbacks."""
    vals = []
    for sg in (1, -1):
        poses = f_poses(sg * h) if f_poses else w.poses_init
        sensors = f_sens(sg * h) if f_sens else None
        chans = f_chan(sg) if f_chan else None
        vals.append(_oracle_cost(O, w, poses, chans, sensors))
    assert vals[0][1] == vals[1][1], "validity changed under the finite-difference step"
    return vals


@pytest.mark.parametrize("which", ["room3", "street3"])
def test_pose_gradient_matches_finite_differences(oracle_lib, which, request):
    w = request.getfixturevalue(which)
    p = _problem(w)
    cost, n, dP, _, _ = p.cost_gradient(poses=True, extrinsics=False)
    g = dP.cpu().numpy()
    fd = np.zeros_like(g)
    h = 1e-7
    for k in range(w.n_frames):
        for r in range(3):
            for c in range(4):
                def fp(eps, k=k, r=r, c=c):
                    P = w.poses_init.copy()
                    P[k, r, c] += eps
                    return P
                v = _fd(oracle_lib, w, f_poses=fp, h=h)
                fd[k, r, c] = (v[0][0] - v[1][0]) / (2 * h)
    assert rel(g, fd) <= TOL
    p.close()


def test_tangent_gradient_is_twice_b(oracle_lib, room3):
    import torch
    from paper_2303_16878_gb300.autograd import tangent_gradient
    w = room3
    params = dict(w.params, grad_mode=1)
    ref = oracle_lib.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs, params)
    p = _problem(w)
    _, _, dP, _, _ = p.cost_gradient(poses=True, extrinsics=False)
    gt = tangent_gradient(p, torch.from_numpy(w.poses_init).to(dP.device), dP).cpu().numpy().reshape(-1)
    assert rel(gt, 2.0 * ref["b"]) <= TOL
    p.close()


def test_extrinsic_gradient_matches_finite_differences(oracle_lib, room3):
    from paper_2303_16878_gb300 import synth
    w = synth.with_extrinsic(room3, synth.offset_transform(0.05, 3.0, seed=11))
    p = _problem(w)
    _, _, _, dE, _ = p.cost_gradient(poses=False, extrinsics=True)
    g = dE.cpu().numpy()[0]
    fd = np.zeros((3, 4))
    h = 1e-7
    for r in range(3):
        for c in range(4):
            def fs(eps, r=r, c=c):
                Xo = np.array(w.sensors[0].extrinsic, dtype=np.float64).reshape(3, 4).copy()
                Xo[r, c] += eps
                return [synth.Sensor(**{**w.sensors[0].__dict__, "extrinsic": Xo})]
            v = _fd(oracle_lib, w, f_sens=fs, h=h)
            fd[r, c] = (v[0][0] - v[1][0]) / (2 * h)
    assert rel(g, fd) <= TOL
    p.close()


def test_image_gradient_matches_finite_differences(oracle_lib, room3):
    """Sampled target and source pixels: perturb one channel value of one
    pixel in the oracle's float32 input and difference F (the step is the
    float32-rounded one actually applied)."""
    w = room3
    p = _problem(w)
    _, _, _, _, dI = p.cost_gradient(poses=False, extrinsics=False, images=True)
    g = dI.cpu().numpy().reshape(w.n_frames, 120, 160, 5)
    rng = np.random.default_rng(3)
    cand = np.argwhere(np.abs(g) > 1e-3 * np.abs(g).max())
    picks = cand[rng.choice(len(cand), size=min(24, len(cand)), replace=False)]
    errs, refs = [], []
    for f, r, c, ch in picks.tolist():
        base = w.channels[f][r, c, ch]
        step = np.float32(max(abs(base) * 2.0 ** -12, 2.0 ** -16))
        hi, lo = np.float32(base + step), np.float32(base - step)

        def fc(sg, f=f, r=r, c=c, ch=ch):
            chans = [x.copy() for x in w.channels]
            chans[f][r, c, ch] = hi if sg > 0 else lo
            return chans
        v = _fd(oracle_lib, w, f_chan=fc)
        fd = (v[0][0] - v[1][0]) / (float(hi) - float(lo))
        errs.append(g[f, r, c, ch] - fd)
        refs.append(fd)
    assert np.linalg.norm(errs) <= TOL * np.linalg.norm(refs)
    p.close()


def test_autograd_function_matches_and_descends(room3):
    import torch
    from paper_2303_16878_gb300.autograd import photometric_cost
    w = room3
    p = _problem(w)
    dev = torch.device("cuda")
    poses = torch.from_numpy(w.poses_init.copy()).to(dev).requires_grad_(True)
    ext = torch.from_numpy(np.array(w.sensors[0].extrinsic, dtype=np.float64).reshape(1, 3, 4)).to(dev)
    ext.requires_grad_(True)
    chans = torch.from_numpy(np.stack(w.channels)).to(dev).requires_grad_(True)
    F = photometric_cost(p, poses, ext, chans)
    F.backward()
    _, _, dP, dE, dI = p.cost_gradient(poses=True, extrinsics=True, images=True)
    assert torch.allclose(poses.grad, dP) and torch.allclose(ext.grad, dE)
    # the image gradient accumulates with FP32 atomics: two calls agree up to the summation order
    gi = chans.grad.reshape(-1)
    assert float(torch.linalg.norm(gi - dI)) <= 1e-5 * float(torch.linalg.norm(dI))
    # a small step against the se(3) gradient lowers F
    from paper_2303_16878_gb300.autograd import tangent_gradient
    import oracle
    gt = tangent_gradient(p, poses.detach(), poses.grad).cpu().numpy()
    gt[0] = 0.0
    step = -1e-4 / np.abs(gt).max() * gt
    new = np.stack([oracle.boxplus(w.poses_init[k], step[k]) for k in range(w.n_frames)])
    F2 = photometric_cost(p, torch.from_numpy(new).to(dev), ext.detach(), chans.detach())
    assert F2.item() < F.item()
    p.close()
