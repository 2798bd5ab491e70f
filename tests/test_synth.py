"""The torch renderer and overlap ratio (used to generate the large
configurations on the GPU) reproduce the numpy ones bit for bit (CPU)."""
import numpy as np


def test_torch_renderer_matches_numpy():
    import torch
    from paper_2303_16878_gb300 import synth
    room = synth._room_scene(1001)
    cam = synth.pinhole_sensor(64, 48, 50.0, 31.5, 23.5)
    pose = synth.look_at([0.5, 0.3, 1.5], [0.0, 2.5, 1.3])
    cases = [(room, cam, pose, 0.5, 5.0)]
    street = synth._street_scene(1002, 0.0, 20.0)
    lidar = synth.spherical_sensor(128, 16, 16.6, -16.6)
    P = synth._street_trajectory(12, 1.0, 2002)
    cases += [(street, lidar, P[k], 1.0, 80.0) for k in (1, 9)]
    hall = synth._hall_scene(1003)
    path = synth._hall_path(6, 2003)
    Xc = np.zeros((3, 4))
    Xc[:, :3] = synth.CAMERA_ON_PLATFORM
    cases += [(hall, cam, synth.compose(path[k], Xc), 0.5, 5.0) for k in (0, 3)]
    cases += [(hall, lidar, path[2], 0.5, 8.0)]
    for scene, s, X, dmin, dmax in cases:
        a = synth.render(scene, s, X, dmin, dmax)
        b = synth.render_t(scene, s, X, dmin, dmax).numpy()
        assert np.array_equal(a, b)
        assert (a[..., 1] > 0).mean() > 0.2


def test_torch_overlap_ratios_match_numpy():
    import torch
    from paper_2303_16878_gb300 import synth
    w = synth.make_lidar_street(n_frames=4, width=128, height=16)
    s = w.sensors[0]
    rays = torch.as_tensor(synth._pixel_rays(s)[0].reshape(-1, 3), dtype=torch.float64)
    ch = [torch.as_tensor(c) for c in w.channels]
    got = synth.overlap_ratios_t(ch[0], ch[1:], s, w.poses_gt[0], w.poses_gt[1:], rays, stride=7)
    ref = [synth.overlap_ratio(w.channels[0], w.channels[j], s, w.poses_gt[0], w.poses_gt[j], stride=7)
           for j in (1, 2, 3)]
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
