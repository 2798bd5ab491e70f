"""Shared fixtures.  GPU tests carry @pytest.mark.gpu; everything else runs on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


_CACHE = {}


def workload(name, **kw):
    """Seeded synthetic workloads, cached per process."""
    from paper_2303_16878_gb300 import synth
    key = (name, tuple(sorted(kw.items())))
    if key not in _CACHE:
        fn = {"room": synth.make_rgbd_room, "street": synth.make_lidar_street,
              "plane": synth.make_plane_shift, "fusion": synth.make_fusion_room}[name]
        _CACHE[key] = fn(**kw)
    return _CACHE[key]


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def room3():
    return workload("room", n_frames=3)


@pytest.fixture(scope="session")
def room8():
    return workload("room")


@pytest.fixture(scope="session")
def room8x(room8):
    """The RGB-D room with the camera mounted at a 2 cm / 0.5 deg offset."""
    from paper_2303_16878_gb300 import synth
    return synth.with_extrinsic(room8, synth.offset_transform(0.02, 0.5, seed=3005))


@pytest.fixture(scope="session")
def street3():
    return workload("street", n_frames=3, width=256, height=32)


@pytest.fixture(scope="session")
def fusion():
    """RGB-D camera + LiDAR on one platform in the room, 4 platform poses, coupled."""
    return workload("fusion")
