"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/pba.h declares (CPU only: no call that needs a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pba.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pba_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_surface():
    from paper_2303_16878_gb300 import _lib
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2303_16878_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_declares_argument_types_without_touching_the_gpu():
    from paper_2303_16878_gb300 import _lib
    lib = _lib.load()
    for name in _lib.EXPORTS:
        assert getattr(lib, name).argtypes is not None
    # no-GPU-safe calls: argument validation happens before any CUDA call, and a
    # failed create leaves its reason for pba_last_error(NULL) on this thread
    assert lib.pba_create(None, None, None) == _lib.PBA_EINVAL
    assert lib.pba_last_error(None).startswith(b"pba_create: null configuration")


def test_without_a_gpu_creation_fails_loudly():
    """The library has no CPU path: on a machine without a CUDA device,
    creating a problem raises with the CUDA runtime's reason."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2303_16878_gb300 as pba
    from paper_2303_16878_gb300 import synth
    w = synth.make_rgbd_room(n_frames=2, width=32, height=24, f=24.0)
    with pytest.raises(pba.PbaError) as err:
        pba.problem_from_workload(w)
    assert err.value.code == pba._lib.PBA_ECUDA
    assert "no usable CUDA device" in str(err.value) and "no CPU path" in str(err.value)


def test_struct_layouts_match_the_header():
    from paper_2303_16878_gb300 import _lib
    # sizes implied by include/pba.h on LP64 (4 x int32 + 16 doubles, ...)
    assert ctypes.sizeof(_lib.PbaSensor) == 16 + 8 * 16
    assert ctypes.sizeof(_lib.PbaConfig) == 8 + 8 + 8 + 9 * 8 + 16
    assert ctypes.sizeof(_lib.PbaIterStats) == 4 * 8 + 8 + 8 + 2 * 8
    assert ctypes.sizeof(_lib.PbaTuning) == 6 * 4 + 2 * 4 + 4
    assert _lib.PbaTuning.reduction.offset == 32


def _config(_lib, sensors, n_frames=2, frame_sensor=None, **over):
    cfg = _lib.PbaConfig()
    cfg.n_frames, cfg.n_sensors = n_frames, len(sensors)
    arr = (_lib.PbaSensor * len(sensors))(*sensors)
    cfg.sensors = ctypes.cast(arr, ctypes.POINTER(_lib.PbaSensor))
    keep = [arr]
    if frame_sensor is not None:
        fs = (ctypes.c_int32 * len(frame_sensor))(*frame_sensor)
        cfg.frame_sensor = ctypes.cast(fs, ctypes.POINTER(ctypes.c_int32))
        keep.append(fs)
    cfg.w_int = cfg.w_depth = cfg.w_normal = 1.0
    cfg.huber_delta, cfg.occ_abs, cfg.occ_rel, cfg.z_min = 0.1, 0.1, 0.05, 0.05
    cfg.range_min, cfg.range_max = 0.0, 1e30
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg, keep


def _sensor(_lib, **over):
    s = _lib.PbaSensor()
    s.model, s.width, s.height = _lib.PBA_PINHOLE, 64, 48
    s.fx = s.fy = 48.0
    s.cx, s.cy = 32.0, 24.0
    for e, v in enumerate((1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0)):
        s.extrinsic[e] = v
    for k, v in over.items():
        setattr(s, k, v)
    return s


def test_create_rejects_bad_configurations_before_touching_the_gpu():
    """Every configuration check of pba_create runs before any CUDA call:
    each bad field gives PBA_EINVAL and names itself in pba_last_error(NULL)."""
    from paper_2303_16878_gb300 import _lib
    lib = _lib.load()
    good = _sensor(_lib)
    cases = [
        (dict(n_frames=0), [good], None, b"n_frames"),
        (dict(huber_delta=0.0), [good], None, b"huber_delta"),
        (dict(huber_delta=float("nan")), [good], None, b"huber_delta"),
        (dict(grad_mode=2), [good], None, b"grad_mode"),
        (dict(texel_precision=5), [good], None, b"texel_precision"),
        (dict(path=7), [good], None, b"path"),
        (dict(solver=9), [good], None, b"solver"),
        ({}, [_sensor(_lib, model=3)], None, b"sensor 0"),
        ({}, [_sensor(_lib, width=3)], None, b"sensor 0"),
        ({}, [good, _sensor(_lib, fx=0.0)], None, b"sensor 1: zero focal length"),
        ({}, [_sensor(_lib, width=1 << 16, height=1 << 15)], None, b"2^30 pixels"),
        ({}, [good], [0, 1], b"frame_sensor[1] out of range"),
        ({}, [good, good], [-1, 0], b"frame_sensor[0] out of range"),
    ]
    for over, sensors, fs, needle in cases:
        n_frames = over.pop("n_frames", 2)
        cfg, keep = _config(_lib, sensors, n_frames=n_frames, frame_sensor=fs, **over)
        h = ctypes.c_void_p()
        assert lib.pba_create(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.PBA_EINVAL, needle
        assert not h.value
        msg = lib.pba_last_error(None)
        assert msg.startswith(b"pba_create: ") and needle in msg, (needle, msg)


def test_header_compiles_as_c99_and_links(tmp_path):
    """include/pba.h is plain C: a C99 program includes it, links libpba.so and
    calls the entry points that need no GPU."""
    import shutil
    import subprocess
    import pytest
    from paper_2303_16878_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "pba.h"
int main(void) {
    pba_problem* p = NULL;
    pba_config cfg;
    memset(&cfg, 0, sizeof cfg);
    if (pba_create(NULL, NULL, &p) != PBA_EINVAL) return 1;
    if (strncmp(pba_last_error(NULL), "pba_create: ", 12) != 0) return 2;
    if (pba_create(&cfg, NULL, &p) != PBA_EINVAL || p != NULL) return 3;
    if (pba_set_lambda(NULL, 1.0) != PBA_EINVAL) return 4;
    pba_destroy(NULL);
    if (sizeof(pba_tuning) != 36 || offsetof(pba_tuning, reduction) != 32) return 5;
    printf("%d %d %d %s\n", (int)sizeof(pba_sensor), (int)sizeof(pba_config), (int)sizeof(pba_iter_stats),
           pba_last_error(NULL));
    return 0;
}
""")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lpba", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    size_s, size_c, size_i, msg = r.stdout.split(" ", 3)
    assert (int(size_s), int(size_c), int(size_i)) == (16 + 8 * 16, 8 + 8 + 8 + 9 * 8 + 16, 4 * 8 + 8 + 8 + 2 * 8)
    assert msg.startswith("pba_create: n_frames")
