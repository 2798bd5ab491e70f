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
    assert ctypes.sizeof(_lib.PbaIterStats) == 4 * 8 + 8 + 8
