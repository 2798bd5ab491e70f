"""Argument marshalling of the Python binding, checked on the CPU against a
recording stand-in for libpba (no GPU, no library call reaches the device)."""
import ctypes

import numpy as np
import pytest


class _Recorder:
    """Records pba_set_poses calls: the pointer's 12 N doubles and is_device."""

    def __init__(self, n):
        self.n, self.calls = n, []

    def pba_set_poses(self, h, ptr, is_device):
        addr = ptr.value if isinstance(ptr, ctypes.c_void_p) else ptr
        vals = np.ctypeslib.as_array((ctypes.c_double * (12 * self.n)).from_address(addr)).copy()
        self.calls.append((vals, is_device))
        return 0

    def pba_last_error(self, h):
        return b""


def _problem(n):
    import paper_2303_16878_gb300 as pba
    p = object.__new__(pba.Problem)
    p._lib, p._h, p.n_frames = _Recorder(n), ctypes.c_void_p(), n
    return p


def test_set_poses_marshals_every_accepted_form():
    torch = pytest.importorskip("torch")
    n = 3
    X = np.random.default_rng(0).normal(size=(n, 3, 4))
    p = _problem(n)
    forms = [X, X.reshape(n, 12), X.astype(np.float32), torch.from_numpy(X), torch.from_numpy(X).float(),
             torch.from_numpy(X.transpose(0, 2, 1).copy()).transpose(1, 2)]   # non-contiguous view
    for f in forms:
        p.set_poses(f)
        vals, is_device = p._lib.calls[-1]
        tol = 1e-6 if str(getattr(f, "dtype", "")) in ("float32", "torch.float32") else 0.0
        assert is_device == 0 and np.abs(vals - X.reshape(-1)).max() <= tol


def test_set_poses_rejects_the_wrong_size():
    torch = pytest.importorskip("torch")
    p = _problem(3)
    for bad in (np.zeros((2, 3, 4)), torch.zeros(3, 3, 3, dtype=torch.float64), np.zeros(35)):
        with pytest.raises(ValueError):
            p.set_poses(bad)
    assert p._lib.calls == []
