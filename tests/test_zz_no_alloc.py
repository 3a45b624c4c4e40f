"""The allocation-free spectral forward (fno_spectral_fwd_static).

Some callers cannot allocate device memory for a workspace (a host program whose
pool owns all device memory, or a runtime that forbids allocation after start-up).
fno_spectral_fwd_static serves them from a fixed 16 MiB device array inside the
library.  These tests call it through the C ABI, twice in a row on different
inputs and sizes, and compare each result with the workspace-taking
fno_spectral_fwd on the same inputs, within the FP32 tolerance used elsewhere
(rel-L2 <= 1e-5).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2211_12709_gb300 import _lib, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _relerr(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm().clamp_min(1e-300))


def _case(B, Ci, Co, grid, m, seed):
    d = _lib.make_dims(B, Ci, Co, *grid, *m)
    modes = (2 * m[0], 2 * m[1], 2 * m[2], m[3])
    x = torch.from_numpy(inputs.normal((B, Ci) + tuple(grid), seed)).cuda()
    w = torch.from_numpy(inputs.spectral_weights(Ci, Co, modes, seed + 1)).cuda()
    return d, x, w


def _with_workspace(d, x, w, Co):
    y = torch.empty((x.shape[0], Co) + tuple(x.shape[2:]), device="cuda")
    n = _lib.fno_workspace_bytes(d, _lib.FNO_FP32, _lib.FNO_OP_SPECTRAL_FWD)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    _lib.fno_spectral_fwd(d, _lib.FNO_FP32, x.data_ptr(), w.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), n, s)
    return y


def _static(d, x, w, Co):
    y = torch.full((x.shape[0], Co) + tuple(x.shape[2:]), float("nan"), device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    _lib.fno_spectral_fwd_static(d, _lib.FNO_FP32, x.data_ptr(), w.data_ptr(), y.data_ptr(), s)
    return y


def test_static_scratch_matches_workspace_entry_on_two_calls_in_a_row():
    cases = [
        (2, 6, 5, (16, 12, 16, 8), (4, 3, 4, 4), 71),
        (1, 8, 8, (16, 16, 16, 8), (4, 4, 4, 4), 72),
    ]
    for B, Ci, Co, grid, m, seed in cases:
        d, x, w = _case(B, Ci, Co, grid, m, seed)
        need = _lib.fno_workspace_bytes(d, _lib.FNO_FP32, _lib.FNO_OP_SPECTRAL_FWD)
        assert need <= _lib.FNO_STATIC_SCRATCH_BYTES
        got = _static(d, x, w, Co)
        ref = _with_workspace(d, x, w, Co)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        err = _relerr(got, ref)
        assert err <= TOL, (grid, err)


def test_static_scratch_refuses_sizes_beyond_its_limit():
    d = _lib.make_dims(2, 20, 20, 64, 64, 64, 16, 8, 8, 8, 6)
    need = _lib.fno_workspace_bytes(d, _lib.FNO_FP32, _lib.FNO_OP_SPECTRAL_FWD)
    assert need > _lib.FNO_STATIC_SCRATCH_BYTES
    lib = _lib.load()
    rc = lib.fno_spectral_fwd_static(ctypes.byref(d), _lib.FNO_FP32, 256, 256, 256, None)
    assert rc == -2
    assert "static scratch" in _lib.fno_last_error()
