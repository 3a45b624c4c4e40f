"""The allocation-free spectral forward (fno_spectral_fwd_static).

Some callers cannot allocate device memory for a workspace: a host program whose
own pool has reserved all device memory up front, or a runtime that forbids any
allocation once it has started.  fno_spectral_fwd_static serves them from a
fixed 16 MiB device array inside the library.  These tests call it through the C
ABI, twice in a row on different inputs and sizes, in the FP32 plain form and in
the tensor-core precisions (split BF16, TF32), and compare each result with the
workspace-taking fno_spectral_fwd on the same inputs (rel-L2 <= 1e-5; the two run
the same kernels).  After every call the status word in the static array is read
back through fno_static_status, and once fno_static_prepare has loaded the
library's device code, repeated calls leave the free device memory unchanged.
This file is collected last on purpose.
"""
import ctypes

import pytest

from paper_2211_12709_gb300 import _lib, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5
CASES = [
    (2, 6, 5, (16, 12, 16, 8), (4, 3, 4, 4), 71),
    (1, 8, 8, (16, 16, 16, 8), (4, 4, 4, 4), 72),
    # Nt = 32, Nz = 16: the tcgen05 epilogue's tiling (spectral-only mode)
    (1, 6, 8, (12, 10, 16, 32), (3, 4, 4, 8), 73),
]
PRECISIONS = {"fp32": _lib.FNO_FP32, "bf16x3": _lib.FNO_BF16X3, "tf32": _lib.FNO_TF32}


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


def _with_workspace(d, prec, x, w, Co):
    y = torch.empty((x.shape[0], Co) + tuple(x.shape[2:]), device="cuda")
    n = _lib.fno_workspace_bytes(d, prec, _lib.FNO_OP_SPECTRAL_FWD)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    _lib.fno_spectral_fwd(d, prec, x.data_ptr(), w.data_ptr(), y.data_ptr(), ws.data_ptr(), n, s)
    _lib.fno_workspace_status(ws.data_ptr(), s)
    return y


def _static_into(d, prec, x, w, y):
    s = torch.cuda.current_stream().cuda_stream
    _lib.fno_spectral_fwd_static(d, prec, x.data_ptr(), w.data_ptr(), y.data_ptr(), s)
    _lib.fno_static_status(s)  # raises on a timed-out wait or a refused launch


@pytest.mark.parametrize("prec_name", sorted(PRECISIONS))
def test_static_scratch_matches_workspace_entry_on_two_calls_in_a_row(prec_name):
    prec = PRECISIONS[prec_name]
    for B, Ci, Co, grid, m, seed in CASES:
        d, x, w = _case(B, Ci, Co, grid, m, seed)
        need = _lib.fno_workspace_bytes(d, prec, _lib.FNO_OP_SPECTRAL_FWD)
        assert need <= _lib.FNO_STATIC_SCRATCH_BYTES
        got = torch.full((B, Co) + tuple(grid), float("nan"), device="cuda")
        _static_into(d, prec, x, w, got)
        ref = _with_workspace(d, prec, x, w, Co)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        err = _relerr(got, ref)
        assert err <= TOL, (prec_name, grid, err)


def test_static_calls_allocate_nothing_once_prepared():
    _lib.fno_static_prepare()
    B, Ci, Co, grid, m, seed = CASES[2]
    d, x, w = _case(B, Ci, Co, grid, m, seed)
    y = torch.empty((B, Co) + tuple(grid), device="cuda")
    # one call per precision loads every kernel the later calls use
    for prec in PRECISIONS.values():
        _static_into(d, prec, x, w, y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for prec in PRECISIONS.values():
            _static_into(d, prec, x, w, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_refuses_sizes_beyond_its_limit():
    d = _lib.make_dims(2, 20, 20, 64, 64, 64, 16, 8, 8, 8, 6)
    need = _lib.fno_workspace_bytes(d, _lib.FNO_FP32, _lib.FNO_OP_SPECTRAL_FWD)
    assert need > _lib.FNO_STATIC_SCRATCH_BYTES
    lib = _lib.load()
    rc = lib.fno_spectral_fwd_static(ctypes.byref(d), _lib.FNO_FP32, 256, 256, 256, None)
    assert rc == -2
    assert "static scratch" in _lib.fno_last_error()
