"""Host-side checks of libfno that need no GPU: the library loads, exports every
symbol include/fno.h declares, and rejects bad arguments before any launch."""
import ctypes
import os
import re

import pytest

from paper_2211_12709_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fno.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(fno_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_documented_entry_points():
    names = declared_symbols()
    for n in ("fno_spectral_fwd", "fno_spectral_bwd", "fno_block_fwd", "fno_block_bwd",
              "fno_workspace_bytes", "fno_last_error"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    lib = _lib.load()
    for n in declared_symbols():
        assert hasattr(lib, n), n
    assert set(declared_symbols()) <= set(_lib.EXPORTS) | {"fno_version"}
    assert _lib.fno_version() >= 100


def raw_ws(d, p, op):
    return _lib.load().fno_workspace_bytes(ctypes.byref(d), p, op)


def C1():
    return _lib.make_dims(1, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4)


def test_workspace_query_is_deterministic_and_grows_with_batch():
    a = _lib.fno_workspace_bytes(C1(), _lib.FNO_FP32, _lib.FNO_OP_BLOCK_BWD)
    b = _lib.fno_workspace_bytes(C1(), _lib.FNO_FP32, _lib.FNO_OP_BLOCK_BWD)
    assert a == b and a > 0 and a % 256 == 0
    d2 = C1()
    d2.B = 4
    assert _lib.fno_workspace_bytes(d2, _lib.FNO_FP32, _lib.FNO_OP_BLOCK_BWD) > a
    f = _lib.fno_workspace_bytes(C1(), _lib.FNO_FP32, _lib.FNO_OP_SPECTRAL_FWD)
    assert 0 < f < a


@pytest.mark.parametrize("field,value", [("Nx", 0), ("C_in", 0), ("mx", 9), ("mt", 6), ("B", -1),
                                         ("mz", 0)])
def test_invalid_dims_are_rejected_on_the_host(field, value):
    d = C1()
    setattr(d, field, value)
    assert raw_ws(d, _lib.FNO_FP32, _lib.FNO_OP_BLOCK_FWD) == 0
    lib = _lib.load()
    rc = lib.fno_block_fwd(ctypes.byref(d), 0, None, None, None, None, None, None, 0, None)
    assert rc == -1
    assert _lib.fno_last_error()


def test_null_and_misaligned_pointers_and_small_workspace_are_rejected():
    lib = _lib.load()
    d = C1()
    need = _lib.fno_workspace_bytes(d, 0, _lib.FNO_OP_BLOCK_FWD)
    # workspace too small: refused before touching any pointer
    rc = lib.fno_block_fwd(ctypes.byref(d), 0, 256, 256, 256, 256, 256, 256, need - 256, None)
    assert rc == -3
    # misaligned workspace
    rc = lib.fno_block_fwd(ctypes.byref(d), 0, 256, 256, 256, 256, 256, 257, need, None)
    assert rc == -3
    # null weights
    rc = lib.fno_block_fwd(ctypes.byref(d), 0, 256, None, 256, 256, 256, 256, need, None)
    assert rc == -1 and "w is NULL" in _lib.fno_last_error()
    # misaligned x
    rc = lib.fno_block_fwd(ctypes.byref(d), 0, 260, 256, 256, 256, 256, 256, need, None)
    assert rc == -1 and "aligned" in _lib.fno_last_error()
    # spectral backward needs at least one output
    need_b = _lib.fno_workspace_bytes(d, 0, _lib.FNO_OP_SPECTRAL_BWD)
    rc = lib.fno_spectral_bwd(ctypes.byref(d), 0, 256, 256, 256, None, None, 256, need_b, None)
    assert rc == -1


def test_bad_precision_and_op_codes():
    assert raw_ws(C1(), 7, _lib.FNO_OP_BLOCK_FWD) == 0
    assert raw_ws(C1(), 0, 9) == 0
    lib = _lib.load()
    rc = lib.fno_block_fwd(ctypes.byref(C1()), 7, 256, 256, 256, 256, 256, 256, 1 << 30, None)
    assert rc == -1


def test_too_many_channels_is_unsupported_not_a_crash():
    d = C1()
    d.C_in = 65
    assert raw_ws(d, 0, _lib.FNO_OP_BLOCK_FWD) == 0
    assert "<=" in _lib.fno_last_error()


def test_training_workspace_is_the_backward_one_plus_gelu_derivative():
    d = C1()
    bwd = _lib.fno_workspace_bytes(d, 0, _lib.FNO_OP_BLOCK_BWD)
    train = _lib.fno_workspace_bytes(d, 0, _lib.FNO_OP_BLOCK_TRAIN)
    n = d.B * d.C_out * d.Nx * d.Ny * d.Nz * d.Nt
    assert train == bwd + (4 * n + 255) // 256 * 256
    lib = _lib.load()
    # a backward-sized workspace is refused before any pointer is touched
    rc = lib.fno_block_fwd_train(ctypes.byref(d), 0, 256, 256, 256, 256, 256, 256, bwd, None)
    assert rc == -3 and str(train) in _lib.fno_last_error()
    assert raw_ws(d, 0, 5) == 0  # no op 5


def test_more_than_16_t_modes_is_unsupported_not_wrong():
    # the epilogues keep the inverse-t factors of at most 16 modes in registers
    d = C1()
    d.Nt, d.mt = 40, 17
    assert raw_ws(d, 0, _lib.FNO_OP_BLOCK_FWD) == 0
    assert "mt = 17" in _lib.fno_last_error()
    d.mt = 16
    assert raw_ws(d, 0, _lib.FNO_OP_BLOCK_FWD) > 0


def test_pointwise_and_loss_arguments_are_checked_on_the_host():
    lib = _lib.load()
    d = _lib.make_pw_dims(1, 3, 20, 4096)
    need = _lib.fno_pointwise_workspace_bytes(d)
    assert need > 0 and need % 256 == 0
    # channel counts outside 1..64
    for ci, co in ((0, 4), (4, 0), (65, 4), (4, 65)):
        bad = _lib.make_pw_dims(1, ci, co, 16)
        assert lib.fno_pointwise_workspace_bytes(ctypes.byref(bad)) == 0
        assert lib.fno_pointwise_fwd(ctypes.byref(bad), 1, 256, 256, None, 256, None) == -1
    # negative sizes
    assert lib.fno_pointwise_fwd(ctypes.byref(_lib.make_pw_dims(-1, 3, 4, 16)), 1, 256, 256, None,
                                 256, None) == -1
    assert lib.fno_pointwise_fwd(ctypes.byref(_lib.make_pw_dims(1, 3, 4, -16)), 1, 256, 256,
                                 None, 256, None) == -1
    # unknown activation, null weight, misaligned x
    assert lib.fno_pointwise_fwd(ctypes.byref(d), 2, 256, 256, None, 256, None) == -1
    assert lib.fno_pointwise_fwd(ctypes.byref(d), 1, 256, None, None, 256, None) == -1
    assert "w is NULL" in _lib.fno_last_error()
    assert lib.fno_pointwise_fwd(ctypes.byref(d), 1, 258, 256, None, 256, None) == -1
    # an empty input needs no launch and succeeds without a GPU
    assert lib.fno_pointwise_fwd(ctypes.byref(_lib.make_pw_dims(0, 3, 4, 16)), 1, None, 256,
                                 None, None, None) == 0
    # backward: workspace too small or misaligned, null dw
    assert lib.fno_pointwise_bwd(ctypes.byref(d), 1, 256, 256, None, 256, None, 256, None, 256,
                                 need - 256, None) == -3
    assert lib.fno_pointwise_bwd(ctypes.byref(d), 1, 256, 256, None, 256, None, 256, None, 512 + 4,
                                 need, None) == -3
    assert lib.fno_pointwise_bwd(ctypes.byref(d), 1, 256, 256, None, 256, None, None, None, 256,
                                 need, None) == -1
    # loss: n >= 1, required pointers, workspace size
    assert lib.fno_mse_workspace_bytes(0) == 0
    nm = _lib.fno_mse_workspace_bytes(1000)
    assert lib.fno_mse_loss(0, 256, 256, 256, None, 256, nm, None) == -1
    assert lib.fno_mse_loss(1000, None, 256, 256, None, 256, nm, None) == -1
    assert lib.fno_mse_loss(1000, 256, 256, None, None, 256, nm, None) == -1
    assert lib.fno_mse_loss(1000, 256, 256, 256, None, 256, nm - 256, None) == -3


def test_saved_backward_without_a_recorded_forward_is_refused():
    lib = _lib.load()
    d = C1()
    need = _lib.fno_workspace_bytes(d, 0, _lib.FNO_OP_BLOCK_BWD)
    rc = lib.fno_block_bwd_saved(ctypes.byref(d), 0, 256, 256, 256, 256, 256, 512, 256, 256, 256,
                                 1024, need, None)
    assert rc == -1 and "fno_block_fwd" in _lib.fno_last_error()


def test_adam_arguments_are_checked_on_the_host():
    lib = _lib.load()
    ok = (256, 256, 256, 256)
    assert lib.fno_adam_step(16, *ok, 1e-3, 0.9, 0.999, 1e-8, 0, None) == -1   # step 0
    assert lib.fno_adam_step(16, *ok, 1e-3, 1.0, 0.999, 1e-8, 1, None) == -1   # beta1 = 1
    assert lib.fno_adam_step(16, *ok, 1e-3, 0.9, 0.999, 0.0, 1, None) == -1    # eps = 0
    assert lib.fno_adam_step(16, *ok, -1.0, 0.9, 0.999, 1e-8, 1, None) == -1   # lr < 0
    assert lib.fno_adam_step(16, None, 256, 256, 256, 1e-3, 0.9, 0.999, 1e-8, 1, None) == -1
    assert lib.fno_adam_step(0, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == 0


def test_workspace_holds_the_synthesis_region_only_outside_the_fused_tiling():
    # Nt = 32 is tiled by the fused epilogues; Nt = 30 takes the synthesis path,
    # whose inverse z stage needs B * C * Nx * Ny * Nz * mt complex64 values
    def ws(nt):
        d = _lib.make_dims(1, 8, 8, 16, 16, 32, nt, 4, 4, 4, 8)
        return _lib.fno_workspace_bytes(d, _lib.FNO_BF16X3, _lib.FNO_OP_SPECTRAL_FWD)
    v = 8 * 1 * 8 * 16 * 16 * 32 * 8
    diff = ws(30) - ws(32)
    # the t tables (Jt x Nt) and the fused epilogues' basis tables differ by a few KB
    assert abs(diff - v) < (1 << 20), (diff, v)
