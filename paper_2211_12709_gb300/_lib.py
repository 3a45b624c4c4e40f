"""ctypes binding of libfno.so: the C ABI of include/fno.h with the same names.

Argument marshalling only.  Every pointer argument is a plain integer address
(device memory for tensors, any host address for ``dims``); ``stream`` is a
cudaStream_t handle as an integer (0 = legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

FNO_FP32, FNO_TF32, FNO_BF16, FNO_BF16X3 = 0, 1, 2, 3
FNO_OP_SPECTRAL_FWD, FNO_OP_SPECTRAL_BWD, FNO_OP_BLOCK_FWD, FNO_OP_BLOCK_BWD = 0, 1, 2, 3
FNO_OP_BLOCK_TRAIN = 4
FNO_OK = 0
STATUS_NAMES = {0: "FNO_OK", -1: "FNO_ERR_INVALID_ARG", -2: "FNO_ERR_UNSUPPORTED",
                -3: "FNO_ERR_WORKSPACE", -4: "FNO_ERR_CUDA", -5: "FNO_ERR_TIMEOUT"}
PRECISIONS = {"fp32": FNO_FP32, "tf32": FNO_TF32, "bf16": FNO_BF16, "bf16x3": FNO_BF16X3}

EXPORTS = (
    "fno_workspace_bytes", "fno_spectral_fwd", "fno_spectral_bwd", "fno_block_fwd",
    "fno_block_bwd", "fno_last_error", "fno_version", "fno_launch_count", "fno_profile_start",
    "fno_profile_stop", "fno_profile_count", "fno_profile_entry", "fno_spectral_fwd_static", "fno_workspace_status", "fno_last_status",
    "fno_pointwise_fwd", "fno_pointwise_workspace_bytes", "fno_pointwise_bwd",
    "fno_mse_workspace_bytes", "fno_mse_loss", "fno_block_bwd_saved", "fno_adam_step",
    "fno_block_fwd_train", "fno_static_prepare", "fno_static_status",
)
FNO_ACT_NONE, FNO_ACT_GELU = 0, 1
FNO_STATIC_SCRATCH_BYTES = 16 << 20


class fno_dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("B", "C_in", "C_out", "Nx", "Ny", "Nz", "Nt", "mx", "my", "mz", "mt")]


class fno_pw_dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("B", "C_in", "C_out", "P")]


class FnoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libfno.so (compiling it in-tree first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libfno.so not found at {_build.LIB}; run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        vp, sz, ci, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int64
        dp = ctypes.POINTER(fno_dims)
        lib.fno_workspace_bytes.argtypes = [dp, ci, ci]
        lib.fno_workspace_bytes.restype = sz
        lib.fno_spectral_fwd.argtypes = [dp, ci, vp, vp, vp, vp, sz, vp]
        lib.fno_spectral_bwd.argtypes = [dp, ci, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_block_fwd.argtypes = [dp, ci, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_block_fwd_train.argtypes = [dp, ci, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_spectral_fwd_static.argtypes = [dp, ci, vp, vp, vp, vp]
        lib.fno_spectral_fwd_static.restype = ci
        lib.fno_static_prepare.argtypes = []
        lib.fno_static_prepare.restype = ci
        lib.fno_static_status.argtypes = [vp]
        lib.fno_static_status.restype = ci
        lib.fno_block_bwd.argtypes = [dp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_block_bwd_saved.argtypes = [dp, ci, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        for f in (lib.fno_spectral_fwd, lib.fno_spectral_bwd, lib.fno_block_fwd, lib.fno_block_bwd,
                  lib.fno_block_bwd_saved, lib.fno_block_fwd_train):
            f.restype = ci
        lib.fno_workspace_status.argtypes = [vp, vp]
        lib.fno_workspace_status.restype = ci
        lib.fno_last_status.argtypes = []
        lib.fno_last_status.restype = ci
        lib.fno_last_error.argtypes = []
        lib.fno_last_error.restype = ctypes.c_char_p
        lib.fno_version.restype = ci
        lib.fno_launch_count.restype = i64
        lib.fno_profile_start.restype = ci
        lib.fno_profile_stop.restype = ci
        lib.fno_profile_count.restype = ci
        lib.fno_profile_entry.argtypes = [ci, ctypes.POINTER(ctypes.c_char_p),
                                          ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
        lib.fno_profile_entry.restype = ci
        pp = ctypes.POINTER(fno_pw_dims)
        lib.fno_pointwise_fwd.argtypes = [pp, ci, vp, vp, vp, vp, vp]
        lib.fno_pointwise_fwd.restype = ci
        lib.fno_pointwise_workspace_bytes.argtypes = [pp]
        lib.fno_pointwise_workspace_bytes.restype = sz
        lib.fno_pointwise_bwd.argtypes = [pp, ci, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_pointwise_bwd.restype = ci
        lib.fno_mse_workspace_bytes.argtypes = [i64]
        lib.fno_mse_workspace_bytes.restype = sz
        lib.fno_mse_loss.argtypes = [i64, vp, vp, vp, vp, vp, sz, vp]
        lib.fno_mse_loss.restype = ci
        fl = ctypes.c_float
        lib.fno_adam_step.argtypes = [i64, vp, vp, vp, vp, fl, fl, fl, fl, i64, vp]
        lib.fno_adam_step.restype = ci
        _lib = lib
        return lib


def make_dims(B, C_in, C_out, Nx, Ny, Nz, Nt, mx, my, mz, mt) -> fno_dims:
    return fno_dims(int(B), int(C_in), int(C_out), int(Nx), int(Ny), int(Nz), int(Nt),
                    int(mx), int(my), int(mz), int(mt))


def _check(rc: int):
    if rc != FNO_OK:
        msg = load().fno_last_error()
        raise FnoError(rc, msg.decode() if msg else "")


def fno_last_error() -> str:
    m = load().fno_last_error()
    return m.decode() if m else ""


def fno_workspace_bytes(dims: fno_dims, precision: int, op: int) -> int:
    lib = load()
    n = lib.fno_workspace_bytes(ctypes.byref(dims), int(precision), int(op))
    if n == 0:
        raise FnoError(int(lib.fno_last_status()), fno_last_error())
    return int(n)


def fno_spectral_fwd(dims, precision, x, w, y, ws, ws_bytes, stream=0):
    _check(load().fno_spectral_fwd(ctypes.byref(dims), int(precision), x, w, y, ws, ws_bytes,
                                   stream))


def fno_spectral_fwd_static(dims, precision, x, w, y, stream=0):
    """fno_spectral_fwd with the library's static device scratch (no workspace argument)."""
    _check(load().fno_spectral_fwd_static(ctypes.byref(dims), int(precision), x, w, y, stream))


def fno_static_prepare():
    """Load the library's device code on the current device (commits the static scratch)."""
    _check(load().fno_static_prepare())


def fno_static_status(stream=0):
    """Raise FnoError if the last fno_spectral_fwd_static call left an error status."""
    _check(load().fno_static_status(stream))


def fno_spectral_bwd(dims, precision, x, w, dy, dx, dw, ws, ws_bytes, stream=0):
    _check(load().fno_spectral_bwd(ctypes.byref(dims), int(precision), x, w, dy, dx, dw, ws,
                                   ws_bytes, stream))


def fno_block_fwd(dims, precision, x, w, w_lin, bias, z, ws, ws_bytes, stream=0):
    _check(load().fno_block_fwd(ctypes.byref(dims), int(precision), x, w, w_lin, bias, z, ws,
                                ws_bytes, stream))


def fno_block_fwd_train(dims, precision, x, w, w_lin, bias, z, ws, ws_bytes, stream=0):
    """fno_block_fwd that also keeps GELU'(A) in ws (sized for FNO_OP_BLOCK_TRAIN)."""
    _check(load().fno_block_fwd_train(ctypes.byref(dims), int(precision), x, w, w_lin, bias, z,
                                      ws, ws_bytes, stream))


def fno_block_bwd(dims, precision, x, w, w_lin, bias, dz, dx, dw, dw_lin, db, ws, ws_bytes,
                  stream=0):
    _check(load().fno_block_bwd(ctypes.byref(dims), int(precision), x, w, w_lin, bias, dz, dx, dw,
                                dw_lin, db, ws, ws_bytes, stream))


def fno_block_bwd_saved(dims, precision, x, w, w_lin, bias, dz, dx, dw, dw_lin, db, ws, ws_bytes,
                        stream=0):
    """fno_block_bwd reusing the state the last fno_block_fwd(_train) left in ws."""
    _check(load().fno_block_bwd_saved(ctypes.byref(dims), int(precision), x, w, w_lin, bias, dz,
                                      dx, dw, dw_lin, db, ws, ws_bytes, stream))


def fno_workspace_status(ws, stream=0):
    """Raise FnoError(FNO_ERR_TIMEOUT) if the call that used ws hit a bounded-wait timeout."""
    _check(load().fno_workspace_status(ws, stream))


def fno_version() -> int:
    return int(load().fno_version())


def fno_launch_count() -> int:
    return int(load().fno_launch_count())


def fno_profile_start():
    _check(load().fno_profile_start())


def fno_profile_stop():
    """Stop timing and return {kernel name: (launches, total_ms)}."""
    lib = load()
    _check(lib.fno_profile_stop())
    out = {}
    for i in range(lib.fno_profile_count()):
        name = ctypes.c_char_p()
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(lib.fno_profile_entry(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)))
        out[name.value.decode()] = (int(n.value), float(ms.value))
    return out


def make_pw_dims(B, C_in, C_out, P) -> fno_pw_dims:
    return fno_pw_dims(int(B), int(C_in), int(C_out), int(P))


def fno_pointwise_fwd(dims, act, x, w, bias, y, stream=0):
    _check(load().fno_pointwise_fwd(ctypes.byref(dims), int(act), x, w, bias, y, stream))


def fno_pointwise_workspace_bytes(dims) -> int:
    lib = load()
    n = lib.fno_pointwise_workspace_bytes(ctypes.byref(dims))
    if n == 0:
        raise FnoError(int(lib.fno_last_status()), fno_last_error())
    return int(n)


def fno_pointwise_bwd(dims, act, x, w, bias, dy, dx, dw, db, ws, ws_bytes, stream=0):
    _check(load().fno_pointwise_bwd(ctypes.byref(dims), int(act), x, w, bias, dy, dx, dw, db, ws,
                                    ws_bytes, stream))


def fno_mse_workspace_bytes(n: int) -> int:
    lib = load()
    r = lib.fno_mse_workspace_bytes(int(n))
    if r == 0:
        raise FnoError(int(lib.fno_last_status()), fno_last_error())
    return int(r)


def fno_mse_loss(n, y, target, loss, dy, ws, ws_bytes, stream=0):
    _check(load().fno_mse_loss(int(n), y, target, loss, dy, ws, ws_bytes, stream))


def fno_adam_step(n, param, grad, m, v, lr, beta1, beta2, eps, step, stream=0):
    _check(load().fno_adam_step(int(n), param, grad, m, v, float(lr), float(beta1), float(beta2),
                                float(eps), int(step), stream))
