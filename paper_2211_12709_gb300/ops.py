"""PyTorch-facing wrappers of libfno (marshalling only: every step runs in the CUDA kernels).

Tensors are FP32 CUDA tensors in the layouts of include/fno.h:
  x  [B, C_in, Nx, Ny, Nz, Nt],  w [C_in, C_out, 2mx, 2my, 2mz, mt, 2] (re, im),
  w_lin [C_in, C_out],  bias [C_out].
``modes`` is (mx, my, mz, mt).  PyTorch provides device memory (outputs and the
workspace come from its caching allocator) and the current stream.

``SpectralConv4dFn`` and ``FNOBlock4dFn`` are autograd Functions whose backward
calls the hand-written adjoint kernels.  The block keeps only its input between
the passes (the backward recomputes the forward spectrum: per-block activation
checkpointing), so a stack of blocks holds one activation per block.
"""
from __future__ import annotations

import torch

from . import _lib

OP_SPECTRAL_FWD = _lib.FNO_OP_SPECTRAL_FWD
OP_SPECTRAL_BWD = _lib.FNO_OP_SPECTRAL_BWD
OP_BLOCK_FWD = _lib.FNO_OP_BLOCK_FWD
OP_BLOCK_BWD = _lib.FNO_OP_BLOCK_BWD
OP_BLOCK_TRAIN = _lib.FNO_OP_BLOCK_TRAIN

# When set, every call waits for its stream and raises if a device-side bounded
# wait gave up (FNO_ERR_TIMEOUT).  For tests and debugging; off by default.
CHECK_STATUS = False


def _status(ws, dev):
    if CHECK_STATUS:
        _lib.fno_workspace_status(ws.data_ptr(), _stream_handle(dev))


def precision_code(p) -> int:
    if isinstance(p, int):
        return p
    try:
        return _lib.PRECISIONS[p]
    except KeyError:
        raise ValueError(f"unknown precision {p!r}; one of {sorted(_lib.PRECISIONS)}") from None


def dims_of(x: torch.Tensor, C_out: int, modes) -> _lib.fno_dims:
    if x.dim() != 6:
        raise ValueError(f"x must be [B, C, Nx, Ny, Nz, Nt], got shape {tuple(x.shape)}")
    B, Ci, Nx, Ny, Nz, Nt = (int(v) for v in x.shape)
    mx, my, mz, mt = (int(v) for v in modes)
    return _lib.make_dims(B, Ci, C_out, Nx, Ny, Nz, Nt, mx, my, mz, mt)


def _req(t: torch.Tensor, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor (libfno has no CPU path)")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


def _stream_handle(dev) -> int:
    return int(torch.cuda.current_stream(dev).cuda_stream)


def workspace(dims, precision, op, device) -> torch.Tensor:
    n = _lib.fno_workspace_bytes(dims, precision_code(precision), op)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def _wshape(Ci, Co, modes):
    mx, my, mz, mt = modes
    return (Ci, Co, 2 * mx, 2 * my, 2 * mz, mt, 2)


def spectral_fwd(x, w, modes, precision="fp32", ws=None):
    x = _req(x, "x")
    Ci = x.shape[1]
    Co = w.shape[1]
    w = _req(w, "w", _wshape(Ci, Co, modes))
    d = dims_of(x, Co, modes)
    p = precision_code(precision)
    y = torch.empty((x.shape[0], Co) + tuple(x.shape[2:]), dtype=torch.float32, device=x.device)
    if ws is None:
        ws = workspace(d, p, OP_SPECTRAL_FWD, x.device)
    _lib.fno_spectral_fwd(d, p, x.data_ptr(), w.data_ptr(), y.data_ptr(), ws.data_ptr(),
                          ws.numel(), _stream_handle(x.device))
    _status(ws, x.device)
    return y


def spectral_bwd(x, w, dy, modes, need_dx=True, need_dw=True, precision="fp32", ws=None):
    x = _req(x, "x")
    Ci, Co = x.shape[1], w.shape[1]
    w = _req(w, "w", _wshape(Ci, Co, modes))
    dy = _req(dy, "dy", (x.shape[0], Co) + tuple(x.shape[2:]))
    d = dims_of(x, Co, modes)
    p = precision_code(precision)
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty_like(w) if need_dw else None
    if ws is None:
        ws = workspace(d, p, OP_SPECTRAL_BWD, x.device)
    _lib.fno_spectral_bwd(d, p, x.data_ptr(), w.data_ptr(), dy.data_ptr(),
                          dx.data_ptr() if dx is not None else None,
                          dw.data_ptr() if dw is not None else None,
                          ws.data_ptr(), ws.numel(), _stream_handle(x.device))
    _status(ws, x.device)
    return dx, dw


def block_fwd(x, w, w_lin, bias, modes, precision="fp32", ws=None, train=False):
    """Block forward.  train=True also keeps GELU'(A) in ws (sized for
    OP_BLOCK_TRAIN) for a following block_bwd(..., saved=True)."""
    x = _req(x, "x")
    Ci, Co = x.shape[1], w.shape[1]
    w = _req(w, "w", _wshape(Ci, Co, modes))
    w_lin = _req(w_lin, "w_lin", (Ci, Co))
    bias = _req(bias, "bias", (Co,))
    d = dims_of(x, Co, modes)
    p = precision_code(precision)
    z = torch.empty((x.shape[0], Co) + tuple(x.shape[2:]), dtype=torch.float32, device=x.device)
    if ws is None:
        ws = workspace(d, p, OP_BLOCK_TRAIN if train else OP_BLOCK_FWD, x.device)
    fn = _lib.fno_block_fwd_train if train else _lib.fno_block_fwd
    fn(d, p, x.data_ptr(), w.data_ptr(), w_lin.data_ptr(), bias.data_ptr(), z.data_ptr(),
       ws.data_ptr(), ws.numel(), _stream_handle(x.device))
    _status(ws, x.device)
    return z


def block_bwd(x, w, w_lin, bias, dz, modes, precision="fp32", ws=None, saved=False):
    """Block backward.  saved=True reuses the state the last block_fwd left in ws
    (the workspace of that call, sized for OP_BLOCK_BWD, or OP_BLOCK_TRAIN after a
    training forward) instead of recomputing it."""
    x = _req(x, "x")
    Ci, Co = x.shape[1], w.shape[1]
    w = _req(w, "w", _wshape(Ci, Co, modes))
    w_lin = _req(w_lin, "w_lin", (Ci, Co))
    bias = _req(bias, "bias", (Co,))
    dz = _req(dz, "dz", (x.shape[0], Co) + tuple(x.shape[2:]))
    d = dims_of(x, Co, modes)
    p = precision_code(precision)
    dx = torch.empty_like(x)
    dw = torch.empty_like(w)
    dwl = torch.empty_like(w_lin)
    db = torch.empty_like(bias)
    if ws is None:
        if saved:
            raise ValueError("saved=True needs the workspace of the forward call")
        ws = workspace(d, p, OP_BLOCK_BWD, x.device)
    fn = _lib.fno_block_bwd_saved if saved else _lib.fno_block_bwd
    fn(d, p, x.data_ptr(), w.data_ptr(), w_lin.data_ptr(), bias.data_ptr(), dz.data_ptr(),
       dx.data_ptr(), dw.data_ptr(), dwl.data_ptr(), db.data_ptr(), ws.data_ptr(), ws.numel(),
       _stream_handle(x.device))
    _status(ws, x.device)
    return dx, dw, dwl, db


class SpectralConv4dFn(torch.autograd.Function):
    """y = S(x; w): truncated DFT, per-mode complex mixing, inverse DFT (Alg. 2)."""

    @staticmethod
    def forward(ctx, x, w, modes, precision="fp32"):
        ctx.modes = tuple(int(m) for m in modes)
        ctx.precision = precision
        ctx.save_for_backward(x, w)
        return spectral_fwd(x, w, ctx.modes, precision)

    @staticmethod
    def backward(ctx, dy):
        x, w = ctx.saved_tensors
        dx, dw = spectral_bwd(x, w, dy.contiguous(), ctx.modes, ctx.needs_input_grad[0],
                              ctx.needs_input_grad[1] or not ctx.needs_input_grad[0],
                              ctx.precision)
        return dx, (dw if ctx.needs_input_grad[1] else None), None, None


class FNOBlock4dFn(torch.autograd.Function):
    """z = GELU(S(x; w) + w_lin^T x + bias).

    Between the passes the block keeps its input and the forward's workspace,
    which holds the truncated spectra (X̂ and the inverse x, y partial U1, a
    small fraction of x) and GELU'(A) (one output-sized tensor); the backward
    reuses them.  A second backward through the same graph finds the workspace
    spent and recomputes the spectra.
    """

    @staticmethod
    def forward(ctx, x, w, w_lin, bias, modes, precision="fp32"):
        ctx.modes = tuple(int(m) for m in modes)
        ctx.precision = precision
        ctx.save_for_backward(x, w, w_lin, bias)
        x = _req(x, "x")
        d = dims_of(x, int(w.shape[1]), ctx.modes)
        ctx.ws = workspace(d, precision, OP_BLOCK_TRAIN, x.device)
        return block_fwd(x, w, w_lin, bias, ctx.modes, precision, ws=ctx.ws, train=True)

    @staticmethod
    def backward(ctx, dz):
        x, w, w_lin, bias = ctx.saved_tensors
        dz = dz.contiguous()
        try:
            out = block_bwd(x, w, w_lin, bias, dz, ctx.modes, ctx.precision, ws=ctx.ws, saved=True)
        except _lib.FnoError as e:
            if e.status != -1:
                raise
            out = block_bwd(x, w, w_lin, bias, dz, ctx.modes, ctx.precision)
        dx, dw, dwl, db = out
        return dx, dw, dwl, db, None, None


class FNOBlock4d(torch.nn.Module):
    """One 4-D FNO block with its parameters (spectral weights, 1x1 weight, bias)."""

    def __init__(self, width: int, modes, precision="fp32", device=None, seed=None):
        super().__init__()
        mx, my, mz, mt = (int(m) for m in modes)
        self.modes = (mx, my, mz, mt)
        self.precision = precision
        g = torch.Generator(device="cpu")
        if seed is not None:
            g.manual_seed(int(seed))
        scale = 1.0 / (width * width)
        w = (torch.rand(_wshape(width, width, self.modes), generator=g) * 2 - 1) * scale
        s = width ** -0.5
        wl = (torch.rand((width, width), generator=g) * 2 - 1) * s
        b = (torch.rand((width,), generator=g) * 2 - 1) * s
        self.weight = torch.nn.Parameter(w.to(device))
        self.w_lin = torch.nn.Parameter(wl.to(device))
        self.bias = torch.nn.Parameter(b.to(device))

    def forward(self, x):
        return FNOBlock4dFn.apply(x, self.weight, self.w_lin, self.bias, self.modes, self.precision)


# ---------------------------------------------------------------------------
# Layers around the blocks (Alg. 1): pointwise encoder/decoder, MSE loss
# ---------------------------------------------------------------------------
ACT = {"none": _lib.FNO_ACT_NONE, "gelu": _lib.FNO_ACT_GELU}


def _act_code(act) -> int:
    if isinstance(act, int):
        return act
    try:
        return ACT[act]
    except KeyError:
        raise ValueError(f"unknown activation {act!r}; one of {sorted(ACT)}") from None


def _pw_dims(x: torch.Tensor, C_out: int):
    if x.dim() < 2:
        raise ValueError(f"x must be [B, C, ...], got shape {tuple(x.shape)}")
    B, Ci = int(x.shape[0]), int(x.shape[1])
    P = 1
    for v in x.shape[2:]:
        P *= int(v)
    return _lib.make_pw_dims(B, Ci, C_out, P)


def pointwise_fwd(x, w, bias=None, act="gelu"):
    """y[b,o,...] = act(sum_i x[b,i,...] w[i,o] + bias[o]): the 1x1 layers of Alg. 1."""
    x = _req(x, "x")
    Ci, Co = int(x.shape[1]), int(w.shape[1])
    w = _req(w, "w", (Ci, Co))
    bias = None if bias is None else _req(bias, "bias", (Co,))
    d = _pw_dims(x, Co)
    y = torch.empty((x.shape[0], Co) + tuple(x.shape[2:]), dtype=torch.float32, device=x.device)
    _lib.fno_pointwise_fwd(d, _act_code(act), x.data_ptr(), w.data_ptr(),
                           None if bias is None else bias.data_ptr(), y.data_ptr(),
                           _stream_handle(x.device))
    return y


def pointwise_bwd(x, w, bias, dy, act="gelu", need_dx=True):
    """(dx or None, dw, db or None) of ``pointwise_fwd`` for upstream dy."""
    x = _req(x, "x")
    Ci, Co = int(x.shape[1]), int(w.shape[1])
    w = _req(w, "w", (Ci, Co))
    bias = None if bias is None else _req(bias, "bias", (Co,))
    dy = _req(dy, "dy", (x.shape[0], Co) + tuple(x.shape[2:]))
    d = _pw_dims(x, Co)
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty_like(w)
    db = None if bias is None else torch.empty_like(bias)
    n = _lib.fno_pointwise_workspace_bytes(d)
    ws = torch.empty(n, dtype=torch.uint8, device=x.device)
    _lib.fno_pointwise_bwd(d, _act_code(act), x.data_ptr(), w.data_ptr(),
                           None if bias is None else bias.data_ptr(), dy.data_ptr(),
                           None if dx is None else dx.data_ptr(), dw.data_ptr(),
                           None if db is None else db.data_ptr(), ws.data_ptr(), n,
                           _stream_handle(x.device))
    return dx, dw, db


def mse_loss(y, target, need_grad=True):
    """(loss [1] device tensor, dL/dy or None) of mean((y - target)^2)."""
    y = _req(y, "y")
    target = _req(target, "target", tuple(y.shape))
    n = y.numel()
    loss = torch.empty(1, dtype=torch.float32, device=y.device)
    dy = torch.empty_like(y) if need_grad else None
    nb = _lib.fno_mse_workspace_bytes(n)
    ws = torch.empty(nb, dtype=torch.uint8, device=y.device)
    _lib.fno_mse_loss(n, y.data_ptr(), target.data_ptr(), loss.data_ptr(),
                      None if dy is None else dy.data_ptr(), ws.data_ptr(), nb,
                      _stream_handle(y.device))
    return loss, dy


class PointwiseFn(torch.autograd.Function):
    """The encoder / decoder 1x1 layer with sigma.  Only its input is kept."""

    @staticmethod
    def forward(ctx, x, w, bias, act="gelu"):
        ctx.act = act
        ctx.has_bias = bias is not None
        ctx.save_for_backward(x, w, bias)
        return pointwise_fwd(x, w, bias, act)

    @staticmethod
    def backward(ctx, dy):
        x, w, bias = ctx.saved_tensors
        dx, dw, db = pointwise_bwd(x, w, bias if ctx.has_bias else None, dy.contiguous(),
                                   ctx.act, need_dx=ctx.needs_input_grad[0])
        return dx, dw, db, None


class MSELossFn(torch.autograd.Function):
    """mean((y - target)^2); the gradient with respect to y is formed in the forward."""

    @staticmethod
    def forward(ctx, y, target):
        loss, dy = mse_loss(y, target, need_grad=ctx.needs_input_grad[0])
        ctx.save_for_backward(dy if dy is not None else loss)
        return loss.reshape(())

    @staticmethod
    def backward(ctx, g):
        (dy,) = ctx.saved_tensors
        if not ctx.needs_input_grad[0]:
            return None, None
        return dy * g, None
