"""The FNO stack of Alg. 1 (Sec. IV-C): encoder, FNO blocks, decoder, MSE loss.

    X1      = GELU(x0 W_e + b_e)                     encoder: 1x1 lift C_in -> width
    X_{k+1} = GELU(S_k(X_k) + W_l,k^T X_k + b_k)     FNO block k = 1..L (Alg. 2)
    Y       = sigma(X_{L+1} W_d + b_d)               decoder: 1x1 projection width -> C_out
    L       = mean((Y - target)^2)

Alg. 1 applies sigma after the decoder too; ``decoder_act="none"`` drops it.

Two ways to run it, both marshalling only (every step is a libfno kernel):

* ``FNO4d``: a ``torch.nn.Module`` of autograd Functions.  Each layer keeps
  only its input for the backward pass, and each block's backward recomputes
  its forward spectrum, so the stack holds one activation per block (per-block
  activation checkpointing).
* ``StackRunner``: one pass (forward, loss, backward; ``train_step`` adds the
  Adam update of every parameter, ``fno_adam_step``) issued straight
  through the C ABI with preallocated checkpoints, gradients and workspaces: no
  autograd bookkeeping and no allocation inside the pass, so it can be timed
  or captured as it stands.

In both, each block's forward workspace carries its truncated spectra to the
block's backward, which reuses them (``fno_block_bwd_saved``) instead of
recomputing them from the checkpointed input.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib, ops


class FNO4d(torch.nn.Module):
    """Alg. 1 with ``n_blocks`` FNO blocks of width ``width`` (autograd path)."""

    def __init__(self, c_in: int, width: int, c_out: int, modes, n_blocks: int = 4,
                 precision="bf16x3", decoder_act="gelu", device=None, seed=0):
        super().__init__()
        self.modes = tuple(int(m) for m in modes)
        self.precision = precision
        self.decoder_act = decoder_act
        g = torch.Generator(device="cpu")
        g.manual_seed(int(seed))

        def uni(shape, s):
            return ((torch.rand(shape, generator=g) * 2 - 1) * s).to(device)

        self.enc_w = torch.nn.Parameter(uni((c_in, width), c_in ** -0.5))
        self.enc_b = torch.nn.Parameter(uni((width,), c_in ** -0.5))
        self.blocks = torch.nn.ModuleList(
            [ops.FNOBlock4d(width, self.modes, precision, device=device, seed=int(seed) + 1 + k)
             for k in range(n_blocks)])
        self.dec_w = torch.nn.Parameter(uni((width, c_out), width ** -0.5))
        self.dec_b = torch.nn.Parameter(uni((c_out,), width ** -0.5))

    def load_arrays(self, enc, blocks, dec):
        """Set every parameter from arrays: enc = (W_e, b_e), blocks = [(W, W_l, b)], dec = (W_d, b_d)."""
        with torch.no_grad():
            for p, a in zip((self.enc_w, self.enc_b), enc):
                p.copy_(torch.as_tensor(np.asarray(a, dtype=np.float32)))
            for blk, (w, wl, b) in zip(self.blocks, blocks):
                for p, a in zip((blk.weight, blk.w_lin, blk.bias), (w, wl, b)):
                    p.copy_(torch.as_tensor(np.asarray(a, dtype=np.float32)))
            for p, a in zip((self.dec_w, self.dec_b), dec):
                p.copy_(torch.as_tensor(np.asarray(a, dtype=np.float32)))
        return self

    def forward(self, x):
        h = ops.PointwiseFn.apply(x, self.enc_w, self.enc_b, "gelu")
        for blk in self.blocks:
            h = blk(h)
        return ops.PointwiseFn.apply(h, self.dec_w, self.dec_b, self.decoder_act)

    def loss(self, x, target):
        return ops.MSELossFn.apply(self(x), target)


class StackRunner:
    """Forward + MSE loss + backward of the Alg. 1 stack through the C ABI.

    ``params``: dict of float32 CUDA tensors ``enc_w`` [C_in, width], ``enc_b``,
    ``blocks`` = [(w, w_lin, bias), ...], ``dec_w`` [width, C_out], ``dec_b``.
    ``grid`` = (Nx, Ny, Nz, Nt); ``modes`` = (mx, my, mz, mt), the kept
    frequencies per side (stored counts 2mx, 2my, 2mz, mt).  Every tensor's shape
    is checked against these sizes before any launch.  Buffers: the L + 1 block
    inputs (the only activations kept between the passes), the output, two
    gradient buffers used in turn, the parameter gradients, and one workspace
    per kind of call.
    """

    def __init__(self, B: int, c_in: int, grid, params, modes, precision="bf16x3",
                 decoder_act="gelu", device=None):
        self.dev = torch.device(device if device is not None else "cuda")
        self.B = int(B)
        self.c_in = int(c_in)
        self.grid = tuple(int(v) for v in grid)
        self.P = int(np.prod(self.grid))
        self.modes = tuple(int(m) for m in modes)
        self.prec = ops.precision_code(precision)
        self.dec_act = ops._act_code(decoder_act)
        self.p = params
        self.width = int(params["enc_w"].shape[1])
        self.c_out = int(params["dec_w"].shape[1])
        self.L = len(params["blocks"])
        W, Co, dev, sh = self.width, self.c_out, self.dev, (self.B,)
        # the C ABI takes raw pointers: every parameter's shape is checked here
        ops._req(params["enc_w"], "enc_w", (self.c_in, W))
        ops._req(params["enc_b"], "enc_b", (W,))
        ops._req(params["dec_w"], "dec_w", (W, Co))
        ops._req(params["dec_b"], "dec_b", (Co,))
        for k, (w, wl, b) in enumerate(params["blocks"]):
            ops._req(w, f"blocks[{k}].w", ops._wshape(W, W, self.modes))
            ops._req(wl, f"blocks[{k}].w_lin", (W, W))
            ops._req(b, f"blocks[{k}].bias", (W,))
            for t in (w, wl, b):
                if not t.is_contiguous():
                    raise ValueError(f"blocks[{k}] parameters must be contiguous")
        for t in (params["enc_w"], params["enc_b"], params["dec_w"], params["dec_b"]):
            if not t.is_contiguous():
                raise ValueError("encoder/decoder parameters must be contiguous")
        f32 = dict(dtype=torch.float32, device=dev)
        self.h = [torch.empty(sh + (W,) + self.grid, **f32) for _ in range(self.L + 1)]
        self.y = torch.empty(sh + (Co,) + self.grid, **f32)
        self.dy = torch.empty_like(self.y)
        self.g = [torch.empty_like(self.h[0]) for _ in range(2)]
        self.loss = torch.empty(1, **f32)
        self.grads = {
            "enc_w": torch.empty_like(params["enc_w"]), "enc_b": torch.empty_like(params["enc_b"]),
            "blocks": [tuple(torch.empty_like(t) for t in blk) for blk in params["blocks"]],
            "dec_w": torch.empty_like(params["dec_w"]), "dec_b": torch.empty_like(params["dec_b"]),
        }
        mx, my, mz, mt = self.modes
        self.bd = _lib.make_dims(self.B, W, W, *self.grid, mx, my, mz, mt)
        nb = _lib.fno_workspace_bytes(self.bd, self.prec, ops.OP_BLOCK_TRAIN)
        # one workspace per block (the training size covers the forward and the
        # backward): it carries the block's truncated spectra and GELU'(A) from
        # the forward to the backward (fno_block_bwd_saved)
        self.ws_block = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(self.L)]
        self.ed = _lib.make_pw_dims(self.B, self.c_in, W, self.P)
        self.dd = _lib.make_pw_dims(self.B, W, Co, self.P)
        npw = max(_lib.fno_pointwise_workspace_bytes(self.ed),
                  _lib.fno_pointwise_workspace_bytes(self.dd))
        self.ws_pw = torch.empty(npw, dtype=torch.uint8, device=dev)
        nm = _lib.fno_mse_workspace_bytes(self.B * Co * self.P)
        self.ws_mse = torch.empty(nm, dtype=torch.uint8, device=dev)

    def bytes_held(self) -> int:
        ts = self.h + [self.y, self.dy, self.loss, self.ws_pw, self.ws_mse] + self.g + self.ws_block
        return int(sum(t.numel() * t.element_size() for t in ts))

    def _check_io(self, x0, target=None):
        ops._req(x0, "x0", (self.B, self.c_in) + self.grid)
        if not x0.is_contiguous():
            raise ValueError("x0 must be contiguous")
        if target is not None:
            ops._req(target, "target", (self.B, self.c_out) + self.grid)
            if not target.is_contiguous():
                raise ValueError("target must be contiguous")

    def forward(self, x0, stream=None, train=False):
        """Y for input x0 [B, C_in, *grid]; fills the block-input checkpoints
        (train=True: the blocks also keep GELU'(A) for the backward)."""
        self._check_io(x0)
        s = stream if stream is not None else int(torch.cuda.current_stream(self.dev).cuda_stream)
        p = self.p
        _lib.fno_pointwise_fwd(self.ed, _lib.FNO_ACT_GELU, x0.data_ptr(), p["enc_w"].data_ptr(),
                               p["enc_b"].data_ptr(), self.h[0].data_ptr(), s)
        for k, (w, wl, b) in enumerate(p["blocks"]):
            ws = self.ws_block[k]
            fwd = _lib.fno_block_fwd_train if train else _lib.fno_block_fwd
            fwd(self.bd, self.prec, self.h[k].data_ptr(), w.data_ptr(), wl.data_ptr(),
                b.data_ptr(), self.h[k + 1].data_ptr(), ws.data_ptr(), ws.numel(), s)
        _lib.fno_pointwise_fwd(self.dd, self.dec_act, self.h[-1].data_ptr(), p["dec_w"].data_ptr(),
                               p["dec_b"].data_ptr(), self.y.data_ptr(), s)
        return self.y

    def step(self, x0, target, stream=None):
        """One training pass: returns the device loss [1]; gradients land in ``grads``."""
        self._check_io(x0, target)
        s = stream if stream is not None else int(torch.cuda.current_stream(self.dev).cuda_stream)
        p, gr = self.p, self.grads
        self.forward(x0, s, train=True)
        n = self.y.numel()
        _lib.fno_mse_loss(n, self.y.data_ptr(), target.data_ptr(), self.loss.data_ptr(),
                          self.dy.data_ptr(), self.ws_mse.data_ptr(), self.ws_mse.numel(), s)
        npw = self.ws_pw.numel()
        _lib.fno_pointwise_bwd(self.dd, self.dec_act, self.h[-1].data_ptr(), p["dec_w"].data_ptr(),
                               p["dec_b"].data_ptr(), self.dy.data_ptr(), self.g[0].data_ptr(),
                               gr["dec_w"].data_ptr(), gr["dec_b"].data_ptr(),
                               self.ws_pw.data_ptr(), npw, s)
        cur = 0
        for k in range(self.L - 1, -1, -1):
            w, wl, b = p["blocks"][k]
            dw, dwl, db = gr["blocks"][k]
            ws = self.ws_block[k]
            _lib.fno_block_bwd_saved(self.bd, self.prec, self.h[k].data_ptr(), w.data_ptr(),
                                     wl.data_ptr(), b.data_ptr(), self.g[cur].data_ptr(),
                                     self.g[1 - cur].data_ptr(), dw.data_ptr(), dwl.data_ptr(),
                                     db.data_ptr(), ws.data_ptr(), ws.numel(), s)
            cur = 1 - cur
        _lib.fno_pointwise_bwd(self.ed, _lib.FNO_ACT_GELU, x0.data_ptr(), p["enc_w"].data_ptr(),
                               p["enc_b"].data_ptr(), self.g[cur].data_ptr(), None,
                               gr["enc_w"].data_ptr(), gr["enc_b"].data_ptr(),
                               self.ws_pw.data_ptr(), npw, s)
        return self.loss

    # ---- training step ------------------------------------------------------
    def params_and_grads(self):
        """(parameter, gradient) pairs in a fixed order."""
        p, g = self.p, self.grads
        pairs = [(p["enc_w"], g["enc_w"]), (p["enc_b"], g["enc_b"])]
        for blk, gb in zip(p["blocks"], g["blocks"]):
            pairs += list(zip(blk, gb))
        pairs += [(p["dec_w"], g["dec_w"]), (p["dec_b"], g["dec_b"])]
        return pairs

    def train_step(self, x0, target, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, stream=None):
        """step() followed by an Adam update of every parameter (fno_adam_step)."""
        s = stream if stream is not None else int(torch.cuda.current_stream(self.dev).cuda_stream)
        loss = self.step(x0, target, s)
        if not hasattr(self, "_adam"):
            self._adam = [(torch.zeros_like(q), torch.zeros_like(q)) for q, _ in self.params_and_grads()]
            self._t = 0
        self._t += 1
        for (q, gq), (m, v) in zip(self.params_and_grads(), self._adam):
            _lib.fno_adam_step(q.numel(), q.data_ptr(), gq.data_ptr(), m.data_ptr(), v.data_ptr(),
                               lr, betas[0], betas[1], eps, self._t, s)
        return loss
