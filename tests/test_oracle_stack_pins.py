"""Pins of the oracle's Alg. 1 layers around the blocks (CPU only).

The encoder/decoder pointwise layers and the loss are checked against PyTorch's
CPU FP64 library routines (``matmul``, ``gelu`` in its exact erf form,
``mse_loss``) and their autograd; the composed stack (encoder, FNO blocks,
decoder, loss) is checked against an independent PyTorch model built on
``torch.fft.rfftn`` / ``irfftn`` with autograd, and against central finite
differences of the oracle's own loss.  Each is a check by different code or by
mathematics, not a retyping of the oracle's formulas.
"""
import numpy as np
import pytest

import oracle
from oracle import Dims

torch = pytest.importorskip("torch")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _torch_pointwise(x, w, b, act):
    a = torch.einsum("bi...,io->bo...", x, w)
    if b is not None:
        a = a + b.reshape((1, -1) + (1,) * (x.dim() - 2))
    return torch.nn.functional.gelu(a) if act else a


@pytest.mark.parametrize("act", [0, 1])
def test_pointwise_forward_equals_torch_linear_and_gelu(act):
    g = _rng(11)
    x = g.standard_normal((2, 3, 5, 4, 3, 2))
    w = g.standard_normal((3, 7))
    b = g.standard_normal(7)
    y = oracle.pointwise_fwd(x, w, b, act=act)
    ref = _torch_pointwise(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), act)
    assert _rel(y, ref.numpy()) < 1e-13
    # without a bias the layer is the plain channel contraction
    y0 = oracle.pointwise_fwd(x, w, None, act=act)
    ref0 = _torch_pointwise(torch.from_numpy(x), torch.from_numpy(w), None, act)
    assert _rel(y0, ref0.numpy()) < 1e-13


@pytest.mark.parametrize("act", [0, 1])
def test_pointwise_gradient_equals_torch_autograd(act):
    g = _rng(12)
    x = g.standard_normal((2, 4, 3, 5, 2, 3))
    w = g.standard_normal((4, 3))
    b = g.standard_normal(3)
    dy = g.standard_normal((2, 3, 3, 5, 2, 3))
    r = oracle.pointwise_bwd(x, w, dy, b, act=act)
    tx, tw, tb = (torch.tensor(v, requires_grad=True) for v in (x, w, b))
    _torch_pointwise(tx, tw, tb, act).backward(torch.from_numpy(dy))
    assert _rel(r["dx"], tx.grad.numpy()) < 1e-13
    assert _rel(r["dw"], tw.grad.numpy()) < 1e-13
    assert _rel(r["db"], tb.grad.numpy()) < 1e-13


def test_mse_equals_torch_mse_loss_and_its_gradient():
    g = _rng(13)
    y = g.standard_normal((3, 2, 4, 5))
    t = g.standard_normal((3, 2, 4, 5))
    loss, dy = oracle.mse(y, t)
    ty = torch.tensor(y, requires_grad=True)
    tl = torch.nn.functional.mse_loss(ty, torch.from_numpy(t))
    tl.backward()
    assert abs(loss - tl.item()) <= 1e-14 * abs(tl.item())
    assert _rel(dy, ty.grad.numpy()) < 1e-14


# ---- the composed stack ----------------------------------------------------
D_STACK = Dims(1, 4, 4, 8, 6, 8, 4, 2, 2, 2, 2)   # width 4, two blocks below
C0, COUT = 3, 1


def _stack_params(seed):
    g = _rng(seed)
    d = D_STACK
    x0 = g.standard_normal((d.B, C0) + d.grid)
    target = g.uniform(0.0, 1.0, (d.B, COUT) + d.grid)
    enc = (g.uniform(-1, 1, (C0, d.Ci)) / np.sqrt(C0), g.uniform(-0.5, 0.5, d.Ci))
    blocks = []
    for _ in range(2):
        w = g.uniform(-1, 1, (d.Ci, d.Co) + d.modes + (2,)) / (d.Ci * d.Co) * 8.0
        wl = g.uniform(-1, 1, (d.Ci, d.Co)) / np.sqrt(d.Ci)
        bb = g.uniform(-0.5, 0.5, d.Co)
        blocks.append((w, wl, bb))
    dec = (g.uniform(-1, 1, (d.Ci, COUT)) / np.sqrt(d.Ci), g.uniform(-0.5, 0.5, COUT))
    return x0, target, enc, blocks, dec


def _torch_spectral(x, w, d):
    """S(x) by the library FFTs: rfftn, keep the corner modes, mix, zero-pad, irfftn."""
    grid = d.grid
    X = torch.fft.rfftn(x, dim=(-4, -3, -2, -1))

    def keep(m, n):
        return torch.cat([torch.arange(m), torch.arange(n - m, n)])

    ix, iy, iz = keep(d.mx, d.Nx), keep(d.my, d.Ny), keep(d.mz, d.Nz)
    it = torch.arange(d.mt)
    sel = (ix[:, None, None, None], iy[None, :, None, None], iz[None, None, :, None],
           it[None, None, None, :])
    Xk = X[(slice(None), slice(None)) + sel]
    W = torch.complex(w[..., 0], w[..., 1])
    Yk = torch.einsum("bixyzt,ioxyzt->boxyzt", Xk, W)
    Y = torch.zeros((x.shape[0], W.shape[1]) + X.shape[2:], dtype=Yk.dtype)
    Y[(slice(None), slice(None)) + sel] = Yk
    return torch.fft.irfftn(Y, s=grid, dim=(-4, -3, -2, -1))


def _torch_stack_loss(x0, target, enc, blocks, dec, d, dec_act):
    h = _torch_pointwise(x0, enc[0], enc[1], 1)
    for (w, wl, b) in blocks:
        a = _torch_spectral(h, w, d) + _torch_pointwise(h, wl, b, 0)
        h = torch.nn.functional.gelu(a)
    y = _torch_pointwise(h, dec[0], dec[1], dec_act)
    return torch.nn.functional.mse_loss(y, target)


@pytest.mark.parametrize("dec_act", [1, 0])
def test_stack_loss_and_gradients_equal_torch_fft_model(dec_act):
    d = D_STACK
    x0, target, enc, blocks, dec = _stack_params(21)
    loss, gr = oracle.stack_loss_and_grads(d, x0, target, enc, blocks, dec, dec_act=dec_act)
    T = lambda a: torch.tensor(a, requires_grad=True)
    tx0 = T(x0)
    tenc = (T(enc[0]), T(enc[1]))
    tblocks = [(T(w), T(wl), T(b)) for (w, wl, b) in blocks]
    tdec = (T(dec[0]), T(dec[1]))
    tl = _torch_stack_loss(tx0, torch.from_numpy(target), tenc, tblocks, tdec, d, dec_act)
    tl.backward()
    assert abs(loss - tl.item()) <= 1e-12 * abs(tl.item())
    assert _rel(gr["x0"], tx0.grad.numpy()) < 1e-10
    for a, t in zip(gr["enc"] + gr["dec"], tenc + tdec):
        assert _rel(a, t.grad.numpy()) < 1e-10
    for (dw, dwl, db), (tw, twl, tb) in zip(gr["blocks"], tblocks):
        assert _rel(dw, tw.grad.numpy()) < 1e-10
        assert _rel(dwl, twl.grad.numpy()) < 1e-10
        assert _rel(db, tb.grad.numpy()) < 1e-10


def test_stack_gradient_central_finite_differences():
    """(L(p + eps v) - L(p - eps v)) / 2 eps against <dL/dp, v>, eps = 1e-4, FP64.

    One seeded direction per parameter group.  The central difference errs by
    O(eps^2) through the third derivatives of the three stacked GELUs (about
    3e-6 relative at eps = 1e-3 on this stack, so eps is 1e-4); rounding adds
    about 1e-16 L / eps.
    """
    d = D_STACK
    x0, target, enc, blocks, dec = _stack_params(22)
    loss, gr = oracle.stack_loss_and_grads(d, x0, target, enc, blocks, dec)
    g = _rng(23)
    eps = 1e-4

    def L(x0_, enc_, blocks_, dec_):
        return oracle.stack_loss_and_grads(d, x0_, target, enc_, blocks_, dec_)[0]

    checks = []
    v = g.standard_normal(x0.shape)
    checks.append((L(x0 + eps * v, enc, blocks, dec) - L(x0 - eps * v, enc, blocks, dec),
                   float(np.sum(gr["x0"] * v))))
    for k in range(2):
        v = g.standard_normal(enc[k].shape)
        ep = tuple(e + eps * v if j == k else e for j, e in enumerate(enc))
        em = tuple(e - eps * v if j == k else e for j, e in enumerate(enc))
        checks.append((L(x0, ep, blocks, dec) - L(x0, em, blocks, dec),
                       float(np.sum(gr["enc"][k] * v))))
        v = g.standard_normal(dec[k].shape)
        dp = tuple(e + eps * v if j == k else e for j, e in enumerate(dec))
        dm = tuple(e - eps * v if j == k else e for j, e in enumerate(dec))
        checks.append((L(x0, enc, blocks, dp) - L(x0, enc, blocks, dm),
                       float(np.sum(gr["dec"][k] * v))))
    for bi in range(2):
        for k in range(3):
            v = g.standard_normal(blocks[bi][k].shape)
            bp = [tuple(e + eps * v if (i == bi and j == k) else e for j, e in enumerate(blk))
                  for i, blk in enumerate(blocks)]
            bm = [tuple(e - eps * v if (i == bi and j == k) else e for j, e in enumerate(blk))
                  for i, blk in enumerate(blocks)]
            checks.append((L(x0, enc, bp, dec) - L(x0, enc, bm, dec),
                           float(np.sum(gr["blocks"][bi][k] * v))))
    for diff, an in checks:
        fd = diff / (2 * eps)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * loss), (fd, an)


def test_adam_matches_torch_optim_adam():
    """Three Adam steps against torch.optim.Adam in FP64 (a library routine)."""
    g = _rng(31)
    p0 = g.standard_normal(257)
    grads = [g.standard_normal(257) * s for s in (1.0, 0.3, 2.0)]
    p, m, v = p0.copy(), np.zeros(257), np.zeros(257)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.85, 0.995), eps=1e-7)
    for t, gr in enumerate(grads, start=1):
        oracle.adam(p, gr, m, v, t, lr=3e-3, b1=0.85, b2=0.995, eps=1e-7)
        opt.zero_grad()
        tp.grad = torch.from_numpy(gr.copy())
        opt.step()
    assert _rel(p - p0, tp.detach().numpy() - p0) < 1e-12


def test_adam_first_step_moves_every_coordinate_by_about_lr():
    """At t = 1 the bias-corrected ratio is g / (|g| + eps): a step of lr against g's sign."""
    g = _rng(32)
    p0 = g.standard_normal(100)
    gr = g.standard_normal(100)
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    oracle.adam(p, gr, m, v, 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(p0 - p, 0.01 * np.sign(gr), rtol=1e-9)
