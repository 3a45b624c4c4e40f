"""GPU parity of the Alg. 1 layers around the blocks and of the whole stack.

The pointwise encoder/decoder layer (forward and backward) and the MSE loss run
through the C ABI and are compared element by element with the FP64 oracle on
the same seeded inputs: shapes with several 256-point tiles and a ragged tail,
point counts that are not a multiple of 4 (the scalar path), the largest
channel counts (64 x 64), one channel on either side, no bias, no input
gradient, and an empty batch.  The stack (encoder, FNO blocks, decoder, loss)
runs through ``StackRunner`` and through the autograd module ``FNO4d``; both
are compared with ``oracle.stack_loss_and_grads``.  Tolerances (rel-L2 per
tensor): the FP32 layers 1e-6; the stack 1e-5 for FP32 and split BF16 blocks,
2e-2 for BF16 blocks.
"""
import numpy as np
import pytest

import oracle
from oracle import Dims
from paper_2211_12709_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


PW_CASES = [
    # B, Ci, Co, grid, act, bias, need_dx, label
    (1, 3, 20, (16, 16, 16, 8), 1, True, False, "encoder 3 -> 20, 128 tiles"),
    (2, 20, 1, (8, 8, 8, 4), 1, True, True, "decoder 20 -> 1"),
    (2, 5, 7, (3, 5, 7, 3), 0, False, True, "P = 315: scalar path, ragged tile, no bias"),
    (1, 64, 64, (8, 8, 4, 4), 1, True, True, "64 x 64 channels (four pair blocks per thread)"),
    (3, 1, 1, (5, 5, 5, 5), 1, True, True, "one channel each side, P = 625"),
    (1, 20, 33, (1, 1, 1, 785), 1, True, True, "P = 3 tiles + 17"),
    (2, 8, 20, (16, 8, 8, 8), 0, True, True, "identity activation"),
]


@pytest.mark.parametrize("case", PW_CASES, ids=[c[-1] for c in PW_CASES])
def test_pointwise_layer_matches_oracle(case):
    from paper_2211_12709_gb300 import ops
    B, Ci, Co, grid, act, with_bias, need_dx, _ = case
    x = inputs.normal((B, Ci) + grid, 600 + Ci)
    w, b = inputs.linear_params(Ci, Co, 700 + Co)
    if not with_bias:
        b = None
    dy = inputs.normal((B, Co) + grid, 800 + Co)
    X, W, DY = (torch.from_numpy(a).to(DEV) for a in (x, w, dy))
    Bb = None if b is None else torch.from_numpy(b).to(DEV)
    y = ops.pointwise_fwd(X, W, Bb, act)
    dx, dw, db = ops.pointwise_bwd(X, W, Bb, DY, act, need_dx=need_dx)
    torch.cuda.synchronize()
    ry = oracle.pointwise_fwd(x, w, b, act=act)
    rb = oracle.pointwise_bwd(x, w, dy, b, act=act, need_dx=need_dx)
    errs = {"y": relerr(y.cpu().numpy(), ry), "dw": relerr(dw.cpu().numpy(), rb["dw"])}
    if need_dx:
        errs["dx"] = relerr(dx.cpu().numpy(), rb["dx"])
    else:
        assert dx is None
    if b is not None:
        errs["db"] = relerr(db.cpu().numpy(), rb["db"])
    print(case[-1], errs)
    assert all(v <= 1e-6 for v in errs.values()), errs


def test_pointwise_empty_batch_gives_zero_gradients():
    from paper_2211_12709_gb300 import ops
    X = torch.empty((0, 3, 4, 4, 4, 4), device=DEV)
    W = torch.randn(3, 5, device=DEV)
    Bb = torch.randn(5, device=DEV)
    y = ops.pointwise_fwd(X, W, Bb, "gelu")
    assert y.shape == (0, 5, 4, 4, 4, 4)
    dx, dw, db = ops.pointwise_bwd(X, W, Bb, torch.empty((0, 5, 4, 4, 4, 4), device=DEV), "gelu")
    torch.cuda.synchronize()
    assert torch.count_nonzero(dw).item() == 0 and torch.count_nonzero(db).item() == 0


@pytest.mark.parametrize("n", [1, 1001, 1 << 20, (1 << 20) + 3])
def test_mse_loss_matches_oracle(n):
    from paper_2211_12709_gb300 import ops
    y = inputs.normal((n,), 900 + n % 97)
    t = inputs.normal((n,), 901 + n % 89)
    Y, T = torch.from_numpy(y).to(DEV), torch.from_numpy(t).to(DEV)
    loss, dy = ops.mse_loss(Y, T)
    torch.cuda.synchronize()
    rl, rdy = oracle.mse(y, t)
    assert abs(loss.item() - rl) <= 1e-6 * rl, (loss.item(), rl)
    assert relerr(dy.cpu().numpy(), rdy) <= 1e-6


# ---- the stack -------------------------------------------------------------
STACK = Dims(1, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4)   # width 8
MODES = (STACK.mx, STACK.my, STACK.mz, STACK.mt)   # kept frequencies per side
C0, COUT, NBLK = 3, 1, 3
TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 2e-2, "tf32": 5e-3}


def _stack_arrays(d, seed=31):
    x0 = inputs.grf((d.B, C0), d.grid, (4.0, 4.0, 4.0, 2.0), seed)
    target = inputs.normal((d.B, COUT) + d.grid, seed + 1) * 0.1 + 0.5
    ew, eb = inputs.linear_params(C0, d.Ci, seed + 2)
    blocks = []
    for k in range(NBLK):
        w = inputs.spectral_weights(d.Ci, d.Co, d.modes, seed + 10 + k)
        wl, b = inputs.linear_params(d.Ci, d.Co, seed + 20 + k)
        blocks.append((w, wl, b))
    dw_, db_ = inputs.linear_params(d.Ci, COUT, seed + 3)
    return x0, target, (ew, eb), blocks, (dw_, db_)


@pytest.fixture(scope="module")
def stack_case():
    d = STACK
    x0, target, enc, blocks, dec = _stack_arrays(d)
    loss, gr = oracle.stack_loss_and_grads(d, x0, target, enc, blocks, dec)
    return d, x0, target, enc, blocks, dec, loss, gr


def _stack_errs(loss, grads, ref_loss, ref):
    errs = {"loss": abs(loss - ref_loss) / abs(ref_loss),
            "enc_w": relerr(grads["enc_w"], ref["enc"][0]),
            "enc_b": relerr(grads["enc_b"], ref["enc"][1]),
            "dec_w": relerr(grads["dec_w"], ref["dec"][0]),
            "dec_b": relerr(grads["dec_b"], ref["dec"][1])}
    for k, (g, r) in enumerate(zip(grads["blocks"], ref["blocks"])):
        for name, a, b in zip(("dw", "dwl", "db"), g, r):
            errs[f"b{k}.{name}"] = relerr(a, b)
    return errs


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16"])
def test_stack_runner_matches_oracle(stack_case, precision):
    from paper_2211_12709_gb300.stack import StackRunner
    d, x0, target, enc, blocks, dec, ref_loss, ref = stack_case
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    params = {"enc_w": T(enc[0]), "enc_b": T(enc[1]), "dec_w": T(dec[0]), "dec_b": T(dec[1]),
              "blocks": [tuple(T(a) for a in blk) for blk in blocks]}
    r = StackRunner(d.B, C0, d.grid, params, MODES, precision, device=DEV)
    X0, TG = T(x0), T(target)
    loss = r.step(X0, TG)
    torch.cuda.synchronize()
    grads = {"enc_w": r.grads["enc_w"].cpu().numpy(), "enc_b": r.grads["enc_b"].cpu().numpy(),
             "dec_w": r.grads["dec_w"].cpu().numpy(), "dec_b": r.grads["dec_b"].cpu().numpy(),
             "blocks": [tuple(t.cpu().numpy() for t in blk) for blk in r.grads["blocks"]]}
    errs = _stack_errs(loss.item(), grads, ref_loss, ref)
    # the checkpoints are the oracle's block inputs
    for k in range(NBLK + 1):
        errs[f"h{k}"] = relerr(r.h[k].cpu().numpy(), ref["h"][k])
    print(precision, {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(np.isfinite(v) and v <= TOL[precision] for v in errs.values()), errs
    # a second pass on the same inputs is bitwise identical (fixed-order reductions)
    g0 = [t.clone() for t in (r.grads["enc_w"], r.grads["dec_w"], r.grads["blocks"][0][0])]
    l0 = loss.clone()
    loss2 = r.step(X0, TG)
    torch.cuda.synchronize()
    assert torch.equal(l0, loss2)
    for a, b in zip(g0, (r.grads["enc_w"], r.grads["dec_w"], r.grads["blocks"][0][0])):
        assert torch.equal(a, b)


def test_stack_runner_rejects_weights_of_other_mode_counts(stack_case):
    """Stored mode counts (2mx, 2my, 2mz, mt) passed as modes: refused on the host."""
    from paper_2211_12709_gb300.stack import StackRunner
    d, x0, target, enc, blocks, dec, ref_loss, ref = stack_case
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    params = {"enc_w": T(enc[0]), "enc_b": T(enc[1]), "dec_w": T(dec[0]), "dec_b": T(dec[1]),
              "blocks": [tuple(T(a) for a in blk) for blk in blocks]}
    with pytest.raises(ValueError, match="blocks\\[0\\].w"):
        StackRunner(d.B, C0, d.grid, params, d.modes, "fp32", device=DEV)
    r = StackRunner(d.B, C0, d.grid, params, MODES, "fp32", device=DEV)
    with pytest.raises(ValueError, match="x0"):
        r.step(T(x0[:, :2]), T(target))


def test_autograd_module_equals_runner(stack_case):
    from paper_2211_12709_gb300.stack import FNO4d, StackRunner
    d, x0, target, enc, blocks, dec, ref_loss, ref = stack_case
    m = FNO4d(C0, d.Ci, COUT, MODES, n_blocks=NBLK, precision="bf16x3", device=DEV)
    m.load_arrays(enc, blocks, dec)
    X0 = torch.from_numpy(x0.astype(np.float32)).to(DEV)
    TG = torch.from_numpy(target.astype(np.float32)).to(DEV)
    loss = m.loss(X0, TG)
    loss.backward()
    params = {"enc_w": m.enc_w.detach(), "enc_b": m.enc_b.detach(), "dec_w": m.dec_w.detach(),
              "dec_b": m.dec_b.detach(),
              "blocks": [(b.weight.detach(), b.w_lin.detach(), b.bias.detach()) for b in m.blocks]}
    r = StackRunner(d.B, C0, d.grid, params, MODES, "bf16x3", device=DEV)
    l2 = r.step(X0, TG)
    torch.cuda.synchronize()
    assert loss.item() == l2.item()
    assert torch.equal(m.enc_w.grad, r.grads["enc_w"])
    assert torch.equal(m.dec_b.grad, r.grads["dec_b"])
    for blk, g in zip(m.blocks, r.grads["blocks"]):
        assert torch.equal(blk.weight.grad, g[0])
        assert torch.equal(blk.w_lin.grad, g[1])
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss


# ---- training step (Adam) ----------------------------------------------------
@pytest.mark.parametrize("n", [1, 1001, 1 << 20])
def test_adam_step_matches_oracle(n):
    from paper_2211_12709_gb300 import _lib
    g = np.random.Generator(np.random.PCG64(70 + n % 11))
    p0 = g.standard_normal(n).astype(np.float32)
    gr = g.standard_normal(n).astype(np.float32)
    m0 = (0.1 * g.standard_normal(n)).astype(np.float32)
    v0 = (0.01 * g.random(n)).astype(np.float32)
    P, G, M, V = (torch.from_numpy(a.copy()).to(DEV) for a in (p0, gr, m0, v0))
    # a large step (lr 0.1), so that the update is large against one FP32 rounding of p
    _lib.fno_adam_step(n, P.data_ptr(), G.data_ptr(), M.data_ptr(), V.data_ptr(), 0.1, 0.9, 0.999,
                       1e-8, 7, int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    rp, rm, rv = (a.astype(np.float64) for a in (p0, m0, v0))
    # the oracle takes the hyperparameters the kernel receives (FP32 values)
    f = lambda c: float(np.float32(c))
    oracle.adam(rp, gr, rm, rv, 7, lr=f(0.1), b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    # FP32 state: the update p - p0 within the FP32 bar, 1e-5 rel-L2.  Its error
    # budget: one FP32 rounding of the stored p (about 6e-7 of an update of size
    # 0.1 on |p| ~ 1) and a few roundings in the update's arithmetic; where
    # b1 m and (1 - b1) g nearly cancel, m has a large relative error in any
    # FP32 implementation, but a small absolute one
    pg = P.cpu().numpy().astype(np.float64)
    assert relerr(pg - p0, rp - p0) <= 1e-5
    assert relerr(M.cpu().numpy(), rm) <= 1e-6
    assert relerr(V.cpu().numpy(), rv) <= 1e-6


def test_training_steps_reduce_the_loss(stack_case):
    """Forty Adam steps on one synthetic batch: the loss falls well below its start."""
    from paper_2211_12709_gb300.stack import StackRunner
    d, x0, target, enc, blocks, dec, ref_loss, ref = stack_case
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    params = {"enc_w": T(enc[0]), "enc_b": T(enc[1]), "dec_w": T(dec[0]), "dec_b": T(dec[1]),
              "blocks": [tuple(T(a) for a in blk) for blk in blocks]}
    r = StackRunner(d.B, C0, d.grid, params, MODES, "bf16x3", device=DEV)
    X0, TG = T(x0), T(target)
    losses = [r.train_step(X0, TG, lr=3e-3).item() for _ in range(40)]
    print("losses", losses[0], losses[9], losses[19], losses[-1])
    assert abs(losses[0] - ref_loss) <= 1e-5 * ref_loss   # the first loss is the oracle's
    assert losses[-1] < 0.5 * losses[0]
    assert sum(b < a for a, b in zip(losses, losses[1:])) >= 30
