"""fno_block_bwd_saved: the backward that reuses the forward's state.

After fno_block_fwd it must give bitwise the results of fno_block_bwd (the same
kernels see the same spectra, recomputed or kept).  After fno_block_fwd_train it
takes GELU'(A) from the forward instead of evaluating A again: z is bitwise the
plain forward's, and the gradients match the FP64 oracle within each
precision's bound.  The library must refuse the saved backward whenever its
record of the workspace does not match: no forward, another call on the
workspace in between, another x or w, a second use after the state is spent, or
a workspace smaller than the training layout after a training forward.
"""
import numpy as np
import pytest

import oracle
from oracle import Dims
from paper_2211_12709_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
CASES = [
    (Dims(2, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4), "fp32"),
    (Dims(2, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4), "bf16x3"),
    (Dims(1, 20, 20, 32, 32, 32, 32, 6, 6, 6, 8), "bf16x3"),
    (Dims(3, 5, 7, 12, 10, 9, 6, 3, 2, 4, 4), "fp32"),
]


TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 2e-2, "tf32": 5e-3}


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def _case(d, seed=5):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    x = T(inputs.normal((d.B, d.Ci) + d.grid, seed))
    w = T(inputs.spectral_weights(d.Ci, d.Co, d.modes, seed + 1))
    wl, b = (T(a) for a in inputs.linear_params(d.Ci, d.Co, seed + 2))
    dz = T(inputs.normal((d.B, d.Co) + d.grid, seed + 3))
    return x, w, wl, b, dz


@pytest.mark.parametrize("d,precision", CASES, ids=[f"{c[1]}-{c[0].grid}" for c in CASES])
def test_saved_backward_is_bitwise_the_recompute_backward(d, precision):
    from paper_2211_12709_gb300 import ops
    modes = (d.mx, d.my, d.mz, d.mt)
    x, w, wl, b, dz = _case(d)
    dims = ops.dims_of(x, d.Co, modes)
    ws = ops.workspace(dims, precision, ops.OP_BLOCK_BWD, x.device)
    z = ops.block_fwd(x, w, wl, b, modes, precision, ws=ws)
    got = ops.block_bwd(x, w, wl, b, dz, modes, precision, ws=ws, saved=True)
    ref = ops.block_bwd(x, w, wl, b, dz, modes, precision)
    torch.cuda.synchronize()
    for g, r, name in zip(got, ref, ("dx", "dw", "dwl", "db")):
        assert torch.equal(g, r), name
    assert torch.isfinite(z).all()


TRAIN_CASES = [
    (Dims(2, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4), "single-layer 16^3x8"),
    (Dims(3, 5, 7, 12, 10, 10, 6, 3, 2, 4, 3), "5 -> 7 channels, Nt=6"),
    (Dims(2, 2, 1, 4, 6, 32, 16, 2, 3, 5, 8), "one output channel"),
    (Dims(1, 20, 20, 8, 8, 16, 32, 2, 2, 4, 8), "width 20, Nt=32 (the tensor-core epilogue)"),
    (Dims(1, 3, 3, 6, 5, 26, 22, 2, 2, 5, 6), "Nz=26, Nt=22 (the FP32 epilogue beside tensor-core stages)"),
    # N = 735: rows of the dA pass are not 16-byte aligned (4-byte copies);
    # outside the tensor-core tilings (odd Nt), so FP32 only
    (Dims(2, 3, 2, 5, 7, 3, 7, 2, 3, 1, 4), "odd N: 4-byte staged copies"),
    # past 31 inputs or 24 outputs the dA pass contracts dW_lin on the CUDA cores
    (Dims(1, 40, 36, 6, 4, 16, 16, 2, 2, 4, 6), "40 -> 36 channels: the FP32 dA pass"),
    # 32 channels: the tensor-core precisions keep the tensor-core dA epilogue
    # (no GELU'(A) stored), FP32 takes the FP32 dA pass
    (Dims(1, 32, 32, 4, 4, 16, 16, 2, 2, 4, 6), "32 channels: dA epilogue in the tensor-core precisions"),
    # the fused dA + t,z pass: 31 -> 24 channels and 32 kept z modes (its limits),
    # 312 columns over at most 152 CTAs, Nt = 16 (two 8-plane n-tiles per chunk)
    (Dims(2, 31, 24, 12, 13, 32, 16, 3, 3, 16, 8), "31 -> 24 channels, Jz = 32: fused dA + t,z at its limits"),
    # Nt = 32: a 16-plane z k-step spans two chunks; eight chunks per column
    (Dims(1, 20, 20, 16, 10, 64, 32, 4, 4, 8, 8), "width 20, 64 x 32 columns: fused dA + t,z over 8 chunks"),
]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("d,label", TRAIN_CASES, ids=[c[1] for c in TRAIN_CASES])
def test_training_forward_then_saved_backward_matches_the_oracle(d, label, precision):
    from paper_2211_12709_gb300 import _lib, ops
    modes = (d.mx, d.my, d.mz, d.mt)
    x, w, wl, b, dz = _case(d, seed=21)
    dims = ops.dims_of(x, d.Co, modes)
    try:
        _lib.fno_workspace_bytes(dims, ops.precision_code(precision), ops.OP_BLOCK_TRAIN)
    except _lib.FnoError as e:
        assert precision != "fp32" and e.status == -2
        pytest.skip(f"shape outside the tensor-core tilings: {e}")
    ws = ops.workspace(dims, precision, ops.OP_BLOCK_TRAIN, x.device)
    z = ops.block_fwd(x, w, wl, b, modes, precision, ws=ws, train=True)
    z_plain = ops.block_fwd(x, w, wl, b, modes, precision)
    z_saved = z.clone()
    ops.block_fwd(x, w, wl, b, modes, precision, ws=ws, train=True)  # the state the backward uses
    dx, dw, dwl, db = ops.block_bwd(x, w, wl, b, dz, modes, precision, ws=ws, saved=True)
    ref = ops.block_bwd(x, w, wl, b, dz, modes, precision)
    torch.cuda.synchronize()
    assert torch.equal(z_saved, z_plain)
    if precision == "fp32":
        # the FP32 epilogue forms A the same way in both modes: dA, and with it
        # dx and dw, are bitwise those of the recompute path
        assert torch.equal(dx, ref[0]) and torch.equal(dw, ref[1])
    h = lambda t: t.detach().cpu().numpy()
    rz, _ = oracle.block_fwd(d, h(x), h(w), h(wl), h(b))
    rg = oracle.block_bwd(d, h(x), h(w), h(dz), h(wl), h(b))
    errs = {"z": relerr(h(z_saved), rz), "dx": relerr(h(dx), rg["dx"]), "dw": relerr(h(dw), rg["dw"]),
            "dwl": relerr(h(dwl), rg["dwl"]), "db": relerr(h(db), rg["db"])}
    print(label, precision, errs)
    assert all(v <= TOL[precision] for v in errs.values()), errs


def test_saved_backward_is_refused_when_the_workspace_state_does_not_match():
    from paper_2211_12709_gb300 import _lib, ops
    d = CASES[0][0]
    modes = (d.mx, d.my, d.mz, d.mt)
    x, w, wl, b, dz = _case(d)
    dims = ops.dims_of(x, d.Co, modes)
    ws = ops.workspace(dims, "fp32", ops.OP_BLOCK_BWD, x.device)

    def saved(xx=x, ww=w):
        return ops.block_bwd(xx, ww, wl, b, dz, modes, "fp32", ws=ws, saved=True)

    def refused(fn):
        with pytest.raises(_lib.FnoError) as ei:
            fn()
        assert ei.value.status == -1

    refused(saved)                                   # no forward yet
    ops.block_fwd(x, w, wl, b, modes, "fp32", ws=ws)
    saved()                                          # the matching use
    refused(saved)                                   # the state is spent
    ops.block_fwd(x, w, wl, b, modes, "fp32", ws=ws)
    ops.spectral_fwd(x, w, modes, "fp32", ws=ws)     # another call on the workspace
    refused(saved)
    ops.block_fwd(x, w, wl, b, modes, "fp32", ws=ws)
    refused(lambda: saved(xx=x.clone()))             # another x
    ops.block_fwd(x, w, wl, b, modes, "fp32", ws=ws)
    refused(lambda: saved(ww=w.clone()))             # another w
    # a training forward needs the training layout, and so does the backward after it
    with pytest.raises(_lib.FnoError) as ei:
        ops.block_fwd(x, w, wl, b, modes, "fp32", ws=ws, train=True)
    assert ei.value.status == -3
    wt = ops.workspace(dims, "fp32", ops.OP_BLOCK_TRAIN, x.device)
    assert wt.numel() > ws.numel()
    ops.block_fwd(x, w, wl, b, modes, "fp32", ws=wt, train=True)
    with pytest.raises(_lib.FnoError) as ei:
        ops.block_bwd(x, w, wl, b, dz, modes, "fp32", ws=wt[:ws.numel()], saved=True)
    assert ei.value.status == -3
    torch.cuda.synchronize()


def test_autograd_block_reuses_its_forward_workspace_and_survives_a_second_backward():
    # the first backward takes GELU'(A) from the training forward; the second
    # finds the state spent and recomputes, bitwise the plain backward
    from paper_2211_12709_gb300 import ops
    d = CASES[1][0]
    modes = (d.mx, d.my, d.mz, d.mt)
    x, w, wl, b, dz = _case(d)
    X = x.clone().requires_grad_(True)
    W, WL, Bb = (t.clone().requires_grad_(True) for t in (w, wl, b))
    z = ops.FNOBlock4dFn.apply(X, W, WL, Bb, modes, "bf16x3")
    z.backward(dz, retain_graph=True)
    g1 = [t.grad.clone() for t in (X, W, WL, Bb)]
    for t in (X, W, WL, Bb):
        t.grad = None
    z.backward(dz)  # the forward state is spent: this one recomputes the spectra
    g2 = [t.grad for t in (X, W, WL, Bb)]
    ref = ops.block_bwd(x, w, wl, b, dz, modes, "bf16x3")
    torch.cuda.synchronize()
    for a, c, r in zip(g1, g2, ref):
        assert torch.equal(c, r)
        assert float((a - r).norm() / r.norm()) <= 2e-6
