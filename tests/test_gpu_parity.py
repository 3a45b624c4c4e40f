"""CUDA path (through the C ABI) vs the FP64 oracle, element by element.

Every input comes from the seeded generators of paper_2211_12709_gb300.inputs;
every expected value comes from oracle/.  Tolerance: rel-L2 <= 1e-5 per tensor
(Z or y, dX, dW, dW_lin, db) for the FP32 plain form.
"""
import numpy as np
import pytest

import oracle
from oracle import Dims
from paper_2211_12709_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5}


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def make_case(d: Dims, cfg: int, field="normal"):
    if field == "grf":
        x = inputs.grf((d.B, d.Ci), d.grid, (8.0, 8.0, 8.0, 8.0), inputs.SEED_INPUT + cfg)
    else:
        x = inputs.normal((d.B, d.Ci) + d.grid, inputs.SEED_INPUT + cfg)
    w = inputs.spectral_weights(d.Ci, d.Co, d.modes, inputs.SEED_SPECTRAL_W + cfg)
    wl, b = inputs.linear_params(d.Ci, d.Co, inputs.SEED_LINEAR + cfg)
    dz = inputs.normal((d.B, d.Co) + d.grid, inputs.SEED_UPSTREAM + cfg)
    return x, w, wl, b, dz


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy() if t is not None else None


def modes_of(d):
    return (d.mx, d.my, d.mz, d.mt)


def run_block(d, x, w, wl, b, dz, precision):
    from paper_2211_12709_gb300 import ops
    X, W, WL, Bb, DZ = gpu(x), gpu(w), gpu(wl), gpu(b), gpu(dz)
    z = ops.block_fwd(X, W, WL, Bb, modes_of(d), precision)
    dx, dw, dwl, db = ops.block_bwd(X, W, WL, Bb, DZ, modes_of(d), precision)
    torch.cuda.synchronize()
    return host(z), host(dx), host(dw), host(dwl), host(db)


def run_spectral(d, x, w, dy, precision):
    from paper_2211_12709_gb300 import ops
    X, W, DY = gpu(x), gpu(w), gpu(dy)
    y = ops.spectral_fwd(X, W, modes_of(d), precision)
    dx, dw = ops.spectral_bwd(X, W, DY, modes_of(d), True, True, precision)
    torch.cuda.synchronize()
    return host(y), host(dx), host(dw)


SMALL = [
    # (dims, label)
    (Dims(1, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4), "single-layer 16^3x8"),
    (Dims(3, 5, 7, 12, 10, 9, 6, 3, 2, 4, 4), "ragged: odd Nz, Nt%4!=0... Nt=6, mt=Nt/2+1, Ci!=Co"),
    (Dims(2, 3, 3, 8, 6, 10, 7, 4, 3, 5, 3), "2m = N on every spatial axis, odd Nt"),
    (Dims(1, 2, 4, 5, 7, 3, 12, 1, 2, 1, 7), "tiny odd grid, mt = Nt/2+1 with Nyquist"),
    (Dims(2, 17, 9, 20, 8, 40, 8, 5, 3, 7, 2), "tails: 17 channels, Nz=40"),
    (Dims(10, 3, 2, 8, 6, 8, 4, 2, 2, 2, 2), "batch of 10: two batch chunks in the mixing"),
    # the dW_lin/db reduction works on 4x4 (input + ones row, output) blocks,
    # one per thread of a 128-thread CTA up to 128 blocks; past that threads
    # own several: 11 x 12 = 132 blocks, and 17 x 16 = 272 at the 64-channel limit
    (Dims(2, 40, 48, 6, 4, 16, 16, 2, 2, 4, 6), "40 -> 48 channels: 132 dW_lin blocks"),
    (Dims(1, 64, 64, 6, 5, 8, 8, 2, 2, 3, 3), "64 -> 64 channels (the limit): 272 dW_lin blocks"),
    # the epilogue tiles each (b, x, y) column in runs of 128 points: with Nt
    # not dividing 128 they start and end inside z-planes, with Nt > 128 a
    # tile is part of one plane
    (Dims(2, 3, 4, 4, 3, 20, 22, 2, 1, 5, 6), "Nt=22: tiles start inside z-planes"),
    (Dims(1, 3, 2, 4, 4, 4, 160, 1, 1, 2, 7), "Nt=160 > 128: a tile is part of a plane"),
    (Dims(1, 2, 3, 4, 4, 6, 40, 1, 1, 3, 16), "mt=16, the most t modes the epilogue takes"),
]


@pytest.mark.parametrize("d,label", SMALL, ids=[s[1] for s in SMALL])
@pytest.mark.parametrize("precision", ["fp32"])
def test_spectral_conv_matches_oracle(d, label, precision):
    x, w, _, _, dy = make_case(d, 1)
    y, dx, dw = run_spectral(d, x, w, dy, precision)
    ry, _ = oracle.block_fwd(d, x, w)
    rg = oracle.block_bwd(d, x, w, dy)
    tol = TOL[precision]
    assert relerr(y, ry) <= tol, relerr(y, ry)
    assert relerr(dx, rg["dx"]) <= tol, relerr(dx, rg["dx"])
    assert relerr(dw, rg["dw"]) <= tol, relerr(dw, rg["dw"])


@pytest.mark.parametrize("d,label", SMALL, ids=[s[1] for s in SMALL])
@pytest.mark.parametrize("precision", ["fp32"])
def test_block_matches_oracle(d, label, precision):
    x, w, wl, b, dz = make_case(d, 2)
    z, dx, dw, dwl, db = run_block(d, x, w, wl, b, dz, precision)
    rz, _ = oracle.block_fwd(d, x, w, wl, b)
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    tol = TOL[precision]
    errs = {"z": relerr(z, rz), "dx": relerr(dx, rg["dx"]), "dw": relerr(dw, rg["dw"]),
            "dwl": relerr(dwl, rg["dwl"]), "db": relerr(db, rg["db"])}
    assert all(v <= tol for v in errs.values()), errs


@pytest.mark.parametrize("precision", ["fp32"])
def test_full_block_grf_64cube_matches_oracle(precision):
    # block on 2 x 20 channels of a 64^3 x 16 smooth GRF (correlation 8 cells), modes 8/8/8/6
    d = Dims(2, 20, 20, 64, 64, 64, 16, 8, 8, 8, 6)
    x, w, wl, b, dz = make_case(d, 2, field="grf")
    z, dx, dw, dwl, db = run_block(d, x, w, wl, b, dz, precision)
    rz, _ = oracle.block_fwd(d, x, w, wl, b)
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    tol = TOL[precision]
    errs = {"z": relerr(z, rz), "dx": relerr(dx, rg["dx"]), "dw": relerr(dw, rg["dw"]),
            "dwl": relerr(dwl, rg["dwl"]), "db": relerr(db, rg["db"])}
    print("64^3x16 block errors", precision, errs)
    assert all(v <= tol for v in errs.values()), errs


def test_autograd_function_matches_direct_calls():
    from paper_2211_12709_gb300 import ops
    d = Dims(2, 4, 4, 8, 8, 8, 8, 2, 2, 2, 3)
    x, w, wl, b, dz = make_case(d, 5)
    X = gpu(x).requires_grad_(True)
    W = gpu(w).requires_grad_(True)
    WL = gpu(wl).requires_grad_(True)
    Bb = gpu(b).requires_grad_(True)
    z = ops.FNOBlock4dFn.apply(X, W, WL, Bb, modes_of(d), "fp32")
    z.backward(gpu(dz))
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    assert relerr(host(X.grad), rg["dx"]) <= 1e-5
    assert relerr(host(W.grad), rg["dw"]) <= 1e-5
    assert relerr(host(WL.grad), rg["dwl"]) <= 1e-5
    assert relerr(host(Bb.grad), rg["db"]) <= 1e-5
    # two stacked blocks: the autograd graph keeps only the block inputs
    blk1 = ops.FNOBlock4d(4, modes_of(d), device="cuda", seed=1)
    blk2 = ops.FNOBlock4d(4, modes_of(d), device="cuda", seed=2)
    out = blk2(blk1(gpu(x)))
    out.square().mean().backward()
    assert torch.isfinite(blk1.weight.grad).all() and blk1.weight.grad.abs().sum() > 0


def test_empty_batch_gives_empty_outputs_and_zero_gradients():
    from paper_2211_12709_gb300 import ops
    d = Dims(0, 3, 2, 8, 8, 8, 8, 2, 2, 2, 3)
    x = torch.zeros((0, 3, 8, 8, 8, 8), device="cuda")
    w = gpu(inputs.spectral_weights(3, 2, d.modes, 7))
    wl, b = (gpu(a) for a in inputs.linear_params(3, 2, 7))
    z = ops.block_fwd(x, w, wl, b, modes_of(d))
    assert z.shape == (0, 2, 8, 8, 8, 8)
    dx, dw, dwl, db = ops.block_bwd(x, w, wl, b, torch.zeros((0, 2, 8, 8, 8, 8), device="cuda"),
                                    modes_of(d))
    torch.cuda.synchronize()
    assert dx.shape == x.shape
    assert float(dw.abs().sum()) == 0.0 and float(dwl.abs().sum()) == 0.0 and float(db.abs().sum()) == 0.0


def test_repeated_calls_are_bitwise_deterministic():
    d = Dims(2, 6, 6, 16, 12, 16, 8, 4, 3, 4, 4)
    x, w, wl, b, dz = make_case(d, 6)
    a = run_block(d, x, w, wl, b, dz, "fp32")
    c = run_block(d, x, w, wl, b, dz, "fp32")
    for u, v in zip(a, c):
        assert np.array_equal(u, v)


def test_workspace_status_word_reports_timeout_and_misalignment_codes():
    # The status word at the start of the workspace is what a kernel sets when a
    # bounded wait gives up (1) or its shared window is misaligned (2); planting
    # the codes by hand checks the host-side reporting without any kernel failing.
    from paper_2211_12709_gb300 import _lib
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    status = ws.view(torch.int32)
    _lib.fno_workspace_status(ws.data_ptr(), 0)                 # 0: OK
    status[0] = 1
    with pytest.raises(_lib.FnoError) as ei:
        _lib.fno_workspace_status(ws.data_ptr(), 0)
    assert ei.value.status == -5                                # FNO_ERR_TIMEOUT
    status[0] = 2
    with pytest.raises(_lib.FnoError) as ei:
        _lib.fno_workspace_status(ws.data_ptr(), 0)
    assert ei.value.status == -4                                # FNO_ERR_CUDA
