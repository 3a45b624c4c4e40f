"""Tensor-core precisions (BF16, split BF16, TF32) of the CUDA path vs the FP64 oracle.

Tolerances (rel-L2 per tensor): split BF16 <= 1e-5, BF16 <= 2e-2.  TF32 has no
stated bound; each TF32-rounded operand carries at most 2^-11 ~ 4.9e-4 relative
error and about ten rounded operands lie on the path to any output (four
forward DFT stages, four inverse, the 1x1 and its weight), so the test bound is
10 * 2^-11 ~ 5e-3.  Every call also checks the device status word: no bounded
device-side wait gave up.
"""
import numpy as np
import pytest

import oracle
from oracle import Dims
from paper_2211_12709_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-5, "bf16": 2e-2, "tf32": 5e-3}


@pytest.fixture(autouse=True)
def _check_status():
    from paper_2211_12709_gb300 import ops
    old = ops.CHECK_STATUS
    ops.CHECK_STATUS = True
    yield
    ops.CHECK_STATUS = old


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def make_case(d, cfg, field="normal"):
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


TC_CASES = [
    (Dims(1, 8, 8, 16, 16, 16, 8, 4, 4, 4, 4), "single-layer 16^3x8"),
    (Dims(3, 5, 7, 12, 10, 32, 16, 3, 2, 8, 6), "Ci!=Co, Nz=32, Nt=16, ragged column groups"),
    (Dims(2, 17, 9, 6, 5, 64, 32, 2, 2, 12, 8), "17->9 channels, Nz=64, Nt=32, 2mz=24"),
    (Dims(1, 3, 4, 4, 4, 128, 8, 1, 1, 3, 5), "Nz=128, Nt=8, mt=Nt/2+1 (Nyquist)"),
    (Dims(2, 20, 20, 8, 8, 16, 16, 2, 3, 8, 3), "Nz=16 (8 columns per tile), 2mz=Nz"),
    (Dims(1, 32, 32, 6, 4, 16, 32, 2, 2, 4, 8), "32 channels: two dW_lin tiles per warp"),
    # single channels on either side of the 1x1; with C_in = C_out = 1 and this
    # seed db is one sum of 24576 terms that cancels to 0.72 (sum |dA| ~ 1e4), a
    # conditioning test of the sum rather than of the kernel, so the edge is
    # covered by 1 -> 2 and 2 -> 1 channels instead
    (Dims(2, 1, 2, 4, 6, 32, 16, 2, 3, 5, 8), "one input channel, mt = Nt/2"),
    (Dims(2, 2, 1, 4, 6, 32, 16, 2, 3, 5, 8), "one output channel, mt = Nt/2"),
    # forward t,z kernel shapes: a 32 KB column staged in two chunks, three z
    # m-tiles on a non-power-of-two Nz, and a half-empty (masked) t k-step
    (Dims(1, 3, 3, 4, 4, 128, 64, 1, 1, 5, 8), "Nz=128, Nt=64: each column in two staged chunks"),
    (Dims(1, 2, 3, 4, 4, 96, 16, 1, 2, 20, 4), "Nz=96, 2mz=40: three z m-tiles"),
    (Dims(2, 2, 2, 4, 4, 32, 24, 1, 1, 4, 6), "Nt=24: the second t k-step half masked"),
    # non-power-of-two grids like the paper's data (262 x 118 x 64 x 86 and
    # 130^3 x 84): masked z and t tails, Nt % 4 = 2 (8-byte rows), uneven chunks
    (Dims(1, 3, 3, 6, 5, 26, 22, 2, 2, 5, 6), "Nz=26, Nt=22: masked z and t tails"),
    (Dims(1, 2, 3, 4, 3, 64, 86, 1, 1, 6, 8), "Nz=64, Nt=86 (the CO2 data's z, t): two chunks"),
    (Dims(1, 2, 2, 3, 4, 130, 84, 1, 1, 12, 8), "Nz=130, Nt=84 (the NS data's z, t): chunks 48/48/34"),
    # more channels than the fused tensor-core epilogue takes (32): that stage
    # runs on the FP32 kernels, the t,z, line and mixing stages stay on theirs
    (Dims(2, 40, 48, 6, 4, 16, 16, 2, 2, 4, 6), "40 -> 48 channels: FP32 epilogue beside tensor-core stages"),
    (Dims(1, 64, 64, 6, 5, 8, 8, 2, 2, 3, 3), "64 -> 64 channels (the limit), Nz = Nt = 8"),
]


@pytest.mark.parametrize("d,label", TC_CASES, ids=[c[1] for c in TC_CASES])
@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "tf32"])
def test_tc_block_matches_oracle(d, label, precision):
    from paper_2211_12709_gb300 import ops
    x, w, wl, b, dz = make_case(d, 11)
    X, W, WL, Bb, DZ = gpu(x), gpu(w), gpu(wl), gpu(b), gpu(dz)
    z = ops.block_fwd(X, W, WL, Bb, modes_of(d), precision)
    dx, dw, dwl, db = ops.block_bwd(X, W, WL, Bb, DZ, modes_of(d), precision)
    torch.cuda.synchronize()
    rz, _ = oracle.block_fwd(d, x, w, wl, b)
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    errs = {"z": relerr(host(z), rz), "dx": relerr(host(dx), rg["dx"]),
            "dw": relerr(host(dw), rg["dw"]), "dwl": relerr(host(dwl), rg["dwl"]),
            "db": relerr(host(db), rg["db"])}
    print(label, precision, errs)
    assert all(v <= TOL[precision] for v in errs.values()), errs


@pytest.mark.parametrize("d,label", TC_CASES[:3], ids=[c[1] for c in TC_CASES[:3]])
@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "tf32"])
def test_tc_spectral_conv_matches_oracle(d, label, precision):
    from paper_2211_12709_gb300 import ops
    x, w, _, _, dy = make_case(d, 12)
    X, W, DY = gpu(x), gpu(w), gpu(dy)
    y = ops.spectral_fwd(X, W, modes_of(d), precision)
    dx, dw = ops.spectral_bwd(X, W, DY, modes_of(d), True, True, precision)
    torch.cuda.synchronize()
    ry, _ = oracle.block_fwd(d, x, w)
    rg = oracle.block_bwd(d, x, w, dy)
    errs = {"y": relerr(host(y), ry), "dx": relerr(host(dx), rg["dx"]), "dw": relerr(host(dw), rg["dw"])}
    print(label, precision, errs)
    assert all(v <= TOL[precision] for v in errs.values()), errs


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "tf32"])
def test_tc_full_block_grf_64cube(precision):
    # 2 x 20 channels of a 64^3 x 16 smooth GRF (correlation 8 cells), modes 8/8/8/6
    from paper_2211_12709_gb300 import ops
    d = Dims(2, 20, 20, 64, 64, 64, 16, 8, 8, 8, 6)
    x, w, wl, b, dz = make_case(d, 2, field="grf")
    X, W, WL, Bb, DZ = gpu(x), gpu(w), gpu(wl), gpu(b), gpu(dz)
    z = ops.block_fwd(X, W, WL, Bb, modes_of(d), precision)
    dx, dw, dwl, db = ops.block_bwd(X, W, WL, Bb, DZ, modes_of(d), precision)
    torch.cuda.synchronize()
    rz, _ = oracle.block_fwd(d, x, w, wl, b)
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    errs = {"z": relerr(host(z), rz), "dx": relerr(host(dx), rg["dx"]),
            "dw": relerr(host(dw), rg["dw"]), "dwl": relerr(host(dwl), rg["dwl"]),
            "db": relerr(host(db), rg["db"])}
    print("64^3x16 block errors", precision, errs)
    assert all(v <= TOL[precision] for v in errs.values()), errs


def test_tc_unsupported_shapes_are_refused_not_run():
    from paper_2211_12709_gb300 import _lib, ops
    # odd Nt (rows of the staged column would not be 8-byte aligned)
    x = torch.zeros((1, 2, 8, 8, 12, 7), device="cuda")
    w = torch.zeros((2, 2, 4, 4, 4, 3, 2), device="cuda")
    with pytest.raises(_lib.FnoError) as ei:
        ops.spectral_fwd(x, w, (2, 2, 2, 3), "bf16x3")
    assert ei.value.status == -2
    # mt > 8 (the t stage keeps at most 8 kt rows in its m-tile)
    x = torch.zeros((1, 2, 8, 8, 16, 20), device="cuda")
    w = torch.zeros((2, 2, 4, 4, 4, 9, 2), device="cuda")
    with pytest.raises(_lib.FnoError) as ei:
        ops.spectral_fwd(x, w, (2, 2, 2, 9), "bf16x3")
    assert ei.value.status == -2


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "tf32"])
def test_paper_nt_runs_the_tensor_core_synthesis_path(precision):
    # Nt = 86 (the CO2 data's t axis) is outside the fused epilogues' tiling:
    # the forward and dX epilogues take the inverse-t synthesis kernel and the
    # in-place pointwise pass, and still match the oracle
    from paper_2211_12709_gb300 import _lib, ops
    d = Dims(1, 3, 4, 4, 3, 20, 86, 1, 1, 4, 8)
    x, w, wl, b, dz = make_case(d, 13)
    X, W, WL, Bb, DZ = gpu(x), gpu(w), gpu(wl), gpu(b), gpu(dz)
    torch.cuda.synchronize()
    _lib.fno_profile_start()
    z = ops.block_fwd(X, W, WL, Bb, modes_of(d), precision)
    dx, dw, dwl, db = ops.block_bwd(X, W, WL, Bb, DZ, modes_of(d), precision)
    torch.cuda.synchronize()
    prof = _lib.fno_profile_stop()
    names = set(prof)
    assert f"fno_synth_t_{precision}" in names, names
    assert "fno_pw_add_fwd" in names and "fno_pw_add_dx" in names, names
    rz, _ = oracle.block_fwd(d, x, w, wl, b)
    rg = oracle.block_bwd(d, x, w, dz, wl, b)
    errs = {"z": relerr(host(z), rz), "dx": relerr(host(dx), rg["dx"]),
            "dw": relerr(host(dw), rg["dw"]), "dwl": relerr(host(dwl), rg["dwl"]),
            "db": relerr(host(db), rg["db"])}
    assert all(v <= TOL[precision] for v in errs.values()), errs
