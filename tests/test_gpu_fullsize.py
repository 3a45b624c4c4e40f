"""Full-size parity on the benchmark workload, on sampled outputs.

The CO2-like block: B = 1, width 20, grid 128 x 128 x 128 x 32 (2.1 M cells x
32 steps), kept modes 12/12/8/8, input the same seeded anisotropic Gaussian
random field that bench.py times (correlation 20 x 20 x 4 cells, 8 steps),
upstream gradient N(0, 1).  The GPU runs, through the C ABI with one workspace,
fno_block_fwd_train + fno_block_bwd_saved (the step the benchmark times) and
fno_block_fwd + fno_block_bwd (the recompute form).  The FP64 oracle computes
the full kept spectra (Alg. 2) and evaluates Z and dX at 96 sampled grid points
(corners and edges of every axis included); dW, dW_lin and db are compared in
full.  Tolerance: rel-L2 per tensor, FP32 and split BF16 <= 1e-5, BF16 <= 2e-2,
TF32 <= 5e-3 (ten TF32-rounded operands on a path, 2^-11 each).  A second
workload, 64^3 x 16 with batch 2, runs the training step in split BF16 and
TF32 the same way (see test_training_step_at_64c_t16_full_size_sampled).
"""
import numpy as np
import pytest

import oracle
from oracle import Dims
from paper_2211_12709_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 2e-2, "tf32": 5e-3}
D = Dims(1, 20, 20, 128, 128, 128, 32, 12, 12, 8, 8)
ELL = (20.0, 20.0, 4.0, 8.0)
CFG = 4


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def sample_points(d, n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    pts = np.stack([g.integers(0, s, n) for s in d.grid], axis=1)
    edges = []
    for a, s in enumerate(d.grid):
        for v in (0, s - 1):
            p = [s2 // 2 for s2 in d.grid]
            p[a] = v
            edges.append(p)
    edges.append([0, 0, 0, 0])
    edges.append([s - 1 for s in d.grid])
    return np.concatenate([np.array(edges, dtype=np.int64), pts.astype(np.int64)])[:96]


@pytest.fixture(scope="module")
def case():
    d = D
    x = inputs.grf((d.B, d.Ci), d.grid, ELL, inputs.SEED_INPUT + CFG)
    w = inputs.spectral_weights(d.Ci, d.Co, d.modes, inputs.SEED_SPECTRAL_W + CFG)
    wl, b = inputs.linear_params(d.Ci, d.Co, inputs.SEED_LINEAR + CFG)
    dz = inputs.normal((d.B, d.Co) + d.grid, inputs.SEED_UPSTREAM + CFG)
    pts = sample_points(d, 96, 77)
    _, zp = oracle.block_fwd(d, x, w, wl, b, full=False, pts=pts)
    ref = oracle.block_bwd(d, x, w, dz, wl, b, full=False, pts=pts)
    ref["z_pts"] = zp
    return d, x, w, wl, b, dz, pts, ref


@pytest.mark.parametrize("path", ["train+saved", "recompute"])
@pytest.mark.parametrize("precision", ["bf16x3", "fp32", "bf16", "tf32"])
def test_block_fwd_bwd_full_size_sampled(case, precision, path):
    from paper_2211_12709_gb300 import _lib, ops
    d, x, w, wl, b, dz, pts, ref = case
    dev = torch.device("cuda", 0)
    X = torch.from_numpy(x).to(dev)
    DZ = torch.from_numpy(dz).to(dev)
    W = torch.from_numpy(w).to(dev)
    WL = torch.from_numpy(wl).to(dev)
    Bb = torch.from_numpy(b).to(dev)
    Z = torch.empty_like(X)
    DX = torch.empty_like(X)
    DW = torch.empty_like(W)
    DWL = torch.empty_like(WL)
    DB = torch.empty_like(Bb)
    dims = ops.dims_of(X, d.Co, (d.mx, d.my, d.mz, d.mt))
    p = ops.precision_code(precision)
    train = path == "train+saved"
    nws = _lib.fno_workspace_bytes(dims, p, ops.OP_BLOCK_TRAIN if train else ops.OP_BLOCK_BWD)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    sh = int(torch.cuda.current_stream(dev).cuda_stream)
    fwd = _lib.fno_block_fwd_train if train else _lib.fno_block_fwd
    bwd = _lib.fno_block_bwd_saved if train else _lib.fno_block_bwd
    fwd(dims, p, X.data_ptr(), W.data_ptr(), WL.data_ptr(), Bb.data_ptr(), Z.data_ptr(),
        ws.data_ptr(), nws, sh)
    bwd(dims, p, X.data_ptr(), W.data_ptr(), WL.data_ptr(), Bb.data_ptr(), DZ.data_ptr(),
        DX.data_ptr(), DW.data_ptr(), DWL.data_ptr(), DB.data_ptr(), ws.data_ptr(), nws, sh)
    _lib.fno_workspace_status(ws.data_ptr(), sh)
    torch.cuda.synchronize()
    ix = [torch.from_numpy(pts[:, a]).to(dev) for a in range(4)]
    z_pts = Z[:, :, ix[0], ix[1], ix[2], ix[3]].cpu().numpy()
    dx_pts = DX[:, :, ix[0], ix[1], ix[2], ix[3]].cpu().numpy()
    errs = {"z": relerr(z_pts, ref["z_pts"]), "dx": relerr(dx_pts, ref["dx_pts"]),
            "dw": relerr(DW.cpu().numpy(), ref["dw"]), "dwl": relerr(DWL.cpu().numpy(), ref["dwl"]),
            "db": relerr(DB.cpu().numpy(), ref["db"])}
    print("128^3x32 width 20", precision, path, errs)
    assert all(np.isfinite(v) and v <= TOL[precision] for v in errs.values()), errs


# The small benchmark workload at its full size: B = 2, width 20, 64^3 x 16,
# modes 8/8/8/6.  Nt = 16 gives the fused dA + t,z pass two 8-plane n-tiles per
# 256-point chunk and four chunks per column, with batch 2 (8192 columns over
# the CTAs), where the 128^3 x 32 case has one n-tile per chunk and batch 1.
D_NS = Dims(2, 20, 20, 64, 64, 64, 16, 8, 8, 8, 6)


@pytest.fixture(scope="module")
def case_ns():
    d = D_NS
    x = inputs.normal((d.B, d.Ci) + d.grid, inputs.SEED_INPUT + 7)
    w = inputs.spectral_weights(d.Ci, d.Co, d.modes, inputs.SEED_SPECTRAL_W + 7)
    wl, b = inputs.linear_params(d.Ci, d.Co, inputs.SEED_LINEAR + 7)
    dz = inputs.normal((d.B, d.Co) + d.grid, inputs.SEED_UPSTREAM + 7)
    pts = sample_points(d, 96, 78)
    _, zp = oracle.block_fwd(d, x, w, wl, b, full=False, pts=pts)
    ref = oracle.block_bwd(d, x, w, dz, wl, b, full=False, pts=pts)
    ref["z_pts"] = zp
    return d, x, w, wl, b, dz, pts, ref


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
def test_training_step_at_64c_t16_full_size_sampled(case_ns, precision):
    from paper_2211_12709_gb300 import _lib, ops
    d, x, w, wl, b, dz, pts, ref = case_ns
    dev = torch.device("cuda", 0)
    X, DZ, W, WL, Bb = (torch.from_numpy(a).to(dev) for a in (x, dz, w, wl, b))
    Z, DX, DW, DWL, DB = (torch.empty_like(t) for t in (X, X, W, WL, Bb))
    dims = ops.dims_of(X, d.Co, (d.mx, d.my, d.mz, d.mt))
    p = ops.precision_code(precision)
    nws = _lib.fno_workspace_bytes(dims, p, ops.OP_BLOCK_TRAIN)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    sh = int(torch.cuda.current_stream(dev).cuda_stream)
    _lib.fno_block_fwd_train(dims, p, X.data_ptr(), W.data_ptr(), WL.data_ptr(), Bb.data_ptr(), Z.data_ptr(),
                             ws.data_ptr(), nws, sh)
    _lib.fno_block_bwd_saved(dims, p, X.data_ptr(), W.data_ptr(), WL.data_ptr(), Bb.data_ptr(), DZ.data_ptr(),
                             DX.data_ptr(), DW.data_ptr(), DWL.data_ptr(), DB.data_ptr(), ws.data_ptr(), nws, sh)
    _lib.fno_workspace_status(ws.data_ptr(), sh)  # raises if a bounded wait gave up
    torch.cuda.synchronize()
    ix = [torch.from_numpy(pts[:, a]).to(dev) for a in range(4)]
    z_pts = Z[:, :, ix[0], ix[1], ix[2], ix[3]].cpu().numpy()
    dx_pts = DX[:, :, ix[0], ix[1], ix[2], ix[3]].cpu().numpy()
    errs = {"z": relerr(z_pts, ref["z_pts"]), "dx": relerr(dx_pts, ref["dx_pts"]),
            "dw": relerr(DW.cpu().numpy(), ref["dw"]), "dwl": relerr(DWL.cpu().numpy(), ref["dwl"]),
            "db": relerr(DB.cpu().numpy(), ref["db"])}
    print("64^3x16 B=2 width 20", precision, errs)
    assert all(np.isfinite(v) and v <= TOL[precision] for v in errs.values()), errs
