"""fno_block_bwd_saved: the backward that reuses the forward's spectra.

It must give bitwise the results of fno_block_bwd (the same kernels see the
same spectra, recomputed or kept), and the library must refuse it whenever its
record of the workspace does not match: no forward, another call on the
workspace in between, another x or w, or a second use after the state is spent.
"""
import numpy as np
import pytest

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
    torch.cuda.synchronize()


def test_autograd_block_reuses_its_forward_workspace_and_survives_a_second_backward():
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
        assert torch.equal(a, r) and torch.equal(c, r)
