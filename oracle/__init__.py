"""FP64 CPU oracle of the 4-D spectral FNO block (Alg. 2, Sec. IV-C of the paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it; the two share no code.

The arithmetic lives in ``fno_oracle.c`` (plain separable direct summation in
FP64, OpenMP over independent rows); this module only compiles it with the host
``gcc`` and marshals NumPy arrays through ``ctypes``.

Array conventions (all C-contiguous):
  x, dz        [B][Ci|Co][Nx][Ny][Nz][Nt]   float32 or float64
  w            [Ci][Co][2mx][2my][2mz][mt][2]  (re, im)
  wl, bias     [Ci][Co], [Co]
  spectra      [..][2mx][2my][2mz][mt][2]   float64
Stored mode index j < m maps to frequency j, j >= m to j - 2m (x, y, z);
the t axis keeps kt = 0..mt-1.

The layers around the blocks in Alg. 1 (encoder and decoder pointwise 1x1
layers with sigma, the mean-squared-error loss) and the composed stack are
``pointwise_fwd``, ``pointwise_bwd``, ``mse`` and ``stack_loss_and_grads``; the
Adam update of a training step is ``adam``.

Parity notes: every routine is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute-force 4-D sums, NumPy ``rfftn``/``irfftn``,
identity, projector/Parseval, shift equivariance, plane waves, adjoint
dot-products and central finite differences) and ``tests/test_oracle_stack_pins.py``
(the pointwise layers and the loss against PyTorch's CPU ``linear``/``gelu``/
``mse_loss`` and its autograd, the whole stack against a PyTorch ``rfftn``
model and against central finite differences).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fno_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_F64P = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle with the host C compiler (portable flags, no -march).

    ``mutant`` > 0 builds a copy with one planted slip (see ORACLE_MUTANT in
    fno_oracle.c); only the mutation tests ask for one.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    so = _SO if mutant == 0 else os.path.join(_OUT_DIR, f"liboracle_mutant{int(mutant)}.so")
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def mutant(k: int):
    """Run the enclosed calls on a build with planted slip k (mutation tests only)."""
    global _lib
    lib = _bind(ctypes.CDLL(build(mutant=k)))
    with _lock:
        old = _lib
        _lib = lib
    try:
        yield
    finally:
        with _lock:
            _lib = old


def _bind(lib):
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    lib.oracle_threads.argtypes = [ci]
    lib.oracle_threads.restype = ci
    lib.oracle_gelu.argtypes = [ctypes.c_double]
    lib.oracle_gelu.restype = ctypes.c_double
    lib.oracle_gelu_grad.argtypes = [ctypes.c_double]
    lib.oracle_gelu_grad.restype = ctypes.c_double
    for name in ("oracle_spectrum", "oracle_spectrum_bruteforce"):
        fn = getattr(lib, name)
        fn.argtypes = [_I64P, i64, vp, vp, ci]
        fn.restype = ci
    for name in ("oracle_synthesis", "oracle_synthesis_bruteforce"):
        fn = getattr(lib, name)
        fn.argtypes = [_I64P, i64, vp, vp, ci]
        fn.restype = ci
    lib.oracle_synthesis_points.argtypes = [_I64P, i64, vp, i64, vp, vp, ci]
    lib.oracle_synthesis_points.restype = ci
    lib.oracle_mix.argtypes = [_I64P, vp, vp, vp]
    lib.oracle_mix.restype = ci
    lib.oracle_mix_adjoint.argtypes = [_I64P, vp, vp, vp, vp, vp]
    lib.oracle_mix_adjoint.restype = ci
    lib.oracle_block_fwd.argtypes = [_I64P, ci, ci, vp, vp, vp, vp, vp, i64, vp, vp]
    lib.oracle_block_fwd.restype = ci
    lib.oracle_block_bwd.argtypes = [_I64P, ci, ci, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp,
                                     vp, vp]
    lib.oracle_block_bwd.restype = ci
    lib.oracle_pointwise_fwd.argtypes = [i64, i64, i64, i64, ci, ci, vp, vp, vp, vp]
    lib.oracle_pointwise_fwd.restype = ci
    lib.oracle_pointwise_bwd.argtypes = [i64, i64, i64, i64, ci, ci, vp, vp, vp, vp, vp, vp, vp]
    lib.oracle_pointwise_bwd.restype = ci
    lib.oracle_mse.argtypes = [i64, ci, vp, vp, vp, vp]
    lib.oracle_mse.restype = ci
    dbl = ctypes.c_double
    lib.oracle_adam.argtypes = [i64, ci, vp, vp, vp, vp, dbl, dbl, dbl, dbl, i64]
    lib.oracle_adam.restype = ci
    return lib


class Dims:
    """B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt of one block."""

    __slots__ = ("B", "Ci", "Co", "Nx", "Ny", "Nz", "Nt", "mx", "my", "mz", "mt")

    def __init__(self, B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt):
        for k, v in zip(self.__slots__, (B, Ci, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt)):
            setattr(self, k, int(v))

    def array(self):
        return np.array([getattr(self, k) for k in self.__slots__], dtype=np.int64)

    @property
    def grid(self):
        return (self.Nx, self.Ny, self.Nz, self.Nt)

    @property
    def modes(self):
        return (2 * self.mx, 2 * self.my, 2 * self.mz, self.mt)

    @property
    def n_grid(self):
        return self.Nx * self.Ny * self.Nz * self.Nt

    @property
    def n_modes(self):
        return 4 * self.mx * 2 * self.my * self.mz * self.mt

    def __repr__(self):
        return "Dims(" + ", ".join(f"{k}={getattr(self, k)}" for k in self.__slots__) + ")"


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _dptr(d):
    arr = d.array()
    return arr, arr.ctypes.data_as(_I64P)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return _load().oracle_threads(int(n))


def gelu(a: float) -> float:
    return _load().oracle_gelu(float(a))


def gelu_grad(a: float) -> float:
    return _load().oracle_gelu_grad(float(a))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def spectrum(d: Dims, f, adjoint_scale=False, brute_force=False):
    """Kept-mode spectrum of real channels f[..., Nx, Ny, Nz, Nt] -> [..., Jx, Jy, Jz, Jt] complex128."""
    f = _c64(f)
    lead = f.shape[:-4]
    assert f.shape[-4:] == d.grid, (f.shape, d.grid)
    nch = int(np.prod(lead)) if lead else 1
    out = np.empty(lead + d.modes + (2,), dtype=np.float64)
    keep, dp = _dptr(d)
    fn = _load().oracle_spectrum_bruteforce if brute_force else _load().oracle_spectrum
    _check(fn(dp, nch, _ptr(f), _ptr(out), int(bool(adjoint_scale))), "spectrum")
    return out[..., 0] + 1j * out[..., 1]


def _cplx_in(s, d):
    s = np.asarray(s)
    assert s.shape[-4:] == d.modes, (s.shape, d.modes)
    return np.ascontiguousarray(np.stack([s.real, s.imag], axis=-1), dtype=np.float64)


def synthesis(d: Dims, sp, scaled=True, brute_force=False):
    """Real field of kept spectra sp[..., Jx, Jy, Jz, Jt] (complex) -> [..., Nx, Ny, Nz, Nt]."""
    a = _cplx_in(sp, d)
    lead = a.shape[:-5]
    nch = int(np.prod(lead)) if lead else 1
    out = np.empty(lead + d.grid, dtype=np.float64)
    keep, dp = _dptr(d)
    fn = _load().oracle_synthesis_bruteforce if brute_force else _load().oracle_synthesis
    _check(fn(dp, nch, _ptr(a), _ptr(out), int(bool(scaled))), "synthesis")
    return out


def synthesis_points(d: Dims, sp, pts, scaled=True):
    """The synthesis at points pts[n, 4] = (x, y, z, t): returns [..., n]."""
    a = _cplx_in(sp, d)
    lead = a.shape[:-5]
    nch = int(np.prod(lead)) if lead else 1
    pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 4)
    out = np.empty(lead + (pts.shape[0],), dtype=np.float64)
    keep, dp = _dptr(d)
    _check(_load().oracle_synthesis_points(dp, nch, _ptr(a), pts.shape[0], _ptr(pts), _ptr(out),
                                           int(bool(scaled))), "synthesis_points")
    return out


def mix(d: Dims, xh, w):
    """Yh[b,o,j] = sum_i Xh[b,i,j] W[i,o,j] (complex arrays)."""
    a = _cplx_in(xh, d)
    ww = _cplx_in(w, d)
    out = np.empty((d.B, d.Co) + d.modes + (2,), dtype=np.float64)
    keep, dp = _dptr(d)
    _check(_load().oracle_mix(dp, _ptr(a), _ptr(ww), _ptr(out)), "mix")
    return out[..., 0] + 1j * out[..., 1]


def mix_adjoint(d: Dims, xh, w, g):
    """(dW, GXh) of the spectral convolution for the mode gradient g[b,o,j]."""
    a = _cplx_in(xh, d)
    ww = _cplx_in(w, d)
    gg = _cplx_in(g, d)
    dw = np.empty((d.Ci, d.Co) + d.modes + (2,), dtype=np.float64)
    gx = np.empty((d.B, d.Ci) + d.modes + (2,), dtype=np.float64)
    keep, dp = _dptr(d)
    _check(_load().oracle_mix_adjoint(dp, _ptr(a), _ptr(ww), _ptr(gg), _ptr(dw), _ptr(gx)),
           "mix_adjoint")
    return dw[..., 0] + 1j * dw[..., 1], gx[..., 0] + 1j * gx[..., 1]


def _inputs(dtype, *arrs):
    np_t = np.float32 if dtype == 0 else np.float64
    return [None if a is None else np.ascontiguousarray(a, dtype=np_t) for a in arrs]


def _dtype_of(x):
    return 0 if np.asarray(x).dtype == np.float32 else 1


def block_fwd(d: Dims, x, w, wl=None, bias=None, full=True, pts=None):
    """Block forward (wl, bias given) or the spectral convolution alone.

    x is float32 or float64 (all inputs are cast to x's precision);
    w is real [Ci][Co][Jx][Jy][Jz][Jt][2].  Returns (z_full or None, z_pts or None).
    """
    dt = _dtype_of(x)
    x, w, wl, bias = _inputs(dt, x, w, wl, bias)
    with_lin = wl is not None
    z = np.empty((d.B, d.Co) + d.grid, dtype=np.float64) if full else None
    npts = 0
    zp = None
    pp = None
    if pts is not None:
        pp = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 4)
        npts = pp.shape[0]
        zp = np.empty((d.B, d.Co, npts), dtype=np.float64)
    keep, dp = _dptr(d)
    _check(_load().oracle_block_fwd(dp, int(with_lin), dt, _ptr(x), _ptr(w), _ptr(wl), _ptr(bias),
                                    _ptr(z), npts, _ptr(pp), _ptr(zp)), "block_fwd")
    return z, zp


def block_bwd(d: Dims, x, w, dz, wl=None, bias=None, full=True, pts=None):
    """Gradient of the block (wl, bias given) or of the spectral convolution alone.

    Returns dict with dx (full or None), dx_pts (or None), dw (real, [..][2]),
    dwl, db (None without the linear part).
    """
    dt = _dtype_of(x)
    x, w, wl, bias, dz = _inputs(dt, x, w, wl, bias, dz)
    with_lin = wl is not None
    dx = np.empty((d.B, d.Ci) + d.grid, dtype=np.float64) if full else None
    dw = np.empty((d.Ci, d.Co) + d.modes + (2,), dtype=np.float64)
    dwl = np.empty((d.Ci, d.Co), dtype=np.float64) if with_lin else None
    db = np.empty((d.Co,), dtype=np.float64) if with_lin else None
    npts = 0
    pp = None
    dxp = None
    if pts is not None:
        pp = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 4)
        npts = pp.shape[0]
        dxp = np.empty((d.B, d.Ci, npts), dtype=np.float64)
    keep, dp = _dptr(d)
    _check(_load().oracle_block_bwd(dp, int(with_lin), dt, _ptr(x), _ptr(w), _ptr(wl), _ptr(bias),
                                    _ptr(dz), _ptr(dx), npts, _ptr(pp), _ptr(dxp), _ptr(dw),
                                    _ptr(dwl), _ptr(db)), "block_bwd")
    return {"dx": dx, "dx_pts": dxp, "dw": dw, "dwl": dwl, "db": db}


# ---------------------------------------------------------------------------
# Layers around the blocks (Alg. 1) and the composed stack
# ---------------------------------------------------------------------------
def pointwise_fwd(x, w, bias=None, act=1):
    """Y[b,o,p] = sigma(sum_i X[b,i,p] W[i,o] + bias[o]) for x [B, Ci, *grid], w [Ci, Co].

    act 0 = identity, 1 = GELU.  Returns float64 [B, Co, *grid].
    """
    dt = _dtype_of(x)
    x, w, bias = _inputs(dt, x, w, bias)
    B, Ci = x.shape[:2]
    grid = x.shape[2:]
    P = int(np.prod(grid)) if grid else 1
    Co = w.shape[1]
    assert w.shape == (Ci, Co), (w.shape, Ci)
    y = np.empty((B, Co) + tuple(grid), dtype=np.float64)
    _check(_load().oracle_pointwise_fwd(B, Ci, Co, P, int(act), dt, _ptr(x), _ptr(w), _ptr(bias),
                                        _ptr(y)), "pointwise_fwd")
    return y


def pointwise_bwd(x, w, dy, bias=None, act=1, need_dx=True):
    """Gradient of ``pointwise_fwd`` for upstream dy: dict with dx (or None), dw, db."""
    dt = _dtype_of(x)
    x, w, bias, dy = _inputs(dt, x, w, bias, dy)
    B, Ci = x.shape[:2]
    grid = x.shape[2:]
    P = int(np.prod(grid)) if grid else 1
    Co = w.shape[1]
    assert dy.shape == (B, Co) + tuple(grid), (dy.shape, x.shape, w.shape)
    dx = np.empty(x.shape, dtype=np.float64) if need_dx else None
    dw = np.empty((Ci, Co), dtype=np.float64)
    db = np.empty((Co,), dtype=np.float64)
    _check(_load().oracle_pointwise_bwd(B, Ci, Co, P, int(act), dt, _ptr(x), _ptr(w), _ptr(bias),
                                        _ptr(dy), _ptr(dx), _ptr(dw), _ptr(db)), "pointwise_bwd")
    return {"dx": dx, "dw": dw, "db": db}


def mse(y, target):
    """(L, dL/dy) of L = mean((y - target)^2)."""
    dt = _dtype_of(y)
    y, target = _inputs(dt, y, target)
    assert y.shape == target.shape
    loss = np.zeros(1, dtype=np.float64)
    dy = np.empty(y.shape, dtype=np.float64)
    _check(_load().oracle_mse(y.size, dt, _ptr(y), _ptr(target), _ptr(loss), _ptr(dy)), "mse")
    return float(loss[0]), dy


def stack_loss_and_grads(d: Dims, x0, target, enc, blocks, dec, dec_act=1):
    """Loss and gradients of the Alg. 1 stack with an MSE loss.

    d: the block sizes (Ci = Co = width).  x0 [B, C0, *grid]; enc = (W_e [C0, width],
    b_e or None); blocks = [(W [width, width, Jx, Jy, Jz, Jt, 2], W_l, bias), ...];
    dec = (W_d [width, C_out], b_d or None); target [B, C_out, *grid].
    Encoder: X1 = GELU(x0 W_e + b_e); block i: X_{i+1} = GELU(S(X_i) + W_l^T X_i + b);
    decoder: Y = sigma(X W_d + b_d) (sigma = GELU for dec_act 1, identity for 0);
    L = mean((Y - target)^2).  Returns (L, grads) with grads "x0", "enc" (dw, db),
    "blocks" [(dw, dwl, db), ...], "dec" (dw, db), and the activations "h" [X1, ...].
    """
    assert d.Ci == d.Co
    h = [pointwise_fwd(x0, enc[0], enc[1], act=1)]
    for (w, wl, b) in blocks:
        z, _ = block_fwd(d, h[-1], w, wl, b)
        h.append(z)
    y = pointwise_fwd(h[-1], dec[0], dec[1], act=dec_act)
    loss, dy = mse(y, target)
    gd = pointwise_bwd(h[-1], dec[0], dy, dec[1], act=dec_act)
    dh = gd["dx"]
    gblocks = []
    for k in range(len(blocks) - 1, -1, -1):
        w, wl, b = blocks[k]
        r = block_bwd(d, h[k], w, dh, wl, b)
        gblocks.append((r["dw"], r["dwl"], r["db"]))
        dh = r["dx"]
    gblocks.reverse()
    ge = pointwise_bwd(x0, enc[0], dh, enc[1], act=1)
    return loss, {"x0": ge["dx"], "enc": (ge["dw"], ge["db"]), "blocks": gblocks,
                  "dec": (gd["dw"], gd["db"]), "h": h, "y": y}


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1) on float64 arrays p, m, v (updated in place)."""
    dt = _dtype_of(g)
    (g,) = _inputs(dt, g)
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == g.shape
    _check(_load().oracle_adam(g.size, dt, _ptr(p), _ptr(g), _ptr(m), _ptr(v), float(lr),
                               float(b1), float(b2), float(eps), int(t)), "adam")
    return p, m, v
