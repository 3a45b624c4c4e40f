"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test fixes one part of the oracle to a fact that the paper's definition
of the block (Alg. 2, Sec. IV-C; the original-FNO bypass and GELU as read in
the oracle's header) or plain mathematics determines:

* brute-force 4-D sums vs the separable stage-by-stage sums,
* NumPy's rfftn / irfftn (a library special case of the same operator),
* identity with all modes kept, orthogonal-projector and Parseval identities,
* circular-shift equivariance, closed-form plane waves, Hermitian completion,
* adjoint (dot-product) identities and central finite differences of the
  gradient, and textbook GELU values.

A plausible slip in the oracle (a dropped c(kt) weight, a wrong sign of the
exponent, a swapped stored-index map, a transposed weight, a missing 1/N, a
conjugate dropped in the adjoint) fails at least one of these.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Dims

TINY = [
    Dims(1, 2, 3, 4, 6, 5, 7, 2, 2, 2, 3),    # odd Nz, odd Nt (no Nyquist bin), 2m = N in x
    Dims(2, 2, 2, 8, 8, 8, 8, 4, 3, 2, 5),    # all power of two, kt up to the Nyquist bin
    Dims(1, 3, 2, 5, 4, 6, 6, 1, 2, 3, 2),    # odd Nx, 2m = N in y, z
]


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def kept_index(j, m, n):
    k = j if j < m else j - 2 * m
    return k % n


def kept_indices(d):
    ix = [kept_index(j, d.mx, d.Nx) for j in range(2 * d.mx)]
    iy = [kept_index(j, d.my, d.Ny) for j in range(2 * d.my)]
    iz = [kept_index(j, d.mz, d.Nz) for j in range(2 * d.mz)]
    it = list(range(d.mt))
    return ix, iy, iz, it


def cw(kt, Nt):
    return 1.0 if (kt == 0 or (Nt % 2 == 0 and 2 * kt == Nt)) else 2.0


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def rand_w(d, seed, complex_=True):
    g = rng(seed)
    w = g.uniform(-1, 1, size=(d.Ci, d.Co) + d.modes + (2,))
    return w[..., 0] + 1j * w[..., 1] if complex_ else w


def w_real(wc):
    return np.stack([wc.real, wc.imag], axis=-1)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("d", TINY, ids=str)
def test_spectrum_matches_bruteforce_4d_sum(d):
    f = rng(1).standard_normal((2,) + d.grid)
    a = oracle.spectrum(d, f)
    b = oracle.spectrum(d, f, brute_force=True)
    assert relerr(a, b) < 1e-12
    a = oracle.spectrum(d, f, adjoint_scale=True)
    b = oracle.spectrum(d, f, adjoint_scale=True, brute_force=True)
    assert relerr(a, b) < 1e-12


@pytest.mark.parametrize("d", TINY, ids=str)
@pytest.mark.parametrize("scaled", [True, False])
def test_synthesis_matches_bruteforce_4d_sum(d, scaled):
    g = rng(2)
    sp = g.standard_normal((2,) + d.modes) + 1j * g.standard_normal((2,) + d.modes)
    a = oracle.synthesis(d, sp, scaled=scaled)
    b = oracle.synthesis(d, sp, scaled=scaled, brute_force=True)
    assert relerr(a, b) < 1e-12
    pts = np.array([[0, 0, 0, 0], [d.Nx - 1, 1, d.Nz - 1, d.Nt - 1], [1, d.Ny - 1, 2, 3]])
    c = oracle.synthesis_points(d, sp, pts, scaled=scaled)
    assert relerr(c, b[:, pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3]]) < 1e-12


# ------------------------------------------------------- library special case

@pytest.mark.parametrize("d", TINY, ids=str)
def test_spectrum_equals_numpy_rfftn_kept_corners(d):
    f = rng(3).standard_normal(d.grid)
    full = np.fft.rfftn(f, axes=(0, 1, 2, 3))
    ix, iy, iz, it = kept_indices(d)
    ref = full[np.ix_(ix, iy, iz, it)]
    assert relerr(oracle.spectrum(d, f), ref) < 1e-12


@pytest.mark.parametrize("d", TINY, ids=str)
def test_synthesis_equals_numpy_irfftn_of_zero_padded(d):
    g = rng(4)
    sp = g.standard_normal(d.modes) + 1j * g.standard_normal(d.modes)
    pad = np.zeros((d.Nx, d.Ny, d.Nz, d.Nt // 2 + 1), dtype=complex)
    ix, iy, iz, it = kept_indices(d)
    pad[np.ix_(ix, iy, iz, it)] = sp
    ref = np.fft.irfftn(pad, s=d.grid, axes=(0, 1, 2, 3))
    assert relerr(oracle.synthesis(d, sp, scaled=True), ref) < 1e-12


@pytest.mark.parametrize("d", TINY, ids=str)
def test_synthesis_is_real_part_of_hermitian_completed_ifft(d):
    g = rng(5)
    sp = g.standard_normal(d.modes) + 1j * g.standard_normal(d.modes)
    H = np.zeros(d.grid, dtype=complex)
    ix, iy, iz, it = kept_indices(d)
    for a, kx in enumerate(ix):
        for b, ky in enumerate(iy):
            for c, kz in enumerate(iz):
                for e, kt in enumerate(it):
                    v = sp[a, b, c, e]
                    if cw(kt, d.Nt) == 2.0:
                        H[kx, ky, kz, kt] += v
                        H[(-kx) % d.Nx, (-ky) % d.Ny, (-kz) % d.Nz, (-kt) % d.Nt] += np.conj(v)
                    else:
                        H[kx, ky, kz, kt] += v / 2
                        H[(-kx) % d.Nx, (-ky) % d.Ny, (-kz) % d.Nz, (-kt) % d.Nt] += np.conj(v) / 2
    full = np.fft.ifftn(H)
    assert np.max(np.abs(full.imag)) < 1e-12 * max(1.0, np.max(np.abs(full.real)))
    assert relerr(oracle.synthesis(d, sp, scaled=True), full.real) < 1e-12


def test_mix_matches_einsum():
    d = TINY[1]
    g = rng(6)
    xh = g.standard_normal((d.B, d.Ci) + d.modes) + 1j * g.standard_normal((d.B, d.Ci) + d.modes)
    w = rand_w(d, 7)
    ref = np.einsum("bixyzt,ioxyzt->boxyzt", xh, w)
    assert relerr(oracle.mix(d, xh, w), ref) < 1e-13
    gg = g.standard_normal((d.B, d.Co) + d.modes) + 1j * g.standard_normal((d.B, d.Co) + d.modes)
    dw, gx = oracle.mix_adjoint(d, xh, w, gg)
    assert relerr(dw, np.einsum("bixyzt,boxyzt->ioxyzt", np.conj(xh), gg)) < 1e-13
    assert relerr(gx, np.einsum("ioxyzt,boxyzt->bixyzt", np.conj(w), gg)) < 1e-13


# ------------------------------------------------------------ closed forms

def test_identity_with_all_modes_kept():
    for d in (Dims(1, 3, 3, 4, 6, 2, 8, 2, 3, 1, 5), Dims(2, 2, 2, 4, 4, 4, 4, 2, 2, 2, 3)):
        x = rng(8).standard_normal((d.B, d.Ci) + d.grid)
        w = np.zeros((d.Ci, d.Co) + d.modes, dtype=complex)
        for i in range(d.Ci):
            w[i, i] = 1.0
        z, _ = oracle.block_fwd(d, x, w_real(w))
        assert relerr(z, x) < 1e-13


def _projector(d, x):
    w = np.zeros((d.Ci, d.Co) + d.modes, dtype=complex)
    for i in range(d.Ci):
        w[i, i] = 1.0
    return oracle.block_fwd(d, x, w_real(w))[0]


def test_truncation_is_orthogonal_projector_when_spatial_set_is_symmetric():
    # 2m = N on x, y, z: the kept set is closed under k -> -k, so S (W = identity)
    # is the orthogonal projector onto kt < mt (and its conjugates).
    d = Dims(1, 1, 1, 4, 6, 2, 9, 2, 3, 1, 3)
    g = rng(9)
    x = g.standard_normal((1, 1) + d.grid)
    y = g.standard_normal((1, 1) + d.grid)
    px = _projector(d, x)
    py = _projector(d, y)
    assert relerr(_projector(d, px), px) < 1e-12                     # idempotent
    assert abs(np.vdot(px, y) - np.vdot(x, py)) < 1e-12 * np.linalg.norm(px) * np.linalg.norm(y)
    assert abs(np.vdot(px, px) - np.vdot(px, x)) < 1e-12 * np.vdot(px, px)


@pytest.mark.parametrize("d", [Dims(1, 1, 1, 6, 8, 5, 8, 2, 3, 2, 3), Dims(1, 1, 1, 5, 4, 6, 7, 2, 1, 2, 3),
                               Dims(1, 1, 1, 6, 4, 6, 6, 1, 1, 2, 4)], ids=str)
def test_truncation_spectrum_of_eigenvalues_and_parseval(d):
    # The corner set {-m..m-1} is not closed under k -> -k, so on the planes kt = 0
    # (and kt = Nt/2) a mode whose mirror is dropped keeps half its weight: S is
    # self-adjoint with eigenvalues in {0, 1/2, 1}, i.e. 2 S^3 - 3 S^2 + S = 0,
    # and <S x, x> = (1/N) sum_j c(kt) |Xh_j|^2.
    g = rng(9)
    x = g.standard_normal((1, 1) + d.grid)
    y = g.standard_normal((1, 1) + d.grid)
    px = _projector(d, x)
    py = _projector(d, y)
    assert abs(np.vdot(px, y) - np.vdot(x, py)) < 1e-12 * np.linalg.norm(px) * np.linalg.norm(y)
    p2 = _projector(d, px)
    p3 = _projector(d, p2)
    assert np.linalg.norm(2 * p3 - 3 * p2 + px) < 1e-12 * np.linalg.norm(px)
    assert relerr(p2, px) > 1e-3                                      # not a projector here
    xh = oracle.spectrum(d, x[0, 0])
    cws = np.array([cw(kt, d.Nt) for kt in range(d.mt)])
    parseval = np.sum(cws * np.abs(xh) ** 2) / d.n_grid
    assert abs(np.vdot(px, x).real - parseval) < 1e-12 * parseval


@pytest.mark.parametrize("axis", [0, 1, 2, 3])
def test_block_commutes_with_circular_shifts(axis):
    d = Dims(1, 3, 2, 6, 5, 4, 6, 2, 2, 1, 3)
    g = rng(10 + axis)
    x = g.standard_normal((d.B, d.Ci) + d.grid)
    w = rand_w(d, 20)
    wl = g.uniform(-1, 1, (d.Ci, d.Co))
    b = g.uniform(-1, 1, d.Co)
    z, _ = oracle.block_fwd(d, x, w_real(w), wl, b)
    zs, _ = oracle.block_fwd(d, np.roll(x, 2, axis=2 + axis), w_real(w), wl, b)
    assert relerr(zs, np.roll(z, 2, axis=2 + axis)) < 1e-12


def _wave(d, k, phase=0.0):
    x, y, z, t = np.meshgrid(*[np.arange(n) for n in d.grid], indexing="ij")
    th = 2 * np.pi * (k[0] * x / d.Nx + k[1] * y / d.Ny + k[2] * z / d.Nz + k[3] * t / d.Nt)
    return np.cos(th + phase), th


def _stored(j_of_k, k, m):
    return k if k >= 0 else k + 2 * m


def test_plane_wave_closed_forms():
    d = Dims(1, 2, 3, 8, 6, 8, 8, 3, 2, 2, 3)
    g = rng(30)
    w = rand_w(d, 31)
    # 0 < kt < Nt/2: S_o = |W[i0,o,j0]| cos(theta + arg W)
    k0 = (2, -1, 1, 2)
    j0 = (_stored(None, 2, d.mx), _stored(None, -1, d.my), _stored(None, 1, d.mz), 2)
    wave, th = _wave(d, k0)
    x = np.zeros((1, d.Ci) + d.grid)
    x[0, 1] = wave
    z, _ = oracle.block_fwd(d, x, w_real(w))
    for o in range(d.Co):
        wv = w[1, o][j0]
        assert relerr(z[0, o], np.abs(wv) * np.cos(th + np.angle(wv))) < 1e-12
    # kt = 0 with k and -k both kept: S = Re(W(k) e^{i th})/2 + Re(W(-k) e^{-i th})/2
    k1 = (1, 1, -1, 0)
    j1 = (1, 1, _stored(None, -1, d.mz), 0)
    jm1 = (_stored(None, -1, d.mx), _stored(None, -1, d.my), 1, 0)
    wave, th = _wave(d, k1)
    x = np.zeros((1, d.Ci) + d.grid)
    x[0, 0] = wave
    z, _ = oracle.block_fwd(d, x, w_real(w))
    for o in range(d.Co):
        ref = 0.5 * np.real(w[0, o][j1] * np.exp(1j * th)) + 0.5 * np.real(w[0, o][jm1] * np.exp(-1j * th))
        assert relerr(z[0, o], ref) < 1e-12
    # kt = 0 with -k dropped (kz = +mz is not kept): only half of the wave survives
    k2 = (1, 1, -d.mz, 0)
    j2 = (1, 1, _stored(None, -d.mz, d.mz), 0)
    wave, th = _wave(d, k2)
    x = np.zeros((1, d.Ci) + d.grid)
    x[0, 1] = wave
    z, _ = oracle.block_fwd(d, x, w_real(w))
    for o in range(d.Co):
        assert relerr(z[0, o], 0.5 * np.real(w[1, o][j2] * np.exp(1j * th))) < 1e-12
    # a wave outside the kept set (kx = mx is not kept: only -mx..mx-1) vanishes
    wave, _ = _wave(d, (d.mx, 0, 0, 1), phase=0.3)
    x = np.zeros((1, d.Ci) + d.grid)
    x[0, 0] = wave
    z, _ = oracle.block_fwd(d, x, w_real(w))
    assert np.max(np.abs(z)) < 1e-12
    # and so does kt = mt
    wave, _ = _wave(d, (1, 0, 0, d.mt), phase=0.7)
    x[0, 0] = wave
    z, _ = oracle.block_fwd(d, x, w_real(w))
    assert np.max(np.abs(z)) < 1e-12


# --------------------------------------------------------------- gradients

@pytest.mark.parametrize("d", [TINY[0], TINY[2]], ids=str)
def test_spectral_adjoint_dot_products(d):
    g = rng(40)
    x = g.standard_normal((d.B, d.Ci) + d.grid)
    gz = g.standard_normal((d.B, d.Co) + d.grid)
    w = w_real(rand_w(d, 41))
    dw_dir = w_real(rand_w(d, 42))
    sx, _ = oracle.block_fwd(d, x, w)
    gr = oracle.block_bwd(d, x, w, gz)
    lhs = np.vdot(sx, gz)
    assert abs(lhs - np.vdot(x, gr["dx"])) < 1e-12 * (abs(lhs) + np.linalg.norm(sx) * np.linalg.norm(gz))
    s_dw, _ = oracle.block_fwd(d, x, dw_dir)                     # linear in W
    lhs = np.vdot(s_dw, gz)
    assert abs(lhs - np.vdot(dw_dir, gr["dw"])) < 1e-12 * (abs(lhs) + np.linalg.norm(s_dw) * np.linalg.norm(gz))


def test_block_gradient_central_finite_differences():
    d = Dims(2, 3, 2, 6, 5, 4, 6, 2, 2, 1, 3)
    g = rng(50)
    x = g.standard_normal((d.B, d.Ci) + d.grid)
    w = w_real(rand_w(d, 51)) * 0.3
    wl = g.uniform(-1, 1, (d.Ci, d.Co))
    b = g.uniform(-1, 1, d.Co)
    r = g.standard_normal((d.B, d.Co) + d.grid)

    def loss(x_, w_, wl_, b_):
        z, _ = oracle.block_fwd(d, x_, w_, wl_, b_)
        return float(np.vdot(z, r))

    gr = oracle.block_bwd(d, x, w, r, wl, b)
    eps = 1e-3

    def along(name, base, v, h):
        args = dict(x_=x, w_=w, wl_=wl, b_=b)
        args[name + "_"] = base + h * v
        return loss(**args)

    def central(name, base, v):
        # second-order central difference (truncation O(eps^2)) and the
        # fourth-order central stencil (truncation O(eps^4)) with the same eps
        lp, lm = along(name, base, v, eps), along(name, base, v, -eps)
        lp2, lm2 = along(name, base, v, 2 * eps), along(name, base, v, -2 * eps)
        fd2 = (lp - lm) / (2 * eps)
        fd4 = (8 * (lp - lm) - (lp2 - lm2)) / (12 * eps)
        return fd2, fd4

    for name, base, grad in (("x", x, gr["dx"]), ("w", w, gr["dw"]), ("wl", wl, gr["dwl"]), ("b", b, gr["db"])):
        v = g.standard_normal(base.shape)
        fd2, fd4 = central(name, base, v)
        an = float(np.vdot(grad, v))
        assert abs(fd2 - an) <= 1e-4 * max(1.0, abs(an)), (name, fd2, an)
        assert abs(fd4 - an) <= 1e-8 * max(1.0, abs(an)), (name, fd4, an)
    # single coordinates of x and of W
    for name, base, grad in (("x", x, gr["dx"]), ("w", w, gr["dw"])):
        for _ in range(4):
            idx = tuple(int(g.integers(0, s)) for s in base.shape)
            e = np.zeros_like(base)
            e[idx] = 1.0
            fd2, fd4 = central(name, base, e)
            assert abs(fd4 - grad[idx]) <= 1e-8 * max(1.0, abs(grad[idx])), (name, idx, fd4, grad[idx])


def test_points_mode_agrees_with_full_grid():
    d = Dims(2, 3, 2, 6, 5, 4, 6, 2, 2, 1, 3)
    g = rng(60)
    x = g.standard_normal((d.B, d.Ci) + d.grid).astype(np.float32)
    w = w_real(rand_w(d, 61)).astype(np.float32)
    wl = g.uniform(-1, 1, (d.Ci, d.Co)).astype(np.float32)
    b = g.uniform(-1, 1, d.Co).astype(np.float32)
    dz = g.standard_normal((d.B, d.Co) + d.grid).astype(np.float32)
    pts = np.stack([g.integers(0, n, 17) for n in d.grid], axis=1)
    z, zp = oracle.block_fwd(d, x, w, wl, b, full=True, pts=pts)
    assert relerr(zp, z[:, :, pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3]]) < 1e-13
    gr = oracle.block_bwd(d, x, w, dz, wl, b, full=True, pts=pts)
    assert relerr(gr["dx_pts"], gr["dx"][:, :, pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3]]) < 1e-13


def test_gelu_textbook_values():
    assert oracle.gelu(0.0) == 0.0
    assert abs(oracle.gelu_grad(0.0) - 0.5) < 1e-16
    # GELU(1) = Phi(1), the standard normal CDF at 1
    assert abs(oracle.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(oracle.gelu(-1.0) + 1.0 - 0.8413447460685429) < 1e-15
    assert abs(oracle.gelu(12.0) - 12.0) < 1e-12
    assert abs(oracle.gelu(-12.0)) < 1e-12
    for a in (-2.5, -0.3, 0.7, 3.1):
        h = 1e-5
        fd = (oracle.gelu(a + h) - oracle.gelu(a - h)) / (2 * h)
        assert abs(fd - oracle.gelu_grad(a)) < 1e-9


# ------------------------------------------------------- linearity, bypass

def test_spectral_part_is_linear_in_x_and_in_w():
    d = Dims(2, 3, 2, 6, 5, 4, 6, 2, 2, 1, 3)
    g = rng(70)
    x1, x2 = (g.standard_normal((d.B, d.Ci) + d.grid) for _ in range(2))
    w1, w2 = w_real(rand_w(d, 71)), w_real(rand_w(d, 72))
    a, b = 0.7, -1.9
    s1, _ = oracle.block_fwd(d, x1, w1)
    s2, _ = oracle.block_fwd(d, x2, w1)
    s12, _ = oracle.block_fwd(d, a * x1 + b * x2, w1)
    assert relerr(s12, a * s1 + b * s2) < 1e-12
    t2, _ = oracle.block_fwd(d, x1, w2)
    t12, _ = oracle.block_fwd(d, x1, a * w1 + b * w2)
    assert relerr(t12, a * s1 + b * t2) < 1e-12


def test_zero_spectral_weight_reduces_to_torch_linear_gelu():
    # With W = 0 the block is a dense 1x1 layer with exact GELU; PyTorch's CPU
    # FP64 linear + gelu (erf form) and autograd give its value and gradients.
    torch = pytest.importorskip("torch")
    d = Dims(2, 3, 5, 4, 3, 5, 6, 1, 1, 2, 2)
    g = rng(80)
    x = g.standard_normal((d.B, d.Ci) + d.grid)
    wl = g.uniform(-1, 1, (d.Ci, d.Co))
    b = g.uniform(-1, 1, d.Co)
    dz = g.standard_normal((d.B, d.Co) + d.grid)
    w0 = np.zeros((d.Ci, d.Co) + d.modes + (2,))
    z, _ = oracle.block_fwd(d, x, w0, wl, b)
    gr = oracle.block_bwd(d, x, w0, dz, wl, b)
    X = torch.tensor(np.moveaxis(x, 1, -1), dtype=torch.float64, requires_grad=True)
    WL = torch.tensor(wl.T.copy(), dtype=torch.float64, requires_grad=True)   # nn.Linear: [out][in]
    Bb = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    Z = torch.nn.functional.gelu(torch.nn.functional.linear(X, WL, Bb), approximate="none")
    Z.backward(torch.tensor(np.moveaxis(dz, 1, -1)))
    assert relerr(z, np.moveaxis(Z.detach().numpy(), -1, 1)) < 1e-13
    assert relerr(gr["dx"], np.moveaxis(X.grad.numpy(), -1, 1)) < 1e-12
    assert relerr(gr["dwl"], WL.grad.numpy().T) < 1e-12
    assert relerr(gr["db"], Bb.grad.numpy()) < 1e-12
