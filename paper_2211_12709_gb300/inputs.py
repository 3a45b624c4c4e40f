"""Seeded synthetic inputs for the spectral FNO block (host, NumPy PCG64, FP64 -> FP32).

This module holds input generation only -- none of the block's arithmetic -- so
both the CUDA-path tests/bench and the CPU oracle tests draw the same fields
from it.  The paper's datasets (WaterLily vorticity, Sleipner/OPM CO2
saturation; Sec. V-A, V-B) are not available, so these fields stand in for
their shapes and structure:

* ``normal``            i.i.d. N(0, 1) (the single-layer check).
* ``grf``               periodic Gaussian random field with squared-exponential
                        covariance exp(-r^2 / (2 l^2)) per axis, unit variance,
                        independent per channel: white noise filtered by the
                        square root of its power spectrum exp(-2 pi^2 sum l_a^2 f_a^2).
* ``co2_static_fields`` (log-permeability, porosity, injection-well map) as in
                        the CO2 example of Sec. V-B: a log-normal GRF with mean
                        ln(100 mD), std 1 and correlation lengths 20 x 20 x 4
                        cells, a porosity derived from it, and a binary
                        vertical well column; static in time (the paper repeats
                        its 3-D inputs along t).
* ``spectral_weights``  Re, Im ~ U(-1, 1) / (Ci Co).
* ``linear_params``     1x1 weight and bias ~ U(-1/sqrt(Ci), 1/sqrt(Ci)).

Seeds: input 1000 + config, spectral weights 2000 + config, 1x1 weights
3000 + config, upstream gradients / directions 4000 + config.
"""
from __future__ import annotations

import math

import numpy as np
import os

import scipy.fft as _sfft

SEED_INPUT = 1000
SEED_SPECTRAL_W = 2000
SEED_LINEAR = 3000
SEED_UPSTREAM = 4000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def normal(shape, seed: int) -> np.ndarray:
    """i.i.d. standard normal, float32."""
    return _rng(seed).standard_normal(size=tuple(shape), dtype=np.float32)


def spectral_weights(Ci: int, Co: int, modes, seed: int) -> np.ndarray:
    """Complex per-mode weights as real pairs [Ci][Co][Jx][Jy][Jz][Jt][2], U(-1,1)/(Ci*Co)."""
    g = _rng(seed)
    shape = (Ci, Co) + tuple(modes) + (2,)
    return (g.uniform(-1.0, 1.0, size=shape) / float(Ci * Co)).astype(np.float32)


def linear_params(Ci: int, Co: int, seed: int):
    """(Wl[Ci][Co], bias[Co]) ~ U(-1/sqrt(Ci), 1/sqrt(Ci)), float32."""
    g = _rng(seed)
    s = 1.0 / math.sqrt(Ci)
    wl = g.uniform(-s, s, size=(Ci, Co)).astype(np.float32)
    b = g.uniform(-s, s, size=(Co,)).astype(np.float32)
    return wl, b


_WORKERS = max(1, os.cpu_count() or 1)


def _grf_channel(g: np.random.Generator, grid, ell, dtype=np.float64) -> np.ndarray:
    noise = g.standard_normal(size=tuple(grid), dtype=dtype)
    spec = _sfft.rfftn(noise, workers=_WORKERS)
    nd = len(grid)
    for a, (n, l) in enumerate(zip(grid, ell)):
        f = np.fft.rfftfreq(n) if a == nd - 1 else np.fft.fftfreq(n)
        shape = [1] * nd
        shape[a] = f.size
        spec *= np.exp(-math.pi ** 2 * (l ** 2) * f.reshape(shape) ** 2).astype(dtype)
    field = _sfft.irfftn(spec, s=tuple(grid), workers=_WORKERS)
    field -= field.mean(dtype=np.float64)
    sd = float(field.std(dtype=np.float64))
    return field / sd if sd > 0 else field


def grf(lead, grid, ell, seed: int) -> np.ndarray:
    """Periodic squared-exponential GRF, unit variance per channel, float32 [*lead, *grid].

    ``ell`` is one correlation length (cells) per grid axis.  The filter is the
    square root of the power spectrum, so the field's covariance is the
    squared-exponential with length ell on each axis.
    """
    g = _rng(seed)
    lead = tuple(lead)
    out = np.empty(lead + tuple(grid), dtype=np.float32)
    flat = out.reshape((-1,) + tuple(grid))
    # large grids are generated in single precision (the stored field is FP32 anyway)
    work = np.float32 if int(np.prod(grid)) >= (1 << 24) else np.float64
    for c in range(flat.shape[0]):
        flat[c] = _grf_channel(g, grid, ell, work).astype(np.float32)
    return out


def co2_static_fields(Nx: int, Ny: int, Nz: int, seed: int):
    """(standardised log-permeability, porosity, well map), each float32 [Nx][Ny][Nz]."""
    g = _rng(seed)
    z = _grf_channel(g, (Nx, Ny, Nz), (20.0, 20.0, 4.0))
    mu = math.log(100.0)
    logk = mu + 1.0 * z
    phi = np.clip(0.25 + 0.05 * (logk - mu), 0.05, 0.40)
    well = np.zeros((Nx, Ny, Nz), dtype=np.float64)
    wx, wy = int(g.integers(0, Nx)), int(g.integers(0, Ny))
    well[wx, wy, :] = 1.0
    logk_std = (logk - logk.mean()) / logk.std()
    return logk_std.astype(np.float32), phi.astype(np.float32), well.astype(np.float32)


def co2_stack_inputs(B: int, grid, seed: int):
    """Input and target of the CO2 stack: x0 [B][3][Nx][Ny][Nz][Nt], target [B][1][...].

    x0 holds the three static fields of ``co2_static_fields`` repeated along t
    (the paper repeats its 3-D inputs along time); the target saturation is a
    smooth field in [0, 1], the logistic function of a GRF with correlation
    lengths 20 x 20 x 4 cells and 8 steps.
    """
    Nx, Ny, Nz, Nt = (int(v) for v in grid)
    x0 = np.empty((B, 3, Nx, Ny, Nz, Nt), dtype=np.float32)
    for b in range(B):
        for c, f in enumerate(co2_static_fields(Nx, Ny, Nz, seed + 17 * b)):
            x0[b, c] = f[..., None]
    z = grf((B, 1), (Nx, Ny, Nz, Nt), (20.0, 20.0, 4.0, 8.0), seed + 1)
    target = (1.0 / (1.0 + np.exp(-z))).astype(np.float32)
    return x0, target


def ns_stack_inputs(B: int, grid, seed: int, kmax: float = 16.0):
    """Input and target of the Navier-Stokes stack: x0, target [B][4][Nx][Ny][Nz][Nt].

    Channels (u, v, w, |omega|) of a divergence-free random Fourier velocity
    field: complex Gaussian amplitudes projected perpendicular to k, with
    |u_hat(k)|^2 proportional to k^(-5/3) / (4 pi k^2) for 1 <= |k| <= kmax and
    zero beyond, each mode rotating in time as exp(2 pi i f_k t / Nt) with a
    seeded f_k in {0..3}; the vorticity is the spectral curl.  The velocity is
    scaled to unit root-mean-square (one factor for all three components, so
    div u = 0 holds) and |omega| to zero mean and unit standard deviation.  The
    target is the same field one time step later (the next state).
    """
    Nx, Ny, Nz, Nt = (int(v) for v in grid)
    g = _rng(seed)
    ks = [np.fft.fftfreq(n, 1.0 / n) for n in (Nx, Ny, Nz)]
    K = np.stack(np.meshgrid(*ks, indexing="ij"))          # [3][Nx][Ny][Nz]
    kmag = np.sqrt((K ** 2).sum(axis=0))
    keep = (kmag >= 1.0) & (kmag <= kmax)
    amp = np.zeros_like(kmag)
    amp[keep] = np.sqrt(kmag[keep] ** (-5.0 / 3.0) / (4.0 * math.pi * kmag[keep] ** 2))
    khat = K / np.where(kmag > 0, kmag, 1.0)
    x0 = np.empty((B, 4, Nx, Ny, Nz, Nt), dtype=np.float32)
    for b in range(B):
        a = g.standard_normal((3, Nx, Ny, Nz)) + 1j * g.standard_normal((3, Nx, Ny, Nz))
        a -= khat * (a * khat).sum(axis=0)                  # k . u_hat = 0
        uh = a * amp
        f = g.integers(0, 4, size=(Nx, Ny, Nz))
        for t in range(Nt):
            uht = uh * np.exp(2j * math.pi * f * t / Nt)
            u = _sfft.ifftn(uht, axes=(1, 2, 3), workers=_WORKERS).real
            wh = 1j * np.cross(K, uht, axis=0)               # curl in Fourier space
            w = _sfft.ifftn(wh, axes=(1, 2, 3), workers=_WORKERS).real
            x0[b, 0:3, ..., t] = u
            x0[b, 3, ..., t] = np.sqrt((w ** 2).sum(axis=0))
    # one scale for the three velocity components (keeps div u = 0), one for |omega|
    vel = x0[:, 0:3]
    vel /= max(float(np.sqrt((vel.astype(np.float64) ** 2).mean())), 1e-30)
    vort = x0[:, 3]
    vort -= vort.mean(dtype=np.float64)
    vort /= max(float(vort.std(dtype=np.float64)), 1e-30)
    target = np.roll(x0, -1, axis=-1)
    return x0, target
