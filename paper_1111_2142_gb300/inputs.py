"""Seeded synthetic initial conditions, in numpy FP64.

This module holds no LW-ACM arithmetic: it only builds initial fields
(d = rho - 1, u) that both the CUDA library and the FP64 oracle are fed with.
Shapes are (ny, nx) for 2D and (nz, ny, nx) for 3D, x fastest.

Workloads:
  * 2D Taylor-Green vortex with its consistent pressure (closed-form solution of
    the incompressible Navier-Stokes equations; pressure p = rho/3, so
    d = 3 (p - p0)).
  * 3D Taylor-Green vortex u = u0 sin cos cos, v = -u0 cos sin cos, w = 0 with
    p - p0 = (u0^2/16)(cos 2kx + cos 2ky)(cos 2kz + 2).
  * band-limited random divergence-free fields (2D stream function, 3D curl of a
    vector potential), Hermitian so the fields are real, scaled to a target rms.
  * the batched ensemble of independent 2D domains (side lengths log-uniform,
    viscosities uniform).
  * smooth random fields for parity tests on ragged shapes.
  * the generalized (time-periodic, forced) Taylor-Green vortex of Section 3.2:
    its exact solution and its external acceleration, in lattice units.
"""
from __future__ import annotations

import numpy as np


def tgv2d(nx: int, ny: int | None = None, u0: float = 0.01):
    """2D Taylor-Green vortex at t = 0 on integer nodes x = i (k = 2 pi / n)."""
    ny = nx if ny is None else ny
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    ux = u0 * np.sin(kx * x) * np.cos(ky * y)
    uy = -u0 * (kx / ky) * np.cos(kx * x) * np.sin(ky * y)
    p = (u0 * u0 / 4.0) * (np.cos(2 * kx * x) + (kx / ky) ** 2 * np.cos(2 * ky * y))
    d = 3.0 * p
    return d.astype(np.float64), ux.astype(np.float64), uy.astype(np.float64)


def tgv3d(n: int, u0: float = 0.02, ny: int | None = None, nz: int | None = None):
    """Classical 3D Taylor-Green vortex at t = 0 (cubic n^3 unless ny/nz given)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    kx, ky, kz = 2 * np.pi / n, 2 * np.pi / ny, 2 * np.pi / nz
    x = np.arange(n)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    sx, cx = np.sin(kx * x), np.cos(kx * x)
    sy, cy = np.sin(ky * y), np.cos(ky * y)
    cz = np.cos(kz * z)
    ux = u0 * sx * cy * cz
    uy = -u0 * cx * sy * cz
    uz = np.zeros((nz, ny, n))
    p = (u0 * u0 / 16.0) * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * (np.cos(2 * kz * z) + 2.0)
    d = 3.0 * p * np.ones((nz, ny, n))
    return (d.astype(np.float64), ux.astype(np.float64), uy.astype(np.float64),
            uz.astype(np.float64))


def _band_coeffs(rng, shape_k, kmin, kmax, mags):
    amp = rng.standard_normal(shape_k) + 1j * rng.standard_normal(shape_k)
    mask = (mags >= kmin) & (mags <= kmax)
    return amp * mask


def random_divfree_2d(nx: int, ny: int, rms: float = 0.02, kmin: float = 1, kmax: float = 4,
                      seed: int = 0):
    """u = (d psi/dy, -d psi/dx) from a random stream function with integer
    wave numbers kmin <= |m| <= kmax; spectral derivatives, real output."""
    rng = np.random.default_rng(seed)
    mx = np.fft.fftfreq(nx, d=1.0 / nx)[None, :]
    my = np.fft.fftfreq(ny, d=1.0 / ny)[:, None]
    mags = np.sqrt(mx ** 2 + my ** 2)
    psi_hat = _band_coeffs(rng, (ny, nx), kmin, kmax, mags)
    kx = 2j * np.pi * mx / nx
    ky = 2j * np.pi * my / ny
    ux = np.real(np.fft.ifft2(ky * psi_hat))
    uy = np.real(np.fft.ifft2(-kx * psi_hat))
    s = np.sqrt(np.mean(ux ** 2 + uy ** 2))
    if s > 0:
        ux, uy = ux * (rms / s), uy * (rms / s)
    d = np.zeros((ny, nx))
    return d, np.ascontiguousarray(ux), np.ascontiguousarray(uy)


def random_divfree_3d(nx: int, ny: int, nz: int, rms: float = 0.03, kmin: float = 1,
                      kmax: float = 8, seed: int = 0):
    """u = curl A for a random band-limited vector potential A."""
    rng = np.random.default_rng(seed)
    mx = np.fft.fftfreq(nx, d=1.0 / nx)[None, None, :]
    my = np.fft.fftfreq(ny, d=1.0 / ny)[None, :, None]
    mz = np.fft.fftfreq(nz, d=1.0 / nz)[:, None, None]
    mags = np.sqrt(mx ** 2 + my ** 2 + mz ** 2)
    shp = (nz, ny, nx)
    A = [_band_coeffs(rng, shp, kmin, kmax, mags) for _ in range(3)]
    kx = 2j * np.pi * mx / nx
    ky = 2j * np.pi * my / ny
    kz = 2j * np.pi * mz / nz
    ux = np.real(np.fft.ifftn(ky * A[2] - kz * A[1]))
    uy = np.real(np.fft.ifftn(kz * A[0] - kx * A[2]))
    uz = np.real(np.fft.ifftn(kx * A[1] - ky * A[0]))
    s = np.sqrt(np.mean(ux ** 2 + uy ** 2 + uz ** 2))
    if s > 0:
        ux, uy, uz = ux * (rms / s), uy * (rms / s), uz * (rms / s)
    return (np.zeros(shp), np.ascontiguousarray(ux), np.ascontiguousarray(uy),
            np.ascontiguousarray(uz))


def smooth_random(shape, seed: int = 0, u_amp: float = 0.03, d_amp: float = 0.01, ncomp=None):
    """Smooth random (d, u...) fields on any (ragged) shape: a few low Fourier
    modes with random phases per component; not divergence-free."""
    rng = np.random.default_rng(seed)
    ncomp = len(shape) if ncomp is None else ncomp
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    out = []
    for amp in [d_amp] + [u_amp] * ncomp:
        f = np.zeros(shape)
        for _ in range(4):
            ph = rng.uniform(0, 2 * np.pi)
            arg = ph
            for g, n in zip(grids, shape):
                arg = arg + 2 * np.pi * rng.integers(-2, 3) * g / n
            f += rng.uniform(-1, 1) * np.cos(arg)
        f += 0.1 * rng.uniform(-1, 1, size=shape)
        out.append(amp * f / max(np.max(np.abs(f)), 1e-30))
    return tuple(np.ascontiguousarray(a) for a in out)


def ensemble_2d(n_domains: int = 256, seed: int = 1, smin: int = 32, smax: int = 512,
                nu_lo: float = 0.002, nu_hi: float = 0.05, rms: float = 0.02,
                kmin: float = 1, kmax: float = 4):
    """Independent periodic D2Q9 domains: side lengths log-uniform on [smin, smax]
    (rounded), nu uniform, initial u band-limited divergence-free with d = 0.

    Returns a list of dicts {nx, ny, nu, d, ux, uy}.
    """
    rng = np.random.default_rng(seed)
    nx = np.rint(np.exp(rng.uniform(np.log(smin), np.log(smax), n_domains))).astype(int)
    ny = np.rint(np.exp(rng.uniform(np.log(smin), np.log(smax), n_domains))).astype(int)
    nus = rng.uniform(nu_lo, nu_hi, n_domains)
    seeds = rng.integers(0, 2 ** 31 - 1, n_domains)
    doms = []
    for b in range(n_domains):
        d, ux, uy = random_divfree_2d(int(nx[b]), int(ny[b]), rms, kmin, kmax, int(seeds[b]))
        doms.append(dict(nx=int(nx[b]), ny=int(ny[b]), nu=float(nus[b]), d=d, ux=ux, uy=uy))
    return doms


# Generalized Taylor-Green vortex (Section 3.2, Eqs. external-force and
# exactsolution): domain [0, 2 pi]^2, periodic, drift (u0, v0) = (0.3, 0.6),
# nu = 0.1, diffusive scaling dx = eps, dt = eps^2 (Section 2.3, Table of units).
GTG_U0, GTG_V0, GTG_NU = 0.3, 0.6, 0.1


def gtg_grid(n: int):
    """Node coordinates x_i = i eps, eps = 2 pi / n, as (X, Y) of shape (n, n)."""
    eps = 2.0 * np.pi / n
    x = np.arange(n) * eps
    X, Y = np.meshgrid(x, x, indexing="xy")
    return eps, X, Y


def gtg_exact(n: int, t: float):
    """Exact (u, v, p) in physical units at time t on the n x n grid."""
    _, X, Y = gtg_grid(n)
    a, b = X - GTG_U0 * t, Y - GTG_V0 * t
    u = GTG_U0 + np.sin(a) * np.cos(b) * np.cos(t)
    v = GTG_V0 - np.cos(a) * np.sin(b) * np.cos(t)
    p = 0.25 * (np.cos(2 * a) + np.cos(2 * b)) * np.cos(t) ** 2
    return u, v, p


def gtg_state(n: int, t: float = 0.0):
    """Lattice fields (d, ux, uy) of the exact solution at time t: u_lattice =
    eps u, p = rho/3 with (p - p0)/eps^2 the physical pressure, so d = 3 eps^2 p."""
    eps = 2.0 * np.pi / n
    u, v, p = gtg_exact(n, t)
    return 3.0 * eps ** 2 * p, eps * u, eps * v


def gtg_force(n: int, t: float):
    """Lattice acceleration (gx, gy) = eps^3 g_bar(t) (Section 2.1: g = eps^3 g_bar
    under diffusive scaling), g_bar of Eq. external-force."""
    eps, X, Y = gtg_grid(n)
    a, b = X - GTG_U0 * t, Y - GTG_V0 * t
    amp = 2.0 * GTG_NU * np.cos(t) - np.sin(t)
    return eps ** 3 * np.sin(a) * np.cos(b) * amp, -eps ** 3 * np.cos(a) * np.sin(b) * amp


def minion_brown(n: int, u_lat: float = 0.04, k: float = 80.0, delta: float = 0.05):
    """Perturbed double shear layer of Section 3.2 (Minion & Brown) on the periodic
    unit square, n x n nodes at x_i = i / n: u = U tanh(k (y - 1/4)) for y <= 1/2,
    U tanh(k (3/4 - y)) above, v = U delta sin(2 pi (x + 1/4)), with the unit speed
    U = u_lat in lattice units (the Mach number Ma of the paper's runs) and d = 0.
    Returns (d, ux, uy) of shape (n, n)."""
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = np.where(Y <= 0.5, np.tanh(k * (Y - 0.25)), np.tanh(k * (0.75 - Y))) * u_lat
    uy = u_lat * delta * np.sin(2.0 * np.pi * (X + 0.25))
    return np.zeros((n, n)), ux, uy


def minion_brown_lattice(n: int, u_lat: float = 0.04, re: float = 1.0e4):
    """Lattice viscosity and the number of steps to t = 1 for the shear layer: with
    dx = 1/n and a unit speed of u_lat lattice units, dt = u_lat / n, so
    nu = (1/Re) dt / dx^2 = u_lat n / Re and t = 1 takes n / u_lat steps."""
    return u_lat * n / re, int(round(n / u_lat))


def gtg_steps(n: int, t_end: float = 60.0) -> int:
    """Number of steps of size eps^2 nearest to t_end."""
    eps = 2.0 * np.pi / n
    return int(round(t_end / eps ** 2))
