"""Seeded synthetic initial conditions for the D3Q19 workloads.

This module holds no lattice Boltzmann arithmetic: it only builds macroscopic
initial fields (density and velocity) from closed-form flows or seeded random
Fourier modes.  Both the GPU library's tests and the CPU oracle's tests take
their inputs from here.

All fields are returned as float64 torch tensors of shape ``rho[nz, ny, nx]``
and ``u[3, nz, ny, nx]`` (x fastest), on the requested device.
"""
import math

import numpy as np
import torch


def _grid(nx, ny, nz, device):
    z = torch.arange(nz, dtype=torch.float64, device=device).view(nz, 1, 1)
    y = torch.arange(ny, dtype=torch.float64, device=device).view(1, ny, 1)
    x = torch.arange(nx, dtype=torch.float64, device=device).view(1, 1, nx)
    return x, y, z


def taylor_green(n, u0=0.05, device="cpu"):
    """3D Taylor-Green vortex on a periodic n^3 box, rho = 1:
    u = u0 (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi x / n at integer nodes."""
    x, y, z = _grid(n, n, n, device)
    X, Y, Z = (2 * math.pi * x / n, 2 * math.pi * y / n, 2 * math.pi * z / n)
    u = torch.zeros((3, n, n, n), dtype=torch.float64, device=device)
    u[0] = u0 * torch.sin(X) * torch.cos(Y) * torch.cos(Z)
    u[1] = -u0 * torch.cos(X) * torch.sin(Y) * torch.cos(Z)
    rho = torch.ones((n, n, n), dtype=torch.float64, device=device)
    return rho, u


def shear_wave(nx, ny, nz, U=(0.0, 0.0, 0.0), amplitude=0.01, device="cpu"):
    """Transverse shear wave u_y = amplitude sin(2 pi x / nx) on a uniform
    background velocity U = (U_x, U_y, U_z); rho = 1."""
    x, _, _ = _grid(nx, ny, nz, device)
    u = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=device)
    for i in range(3):
        u[i] += float(U[i])
    u[1] += amplitude * torch.sin(2 * math.pi * x / nx)
    rho = torch.ones((nz, ny, nx), dtype=torch.float64, device=device)
    return rho, u


def cross_shear(nx, ny, nz, U=0.0, amplitude=0.01, device="cpu"):
    """x-invariant flow u = (U + A sin(2 pi y/ny) sin(2 pi z/nz), 0, 0); rho = 1."""
    _, y, z = _grid(nx, ny, nz, device)
    u = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=device)
    u[0] = U + amplitude * torch.sin(2 * math.pi * y / ny) * torch.sin(2 * math.pi * z / nz)
    rho = torch.ones((nz, ny, nx), dtype=torch.float64, device=device)
    return rho, u


def rest(nx, ny, nz, device="cpu"):
    """Fluid at rest, rho = 1."""
    return (torch.ones((nz, ny, nx), dtype=torch.float64, device=device),
            torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=device))


def _solenoidal_modes(kmax, seed, spectrum):
    """Complex Fourier coefficients c[n] (3-vectors) for integer wave vectors
    |n| <= kmax, drawn in a fixed, grid-independent order, projected onto the
    plane normal to n, with amplitude sqrt(spectrum(|n|) / (4 pi |n|^2))."""
    rng = np.random.default_rng(seed)
    r = np.arange(-kmax, kmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    coef = rng.standard_normal((n.shape[0], 3)) + 1j * rng.standard_normal((n.shape[0], 3))
    k2 = (n * n).sum(axis=1).astype(np.float64)
    keep = (k2 > 0) & (k2 <= kmax * kmax)
    n, coef, k2 = n[keep], coef[keep], k2[keep]
    coef = coef - n * ((coef * n).sum(axis=1) / k2)[:, None]
    k = np.sqrt(k2)
    coef *= np.sqrt(spectrum(k) / (4 * math.pi * k2))[:, None]
    return n, coef


def _synthesize(n, coef, nx, ny, nz, u_rms, device):
    if max(np.abs(n).max() * 2, 0) >= min(nx, ny, nz):
        raise ValueError("grid too small for the requested wave numbers")
    u = torch.zeros((3, nz, ny, nx), dtype=torch.float64, device=device)
    # arrays are [z, y, x]; n = (n_x, n_y, n_z)
    iz = torch.as_tensor(n[:, 2] % nz, device=device)
    iy = torch.as_tensor(n[:, 1] % ny, device=device)
    ix = torch.as_tensor(n[:, 0] % nx, device=device)
    for i in range(3):
        spec = torch.zeros((nz, ny, nx), dtype=torch.complex128, device=device)
        spec[iz, iy, ix] = torch.as_tensor(coef[:, i], device=device)
        u[i] = torch.fft.ifftn(spec).real * (nx * ny * nz)
        del spec
    rms = torch.sqrt((u * u).mean())  # per-component rms, sqrt(<|u|^2> / 3)
    u *= u_rms / rms
    return u


def random_solenoidal(nx, ny, nz, kmax=8, u_rms=0.02, seed=1, device="cpu"):
    """Divergence-free random velocity from Gaussian Fourier modes with
    |n| <= kmax (flat spectrum), scaled to a per-component rms of u_rms; rho = 1."""
    n, coef = _solenoidal_modes(kmax, seed, lambda k: np.ones_like(k))
    u = _synthesize(n, coef, nx, ny, nz, u_rms, device)
    return torch.ones((nz, ny, nx), dtype=torch.float64, device=device), u


def hit_spectrum(nx, ny, nz, u_rms=0.04, seed=4, k0=4.0, kmax=32, device="cpu"):
    """Decaying-turbulence initial field: solenoidal random modes with energy
    spectrum E(k) ~ k^4 exp(-2 (k/k0)^2) for |n| <= kmax, scaled to a
    per-component rms of u_rms; rho = 1.  The same seed gives the same modes on
    every grid that resolves |n| <= kmax, so a coarser grid samples the same
    continuous field."""
    n, coef = _solenoidal_modes(kmax, seed, lambda k: k ** 4 * np.exp(-2.0 * (k / k0) ** 2))
    u = _synthesize(n, coef, nx, ny, nz, u_rms, device)
    return torch.ones((nz, ny, nx), dtype=torch.float64, device=device), u
