"""Seeded synthetic inputs for the EFM collision workloads (NumPy, FP64).

This module only draws distribution functions on the velocity grid; it contains none of the
collision operator's arithmetic and is shared by the tests (CUDA path and oracle alike) and the
benchmark.  Grid convention: per axis j = -N/2 .. N/2-1, v = h j, h = 2L/N, C order.

Workloads (shapes and value distributions):
* ``bigauss2d``: two isotropic unit-temperature Gaussians centred at (+-1.5, 0), total mass 1
  (the shape of the paper's Example 2 with the centres moved to +-1.5).
* ``bkw``: the BKW closed-form solution (2D Example 1 / 3D Example 4 of the paper) at time t,
  optionally scaled to density rho, temperature theta and bulk velocity u:
  rho theta^{-d/2} f_BKW(t rho; (v - u)/sqrt(theta)) (still an exact solution for Maxwell
  molecules, with time scaled by rho).
* ``mixture_cells``: Maxwellians with density U[0.5, 2], bulk velocity |u| <= 1 (uniform in the
  ball), temperature U[0.5, 2], times (1 + 0.3 sum of 3 Gaussian bumps) with centres uniform in
  the ball |c - u| <= 2 sqrt(theta), widths U[0.3, 1] and unit peak, renormalised to the drawn
  density; one seeded generator per cell (seed + cell index).
* ``bkw_family_cells``: BKW cells with t0 ~ U[0.5, 10], rho ~ U[0.5, 2], theta ~ U[0.5, 2],
  |u| <= 1.
"""
from __future__ import annotations

import numpy as np


def grid(d: int, N: int, L: float):
    h = 2.0 * L / N
    v1 = (np.arange(N) - N // 2) * h
    return np.meshgrid(*([v1] * d), indexing="ij")


def _bkw_profile(d: int, t: float, v2):
    if d == 2:
        S = 1.0 - np.exp(-t / 8.0) / 2.0
        return np.exp(-v2 / (2 * S)) / (2 * np.pi * S) * ((2 * S - 1) / S + (1 - S) / (2 * S * S) * v2)
    S = 1.0 - 2.0 * np.exp(-t / 6.0) / 5.0
    return np.exp(-v2 / (2 * S)) / (2 * np.pi * S) ** 1.5 * ((5 * S - 3) / (2 * S) + (1 - S) / (2 * S * S) * v2)


def bkw(d: int, N: int, L: float, t: float, rho: float = 1.0, theta: float = 1.0, u=None) -> np.ndarray:
    V = grid(d, N, L)
    u = np.zeros(d) if u is None else np.asarray(u, dtype=np.float64)
    v2 = sum(((x - ui) ** 2 for x, ui in zip(V, u))) / theta
    return rho * theta ** (-d / 2.0) * _bkw_profile(d, t * rho, v2)


def bigauss2d(N: int, L: float, shift: float = 1.5) -> np.ndarray:
    V = grid(2, N, L)
    a = np.exp(-((V[0] - shift) ** 2 + V[1] ** 2) / 2.0)
    b = np.exp(-((V[0] + shift) ** 2 + V[1] ** 2) / 2.0)
    return (a + b) / (4.0 * np.pi)


def _ball(rng, d, radius):
    x = rng.normal(size=d)
    x /= np.linalg.norm(x)
    return x * radius * rng.uniform() ** (1.0 / d)


def mixture_cell(d: int, N: int, L: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0)
    theta = rng.uniform(0.5, 2.0)
    u = _ball(rng, d, 1.0)
    V = grid(d, N, L)
    h = 2.0 * L / N
    r2 = sum((x - ui) ** 2 for x, ui in zip(V, u))
    F = np.exp(-r2 / (2 * theta)) / (2 * np.pi * theta) ** (d / 2.0)
    bumps = np.zeros_like(F)
    for _ in range(3):
        c = u + _ball(rng, d, 2.0 * np.sqrt(theta))
        w = rng.uniform(0.3, 1.0)
        bumps += np.exp(-sum((x - ci) ** 2 for x, ci in zip(V, c)) / (2 * w * w))
    F = F * (1.0 + 0.3 * bumps)
    return F * (rho / (F.sum() * h ** d))


def mixture_cells(d: int, N_list, L: float, seed: int = 1234) -> list:
    return [mixture_cell(d, int(N), L, seed + i) for i, N in enumerate(N_list)]


def bkw_family_cells(d: int, N: int, L: float, ncells: int, seed: int = 4321) -> np.ndarray:
    out = np.empty((ncells,) + (N,) * d)
    for i in range(ncells):
        rng = np.random.default_rng(seed + i)
        t0 = rng.uniform(0.5, 10.0)
        rho = rng.uniform(0.5, 2.0)
        theta = rng.uniform(0.5, 2.0)
        u = _ball(rng, d, 1.0)
        out[i] = bkw(d, N, L, t0, rho, theta, u)
    return out


def ragged_sizes(ncells: int, choices=(24, 32, 40, 48), seed: int = 1234) -> np.ndarray:
    """Cell sizes N drawn uniformly from ``choices``."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(choices), size=ncells)


def pack(cells) -> np.ndarray:
    """Concatenate cells back to back (cell-major, C order)."""
    return np.concatenate([np.ascontiguousarray(c).ravel() for c in cells])


def bkw_family_params(ncells: int, seed: int = 4321, d: int = 3):
    """Per-cell (t0, rho, theta, u) of the BKW family, drawn exactly as bkw_family_cells does."""
    t0 = np.empty(ncells)
    rho = np.empty(ncells)
    theta = np.empty(ncells)
    u = np.empty((ncells, d))
    for i in range(ncells):
        rng = np.random.default_rng(seed + i)
        t0[i] = rng.uniform(0.5, 10.0)
        rho[i] = rng.uniform(0.5, 2.0)
        theta[i] = rng.uniform(0.5, 2.0)
        u[i] = _ball(rng, d, 1.0)
    return t0, rho, theta, u


def bkw_family_torch(N: int, L: float, ncells: int, seed: int = 4321, device="cuda", dtype=None, out=None):
    """bkw_family_cells evaluated on a torch device (same draws, same formula), [ncells, N, N, N]."""
    import torch
    dtype = dtype or torch.float32
    t0, rho, theta, u = bkw_family_params(ncells, seed, 3)
    h = 2.0 * L / N
    v1 = (torch.arange(N, device=device, dtype=torch.float64) - N // 2) * h
    if out is None:
        out = torch.empty((ncells, N, N, N), device=device, dtype=dtype)
    for c0 in range(0, ncells, 256):
        c1 = min(ncells, c0 + 256)
        uu = torch.as_tensor(u[c0:c1], device=device)
        th = torch.as_tensor(theta[c0:c1], device=device)[:, None, None, None]
        rh = torch.as_tensor(rho[c0:c1], device=device)[:, None, None, None]
        S = 1.0 - 2.0 * torch.exp(-torch.as_tensor(t0[c0:c1] * rho[c0:c1], device=device) / 6.0) / 5.0
        S = S[:, None, None, None]
        x = (v1[None, :] - uu[:, 0:1]) ** 2
        y = (v1[None, :] - uu[:, 1:2]) ** 2
        z = (v1[None, :] - uu[:, 2:3]) ** 2
        v2 = (x[:, :, None, None] + y[:, None, :, None] + z[:, None, None, :]) / th
        f = torch.exp(-v2 / (2 * S)) / (2 * np.pi * S) ** 1.5 * ((5 * S - 3) / (2 * S) + (1 - S) / (2 * S * S) * v2)
        out[c0:c1] = (rh * th ** -1.5 * f).to(dtype)
    return out
