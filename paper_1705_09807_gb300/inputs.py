"""Seeded synthetic initial conditions (workloads), shared by the tests, the benchmark and
the oracle checks.  This module holds no arithmetic of the method itself: it only builds
the fields rho, u, B that a run starts from, as float64 numpy arrays of shape [ny, nx]
(x fastest).  Every random number comes from one counter-based generator (splitmix64 of
seed and cell index), so both sides of a comparison receive identical data.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """U[0,1) doubles: the splitmix64 output (Steele, Lea & Flood 2014) for counters
    ``seed*2^32 + 1 .. seed*2^32 + n``, top 53 bits scaled by 2^-53."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64) + np.uint64((int(seed) & 0xFFFFFFFF) << 32)
        z = idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def kh_jet(n: int, u0: float = 0.05, delta_frac: float = 1.0 / 32, b0: float = 0.02,
           pert: float = 1e-3, noise: float = 1e-5, seed: int = 1, ny: int | None = None):
    """Magnetized Kelvin-Helmholtz double shear layer on an n x ny periodic grid.

    u_x(y) = U0 [tanh((y - N/4)/d) - tanh((y - 3N/4)/d) - 1],  d = delta_frac * N
    u_y    = pert sin(2 pi x / N) + noise (2 U - 1),           U ~ splitmix64(seed, cell)
    B = (B0, 0), rho = 1.
    Returns (rho, ux, uy, bx, by), each [ny, n] float64.
    """
    nx = n
    ny = n if ny is None else ny
    d = delta_frac * ny
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    ux = u0 * (np.tanh((y - ny / 4.0) / d) - np.tanh((y - 3.0 * ny / 4.0) / d) - 1.0)
    ux = np.broadcast_to(ux, (ny, nx)).copy()
    rnd = splitmix64_uniform(seed, nx * ny).reshape(ny, nx)
    uy = pert * np.sin(2.0 * np.pi * x / nx) + noise * (2.0 * rnd - 1.0)
    uy = np.broadcast_to(uy, (ny, nx)).copy()
    rho = np.ones((ny, nx))
    bx = np.full((ny, nx), float(b0))
    by = np.zeros((ny, nx))
    return rho, ux, uy, bx, by


def sech2_jet(n: int, u0: float = 4.88e-2, b0_ratio: float = 0.005, modes: int = 4,
              pert_frac: float = 0.01):
    """The paper's magnetized jet (Sec. 3): U_y = U0 sech^2(2 pi 4 x / L), B_y = B0 = 0.005 U0,
    with 1% mode-4 perturbations U_y += 0.01 U0 sin(2 pi 4 x/L), B_y += 0.01 B0 sin(2 pi 4 x/L),
    U_x = 0.01 U0 sin(2 pi 4 y/L), B_x = 0.01 B0 sin(2 pi 4 y/L); rho = 1."""
    L = float(n)
    b0 = b0_ratio * u0
    y = np.arange(n, dtype=np.float64)[:, None]
    x = np.arange(n, dtype=np.float64)[None, :]
    kx = 2.0 * np.pi * modes * x / L
    ky = 2.0 * np.pi * modes * y / L
    # centre the jet at x = L/2 so the periodic profile is smooth
    arg = 2.0 * np.pi * modes * (x - L / 2.0) / L
    uy = u0 / np.cosh(arg) ** 2 + pert_frac * u0 * np.sin(kx)
    by = b0 + pert_frac * b0 * np.sin(kx)
    ux = pert_frac * u0 * np.sin(ky)
    bx = pert_frac * b0 * np.sin(ky)
    shp = (n, n)
    return (np.ones(shp), np.broadcast_to(ux, shp).copy(), np.broadcast_to(uy, shp).copy(),
            np.broadcast_to(bx, shp).copy(), np.broadcast_to(by, shp).copy())


def block_mean(field: np.ndarray, r: int) -> np.ndarray:
    """r x r block average (box filter of width r followed by downsampling by r)."""
    ny, nx = field.shape
    if ny % r or nx % r:
        raise ValueError("grid not divisible by the block size")
    return field.reshape(ny // r, r, nx // r, r).mean(axis=(1, 3))


def smooth_random_fields(nx: int, ny: int, seed: int, amp_u: float = 0.02, amp_b: float = 0.02,
                         amp_rho: float = 0.01, kmax: int = 3):
    """Smooth random periodic fields (a few low Fourier modes with seeded amplitudes),
    for tests that need a generic non-equilibrium-looking state.  Returns (rho, ux, uy, bx, by)."""
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    r = splitmix64_uniform(seed, 5 * (2 * kmax + 1) ** 2 * 2).reshape(5, -1, 2)
    out = []
    amps = (amp_rho, amp_u, amp_u, amp_b, amp_b)
    for q in range(5):
        fld = np.zeros((ny, nx))
        m = 0
        for kx in range(-kmax, kmax + 1):
            for ky in range(-kmax, kmax + 1):
                a, ph = r[q, m]
                m += 1
                if kx == 0 and ky == 0:
                    continue
                fld += (2 * a - 1) * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + 2 * np.pi * ph)
        fld *= amps[q] / (2 * kmax + 1)
        out.append(fld)
    out[0] = 1.0 + out[0]
    return tuple(out)
