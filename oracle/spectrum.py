"""Plain CPU oracle for the LES-vs-DNS comparison tools (box filter, energy spectra).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): used by the tests and the
benchmark's CPU legs, never by the product path.

* ``block_mean(a, r)``: the box filter of width r cells followed by downsampling by r, i.e.
  the average of each r x r block.  This is the discrete counterpart of the spatial filter of
  Sec. 1 (Eq. VelFilter) with a top-hat kernel G, whose second moment is r^2/12 per direction
  (the Delta^2/12 of Sec. 2.1 with Delta = r).
* ``energy_spectrum(ux, uy, bx, by, nbins)``: shell sums of the Fourier energy,
  E_kin(s) = 1/2 sum_{k in shell s} (|u_x^(k)|^2 + |u_y^(k)|^2) and likewise E_mag with B, where
  a^(k) = n^-2 sum_x a(x) exp(-2 pi i k.x / n) and shell s holds the integer wavevectors with
  (2s - 1)^2 < 4 |k|^2 < (2s + 1)^2 (nearest integer |k|; no ties are possible).  By Parseval
  the sum over all wavevectors equals the mean of |u|^2/2 (resp. |B|^2/2).
"""
from __future__ import annotations

import numpy as np


def block_mean(a: np.ndarray, r: int) -> np.ndarray:
    ny, nx = a.shape
    if nx % r or ny % r:
        raise ValueError("grid not divisible by r")
    out = np.zeros((ny // r, nx // r))
    for j in range(ny // r):
        for i in range(nx // r):
            out[j, i] = a[j * r:(j + 1) * r, i * r:(i + 1) * r].sum() / (r * r)
    return out


def wavenumbers(n: int) -> np.ndarray:
    """Integer wavenumbers in FFT order: 0, 1, ..., n/2 - 1, -n/2, ..., -1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def shell_index(n: int) -> np.ndarray:
    """Shell of every wavevector [ky, kx]: the integer s with (2s-1)^2 < 4|k|^2 < (2s+1)^2."""
    k = wavenumbers(n)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    # f = floor(|k|) is exact for these integers; |k| >= f + 1/2 exactly when 4 k2 > (2f+1)^2
    s = np.floor(np.sqrt(k2)).astype(np.int64)
    s = np.where(4 * k2 >= (2 * s + 1) ** 2, s + 1, s)
    assert np.all(((2 * s - 1) ** 2 < 4 * k2) | (s == 0)) and np.all(4 * k2 < (2 * s + 1) ** 2)
    return s


def energy_spectrum(ux, uy, bx, by, nbins: int):
    n = ux.shape[0]
    assert ux.shape == (n, n)
    s = shell_index(n)
    ek = np.zeros(nbins)
    em = np.zeros(nbins)
    pk = sum(np.abs(np.fft.fft2(a) / (n * n)) ** 2 for a in (ux, uy)) * 0.5
    pm = sum(np.abs(np.fft.fft2(a) / (n * n)) ** 2 for a in (bx, by)) * 0.5
    for b in range(nbins):
        m = s == b
        ek[b] = pk[m].sum()
        em[b] = pm[m].sum()
    return ek, em
