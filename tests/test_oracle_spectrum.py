"""Pins of the oracle's box filter and energy spectra (oracle/spectrum.py) against closed
forms: Parseval's identity, single Fourier modes, and the moments of the discrete top-hat."""
import numpy as np
import pytest

from oracle import spectrum as sp

RNG = np.random.default_rng(7)


@pytest.mark.parametrize("n", [8, 30, 64])
def test_parseval(n):
    f = [RNG.normal(size=(n, n)) for _ in range(4)]
    nb = int(np.ceil(np.sqrt(2) * n / 2)) + 2
    ek, em = sp.energy_spectrum(*f, nbins=nb)
    assert abs(ek.sum() - 0.5 * np.mean(f[0] ** 2 + f[1] ** 2)) < 1e-13
    assert abs(em.sum() - 0.5 * np.mean(f[2] ** 2 + f[3] ** 2)) < 1e-13


@pytest.mark.parametrize("kx,ky,shell", [(3, 4, 5), (1, 0, 1), (0, 7, 7), (5, 5, 7), (2, 3, 4)])
def test_single_mode_lands_in_its_shell(kx, ky, shell):
    n, A, C = 32, 0.3, 0.2
    y, x = np.mgrid[0:n, 0:n]
    ph = 2 * np.pi * (kx * x + ky * y) / n
    z = np.zeros((n, n))
    ek, em = sp.energy_spectrum(A * np.cos(ph), z, z, C * np.sin(ph), nbins=n // 2)
    expect_k = np.zeros(n // 2)
    expect_k[shell] = A * A / 4     # two wavevectors +-k, each |A/2|^2, times 1/2
    expect_m = np.zeros(n // 2)
    expect_m[shell] = C * C / 4
    np.testing.assert_allclose(ek, expect_k, atol=1e-15)
    np.testing.assert_allclose(em, expect_m, atol=1e-15)


def test_shell_boundaries_are_nearest_integer():
    n = 16
    s = sp.shell_index(n)
    k = sp.wavenumbers(n)
    mag = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    assert np.array_equal(s, np.rint(mag).astype(np.int64))


@pytest.mark.parametrize("r", [2, 4, 8])
def test_block_mean_moments_of_the_discrete_top_hat(r):
    """Block means of polynomials: a linear field is reproduced at the block centre, and x^2
    picks up the top-hat's second moment (r^2 - 1)/12 (the discrete form of Delta^2/12)."""
    n = 8 * r
    y, x = np.mgrid[0:n, 0:n].astype(float)
    lin = 0.3 + 0.01 * x - 0.02 * y
    c = (np.arange(n // r) * r + (r - 1) / 2.0)
    np.testing.assert_allclose(sp.block_mean(lin, r), 0.3 + 0.01 * c[None, :] - 0.02 * c[:, None],
                               atol=1e-15)
    np.testing.assert_allclose(sp.block_mean(x * x, r),
                               np.broadcast_to(c[None, :] ** 2 + (r * r - 1) / 12.0, (n // r, n // r)),
                               atol=1e-12)
