"""Pins of the learned-closure oracle (oracle/closure.py): back-propagation against finite
differences of the loss, the convolution against SciPy's periodic 2-D correlation, the subgrid
terms against the exact box-filter identity for linear fields, and the analytic closure against
the closed form of the central difference on sine fields."""
import numpy as np
import pytest

from oracle import closure as oc

RNG = np.random.default_rng(11)


def _small_problem(h=6, w=7, batch=2):
    theta = oc.init_params(3) + 0.01 * RNG.normal(size=oc.num_params())
    x = RNG.normal(size=(batch, 12, h, w))
    t = RNG.normal(size=(batch, 4, h, w)) * 0.3
    return theta, x, t


def test_param_count():
    assert oc.num_params() == 13892


def test_conv_matches_scipy_periodic_correlation():
    signal = pytest.importorskip("scipy.signal")
    a = RNG.normal(size=(1, 3, 8, 9))
    W = RNG.normal(size=(2, 3, 3, 3))
    b = RNG.normal(size=2)
    y = oc.conv3x3(a, W, b)
    for co in range(2):
        ref = b[co] + sum(signal.correlate2d(a[0, ci], W[co, ci], mode="same", boundary="wrap")
                          for ci in range(3))
        np.testing.assert_allclose(y[0, co], ref, atol=1e-12)


def test_backprop_matches_finite_differences():
    theta, x, t = _small_problem()
    L, g = oc.gradient(theta, x, t)
    assert abs(L - oc.loss(theta, x, t)) < 1e-14
    idx = list(RNG.choice(oc.num_params(), 40, replace=False)) + [0, 3455, 3456, 3487, 3488,
                                                                     13000, 13891]
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (oc.loss(theta + e, x, t) - oc.loss(theta - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, i


@pytest.mark.parametrize("r", [2, 4, 8])
def test_subgrid_terms_exact_for_linear_fields(r):
    """Box filter of a product of linear fields: bar(fg) - fbar gbar = (r^2-1)/12 sum_b df_b dg_b
    (the discrete top-hat's variance; the continuous Delta^2/12 of Sec. 2.1)."""
    n = 4 * r
    y, x = np.mgrid[0:n, 0:n].astype(float)
    gj = RNG.uniform(-1e-3, 1e-3, (2, 2))
    gb = RNG.uniform(-1e-3, 1e-3, (2, 2))
    jx = 0.03 + gj[0, 0] * x + gj[0, 1] * y
    jy = -0.02 + gj[1, 0] * x + gj[1, 1] * y
    bx = 0.01 + gb[0, 0] * x + gb[0, 1] * y
    by = 0.02 + gb[1, 0] * x + gb[1, 1] * y
    rho = np.ones((n, n))
    c, _ = oc.subgrid_terms(rho, jx, jy, bx, by, r)
    v = (r * r - 1) / 12.0
    G = lambda a, b: a @ b  # sum over beta of d_beta a d_beta b
    expect = [v * (G(gj[0], gj[1]) - G(gb[0], gb[1])),
              v * (G(gj[0], gj[0]) - G(gj[1], gj[1]) - G(gb[0], gb[0]) + G(gb[1], gb[1])),
              v * (G(gj[0], gj[0]) + G(gj[1], gj[1])),
              v * (G(gj[0], gb[1]) - G(gj[1], gb[0]))]
    for q in range(4):
        np.testing.assert_allclose(c[q], expect[q], atol=1e-16)


def test_analytic_closure_on_sine_fields():
    n, A, C, phi, delta = 16, 0.02, 0.03, 0.7, 2.0
    k = 2 * np.pi / n
    y = np.arange(n)[:, None] * np.ones((1, n))
    z = np.zeros((n, n))
    jx, by = A * np.sin(k * y), C * np.sin(k * y + phi)
    a = oc.analytic(np.ones((n, n)), jx, z, z, by, delta)
    kd = delta ** 2 / 12
    d_jx = A * np.sin(k) * np.cos(k * y)
    d_by = C * np.sin(k) * np.cos(k * y + phi)
    np.testing.assert_allclose(a[0], 0 * y, atol=1e-18)
    np.testing.assert_allclose(a[1], kd * (d_jx ** 2 + d_by ** 2), atol=1e-17)
    np.testing.assert_allclose(a[2], kd * d_jx ** 2, atol=1e-17)
    np.testing.assert_allclose(a[3], kd * d_jx * d_by, atol=1e-17)


# ------------------------------------------------------------------ the corrected step
# The analytic closure a0..a3 is exactly the Delta^2/12 part of the filtered equilibria
# (Eqs. FilterExampleSmall/Large, density gradients dropped as in Sec. 3), written per
# subgrid term.  So one step with Delta = 0 plus the correction a (taken on the same state,
# central differences) must equal one step with Delta = 2 (the oracle's filt_ratio/filt_prod
# route), and each correction channel must land in the equilibrium moments where the k-terms
# of its own products land: c0 in M_3, c1 in M_4, c2 in M_7 and M_8 (times -3), c3 in the
# electric field of N^eq.  This pins oracle_step_corrected against the Delta^2 code path.

import oracle as _or
from paper_1705_09807_gb300.inputs import smooth_random_fields as _smooth

_CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
_CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _generic_state(nx=13, ny=11, seed=21):
    """A non-equilibrium state with O(1e-2) gradients: equilibria of smooth random fields
    advanced by three plain steps."""
    fields = _smooth(nx, ny, seed, amp_u=0.04, amp_b=0.04, amp_rho=0.02)
    f, g = _or.init(*fields)
    return _or.step(f, g, _or.srt_rates(0.01), _or.rate_from_diffusivity(0.01), 0.0, 3)


def _post_collision(f, g):
    """Undo the streaming of a one-step result: f*_i(x) = f_i(x + c_i)."""
    fs = np.stack([np.roll(f[i], (-_CY[i], -_CX[i]), axis=(0, 1)) for i in range(9)])
    gs = np.stack([np.stack([np.roll(g[a, i], (-_CY[i], -_CX[i]), axis=(0, 1)) for i in range(9)])
                   for a in range(2)])
    return fs, gs


def _analytic_of(f, g, delta):
    rho, ux, uy, bx, by = _or.moments(f, g)
    return oc.analytic(rho, rho * ux, rho * uy, bx, by, delta)


_RATES = {"srt": (_or.srt_rates(0.01), _or.rate_from_diffusivity(0.02)),
          "mrt": (np.array([1.0, 1.0, 1.0, 1.6, 1.3, 1.1, 1.2, 1.45, 0.9]), 1.7)}


@pytest.mark.parametrize("rates", ["srt", "mrt"])
def test_corrected_step_with_analytic_terms_equals_filtered_step(rates):
    s, sm = _RATES[rates]
    f, g = _generic_state()
    corr = _analytic_of(f, g, 2.0)
    assert np.abs(corr).max() > 1e-5  # the terms are far above the tolerance below
    f1, g1 = _or.step_corrected(f, g, s, sm, 0.0, 1, corr, stencil=0)
    f2, g2 = _or.step(f, g, s, sm, 2.0, 1, stencil=0)
    np.testing.assert_allclose(f1, f2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-15)
    # and the correction is not a no-op: the plain Delta = 0 step differs by far more
    f0, _ = _or.step(f, g, s, sm, 0.0, 1, stencil=0)
    assert np.abs(f0 - f2).max() > 1e-7


@pytest.mark.parametrize("rates", ["srt", "mrt"])
def test_each_correction_channel_lands_in_its_own_moments(rates):
    """Channel q alone moves exactly the post-collision moments that the Delta^2 terms of its
    products move (rows of Eq. FluidTMatrix / Eq. MagTMatrix), with the same sign, and no other."""
    s, sm = _RATES[rates]
    T = oc_tables()["T"]
    Tm = oc_tables()["Tm"]
    f, g = _generic_state(seed=22)
    a = _analytic_of(f, g, 2.0)

    def moments_after(fn):
        fs, gs = _post_collision(*fn())
        M = np.einsum("ji,ixy->jxy", T, fs)
        N = np.einsum("ji,aixy->ajxy", Tm, gs)
        return M, N

    M0, N0 = moments_after(lambda: _or.step(f, g, s, sm, 0.0, 1))
    M2, N2 = moments_after(lambda: _or.step(f, g, s, sm, 2.0, 1))
    dM, dN = M2 - M0, N2 - N0  # what the Delta^2 terms do, row by row
    rows = {0: [3], 1: [4], 2: [7, 8], 3: []}
    for q in range(4):
        corr = np.zeros_like(a)
        corr[q] = a[q]
        Mq, Nq = moments_after(lambda: _or.step_corrected(f, g, s, sm, 0.0, 1, corr))
        want_M = np.zeros_like(dM)
        want_M[rows[q]] = dM[rows[q]]
        want_N = dN if q == 3 else np.zeros_like(dN)
        np.testing.assert_allclose(Mq - M0, want_M, rtol=0, atol=1e-15, err_msg=f"channel {q}")
        np.testing.assert_allclose(Nq - N0, want_N, rtol=0, atol=1e-15, err_msg=f"channel {q}")
        moved = [j for j in range(9) if np.abs(Mq[j] - M0[j]).max() > 1e-12]
        assert moved == rows[q], (q, moved)
    # every fluid row the Delta^2 terms move belongs to exactly one channel
    assert [j for j in range(9) if np.abs(dM[j]).max() > 1e-12] == [3, 4, 7, 8]
    assert np.abs(dN).max() > 1e-9


def oc_tables():
    return _or.tables()
