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
