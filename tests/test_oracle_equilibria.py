"""Pins of the oracle's equilibria and filtered (Delta^2) equilibrium moments.

* Eq. feq / Eq. geq transformed by the printed T / T_m must give the printed
  Eq. KinMomentEq / Eq. MagMomentEq tables (two independent printed statements agree).
* The Delta^2 terms are pinned by their definition (Sec. 2.1, Eq. FilterExampleSmall and
  FilterExampleLarge): for linear fields and constant density (the density-gradient terms are
  dropped, Sec. 3) a box filter of width Delta, whose second moment is Delta^2/12 in each
  direction, reproduces the O(Delta^2) expansion exactly.  The test integrates the printed,
  unfiltered tables over the box with Gauss-Legendre quadrature, which is exact for these
  quadratics, and compares with the oracle's filtered moments.
* The printed simplified filtered M_3^eq of Sec. 3 is checked term by term.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from golden_io import equilibrium_exprs, paper_tables

RNG = np.random.default_rng(20170527)
SYM = sp.symbols("rho jx jy bx by")


def _table_funcs():
    M_exprs, N_exprs = equilibrium_exprs()
    rho, jx, jy, bx, by = SYM
    ja, ba = sp.symbols("ja ba")
    fM = [sp.lambdify(SYM, e, "numpy") for e in M_exprs]
    fN = []
    for comp, (jc, bc) in enumerate(((jx, bx), (jy, by))):
        fN.append([sp.lambdify(SYM, sp.sympify(e).subs({ja: jc, ba: bc}), "numpy") for e in N_exprs])
    return fM, fN


FM, FN = _table_funcs()


def M_table(rho, J, B):
    return np.array([float(np.broadcast_to(f(rho, J[0], J[1], B[0], B[1]), ())) for f in FM])


def N_table_literal(rho, J, B):
    return np.array([[float(np.broadcast_to(f(rho, J[0], J[1], B[0], B[1]), ())) for f in FN[a]]
                     for a in range(2)])


def N_table_read(rho, J, B):
    """Reading R2: the printed products rho u_b B_a are taken with u = J/rho, i.e. the rows
    that carry a J (rows 1, 2, 6, 7) are divided by rho."""
    N = N_table_literal(rho, J, B)
    N[:, [1, 2, 6, 7]] /= rho
    return N


def random_state():
    rho = RNG.uniform(0.6, 1.4)
    u = RNG.uniform(-0.1, 0.1, 2)
    B = RNG.uniform(-0.1, 0.1, 2)
    return rho, u, B


@pytest.mark.parametrize("trial", range(20))
def test_T_feq_is_the_printed_M_table(trial):
    p = paper_tables()
    rho, u, B = random_state()
    f = oracle.feq(rho, u[0], u[1], B[0], B[1])
    np.testing.assert_allclose(p["T"] @ f, M_table(rho, rho * u, B), rtol=0, atol=2e-15)


@pytest.mark.parametrize("trial", range(20))
def test_Tm_geq_is_the_printed_N_table_with_u(trial):
    p = paper_tables()
    rho, u, B = random_state()
    g = oracle.geq(u[0], u[1], B[0], B[1])
    N = np.stack([p["Tm"] @ g[a] for a in range(2)])
    np.testing.assert_allclose(N, N_table_read(rho, rho * u, B), rtol=0, atol=2e-16)


def test_literal_N_table_needs_the_u_reading():
    """At rho != 1 the N^eq table as printed (rho u) does not equal T_m g^eq; with u it does."""
    p = paper_tables()
    rho, u, B = 1.3, np.array([0.05, -0.02]), np.array([0.03, 0.07])
    g = oracle.geq(u[0], u[1], B[0], B[1])
    N = np.stack([p["Tm"] @ g[a] for a in range(2)])
    assert np.max(np.abs(N - N_table_literal(rho, rho * u, B))) > 1e-4
    assert np.max(np.abs(N - N_table_read(rho, rho * u, B))) < 1e-16


@pytest.mark.parametrize("trial", range(10))
def test_oracle_equilibrium_moments_at_delta0_are_the_tables(trial):
    rho, u, B = random_state()
    J = rho * u
    gJ = RNG.normal(size=4)
    gB = RNG.normal(size=4)
    np.testing.assert_allclose(oracle.meq(rho, J, B, gJ, gB, 0.0), M_table(rho, J, B), atol=2e-16)
    np.testing.assert_allclose(oracle.neq(rho, J, B, gJ, gB, 0.0), N_table_read(rho, J, B),
                               atol=2e-16)


def _box_average(func, delta):
    """Average of func(r) over the square [-delta/2, delta/2]^2 by 3-point Gauss-Legendre per
    direction (exact for polynomials of degree <= 5 in each coordinate)."""
    xg, wg = np.polynomial.legendre.leggauss(3)
    xs = 0.5 * delta * xg
    ws = 0.5 * wg
    acc = 0.0
    for xi, wi in zip(xs, ws):
        for yj, wj in zip(xs, ws):
            acc = acc + wi * wj * func(np.array([xi, yj]))
    return acc


@pytest.mark.parametrize("delta", [0.5, 1.0, 2.0, 3.0])
@pytest.mark.parametrize("trial", range(6))
def test_filtered_moments_equal_box_filter_of_printed_tables(delta, trial):
    """Definition of the filtered equilibrium (Sec. 2.1): bar(M^eq(rho, J, B)) for J, B linear in
    space and rho constant equals M^eq(rho, Jbar, Bbar) + Delta^2 Mbar^(Delta)."""
    rho = RNG.uniform(0.7, 1.3)
    J0 = RNG.uniform(-0.1, 0.1, 2)
    B0 = RNG.uniform(-0.1, 0.1, 2)
    GJ = RNG.uniform(-0.05, 0.05, (2, 2))   # GJ[a, beta] = d_beta J_a
    GB = RNG.uniform(-0.05, 0.05, (2, 2))
    Mbar = _box_average(lambda r: M_table(rho, J0 + GJ @ r, B0 + GB @ r), delta)
    Nbar = _box_average(lambda r: N_table_read(rho, J0 + GJ @ r, B0 + GB @ r), delta)
    Mo = oracle.meq(rho, J0, B0, GJ.ravel(), GB.ravel(), delta)
    No = oracle.neq(rho, J0, B0, GJ.ravel(), GB.ravel(), delta)
    np.testing.assert_allclose(Mo, Mbar, rtol=0, atol=1e-15)
    np.testing.assert_allclose(No, Nbar, rtol=0, atol=1e-15)
    # the filter changes the answer (the terms are really there)
    if delta >= 1.0:
        assert np.max(np.abs(Mo - M_table(rho, J0, B0))) > 1e-5


def test_simplified_filtered_M3_as_printed():
    """Sec. 3, simplified Mbar_3^eq: Jx Jy/rho - Bx By + Delta^2/(12 rho) d_b Jx d_b Jy
    - Delta^2/12 d_b Bx d_b By (every term checked by switching the others off)."""
    rho, delta = 1.2, 2.0
    J = np.array([0.03, -0.04])
    B = np.array([0.02, 0.05])
    GJ = np.array([[0.011, -0.007], [0.005, 0.013]])
    GB = np.array([[-0.004, 0.009], [0.012, -0.006]])
    k = delta ** 2 / 12.0
    expected = (J[0] * J[1] / rho - B[0] * B[1]
                + k / rho * (GJ[0] @ GJ[1]) - k * (GB[0] @ GB[1]))
    got = oracle.meq(rho, J, B, GJ.ravel(), GB.ravel(), delta)[3]
    assert abs(got - expected) < 1e-17
    # Delta^2 terms of M_3 only through these two gradient products
    z = np.zeros(4)
    assert abs(oracle.meq(rho, J, B, z, GB.ravel(), delta)[3]
               - (J[0] * J[1] / rho - B[0] * B[1] - k * (GB[0] @ GB[1]))) < 1e-17
    assert abs(oracle.meq(rho, J, B, GJ.ravel(), z, delta)[3]
               - (J[0] * J[1] / rho - B[0] * B[1] + k / rho * (GJ[0] @ GJ[1]))) < 1e-17


def test_one_dimensional_box_filter_identity():
    """Eq. FilterExampleSmall is exact for linear X, Y under a width-Delta box filter:
    <(a + b x)(c + d x)> = a c + b d Delta^2/12 (the 1/12 is the box's second moment)."""
    xg, wg = np.polynomial.legendre.leggauss(2)
    for delta in (0.5, 1.0, 2.0, 4.0):
        a, b, c, d = RNG.normal(size=4)
        xs = 0.5 * delta * xg
        avg = np.sum(0.5 * wg * (a + b * xs) * (c + d * xs))
        assert abs(avg - (a * c + b * d * delta ** 2 / 12.0)) < 1e-14
