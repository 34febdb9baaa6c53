"""Pins of the oracle's lattice tables against what the paper prints (Sec. 2).

The fixtures in tests/golden/paper_tables.txt are the paper's c_x, c_y lists and the
matrices of Eq. FluidTMatrix and Eq. MagTMatrix, typed in together with the row
definitions printed beside each matrix.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from golden_io import paper_tables


@pytest.fixture(scope="module")
def tabs():
    return oracle.tables(), paper_tables()


def test_velocities_match_paper(tabs):
    o, p = tabs
    np.testing.assert_array_equal(o["cx"], p["cx"])
    np.testing.assert_array_equal(o["cy"], p["cy"])


def test_matrices_match_paper(tabs):
    o, p = tabs
    np.testing.assert_array_equal(o["T"], p["T"])
    np.testing.assert_array_equal(o["Tm"], p["Tm"])


@pytest.mark.parametrize("which", ["T", "Tm"])
def test_printed_matrix_equals_printed_row_polynomials(tabs, which):
    """Each printed matrix row must be its printed polynomial in (c_x, c_y) evaluated on the
    nine lattice vectors: catches a garbled or mistyped entry in either place."""
    _, p = tabs
    cx, cy = sp.symbols("cx cy")
    rows = p["T_rows"] if which == "T" else p["Tm_rows"]
    built = np.array([[float(r.subs({cx: int(a), cy: int(b)})) for a, b in zip(p["cx"], p["cy"])]
                      for r in rows])
    np.testing.assert_array_equal(built, p[which])


def test_T_rows_orthogonal(tabs):
    """T T^T is diagonal (the MRT basis is orthogonal); its diagonal fixes T^{-1} = T^T D^{-1}."""
    _, p = tabs
    G = p["T"] @ p["T"].T
    np.testing.assert_array_equal(G, np.diag(np.diag(G)))
    np.testing.assert_array_equal(np.diag(G), [9, 6, 6, 4, 4, 12, 12, 180, 20])


def test_inverses(tabs):
    o, p = tabs
    I = np.eye(9)
    np.testing.assert_allclose(o["Tinv"] @ p["T"], I, atol=1e-15)
    np.testing.assert_allclose(o["Tminv"] @ p["Tm"], I, atol=1e-15)
    # against LAPACK applied to the printed matrices
    np.testing.assert_allclose(o["Tinv"], np.linalg.inv(p["T"]), atol=1e-15)
    np.testing.assert_allclose(o["Tminv"], np.linalg.inv(p["Tm"]), atol=1e-15)
    # and against the orthogonality closed form T^{-1} = T^T diag(1/9, 1/6, ..., 1/20)
    d = np.array([9, 6, 6, 4, 4, 12, 12, 180, 20], dtype=float)
    np.testing.assert_allclose(o["Tinv"], p["T"].T / d[None, :], atol=1e-16)
    # T_m: det = -64, exact integer
    assert round(np.linalg.det(p["Tm"])) == -64


def test_weights_are_the_isotropic_d2q9_set(tabs):
    """Reading R1: standard D2Q9 weights.  They are the unique weights on this velocity set
    that reproduce the printed equilibria: sum w = 1, sum w c = 0, sum w c_x^2 = 1/3 (N_a4 = B/3)
    and sum w c_x^2 c_y^2 = 1/9 (N_a8 = B/9)."""
    o, p = tabs
    w, cx, cy = o["w"], p["cx"], p["cy"]
    assert abs(w.sum() - 1.0) < 1e-16
    assert abs((w * cx).sum()) < 1e-16 and abs((w * cy).sum()) < 1e-16
    assert abs((w * cx * cx).sum() - 1.0 / 3.0) < 1e-16
    assert abs((w * cy * cy).sum() - 1.0 / 3.0) < 1e-16
    assert abs((w * cx * cy).sum()) < 1e-16
    assert abs((w * cx * cx * cy * cy).sum() - 1.0 / 9.0) < 1e-16
    assert abs((w * cx ** 4).sum() - 1.0 / 3.0) < 1e-16
    # uniqueness: with the lattice symmetries the weights are (w0, wa, wd); the three
    # conditions sum w = 1, sum w cx^2 = 1/3, sum w cx^2 cy^2 = 1/9 fix them.
    A = np.array([[1, 4, 4], [0, 2, 4], [0, 0, 4]], dtype=float)
    w0, wa, wd = np.linalg.solve(A, [1.0, 1.0 / 3.0, 1.0 / 9.0])
    np.testing.assert_allclose(w, [w0] + [wa] * 4 + [wd] * 4, atol=1e-16)
