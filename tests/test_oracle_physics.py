"""Pins of the oracle's full time step against what the paper and the mathematics fix.

* Conservation: M_0, M_1, M_2 and N_a0 are collision invariants (Sec. 2, the remark after
  Eq. geq) and streaming permutes populations, so sum rho, sum J, sum B stay constant.
* Delta = 0 reduces to plain LB-MHD: single-relaxation-time BGK in distribution space toward
  Eq. feq / Eq. geq, written here independently of the oracle's moment-space collision.
* Linear waves: shear and magnetic diffusion decay as exp(-nu k^2 t), exp(-eta k^2 t), with
  nu, eta from the rate relations of Sec. 2; Alfven waves propagate at k B0/sqrt(rho) and damp
  at (nu + eta) k^2/2; sound waves damp at (xi + 4 nu/3) k^2/2 with the paper's bulk viscosity
  xi(s_4, s_7, s_8) (Sec. 2), tested with unequal MRT rates.  All converge at second order.
* Lattice symmetry: 90-degree rotation, reflection and translation commute with the step.
* Solenoidality (Sec. 3 remark on div B): one step from an equilibrium state maps a B field
  that is divergence-free under the isotropic lattice stencil to one that is again
  divergence-free to roundoff, with the Delta^2 terms switched on.
"""
import math

import numpy as np
import pytest

import oracle
from golden_io import paper_tables
from paper_1705_09807_gb300.inputs import kh_jet, smooth_random_fields

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


# ----------------------------------------------------------------------------- helpers
def fsum_field(a):
    return math.fsum(np.asarray(a).ravel().tolist())


def totals(f, g):
    rho = f.sum(axis=0)
    jx = np.tensordot(CX, f, axes=(0, 0))
    jy = np.tensordot(CY, f, axes=(0, 0))
    bx = g[0].sum(axis=0)
    by = g[1].sum(axis=0)
    return [fsum_field(a) for a in (rho, jx, jy, bx, by)]


def mode1(field, axis):
    """Complex amplitude of the first Fourier mode along x (axis=1) or y (axis=0)."""
    n = field.shape[axis]
    prof = field.mean(axis=1 - axis)
    return (prof * np.exp(-2j * np.pi * np.arange(n) / n)).sum() * 2 / n


# ----------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("stencil", [0, 1])
def test_conservation_kh_jet(stencil):
    rho, ux, uy, bx, by = kh_jet(32, seed=3)
    f, g = oracle.init(rho, ux, uy, bx, by)
    t0 = totals(f, g)
    f, g = oracle.step(f, g, oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002), 2.0, 300,
                       stencil=stencil)
    t1 = totals(f, g)
    scale = [1024.0, 1024 * 0.05, 1024 * 0.05, 1024 * 0.02, 1024 * 0.02]
    for a, b, sc in zip(t0, t1, scale):
        assert abs(a - b) <= 1e-13 * sc


# ----------------------------------------------------------------------------- Delta = 0
def bgk_lbmhd(f, g, s, s_m, nsteps):
    """Textbook single-relaxation-time LB-MHD in distribution space: relax toward Eq. feq and
    Eq. geq, then stream (written independently of the oracle)."""
    f = f.copy()
    g = g.copy()
    for _ in range(nsteps):
        rho = f.sum(axis=0)
        ux = np.tensordot(CX, f, axes=(0, 0)) / rho
        uy = np.tensordot(CY, f, axes=(0, 0)) / rho
        bx = g[0].sum(axis=0)
        by = g[1].sum(axis=0)
        cu = CX[:, None, None] * ux + CY[:, None, None] * uy
        cb = CX[:, None, None] * bx + CY[:, None, None] * by
        csq = (CX * CX + CY * CY)[:, None, None]
        wv = W[:, None, None]
        feq = wv * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (ux ** 2 + uy ** 2)) \
            + 4.5 * wv * (0.5 * (bx ** 2 + by ** 2) * csq - cb ** 2)
        gxeq = wv * (bx + 3 * (cu * bx - cb * ux))
        gyeq = wv * (by + 3 * (cu * by - cb * uy))
        f = f - s * (f - feq)
        g = g - s_m * (g - np.stack([gxeq, gyeq]))
        for i in range(9):
            f[i] = np.roll(f[i], (CY[i], CX[i]), axis=(0, 1))
            g[0, i] = np.roll(g[0, i], (CY[i], CX[i]), axis=(0, 1))
            g[1, i] = np.roll(g[1, i], (CY[i], CX[i]), axis=(0, 1))
    return f, g


@pytest.mark.parametrize("shape", [(24, 32), (17, 33)])
def test_delta0_is_plain_bgk_lbmhd(shape):
    ny, nx = shape
    fields = smooth_random_fields(nx, ny, seed=7, amp_u=0.05, amp_b=0.05, amp_rho=0.02)
    f, g = oracle.init(*fields)
    nu, eta = 0.01, 0.02
    s = 1 / (3 * nu + 0.5)
    sm = 1 / (3 * eta + 0.5)
    fo, go = oracle.step(f, g, np.full(9, s), sm, 0.0, 60)
    fb, gb = bgk_lbmhd(f, g, s, sm, 60)
    assert np.max(np.abs(fo - fb)) < 1e-14
    assert np.max(np.abs(go - gb)) < 1e-14
    # with Delta > 0 the answer differs (the Delta^2 terms act)
    fd, gd = oracle.step(f, g, np.full(9, s), sm, 2.0, 60)
    assert np.max(np.abs(fd - fb)) > 1e-8


# ----------------------------------------------------------------------------- linear waves
def _diffusion_rates(n, nu, eta, delta):
    A = 1e-6
    y = np.arange(n)[:, None] * np.ones((1, n))
    x = np.ones((n, 1)) * np.arange(n)[None, :]
    z = np.zeros((n, n))
    f, g = oracle.init(np.ones((n, n)), A * np.sin(2 * np.pi * y / n), z, z,
                       A * np.sin(2 * np.pi * x / n))
    s = oracle.srt_rates(nu)
    sm = oracle.rate_from_diffusivity(eta)
    t1 = 20
    dt = int(0.5 * n * n / (4 * np.pi ** 2 * max(nu, eta)))
    f1, g1 = oracle.step(f, g, s, sm, delta, t1)
    f2, g2 = oracle.step(f1, g1, s, sm, delta, dt)
    m1, m2 = oracle.moments(f1, g1), oracle.moments(f2, g2)
    k2 = (2 * np.pi / n) ** 2
    rate_u = np.log(abs(mode1(m1[1], 0)) / abs(mode1(m2[1], 0))) / dt
    rate_b = np.log(abs(mode1(m1[4], 1)) / abs(mode1(m2[4], 1))) / dt
    return rate_u / (nu * k2), rate_b / (eta * k2)


def test_shear_and_magnetic_diffusion_rates_converge_second_order():
    errs = []
    for n in (16, 32):
        ru, rb = _diffusion_rates(n, 0.02, 0.03, 2.0)
        errs.append((abs(ru - 1), abs(rb - 1)))
    assert errs[1][0] < 5e-3 and errs[1][1] < 5e-3
    for q in range(2):
        ratio = errs[0][q] / errs[1][q]
        assert 3.3 < ratio < 4.8, ratio


@pytest.mark.slow
def test_diffusion_rates_at_64():
    ru, rb = _diffusion_rates(64, 0.02, 0.03, 2.0)
    assert abs(ru - 1) < 1.2e-3 and abs(rb - 1) < 1.2e-3


def test_alfven_wave_speed_and_damping():
    n, nu, eta, B0, A = 32, 0.01, 0.01, 0.05, 1e-6
    k = 2 * np.pi / n
    x = np.ones((n, 1)) * np.arange(n)[None, :]
    z = np.zeros((n, n))
    f, g = oracle.init(np.ones((n, n)), z, A * np.sin(k * x), B0 + z, -A * np.sin(k * x))
    s = oracle.srt_rates(nu)
    sm = oracle.rate_from_diffusivity(eta)
    f, g = oracle.step(f, g, s, sm, 0.0, 10)
    a0 = mode1(oracle.moments(f, g)[2], 1)
    T = int(0.25 * 2 * np.pi / (k * B0))
    f2, g2 = oracle.step(f, g, s, sm, 0.0, T)
    a1 = mode1(oracle.moments(f2, g2)[2], 1)
    omega = -np.angle(a1 / a0) / T
    gamma = np.log(abs(a0) / abs(a1)) / T
    assert abs(omega / (k * B0) - 1) < 2e-4
    assert abs(gamma / ((nu + eta) * k * k / 2) - 1) < 1e-2


@pytest.mark.parametrize("s7,s8", [(None, None), (1.2, 1.6), (1.7, 0.9)])
def test_sound_wave_damping_matches_paper_bulk_viscosity(s7, s8):
    n, nu, A = 64, 0.01, 1e-6
    k = 2 * np.pi / n
    cs = 1 / np.sqrt(3)
    sv = oracle.srt_rates(nu)
    if s7 is not None:
        sv[7], sv[8] = s7, s8
    # bulk viscosity, Sec. 2: xi = -1/9 - 1/(9 s_4) - 1/(15 s_7) + 2/(5 s_8)
    xi = -1 / 9 - 1 / (9 * sv[4]) - 1 / (15 * sv[7]) + 2 / (5 * sv[8])
    x = np.ones((n, 1)) * np.arange(n)[None, :]
    z = np.zeros((n, n))
    f, g = oracle.init(1 + A * np.sin(k * x), cs * A * np.sin(k * x), z, z, z)
    sm = oracle.rate_from_diffusivity(0.01)
    f, g = oracle.step(f, g, sv, sm, 0.0, 10)
    a0 = mode1(oracle.moments(f, g)[0] - 1, 1)
    tq = int(round(0.25 * 2 * np.pi / (k * cs)))
    fq, gq = oracle.step(f, g, sv, sm, 0.0, tq)
    aq = mode1(oracle.moments(fq, gq)[0] - 1, 1)
    assert abs(-np.angle(aq / a0) / tq / (cs * k) - 1) < 2e-2
    T = int(2 * 2 * np.pi / (k * cs))
    f2, g2 = oracle.step(f, g, sv, sm, 0.0, T)
    a1 = mode1(oracle.moments(f2, g2)[0] - 1, 1)
    gamma = np.log(abs(a0) / abs(a1)) / T
    assert abs(gamma / (0.5 * (xi + 4 * nu / 3) * k * k) - 1) < 4e-3


# ----------------------------------------------------------------------------- symmetry
def rot90_fields(rho, ux, uy, bx, by):
    """Rotate a square periodic state by +90 degrees: F'(x', y') = R F(y', -x')."""
    n = rho.shape[0]
    YP, XP = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    src = lambda a: a[(-XP) % n, YP]
    return src(rho), -src(uy), src(ux), -src(by), src(bx)


def reflect_x_fields(rho, ux, uy, bx, by):
    n = rho.shape[1]
    idx = (-np.arange(n)) % n
    return rho[:, idx], -ux[:, idx], uy[:, idx], -bx[:, idx], by[:, idx]


def _run_moments(fields, s, sm, delta, nsteps, stencil):
    f, g = oracle.init(*fields)
    f, g = oracle.step(f, g, s, sm, delta, nsteps, stencil=stencil)
    return oracle.moments(f, g)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("transform", ["rot90", "reflect_x", "translate"])
def test_step_commutes_with_lattice_symmetries(stencil, transform):
    n = 24
    fields = smooth_random_fields(n, n, seed=11, amp_u=0.06, amp_b=0.05, amp_rho=0.02)
    s = oracle.srt_rates(0.01)
    s[5] = s[6] = 1.3       # MRT with s_5 = s_6 keeps the 90-degree symmetry
    s[7], s[8] = 1.4, 1.1
    sm = oracle.rate_from_diffusivity(0.02)
    if transform == "rot90":
        T = rot90_fields
    elif transform == "reflect_x":
        T = reflect_x_fields
    else:
        T = lambda *a: tuple(np.roll(q, (5, -7), axis=(0, 1)) for q in a)
    direct = T(*_run_moments(fields, s, sm, 2.0, 40, stencil))
    mapped = _run_moments(T(*fields), s, sm, 2.0, 40, stencil)
    for a, b in zip(direct, mapped):
        assert np.max(np.abs(a - b)) < 5e-15


# ----------------------------------------------------------------------------- div B
def iso_d(a, axis_c):
    """Isotropic lattice derivative sum_i 3 w_i c_i a(x + c_i) along c = CX or CY."""
    out = np.zeros_like(a)
    for i in range(1, 9):
        if axis_c[i] == 0:
            continue
        out += 3 * W[i] * axis_c[i] * np.roll(a, (-CY[i], -CX[i]), axis=(0, 1))
    return out


@pytest.mark.parametrize("stencil", [0, 1])
def test_one_step_preserves_isotropic_divergence_of_B(stencil):
    """B = (D_y A, -D_x A) is discretely solenoidal (D_x, D_y commute).  From the equilibrium
    state the post-collision g* keeps the form w_i (B + 3 eps c_i E') for any field E', and the
    isotropic divergence of its streamed sum vanishes identically; so after one step with the
    Delta^2 terms on, max |D . B| stays at roundoff while |grad B| is O(1e-2)."""
    n = 32
    rho, ux, uy, _, _ = smooth_random_fields(n, n, seed=5, amp_u=0.05)
    A = smooth_random_fields(n, n, seed=6, amp_rho=0.5)[0] - 1.0
    bx, by = iso_d(A, CY), -iso_d(A, CX)
    div0 = iso_d(bx, CX) + iso_d(by, CY)
    grad0 = max(np.max(np.abs(iso_d(bx, CX))), np.max(np.abs(iso_d(by, CY))))
    assert np.max(np.abs(div0)) < 1e-14 * grad0
    f, g = oracle.init(rho, ux, uy, bx, by)
    f, g = oracle.step(f, g, oracle.srt_rates(0.01), oracle.rate_from_diffusivity(0.01), 2.0, 1,
                       stencil=stencil)
    _, _, _, bx1, by1 = oracle.moments(f, g)
    div1 = iso_d(bx1, CX) + iso_d(by1, CY)
    gradB = max(np.max(np.abs(iso_d(bx1, CX))), np.max(np.abs(iso_d(by1, CY))))
    assert gradB > 1e-3
    assert np.max(np.abs(div1)) < 1e-14 * gradB
    # the central-difference divergence of the same field is not zero: the invariant is the
    # isotropic one
    cdiv = 0.5 * (np.roll(bx1, -1, 1) - np.roll(bx1, 1, 1) + np.roll(by1, -1, 0) - np.roll(by1, 1, 0))
    assert np.max(np.abs(cdiv)) > 1e-6 * gradB


# ----------------------------------------------------------------------------- invariances
def test_uniform_state_stays_uniform():
    n = 8
    z = np.zeros((n, n))
    f, g = oracle.init(1.1 + z, 0.03 + z, -0.02 + z, 0.04 + z, 0.01 + z)
    f1, g1 = oracle.step(f, g, oracle.srt_rates(0.01), 1.5, 2.0, 5)
    assert np.max(np.abs(f1 - f)) < 1e-15 and np.max(np.abs(g1 - g)) < 1e-15


def test_threads_bitwise_identical_and_cell_kernel_consistent():
    fields = kh_jet(32, seed=2)
    f, g = oracle.init(*fields)
    s, sm = oracle.srt_rates(0.002), oracle.rate_from_diffusivity(0.002)
    f, g = oracle.step(f, g, s, sm, 2.0, 30)
    a = oracle.step(f, g, s, sm, 2.0, 7, nthreads=1)
    b = oracle.step(f, g, s, sm, 2.0, 7, nthreads=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for stencil in (0, 1):
        f1, g1 = oracle.step(f, g, s, sm, 2.0, 1, stencil=stencil)
        for (x, y) in ((0, 0), (31, 5), (12, 31)):
            fs, gs = oracle.collide_cell(f, g, s, sm, 2.0, x, y, stencil=stencil)
            for i in range(9):
                xd, yd = (x + CX[i]) % 32, (y + CY[i]) % 32
                assert f1[i, yd, xd] == fs[i]
                assert g1[0, i, yd, xd] == gs[0, i] and g1[1, i, yd, xd] == gs[1, i]


def test_rates_map_to_paper_transport_coefficients():
    """nu = 1/(3 s) - 1/6 and eta = 1/(3 s_m) - 1/6 (Sec. 2) invert the helper's rate."""
    for d in (2e-4, 5e-4, 2e-3, 0.1):
        s = oracle.rate_from_diffusivity(d)
        assert abs(1 / (3 * s) - 1 / 6 - d) < 1e-16
    # the paper's xi at SRT equals 2 nu / 3 (the BGK bulk viscosity)
    s = oracle.rate_from_diffusivity(0.01)
    xi = -1 / 9 - 1 / (9 * s) - 1 / (15 * s) + 2 / (5 * s)
    assert abs(xi - 2 * 0.01 / 3) < 1e-16


@pytest.mark.parametrize("stencil", [0, 1])
def test_gradient_stencil_and_filter_terms_on_sine_fields(stencil):
    """Closed form for the gradient stencil inside the step: for fields varying along y only,
    both stencils give d_y sin(k y) = sin(k) cos(k y).  From an equilibrium state
    f = f^eq, one collision moves the moments by s (Mbar^eq - M^eq), i.e. by s Delta^2/12 times
    the gradient products: M_4 by G_xx = (d_y J_x)^2, M_7 by -3 G_xx, and N_y1 by K_xy."""
    n, A, C, phi, delta = 16, 0.02, 0.03, 0.7, 2.0
    k = 2 * np.pi / n
    y = np.arange(n)[:, None] * np.ones((1, n))
    z = np.zeros((n, n))
    ux = A * np.sin(k * y)
    by = C * np.sin(k * y + phi)
    f, g = oracle.init(1.0 + z, ux, z, z, by)
    s = oracle.srt_rates(0.05)
    sm = 1.3
    p = paper_tables()
    kd = delta ** 2 / 12.0
    for yy in (0, 3, 7):
        fs, gs = oracle.collide_cell(f, g, s, sm, delta, 5, yy, stencil=stencil)
        dM = p["T"] @ (fs - f[:, yy, 5]) / s[0]
        dN = p["Tm"] @ (gs[1] - g[1, :, yy, 5]) / sm
        Gxx = (A * np.sin(k) * np.cos(k * yy)) ** 2
        Hyy = (C * np.sin(k) * np.cos(k * yy + phi)) ** 2
        Kxy = A * C * np.sin(k) ** 2 * np.cos(k * yy) * np.cos(k * yy + phi)
        assert abs(dM[4] - kd * (Gxx + Hyy)) < 1e-15
        assert abs(dM[7] - (-3 * kd * Gxx)) < 1e-15
        assert abs(dM[3]) < 1e-17
        assert abs(dN[1] - kd * Kxy) < 1e-16
