"""Plain FP64 CPU oracle of the learned subgrid correction (test infrastructure only).

Features, targets and network of the learned closure, written from their definitions:

* Subgrid terms.  For a fine state (rho, J = rho u, B) and its r x r box filter (bar), the four
  quantities the analytic closure of Sec. 2.1 / Sec. 3 approximates are
    c0 = bar(J_x J_y / rho) - Jb_x Jb_y / rhob - (bar(B_x B_y) - Bb_x Bb_y)          (enters M_3^eq)
    c1 = bar((J_x^2 - J_y^2)/rho) - (Jb_x^2 - Jb_y^2)/rhob
         - (bar(B_x^2 - B_y^2) - (Bb_x^2 - Bb_y^2))                                  (M_4^eq)
    c2 = bar((J_x^2 + J_y^2)/rho) - (Jb_x^2 + Jb_y^2)/rhob                           (M_7^eq, M_8^eq)
    c3 = bar((J_x B_y - J_y B_x)/rho) - (Jb_x Bb_y - Jb_y Bb_x)/rhob                 (N^eq via E)
  and the analytic closure (Eqs. FilterExampleSmall/Large, density gradients dropped) predicts
    a0 = k (G_xy / rhob - H_xy),  a1 = k ((G_xx - G_yy)/rhob - H_xx + H_yy),
    a2 = k (G_xx + G_yy)/rhob,    a3 = k (K_xy - K_yx)/rhob,        k = Delta^2/12,
  with central-difference gradients of the filtered J, B on the coarse grid (coarse lattice
  units).  The network is trained on the residual c - a.
* Features (12 channels, coarse grid): u_x, u_y, B_x, B_y of the filtered state and their
  central differences d_x, d_y (a(+1) - a(-1))/2 in the order (dx ux, dy ux, dx uy, dy uy, dx Bx,
  dy Bx, dx By, dy By); each channel is divided by its scale.
* Network: three periodic 3x3 convolutions 12 -> 32 -> 32 -> 4 with biases, tanh after the
  first two; weights W[l][co][ci][dy+1][dx+1] act as y[co](x) = b[co] + sum_ci,dy,dx
  W[co][ci][dy+1][dx+1] a[ci](x + (dx, dy)).  Loss: mean over cells and channels of
  (out - target)^2 / 2.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((12, 32), (32, 32), (32, 4))


def num_params() -> int:
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W[co, ci, 3, 3], b[co]), ...] (weights then biases per layer)."""
    out, o = [], 0
    for ci, co in LAYERS:
        W = np.asarray(theta[o:o + co * ci * 9], dtype=np.float64).reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = np.asarray(theta[o:o + co], dtype=np.float64)
        o += co
        out.append((W, b))
    return out


def shifted(a, dx, dy):
    """a(x + dx, y + dy) on the periodic grid (a indexed [..., y, x])."""
    return np.roll(a, (-dy, -dx), axis=(-2, -1))


def conv3x3(a, W, b):
    """a[B, ci, H, W] -> [B, co, H, W]."""
    Bn, ci, H, Wd = a.shape
    co = W.shape[0]
    y = np.zeros((Bn, co, H, Wd)) + b[None, :, None, None]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            s = shifted(a, dx, dy)
            y += np.einsum("oc,bchw->bohw", W[:, :, dy + 1, dx + 1], s)
    return y


def forward(theta, x):
    """Activations [x, a1, a2, out] for inputs x[B, 12, H, W]."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    a1 = np.tanh(conv3x3(x, W1, b1))
    a2 = np.tanh(conv3x3(a1, W2, b2))
    out = conv3x3(a2, W3, b3)
    return [x, a1, a2, out]


def loss(theta, x, target):
    out = forward(theta, x)[-1]
    return 0.5 * np.mean((out - target) ** 2)


def conv3x3_backward(a, W, dy_):
    """Gradients of sum(dy_ * conv3x3(a, W, b)) w.r.t. W, b and a."""
    dW = np.zeros_like(W)
    da = np.zeros_like(a)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            s = shifted(a, dx, dy)
            dW[:, :, dy + 1, dx + 1] = np.einsum("bohw,bchw->oc", dy_, s)
            # y(x) uses a(x + d): a(z) feeds y(z - d)
            da += shifted(np.einsum("oc,bohw->bchw", W[:, :, dy + 1, dx + 1], dy_), -dx, -dy)
    db = dy_.sum(axis=(0, 2, 3))
    return dW, db, da


def gradient(theta, x, target):
    """(loss, flat gradient) by back-propagation."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    x0, a1, a2, out = forward(theta, x)
    n = out.size
    L = 0.5 * np.sum((out - target) ** 2) / n
    d3 = (out - target) / n
    dW3, db3, da2 = conv3x3_backward(a2, W3, d3)
    d2 = da2 * (1 - a2 ** 2)
    dW2, db2, da1 = conv3x3_backward(a1, W2, d2)
    d1 = da1 * (1 - a1 ** 2)
    dW1, db1, _ = conv3x3_backward(x0, W1, d1)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, g


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; splitmix64 numbers."""
    from paper_1705_09807_gb300.inputs import splitmix64_uniform
    u = splitmix64_uniform(seed, num_params())
    theta = np.zeros(num_params())
    o = 0
    for ci, co in LAYERS:
        lim = 1.0 / np.sqrt(ci * 9)
        theta[o:o + co * ci * 9] = (2 * u[o:o + co * ci * 9] - 1) * lim
        o += co * ci * 9 + co
    return theta


# ------------------------------------------------------------------------------ data
def central(a, axis):
    """(a(+1) - a(-1)) / 2 along x (axis=-1) or y (axis=-2), periodic."""
    return 0.5 * (np.roll(a, -1, axis=axis) - np.roll(a, 1, axis=axis))


def box(a, r):
    ny, nx = a.shape
    return a.reshape(ny // r, r, nx // r, r).mean(axis=(1, 3))


def features(rho, ux, uy, bx, by, in_scale):
    """12-channel features of a coarse state (fields [H, W])."""
    ch = [ux, uy, bx, by]
    for a in (ux, uy, bx, by):
        ch += [central(a, -1), central(a, -2)]
    x = np.stack(ch)
    return x / np.asarray(in_scale, dtype=np.float64)[:, None, None]


def analytic(rho, jx, jy, bx, by, delta):
    """The analytic closure a0..a3 on the coarse grid (filtered J, B; central differences)."""
    k = delta * delta / 12.0
    g = {name: (central(f, -1), central(f, -2)) for name, f in (("jx", jx), ("jy", jy), ("bx", bx), ("by", by))}

    def dot(p, q):
        return g[p][0] * g[q][0] + g[p][1] * g[q][1]

    a0 = k * (dot("jx", "jy") / rho - dot("bx", "by"))
    a1 = k * ((dot("jx", "jx") - dot("jy", "jy")) / rho - dot("bx", "bx") + dot("by", "by"))
    a2 = k * (dot("jx", "jx") + dot("jy", "jy")) / rho
    a3 = k * (dot("jx", "by") - dot("jy", "bx")) / rho
    return np.stack([a0, a1, a2, a3])


def subgrid_terms(rho, ux, uy, bx, by, r):
    """True subgrid terms c0..c3 on the coarse grid from a fine state (rho, u, B)."""
    jx, jy = rho * ux, rho * uy
    R, Jx, Jy, Bx, By = (box(a, r) for a in (rho, jx, jy, bx, by))
    c0 = box(jx * jy / rho, r) - Jx * Jy / R - (box(bx * by, r) - Bx * By)
    c1 = (box((jx * jx - jy * jy) / rho, r) - (Jx * Jx - Jy * Jy) / R
          - (box(bx * bx - by * by, r) - (Bx * Bx - By * By)))
    c2 = box((jx * jx + jy * jy) / rho, r) - (Jx * Jx + Jy * Jy) / R
    c3 = box((jx * by - jy * bx) / rho, r) - (Jx * By - Jy * Bx) / R
    return np.stack([c0, c1, c2, c3]), (R, Jx, Jy, Bx, By)


def training_pair(rho, ux, uy, bx, by, r, delta, in_scale, out_scale):
    """(features [12, H, W], target [4, H, W]) from a fine state: target = (c - a) / out_scale."""
    c, (R, Jx, Jy, Bx, By) = subgrid_terms(rho, ux, uy, bx, by, r)
    a = analytic(R, Jx, Jy, Bx, By, delta)
    x = features(R, Jx / R, Jy / R, Bx, By, in_scale)
    t = (c - a) / np.asarray(out_scale, dtype=np.float64)[:, None, None]
    return x, t
