"""Closed-form layer potentials used to pin the oracle (not part of the method).

Double-layer potential of the density cos(k theta) on a circle of radius R (centre c0)
for Lap v - kappa^2 v = 0, with the box Green's function (v = 0 on the boundary of
[-1, 1]^2).  The free-space field solves the interface problem [v] = cos(k theta),
[d_r v] = 0 with decay at infinity:
  kappa = 0:  v_in = 1/2 (r/R)^k cos k theta,   v_out = -1/2 (R/r)^k cos k theta  (k >= 1);
              v = indicator of the disc for k = 0;
  kappa > 0:  v_in = -x K_k'(x) I_k(kappa r) cos k theta,
              v_out = -x I_k'(x) K_k(kappa r) cos k theta,  x = kappa R
(from the two interface conditions and the Wronskian I_k K_k' - I_k' K_k = -1/x).
The box potential adds the smooth w with (Lap - kappa^2) w = 0 in the box and
w = -v_out on its boundary, summed as the textbook sine series of the square.
"""
import numpy as np
from scipy import special


def free_space(k, R, kappa, r, theta, inside):
    if kappa == 0.0:
        if k == 0:
            return np.where(inside, 1.0, 0.0) * np.ones_like(r)
        return np.where(inside, 0.5 * (r / R) ** k, -0.5 * (R / r) ** k) * np.cos(k * theta)
    x = kappa * R
    vin = -x * special.kvp(k, x) * special.iv(k, kappa * r)
    vout = -x * special.ivp(k, x) * special.kv(k, kappa * r)
    return np.where(inside, vin, vout) * np.cos(k * theta)


def box_correction(g_side, kappa, X, Y, terms=160, quad=1200):
    """w at points (X, Y) with (Lap - kappa^2) w = 0 in [-1,1]^2 and w = g_side(side, s)
    on side in {'top','bottom','left','right'} (s the coordinate along the side)."""
    s, wq = np.polynomial.legendre.leggauss(quad)
    m = np.arange(1, terms + 1)
    basis = np.sin(np.outer(m, s + 1.0) * np.pi / 2.0)          # (terms, quad)
    mu = np.sqrt((m * np.pi / 2.0) ** 2 + kappa ** 2)
    w = np.zeros_like(X, dtype=np.float64)
    for side in ("top", "bottom", "left", "right"):
        c = basis @ (wq * g_side(side, s))                      # c_m
        along = X if side in ("top", "bottom") else Y
        if side == "top":
            d = Y + 1.0
        elif side == "bottom":
            d = 1.0 - Y
        elif side == "right":
            d = X + 1.0
        else:
            d = 1.0 - X
        # sinh(mu d)/sinh(2 mu) computed without overflow
        ratio = np.exp(mu[:, None] * (d.reshape(1, -1) - 2.0)) * \
            (1.0 - np.exp(-2.0 * mu[:, None] * d.reshape(1, -1))) / (1.0 - np.exp(-4.0 * mu[:, None]))
        sb = np.sin(np.outer(m, along.reshape(-1) + 1.0) * np.pi / 2.0)
        w += np.sum(c[:, None] * sb * ratio, axis=0).reshape(X.shape)
    return w


def circle_double_layer_plus(k, R, c0, kappa, theta):
    """Exact K_D cos(k theta) = v^+ on the circle at polar angles theta (box potential)."""
    def vout_side(side, s):
        if side == "top":
            x, y = s, np.ones_like(s)
        elif side == "bottom":
            x, y = s, -np.ones_like(s)
        elif side == "right":
            x, y = np.ones_like(s), s
        else:
            x, y = -np.ones_like(s), s
        r = np.hypot(x - c0[0], y - c0[1])
        th = np.arctan2(y - c0[1], x - c0[0])
        return -free_space(k, R, kappa, r, th, np.zeros_like(r, dtype=bool))

    X = c0[0] + R * np.cos(theta)
    Y = c0[1] + R * np.sin(theta)
    vin = free_space(k, R, kappa, np.full_like(theta, R), theta, np.ones_like(theta, dtype=bool))
    return vin + box_correction(vout_side, kappa, X, Y)
