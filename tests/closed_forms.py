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


# ---------------------------------------------------------------------------- sphere (3-D)
def _radial(l, kappa, r):
    """(inside, outside) radial functions and their r-derivatives of the separated
    solutions f(r) Y_l of Lap v - kappa^2 v = 0: r^l and r^-(l+1) for kappa = 0, else the
    modified spherical Bessel functions i_l(kappa r) and k_l(kappa r)."""
    if kappa == 0.0:
        return (r ** l, l * r ** (l - 1.0) if l > 0 else 0.0 * r,
                r ** (-l - 1.0), -(l + 1.0) * r ** (-l - 2.0))
    x = kappa * r
    return (special.spherical_in(l, x), kappa * special.spherical_in(l, x, derivative=True),
            special.spherical_kn(l, x), kappa * special.spherical_kn(l, x, derivative=True))


def sphere_free_space(l, poly, R, c0, kappa, X, inside):
    """Free-space double-layer potential of the density p(x - c0) on the sphere |x - c0| = R,
    p a homogeneous harmonic polynomial of degree l (poly(d) evaluates it on (..., 3)
    offsets): v = f(r) p(d) / r^l with f = A (inside) or B (outside) times the radial
    functions, A and B from [v] = p and [d_r v] = 0 at r = R.  For kappa = 0:
    A R^l = (l + 1)/(2l + 1), B R^-(l+1) = -l/(2l + 1)."""
    d = X - np.asarray(c0)
    r = np.sqrt(np.sum(d * d, axis=-1))
    fi, dfi, fo, dfo = _radial(l, kappa, R)
    # A fi - B fo = R^l,  A dfi - B dfo = 0
    det = -fi * dfo + fo * dfi
    A = -R ** l * dfo / det
    B = -R ** l * dfi / det
    gi, _, go, _ = _radial(l, kappa, r)
    ang = poly(d) / np.where(r > 0, r, 1.0) ** l
    return np.where(inside, A * gi, B * go) * ang


def cube_correction(g_face, kappa, X, terms=40, quad=160):
    """w at points X (..., 3) with (Lap - kappa^2) w = 0 in [-1,1]^3 and w = g_face(axis,
    side, P) on the face x_axis = side (P the (Q, Q, 3) face points): the sum over the six
    faces of the textbook double sine series
      sum_{m,n} c_mn sin(m pi (s+1)/2) sin(n pi (t+1)/2) sinh(mu d) / sinh(2 mu),
      mu = sqrt((pi/2)^2 (m^2 + n^2) + kappa^2), d the distance from the opposite face,
    c_mn by Gauss-Legendre quadrature of the face data."""
    q, wq = np.polynomial.legendre.leggauss(quad)
    m = np.arange(1, terms + 1)
    S = np.sin(np.outer(m, q + 1.0) * np.pi / 2.0) * wq[None, :]      # (terms, quad)
    mu = np.sqrt((np.pi / 2.0) ** 2 * (m[:, None] ** 2 + m[None, :] ** 2) + kappa ** 2)
    Xf = X.reshape(-1, 3)
    w = np.zeros(Xf.shape[0])
    for axis in range(3):
        o1, o2 = [a for a in range(3) if a != axis]
        for side in (-1.0, 1.0):
            P = np.zeros((quad, quad, 3))
            P[..., axis] = side
            P[..., o1] = q[:, None]
            P[..., o2] = q[None, :]
            c = S @ g_face(axis, side, P) @ S.T                        # (terms, terms)
            d = (Xf[:, axis] + 1.0) if side > 0 else (1.0 - Xf[:, axis])
            s1 = np.sin(np.outer(Xf[:, o1] + 1.0, m) * np.pi / 2.0)    # (npts, terms)
            s2 = np.sin(np.outer(Xf[:, o2] + 1.0, m) * np.pi / 2.0)
            # sinh(mu d) / sinh(2 mu) without overflow
            ratio = np.exp(mu[None] * (d[:, None, None] - 2.0)) * \
                (1.0 - np.exp(-2.0 * mu[None] * d[:, None, None])) / (1.0 - np.exp(-4.0 * mu[None]))
            w += np.einsum("pm,pn,mn,pmn->p", s1, s2, c, ratio, optimize=True)
    return w.reshape(X.shape[:-1])


def sphere_double_layer_plus(l, poly, R, c0, kappa, pts):
    """Exact K_D p = v^+ at points pts on the sphere (box potential of [-1,1]^3): the
    inside free-space field plus the cube correction with w = -v_out on the faces."""
    def face(axis, side, P):
        return -sphere_free_space(l, poly, R, c0, kappa, P, np.zeros(P.shape[:-1], dtype=bool))
    vin = sphere_free_space(l, poly, R, c0, kappa, pts, np.ones(pts.shape[:-1], dtype=bool))
    return vin + cube_correction(face, kappa, pts)


# ------------------------------------------------------------------ circle single layer (2-D)
def free_space_single(k, R, kappa, r, theta, inside):
    """Free-space single-layer field of the density cos(k theta) on the circle: [v] = 0 and
    [d_r v] = cos(k theta) (inside minus outside), decaying at infinity:
      kappa = 0 (k >= 1): v_in = R/(2k) (r/R)^k cos k theta, v_out = R/(2k) (R/r)^k cos k theta;
      kappa > 0:          v_in = R K_k(x) I_k(kappa r) cos k theta,
                          v_out = R I_k(x) K_k(kappa r) cos k theta,  x = kappa R
    (continuity by construction; the derivative jump from the Wronskian)."""
    if kappa == 0.0:
        return np.where(inside, R / (2 * k) * (r / R) ** k,
                        R / (2 * k) * (R / r) ** k) * np.cos(k * theta)
    x = kappa * R
    vin = R * special.kv(k, x) * special.iv(k, kappa * r)
    vout = R * special.iv(k, x) * special.kv(k, kappa * r)
    return np.where(inside, vin, vout) * np.cos(k * theta)


def free_space_single_dr_in(k, R, kappa):
    """d_r v_in at r = R of free_space_single, as the factor of cos(k theta)."""
    if kappa == 0.0:
        return 0.5
    x = kappa * R
    return R * kappa * special.kv(k, x) * special.ivp(k, x)


def box_correction_grad(g_side, kappa, X, Y, terms=160, quad=1200):
    """Gradient (wx, wy) at (X, Y) of the box correction w of box_correction: each sine
    series term differentiated along the side and across it."""
    s, wq = np.polynomial.legendre.leggauss(quad)
    m = np.arange(1, terms + 1)
    basis = np.sin(np.outer(m, s + 1.0) * np.pi / 2.0)
    mu = np.sqrt((m * np.pi / 2.0) ** 2 + kappa ** 2)
    wx = np.zeros_like(X, dtype=np.float64)
    wy = np.zeros_like(X, dtype=np.float64)
    for side in ("top", "bottom", "left", "right"):
        c = basis @ (wq * g_side(side, s))
        along = X if side in ("top", "bottom") else Y
        if side == "top":
            d, dd = Y + 1.0, 1.0
        elif side == "bottom":
            d, dd = 1.0 - Y, -1.0
        elif side == "right":
            d, dd = X + 1.0, 1.0
        else:
            d, dd = 1.0 - X, -1.0
        D = d.reshape(1, -1)
        ratio = np.exp(mu[:, None] * (D - 2.0)) * (1.0 - np.exp(-2.0 * mu[:, None] * D)) / \
            (1.0 - np.exp(-4.0 * mu[:, None]))
        dratio = mu[:, None] * np.exp(mu[:, None] * (D - 2.0)) * \
            (1.0 + np.exp(-2.0 * mu[:, None] * D)) / (1.0 - np.exp(-4.0 * mu[:, None]))
        arg = np.outer(m, along.reshape(-1) + 1.0) * np.pi / 2.0
        d_along = np.sum(c[:, None] * (m[:, None] * np.pi / 2.0) * np.cos(arg) * ratio, axis=0)
        d_across = dd * np.sum(c[:, None] * np.sin(arg) * dratio, axis=0)
        if side in ("top", "bottom"):
            wx += d_along.reshape(X.shape)
            wy += d_across.reshape(X.shape)
        else:
            wy += d_along.reshape(X.shape)
            wx += d_across.reshape(X.shape)
    return wx, wy


def circle_single_layer_plus(k, R, c0, kappa, theta):
    """Exact v^+ and d_n v^+ on the circle of the box single-layer potential of cos(k theta)
    (free-space field plus the box correction w = -v_out on the box boundary)."""
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
        return -free_space_single(k, R, kappa, r, th, np.zeros_like(r, dtype=bool))

    X = c0[0] + R * np.cos(theta)
    Y = c0[1] + R * np.sin(theta)
    v = free_space_single(k, R, kappa, np.full_like(theta, R), theta,
                          np.ones_like(theta, dtype=bool)) + box_correction(vout_side, kappa, X, Y)
    wx, wy = box_correction_grad(vout_side, kappa, X, Y)
    dn = free_space_single_dr_in(k, R, kappa) * np.cos(k * theta) + \
        wx * np.cos(theta) + wy * np.sin(theta)
    return v, dn
