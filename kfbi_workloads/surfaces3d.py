"""Seeded synthetic 3-D inputs: closed surfaces given as level sets, their intersections
with the grid lines of a box, and manufactured solutions.

This module holds NO arithmetic of the KFBI method itself: it finds where analytic
surfaces meet the grid lines (bisection on the level-set function), evaluates their
outward unit normals and shape operators there, and evaluates manufactured solutions.

Conventions (shared by every consumer):
  * box B = [lo, hi]^3, N cells per side, nodes x_i = lo + i h, h = (hi - lo)/N; grid
    arrays are (N+1)^3 indexed [k, j, i] = value at (x_i, y_j, z_k), x fastest;
  * the control points are the intersections of the surface with the grid lines: all
    x-lines (y = y_j, z = z_k), then all y-lines, then all z-lines, each line's points in
    increasing coordinate; a point's two off-axis coordinates are exact grid values;
  * normals point out of the enclosed region; the shape operator S is the symmetric
    3x3 map with dn = S dx for tangent vectors dx (S = I/R on a sphere of radius R),
    packed (Sxx, Syy, Szz, Sxy, Sxz, Syz);
  * the PDE is  Lap(u) - kappa^2 u = f.
The surfaces' centres are offset from the origin by a fraction of a cell at any tested N
so that no intersection falls on a grid node.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 15249
CENTER = (0.0131, -0.0217, 0.0173)       # keeps intersections off the grid nodes


@dataclass
class Surface:
    """Level set F < 0 inside; grad and hess of F (callables on (..., 3) arrays)."""
    name: str
    F: callable
    grad: callable
    hess: callable
    bbox: tuple                       # (lo, hi) per axis, a box containing the surface
    param: dict = field(default_factory=dict)


def ellipsoid(a: float = 0.7, b: float = 0.5, c: float = 0.4, center=CENTER) -> Surface:
    ax = np.array([a, b, c], dtype=np.float64)
    cen = np.asarray(center, dtype=np.float64)
    inv2 = 1.0 / (ax * ax)

    def F(X):
        d = X - cen
        return np.sum(d * d * inv2, axis=-1) - 1.0

    def grad(X):
        return 2.0 * (X - cen) * inv2

    def hess(X):
        H = np.zeros(X.shape[:-1] + (3, 3))
        for q in range(3):
            H[..., q, q] = 2.0 * inv2[q]
        return H

    bb = tuple((cen[q] - ax[q], cen[q] + ax[q]) for q in range(3))
    return Surface("ellipsoid", F, grad, hess, bb, dict(a=a, b=b, c=c, center=tuple(cen)))


def sphere(R: float = 0.5, center=CENTER) -> Surface:
    s = ellipsoid(R, R, R, center)
    s.name = "sphere"
    s.param = dict(R=R, center=tuple(np.asarray(center, dtype=np.float64)))
    return s


def star(r0: float = 0.5, amp: float = 0.1, center=CENTER) -> Surface:
    """rho = r0 + amp sin(3 theta) cos(4 phi), theta the polar angle: F = rho - r(theta,
    phi).  Gradient and Hessian by central differences of F (step 1e-4 and 1e-3)."""
    cen = np.asarray(center, dtype=np.float64)

    def F(X):
        d = X - cen
        rho = np.sqrt(np.sum(d * d, axis=-1))
        th = np.arccos(np.clip(d[..., 2] / np.maximum(rho, 1e-300), -1.0, 1.0))
        ph = np.arctan2(d[..., 1], d[..., 0])
        return rho - (r0 + amp * np.sin(3.0 * th) * np.cos(4.0 * ph))

    def grad(X, e=1e-4):
        g = np.zeros_like(X)
        for q in range(3):
            dx = np.zeros(3)
            dx[q] = e
            g[..., q] = (F(X + dx) - F(X - dx)) / (2 * e)
        return g

    def hess(X, e=1e-3):
        H = np.zeros(X.shape[:-1] + (3, 3))
        for q in range(3):
            dx = np.zeros(3)
            dx[q] = e
            H[..., q, :] = (grad(X + dx) - grad(X - dx)) / (2 * e)
        return 0.5 * (H + np.swapaxes(H, -1, -2))

    r = r0 + amp
    bb = tuple((cen[q] - r, cen[q] + r) for q in range(3))
    return Surface("star", F, grad, hess, bb, dict(r0=r0, amp=amp, center=tuple(cen)))


@dataclass
class Interface3D:
    """Grid-line intersection points of a surface: pts, normals (P, 3), shape (P, 6)."""
    pts: np.ndarray
    normals: np.ndarray
    shape: np.ndarray
    N: int
    lo: float
    hi: float
    name: str = ""

    @property
    def P(self) -> int:
        return int(self.pts.shape[0])


def _line_roots(surf: Surface, axis: int, N: int, lo: float, hi: float, sub: int):
    h = (hi - lo) / N
    others = [q for q in range(3) if q != axis]
    xs = lo + np.arange(N + 1) * h
    # lines through the surface's bounding box only
    sel = [xs[(xs >= surf.bbox[q][0] - h) & (xs <= surf.bbox[q][1] + h)] for q in others]
    A, B = np.meshgrid(sel[0], sel[1], indexing="ij")
    A, B = A.ravel(), B.ravel()
    # samples along the line inside the bounding box
    t0 = max(lo, surf.bbox[axis][0] - 2 * h)
    t1 = min(hi, surf.bbox[axis][1] + 2 * h)
    ts = np.linspace(t0, t1, int(math.ceil((t1 - t0) / h)) * sub + 1)
    out = []
    chunk = max(1, 4_000_000 // ts.size)
    for c0 in range(0, A.size, chunk):
        a, b = A[c0:c0 + chunk], B[c0:c0 + chunk]
        X = np.empty((a.size, ts.size, 3))
        X[..., axis] = ts[None, :]
        X[..., others[0]] = a[:, None]
        X[..., others[1]] = b[:, None]
        Fv = surf.F(X)
        sgn = Fv < 0
        li, si = np.nonzero(sgn[:, :-1] != sgn[:, 1:])
        if li.size == 0:
            continue
        tl, tr = ts[si].copy(), ts[si + 1].copy()
        fl = Fv[li, si]
        Y = np.empty((li.size, 3))
        Y[:, others[0]] = a[li]
        Y[:, others[1]] = b[li]
        for _ in range(64):                     # bisection to FP64 resolution
            tm = 0.5 * (tl + tr)
            Y[:, axis] = tm
            fm = surf.F(Y)
            left = (fm < 0) == (fl < 0)
            tl = np.where(left, tm, tl)
            fl = np.where(left, fm, fl)
            tr = np.where(left, tr, tm)
        Y[:, axis] = 0.5 * (tl + tr)
        order = np.lexsort((Y[:, axis], Y[:, others[0]], Y[:, others[1]]))
        out.append(Y[order])
    return np.concatenate(out) if out else np.zeros((0, 3))


def intersect(surf: Surface, N: int, lo: float = -1.0, hi: float = 1.0, sub: int = 4) -> Interface3D:
    """All intersections of the surface with the grid lines of the box (axis by axis,
    line by line), with outward normals and packed shape operators.  Each edge of
    length h is sampled at `sub` sub-intervals before bisection; two crossings inside one
    sub-interval would be missed (the surfaces here are resolved at the tested N)."""
    pts = np.concatenate([_line_roots(surf, a, N, lo, hi, sub) for a in range(3)])
    g = surf.grad(pts)
    gn = np.linalg.norm(g, axis=1)
    n = g / gn[:, None]
    P = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
    S = np.einsum("pab,pbc,pcd->pad", P, surf.hess(pts), P) / gn[:, None, None]
    packed = np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 0, 1], S[:, 0, 2], S[:, 1, 2]], axis=1)
    return Interface3D(pts, n, packed, N, lo, hi, surf.name)


# ---------------------------------------------------------------- manufactured solutions
@dataclass
class Manufactured3D:
    u: callable
    f: callable
    name: str
    kappa: float


def manufactured_sin3(kappa: float = 0.0) -> Manufactured3D:
    """u = sin x sin y sin z; f = -(3 + kappa^2) u."""
    u = lambda x, y, z: np.sin(x) * np.sin(y) * np.sin(z)
    return Manufactured3D(u, lambda x, y, z: -(3.0 + kappa ** 2) * u(x, y, z), "sin3", kappa)


def manufactured_harmonic3() -> Manufactured3D:
    """u = exp(x) cos(y) + z (harmonic, kappa = 0)."""
    u = lambda x, y, z: np.exp(x) * np.cos(y) + z
    return Manufactured3D(u, lambda x, y, z: 0.0 * x, "exp_cos_z", 0.0)


def grid_nodes3(N: int, lo: float = -1.0, hi: float = 1.0):
    """Node coordinates and the (N+1)^3 meshes X, Y, Z indexed [k, j, i]."""
    h = (hi - lo) / N
    xs = lo + np.arange(N + 1, dtype=np.float64) * h
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    return xs, X, Y, Z


@dataclass
class Problem3D:
    iface: Interface3D
    kappa: float
    sol: Manufactured3D

    @property
    def N(self):
        return self.iface.N

    def f_grid(self):
        _, X, Y, Z = grid_nodes3(self.N, self.iface.lo, self.iface.hi)
        return self.sol.f(X, Y, Z)

    def u_grid(self):
        _, X, Y, Z = grid_nodes3(self.N, self.iface.lo, self.iface.hi)
        return self.sol.u(X, Y, Z)

    def f_ctrl(self):
        p = self.iface.pts
        return self.sol.f(p[:, 0], p[:, 1], p[:, 2])

    def g_ctrl(self):
        p = self.iface.pts
        return self.sol.u(p[:, 0], p[:, 1], p[:, 2])


def config_poisson3d(N: int, shape: str = "ellipsoid") -> Problem3D:
    """3-D interior Dirichlet Poisson: ellipsoid (0.7, 0.5, 0.4) or star surface,
    u = sin x sin y sin z (kappa = 0)."""
    surf = ellipsoid() if shape == "ellipsoid" else (sphere() if shape == "sphere" else star())
    return Problem3D(intersect(surf, N), 0.0, manufactured_sin3(0.0))


def config_helmholtz3d(N: int, kappa: float = 2.0, shape: str = "ellipsoid") -> Problem3D:
    surf = ellipsoid() if shape == "ellipsoid" else sphere()
    return Problem3D(intersect(surf, N), float(kappa), manufactured_sin3(kappa))


def random_density3(P: int, pts=None, seed: int = SEED) -> np.ndarray:
    """A smooth density on the points (a low-order polynomial of the position with
    seeded coefficients) or, without pts, seeded normal values."""
    rng = np.random.default_rng(seed)
    if pts is None:
        return rng.standard_normal(P)
    c = rng.standard_normal(10)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z
            + c[7] * x * x + c[8] * np.sin(2 * y) + c[9] * np.cos(3 * z))
