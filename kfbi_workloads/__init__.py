"""Seeded synthetic inputs for the KFBI hot path (curves, manufactured solutions, batches).

This module holds NO arithmetic of the KFBI method itself: it only samples analytic
interfaces (points, outward normals, signed curvature) and manufactured solutions
(u, f = Lu, boundary data g).  Both the FP64 CPU oracle and the CUDA path's tests and
benchmark draw their inputs from here, so neither needs to import the other.

Conventions (shared by every consumer):
  * box B = [lo, hi]^2, N cells per side, grid nodes x_i = lo + i*h, h = (hi-lo)/N,
    grid arrays are (N+1) x (N+1) with x fastest: a[j, i] = value at (x_i, y_j);
  * interface points are sampled counter-clockwise at equispaced parameter
    t_k = 2*pi*k/M, k = 0..M-1, with outward unit normals and the signed curvature
    (positive on convex parts);
  * the PDE is  Lap(u) - kappa^2 u = f  (the paper writes an unsquared kappa, Sec. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 15249


@dataclass
class Interface:
    """Sampled closed curve: pts (M,2), normals (M,2), curv (M,), and the analytic
    parametrisation used to sample it (for drawing extra points in tests)."""
    pts: np.ndarray
    normals: np.ndarray
    curv: np.ndarray
    name: str = ""
    param: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.pts.shape[0])


def _polar_curve(M: int, r, dr, ddr, center=(0.0, 0.0), name="", param=None) -> Interface:
    t = 2.0 * np.pi * np.arange(M, dtype=np.float64) / M
    rr, d1, d2 = r(t), dr(t), ddr(t)
    c, s = np.cos(t), np.sin(t)
    x = center[0] + rr * c
    y = center[1] + rr * s
    xp = d1 * c - rr * s
    yp = d1 * s + rr * c
    sp = np.sqrt(xp * xp + yp * yp)
    normals = np.stack([yp / sp, -xp / sp], axis=1)
    curv = (rr * rr + 2.0 * d1 * d1 - rr * d2) / (rr * rr + d1 * d1) ** 1.5
    return Interface(np.stack([x, y], axis=1), normals, curv, name, dict(param or {}))


def circle(M: int, R: float = 0.5, center=(0.0, 0.0)) -> Interface:
    return _polar_curve(M, lambda t: R + 0 * t, lambda t: 0 * t, lambda t: 0 * t,
                        center, "circle", dict(R=R, center=center))


def flower(M: int, r0: float = 0.5, a: float = 0.15, k: int = 5, center=(0.0, 0.0)) -> Interface:
    """r(t) = r0 + a cos(k t): the 2-D Poisson / Helmholtz test interface."""
    return _polar_curve(M,
                        lambda t: r0 + a * np.cos(k * t),
                        lambda t: -a * k * np.sin(k * t),
                        lambda t: -a * k * k * np.cos(k * t),
                        center, "flower", dict(r0=r0, a=a, k=k, center=center))


def star(M: int, r0: float, amps, phases, center=(0.0, 0.0)) -> Interface:
    """r(t) = r0 + sum_{k=2..} a_k cos(k t + phi_k) (batched random star curves)."""
    ks = np.arange(2, 2 + len(amps), dtype=np.float64)
    amps = np.asarray(amps, dtype=np.float64)
    phases = np.asarray(phases, dtype=np.float64)

    def r(t):
        return r0 + np.sum(amps[:, None] * np.cos(ks[:, None] * t[None, :] + phases[:, None]), axis=0)

    def dr(t):
        return np.sum(-amps[:, None] * ks[:, None] * np.sin(ks[:, None] * t[None, :] + phases[:, None]), axis=0)

    def ddr(t):
        return np.sum(-amps[:, None] * ks[:, None] ** 2 * np.cos(ks[:, None] * t[None, :] + phases[:, None]), axis=0)

    return _polar_curve(M, r, dr, ddr, center, "star",
                        dict(r0=r0, amps=amps.tolist(), phases=phases.tolist(), center=center))


def ellipse(M: int, a: float = 0.7, b: float = 0.4, rot_deg: float = 30.0, center=(0.0, 0.0)) -> Interface:
    """Ellipse with semi-axes (a, b) rotated by rot_deg, sampled at equispaced t."""
    t = 2.0 * np.pi * np.arange(M, dtype=np.float64) / M
    th = math.radians(rot_deg)
    cr, sr = math.cos(th), math.sin(th)
    ex, ey = a * np.cos(t), b * np.sin(t)
    exp_, eyp = -a * np.sin(t), b * np.cos(t)
    x = center[0] + cr * ex - sr * ey
    y = center[1] + sr * ex + cr * ey
    xp = cr * exp_ - sr * eyp
    yp = sr * exp_ + cr * eyp
    sp = np.sqrt(xp * xp + yp * yp)
    normals = np.stack([yp / sp, -xp / sp], axis=1)
    curv = a * b / (a * a * np.sin(t) ** 2 + b * b * np.cos(t) ** 2) ** 1.5
    return Interface(np.stack([x, y], axis=1), normals, curv, "ellipse",
                     dict(a=a, b=b, rot_deg=rot_deg, center=center))


# ---------------------------------------------------------------- manufactured solutions
@dataclass
class Manufactured:
    """u(x, y) and f = Lap(u) - kappa^2 u, both vectorised over numpy arrays; grad(x, y)
    returns (u_x, u_y) (the Neumann data of the Neumann BVP)."""
    u: callable
    f: callable
    name: str
    kappa: float
    grad: callable = None


def manufactured_sinpi(kappa: float = 0.0) -> Manufactured:
    """u = sin(pi x) cos(pi y); f = -(2 pi^2 + kappa^2) u."""
    u = lambda x, y: np.sin(np.pi * x) * np.cos(np.pi * y)
    g = lambda x, y: (np.pi * np.cos(np.pi * x) * np.cos(np.pi * y),
                      -np.pi * np.sin(np.pi * x) * np.sin(np.pi * y))
    return Manufactured(u, lambda x, y: -(2 * np.pi ** 2 + kappa ** 2) * u(x, y), "sinpi", kappa, g)


def manufactured_exp_sin2y(kappa: float) -> Manufactured:
    """u = exp(x) sin(2y); Lap u = (1 - 4) u, so f = -(3 + kappa^2) u."""
    u = lambda x, y: np.exp(x) * np.sin(2 * y)
    g = lambda x, y: (np.exp(x) * np.sin(2 * y), 2.0 * np.exp(x) * np.cos(2 * y))
    return Manufactured(u, lambda x, y: -(3.0 + kappa ** 2) * u(x, y), "exp_sin2y", kappa, g)


def manufactured_sincos(w1: float, w2: float, kappa: float) -> Manufactured:
    """u = sin(w1 x) cos(w2 y); f = -(w1^2 + w2^2 + kappa^2) u."""
    u = lambda x, y: np.sin(w1 * x) * np.cos(w2 * y)
    g = lambda x, y: (w1 * np.cos(w1 * x) * np.cos(w2 * y), -w2 * np.sin(w1 * x) * np.sin(w2 * y))
    return Manufactured(u, lambda x, y: -(w1 * w1 + w2 * w2 + kappa ** 2) * u(x, y),
                        f"sincos({w1:.3f},{w2:.3f})", kappa, g)


def manufactured_harmonic_ctx() -> Manufactured:
    """u = e^x cos y + e^y sin x (harmonic, kappa = 0)."""
    u = lambda x, y: np.exp(x) * np.cos(y) + np.exp(y) * np.sin(x)
    g = lambda x, y: (np.exp(x) * np.cos(y) + np.exp(y) * np.cos(x),
                      -np.exp(x) * np.sin(y) + np.exp(y) * np.sin(x))
    return Manufactured(u, lambda x, y: 0.0 * x, "exp_harmonic", 0.0, g)


def grid_nodes(N: int, lo: float = -1.0, hi: float = 1.0):
    """Node coordinates x_i = lo + i*h (i = 0..N) and the (N+1)^2 mesh, x fastest."""
    h = (hi - lo) / N
    xs = lo + np.arange(N + 1, dtype=np.float64) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")  # X[j, i] = x_i, Y[j, i] = y_j
    return xs, X, Y


@dataclass
class Problem:
    """One 2-D Dirichlet BVP instance: interface + grid size + data on grid and on Gamma."""
    iface: Interface
    N: int
    kappa: float
    sol: Manufactured
    lo: float = -1.0
    hi: float = 1.0

    def f_grid(self) -> np.ndarray:
        _, X, Y = grid_nodes(self.N, self.lo, self.hi)
        return self.sol.f(X, Y)

    def u_grid(self) -> np.ndarray:
        _, X, Y = grid_nodes(self.N, self.lo, self.hi)
        return self.sol.u(X, Y)

    def f_ctrl(self) -> np.ndarray:
        p = self.iface.pts
        return self.sol.f(p[:, 0], p[:, 1])

    def g_ctrl(self) -> np.ndarray:
        p = self.iface.pts
        return self.sol.u(p[:, 0], p[:, 1])

    def gn_ctrl(self) -> np.ndarray:
        """Neumann data d_n u = grad u . n at the control points (outward normals)."""
        p, n = self.iface.pts, self.iface.normals
        gx, gy = self.sol.grad(p[:, 0], p[:, 1])
        return gx * n[:, 0] + gy * n[:, 1]


def config_poisson_flower(N: int = 128, M: int = 256) -> Problem:
    """2-D interior Dirichlet Poisson: flower r = 0.5 + 0.15 cos 5t, u = sin(pi x) cos(pi y)."""
    return Problem(flower(M), N, 0.0, manufactured_sinpi(0.0))


def config_helmholtz(N: int, kappa: float, shape: str = "flower", M: int | None = None) -> Problem:
    """2-D modified Helmholtz: flower or rotated ellipse (0.7, 0.4, 30 deg), M = 2N,
    u = exp(x) sin(2y)."""
    M = 2 * N if M is None else M
    iface = flower(M) if shape == "flower" else ellipse(M)
    return Problem(iface, N, float(kappa), manufactured_exp_sin2y(kappa))


def config_batch(count: int = 256, nrhs: int = 4, seed: int = SEED,
                 sizes=(64, 96, 128, 192, 256, 384, 512, 768, 1024)):
    """Batched 2-D Poisson / Helmholtz problems of uneven size.

    Per problem (drawn in this order from one generator): N ~ U(sizes), r0 ~ U(0.4, 0.6),
    a_k ~ U(0, 0.03) and phi_k ~ U(0, 2 pi) for k = 2..6, kappa ~ U(0, 5); then nrhs
    manufactured solutions u = sin(w1 x) cos(w2 y) with w ~ U(1, 4).  M = 2N.
    Returns a list of (Problem for rhs 0, [Manufactured for each rhs]).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.choice(np.asarray(sizes)))
        r0 = float(rng.uniform(0.4, 0.6))
        amps = rng.uniform(0.0, 0.03, size=5)
        phases = rng.uniform(0.0, 2 * np.pi, size=5)
        kappa = float(rng.uniform(0.0, 5.0))
        sols = []
        for _ in range(nrhs):
            w1, w2 = rng.uniform(1.0, 4.0, size=2)
            sols.append(manufactured_sincos(float(w1), float(w2), kappa))
        iface = star(2 * N, r0, amps, phases)
        out.append((Problem(iface, N, kappa, sols[0]), sols))
    return out


def random_density(M: int, seed: int = SEED, smooth: bool = True) -> np.ndarray:
    """A seeded density on the control points: a random trigonometric polynomial of
    low degree (smooth) or i.i.d. N(0,1) values."""
    rng = np.random.default_rng(seed)
    if not smooth:
        return rng.standard_normal(M)
    t = 2 * np.pi * np.arange(M) / M
    out = np.zeros(M)
    for k in range(0, 8):
        a, b = rng.standard_normal(2) / (1 + k)
        out += a * np.cos(k * t) + b * np.sin(k * t)
    return out
