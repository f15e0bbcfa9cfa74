"""FP64 CPU oracle of the 3-D KFBI method (TEST INFRASTRUCTURE ONLY; see package header).

The same method as kfbi2d (Sec. 2.1-2.2, Alg. 1-5) on the box [lo, hi]^3 with the
7-point Laplacian.  The paper states its 3-D discretisation only by analogy with 2-D;
the readings used here (derived from the interface conditions) are:
  S1  the control points are the intersections of Gamma with the grid lines, given with
      outward unit normals n and the shape operator S (dn = S dx on tangent vectors,
      packed Sxx, Syy, Szz, Sxy, Sxz, Syz); the density lives on these points;
  S2  a point lies on the line of axis a when its two other coordinates are grid values
      to within 1e-9 h; a point on no line or on several (a grid node) is rejected;
      it belongs to the edge x_e < x_q <= x_{e+1} of its line;
  S3  node (i, j, k) is inside iff an odd number of the points of x-line (j, k) have
      x_q <= x_i; the y- and z-line parities must give the same labels; an edge whose
      end labels differ holds exactly one point (two points on one edge are a grid line
      grazing Gamma: the labels agree, the edge is no arm, the points stay control
      points); no inside node within two cells of the box boundary;
  S4  irregular node: interior node with a 7-point neighbour of the other label; the
      arm to that neighbour holds exactly one point q;
  S5  surface derivatives of a density at point p: least-squares quadratic
      c0 + c1 a + c2 b + c3 a^2 + c4 a b + c5 b^2 in the tangent-plane coordinates
      (a, b) = ((X_q - X_p).t1, (X_q - X_p).t2) / h over all points within 2.5 h of p
      (3.5 h when fewer than 10), normal equations by Cholesky; t1 = normalise(e x n)
      with e the coordinate axis least aligned with n (lowest index on ties),
      t2 = n x t1; grad_G = (c1 t1 + c2 t2) / h, Hess_G = [[2 c3, c4], [c4, 2 c5]] / h^2
      in (t1, t2);
  S6  jumps at p in the frame (n, t1, t2), Phi~ and psi~ the fitted values c0:
        [v] = Phi~_p,  grad[v] = psi~ n + grad_G Phi,
        [v_ab] = Hess_G Phi_ab + psi~ II_ab         (a, b tangent, II_ab = t_a . S t_b),
        [v_na] = d_a psi - t_a . S grad_G Phi,
        [v_nn] = [F] + kappa^2 Phi~ - Lap_G Phi - tr(S) psi~;
      (the grid cannot carry a density that varies from point to point faster than the
      grid resolves: with the raw point values in [v] such modes would reach K_D only
      through the in/out split of each interpolation stencil, giving eigenvalues near
      zero; the fit removes them from the interface problem);
  S7  correction along each of the 6 arms exactly as R7 of kfbi2d;
  S8  interpolation at z: nearest node c (round half up), stencil c, c +- e_x, c +- e_y,
      c +- e_z and c + s_a e_a + s_b e_b for the three axis pairs (s = +1 where z >= c);
      outside values get the second-order Taylor expansion of the jump about z (as R8);
      v^+(z) from the 10x10 quadratic fit;
  S9  box solve: sine transforms along z and y, Thomas solve along x per mode pair,
      inverse transforms scaled by 2/N each (Alg. 4);
  S10 K_D phi = v^+[Phi~] + (phi - Phi~) / 2: the double layer acts on the fitted
      density, the identity part 1/2 phi of the BIE (Sec. 2.1) on the point values (for
      a smooth density Phi~ - phi = O(h^3); a point-to-point oscillation is mapped to
      half itself, as by the continuous operator).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_factor, cho_solve
from scipy.sparse import csr_matrix
from scipy.spatial import cKDTree

from .kfbi2d import GeometryError, gmres, sine_matrix

TAG_TOL = 1e-9      # S2, units of h
LS_RADIUS = 2.5     # S5, units of h
LS_RADIUS_WIDE = 3.5
LS_MIN = 10


def unpack_shape(packed):
    """(P, 6) packed shape operators -> (P, 3, 3)."""
    p = np.asarray(packed, dtype=np.float64)
    S = np.empty((p.shape[0], 3, 3))
    S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = p[:, 0], p[:, 1], p[:, 2]
    S[:, 0, 1] = S[:, 1, 0] = p[:, 3]
    S[:, 0, 2] = S[:, 2, 0] = p[:, 4]
    S[:, 1, 2] = S[:, 2, 1] = p[:, 5]
    return S


def tangent_frame(n):
    """t1 = normalise(e x n), e the axis least aligned with n; t2 = n x t1 (S5)."""
    n = np.asarray(n, dtype=np.float64)
    e = np.zeros_like(n)
    e[np.arange(n.shape[0]), np.argmin(np.abs(n), axis=1)] = 1.0
    t1 = np.cross(e, n)
    t1 /= np.linalg.norm(t1, axis=1)[:, None]
    t2 = np.cross(n, t1)
    return t1, t2


def jumps_from_surface(phi, g_phi, H_phi, psi, g_psi, n, t1, t2, S, Fj, kappa2):
    """Cartesian jumps (S6) from the surface data of Phi and psi at the points.

    phi, psi, Fj: (P,); g_phi, g_psi: (P, 2) tangential gradients in (t1, t2); H_phi:
    (P, 2, 2) surface Hessian in (t1, t2); n, t1, t2: (P, 3); S: (P, 3, 3).
    Returns J (P,), G (P, 3), H (P, 3, 3)."""
    T = np.stack([t1, t2], axis=1)                               # (P, 2, 3)
    II = np.einsum("pai,pij,pbj->pab", T, S, T)
    grad_G_phi = np.einsum("pa,pai->pi", g_phi, T)
    tan = H_phi + psi[:, None, None] * II
    mixed = g_psi - np.einsum("pai,pij,pj->pa", T, S, grad_G_phi)
    trS = np.trace(S, axis1=1, axis2=2)
    nn = Fj + kappa2 * phi - (H_phi[:, 0, 0] + H_phi[:, 1, 1]) - trS * psi
    G = psi[:, None] * n + grad_G_phi
    H = nn[:, None, None] * n[:, :, None] * n[:, None, :]
    for a in range(2):
        na = n[:, :, None] * T[:, a, None, :]
        H += mixed[:, a, None, None] * (na + np.transpose(na, (0, 2, 1)))
        for b in range(2):
            H += tan[:, a, b, None, None] * T[:, a, :, None] * T[:, b, None, :]
    return np.asarray(phi, dtype=np.float64).copy(), G, H


class Geometry3D:
    """Point tags, node labels, irregular-node arms, LS stencils and interpolation
    stencils of a 3-D interface given by its grid-line intersection points (S1-S5, S8).

    pts, normals: (P, 3); shape: (P, 6) packed; N cells per side of [lo, hi]^3."""

    def __init__(self, pts, normals, shape, N, kappa, lo=-1.0, hi=1.0):
        self.pts = np.ascontiguousarray(pts, dtype=np.float64)
        self.normals = np.ascontiguousarray(normals, dtype=np.float64)
        self.S = unpack_shape(shape)
        self.P = int(self.pts.shape[0])
        self.N = int(N)
        self.kappa = float(kappa)
        self.kappa2 = self.kappa ** 2
        self.lo, self.hi = float(lo), float(hi)
        self.h = (self.hi - self.lo) / self.N
        self.xs = self.lo + np.arange(self.N + 1) * self.h
        self._tag()
        self._classify()
        self._arms()
        self._ls_stencils()
        self._interp_stencils()

    # --------------------------------------------------------------------------- S2
    def _tag(self):
        g = (self.pts - self.lo) / self.h
        on = np.abs(g - np.round(g)) <= TAG_TOL                   # (P, 3) coordinate on grid
        axis = np.full(self.P, -1)
        for a in range(3):
            o = [q for q in range(3) if q != a]
            sel = on[:, o[0]] & on[:, o[1]] & ~on[:, a]
            axis[sel] = a
        if np.any(axis < 0):
            raise GeometryError("a point lies on no grid line or on a grid node")
        self.axis = axis
        self.line = np.round(g).astype(np.int64)                  # off-axis node indices
        self.edge = np.floor(g[np.arange(self.P), axis]).astype(np.int64)
        if np.any(self.edge < 0) or np.any(self.edge >= self.N):
            raise GeometryError("a point lies outside the box")
        # (axis, two off-axis indices, edge) -> points on that edge
        self.edge_point = {}
        for p in range(self.P):
            a = axis[p]
            o = [q for q in range(3) if q != a]
            key = (a, int(self.line[p, o[0]]), int(self.line[p, o[1]]), int(self.edge[p]))
            self.edge_point.setdefault(key, []).append(p)

    # --------------------------------------------------------------------------- S3
    def _classify(self):
        N = self.N
        labels = []
        for a in range(3):
            D = np.zeros((N + 2,) * 3, dtype=np.int64)            # indexed [x, y, z] here
            sel = self.axis == a
            idx = self.line[sel].copy()
            idx[:, a] = self.edge[sel] + 1
            np.add.at(D, (idx[:, 0], idx[:, 1], idx[:, 2]), 1)
            cnt = np.cumsum(D, axis=a)[: N + 1, : N + 1, : N + 1]
            labels.append((cnt % 2 == 1).transpose(2, 1, 0))      # -> [k, j, i]
        if not (np.array_equal(labels[0], labels[1]) and np.array_equal(labels[0], labels[2])):
            raise GeometryError("node labels from x-, y- and z-lines disagree")
        inside = labels[0]
        band = np.zeros_like(inside)
        band[:3], band[-3:] = True, True
        band[:, :3], band[:, -3:] = True, True
        band[:, :, :3], band[:, :, -3:] = True, True
        if np.any(inside & band):
            raise GeometryError("interface within two cells of the box boundary")
        self.inside = inside

    # --------------------------------------------------------------------------- S4
    def _arms(self):
        N, h, ins = self.N, self.h, self.inside
        arms = []   # (k, j, i, axis, point, delta, sigma)
        idx = np.argwhere(np.ones((N - 1,) * 3, dtype=bool)) + 1
        kk, jj, ii = idx[:, 0], idx[:, 1], idx[:, 2]
        lab = ins[kk, jj, ii]
        irregular = np.zeros((N + 1,) * 3, dtype=bool)
        for a, (dk, dj, di) in enumerate(((0, 0, 1), (0, 1, 0), (1, 0, 0))):
            for sgn in (1, -1):
                nb = ins[kk + sgn * dk, jj + sgn * dj, ii + sgn * di]
                hit = np.nonzero(nb != lab)[0]
                for r in hit:
                    k, j, i = int(kk[r]), int(jj[r]), int(ii[r])
                    node = (i, j, k)
                    e = node[a] if sgn > 0 else node[a] - 1
                    o = [q for q in range(3) if q != a]
                    key = (a, node[o[0]], node[o[1]], e)
                    if len(self.edge_point.get(key, ())) != 1:
                        raise GeometryError("an edge with a label change holds %d points"
                                            % len(self.edge_point.get(key, ())))
                    q = self.edge_point[key][0]
                    nb_coord = self.xs[node[a] + sgn]
                    delta = nb_coord - self.pts[q, a]
                    sigma = -1.0 if lab[r] else 1.0
                    arms.append((k, j, i, a, q, delta, sigma))
                    irregular[k, j, i] = True
        self.arms = arms
        self.irregular = irregular
        A = np.array(arms, dtype=np.float64).reshape(-1, 7)
        self.arm_kji = A[:, :3].astype(np.int64)
        self.arm_axis = A[:, 3].astype(np.int64)
        self.arm_point = A[:, 4].astype(np.int64)
        self.arm_delta = A[:, 5]
        self.arm_sigma = A[:, 6]

    # --------------------------------------------------------------------------- S5
    def _ls_stencils(self):
        h = self.h
        tree = cKDTree(self.pts)
        self.t1, self.t2 = tangent_frame(self.normals)
        self.ls_nbrs, self.ls_w = [], []
        for p in range(self.P):
            nb = sorted(tree.query_ball_point(self.pts[p], LS_RADIUS * h * (1 + 1e-12)))
            if len(nb) < LS_MIN:
                nb = sorted(tree.query_ball_point(self.pts[p], LS_RADIUS_WIDE * h * (1 + 1e-12)))
            if len(nb) < LS_MIN:
                raise GeometryError("fewer than 10 points near a point (surface under-resolved)")
            nb = np.asarray(nb)
            d = self.pts[nb] - self.pts[p]
            a, b = d @ self.t1[p] / h, d @ self.t2[p] / h
            A = np.stack([np.ones_like(a), a, b, a * a, a * b, b * b], axis=1)
            W = cho_solve(cho_factor(A.T @ A), A.T)                # (6, |Q|)
            self.ls_nbrs.append(nb)
            self.ls_w.append(W)
        # the fitted coefficients c1..c5 as sparse linear maps of the density
        rows = np.concatenate([np.full(len(nb), p) for p, nb in enumerate(self.ls_nbrs)])
        cols = np.concatenate(self.ls_nbrs)
        self.ls_maps = [csr_matrix((np.concatenate([W[r] for W in self.ls_w]), (rows, cols)),
                                   shape=(self.P, self.P)) for r in range(6)]

    def fitted(self, dens):
        """The fitted value c0 of a density at every point (S5)."""
        return self.ls_maps[0] @ np.asarray(dens, dtype=np.float64)

    def surface_derivs(self, dens):
        """Fitted value (P,), tangential gradient (P, 2) and surface Hessian (P, 2, 2) of
        a density (S5)."""
        dens = np.asarray(dens, dtype=np.float64)
        c = [m @ dens for m in self.ls_maps]
        h = self.h
        g = np.stack([c[1], c[2]], axis=1) / h
        H = np.stack([np.stack([2 * c[3], c[4]], axis=1), np.stack([c[4], 2 * c[5]], axis=1)],
                     axis=1) / (h * h)
        return c[0], g, H

    def jumps(self, phi=None, psi=None, f_ctrl=None):
        """Cartesian jumps (J, G, H) at every point (S6)."""
        P = self.P
        z = np.zeros(P)
        phi = z if phi is None else np.asarray(phi, dtype=np.float64)
        psi = z if psi is None else np.asarray(psi, dtype=np.float64)
        Fj = z if f_ctrl is None else np.asarray(f_ctrl, dtype=np.float64)
        f_phi, g_phi, H_phi = self.surface_derivs(phi)
        f_psi, g_psi, _ = self.surface_derivs(psi)
        return jumps_from_surface(f_phi, g_phi, H_phi, f_psi, g_psi, self.normals, self.t1,
                                  self.t2, self.S, Fj, self.kappa2)

    # --------------------------------------------------------------------------- S8
    def _interp_stencils(self):
        g = (self.pts - self.lo) / self.h
        c = np.floor(g + 0.5).astype(np.int64)                   # round half up
        s = np.where(self.pts >= self.xs[c], 1, -1)
        offs = [np.zeros((self.P, 3), dtype=np.int64)]
        for a in range(3):
            for sg in (1, -1):
                o = np.zeros((self.P, 3), dtype=np.int64)
                o[:, a] = sg
                offs.append(o)
        for a, b in ((0, 1), (0, 2), (1, 2)):
            o = np.zeros((self.P, 3), dtype=np.int64)
            o[:, a] = s[:, a]
            o[:, b] = s[:, b]
            offs.append(o)
        nodes = c[:, None, :] + np.stack(offs, axis=1)            # (P, 10, 3) as (i, j, k)
        if np.any(nodes < 1) or np.any(nodes > self.N - 1):
            raise GeometryError("interpolation stencil leaves the interior of the box")
        self.interp_nodes = nodes


def correct_rhs(geom: Geometry3D, jumps, F_grid=None):
    """Corrected right-hand side on the (N+1)^3 grid (S7); F_grid outside Omega ignored."""
    N, h = geom.N, geom.h
    b = np.zeros((N + 1,) * 3)
    if F_grid is not None:
        b[1:N, 1:N, 1:N] = np.where(geom.inside[1:N, 1:N, 1:N],
                                    np.asarray(F_grid)[1:N, 1:N, 1:N], 0.0)
    J, G, H = jumps
    q, a, d = geom.arm_point, geom.arm_axis, geom.arm_delta
    T = J[q] + d * G[q, a] + 0.5 * d * d * H[q, a, a]
    kji = geom.arm_kji
    np.add.at(b, (kji[:, 0], kji[:, 1], kji[:, 2]), geom.arm_sigma * T / (h * h))
    return b


# --------------------------------------------------------------------------- Alg. 4
def box_solve_dst(b, N, h, kappa2):
    """(Lap_h - kappa^2) v = b on interior nodes of the (N+1)^3 grid, v = 0 on the box
    boundary: sine transforms along z and y, Thomas along x per mode pair, inverse."""
    S = sine_matrix(N)
    n = N - 1
    Bh = np.einsum("mk,lj,kji->mli", S, S, b[1:N, 1:N, 1:N], optimize=True)
    lam = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, N) / (2.0 * N)) ** 2
    off = 1.0 / (h * h)
    diag = -2.0 / (h * h) + lam[:, None] + lam[None, :] - kappa2   # [m, l]
    cp = np.zeros((n, n, n))
    dp = np.zeros((n, n, n))
    cp[:, :, 0] = off / diag
    dp[:, :, 0] = Bh[:, :, 0] / diag
    for i in range(1, n):
        den = diag - off * cp[:, :, i - 1]
        cp[:, :, i] = off / den
        dp[:, :, i] = (Bh[:, :, i] - off * dp[:, :, i - 1]) / den
    Vh = np.zeros((n, n, n))
    Vh[:, :, n - 1] = dp[:, :, n - 1]
    for i in range(n - 2, -1, -1):
        Vh[:, :, i] = dp[:, :, i] - cp[:, :, i] * Vh[:, :, i + 1]
    v = np.zeros((N + 1,) * 3)
    v[1:N, 1:N, 1:N] = (2.0 / N) ** 2 * np.einsum("mk,lj,mli->kji", S, S, Vh, optimize=True)
    return v


def box_solve_dense(b, N, h, kappa2):
    """The same system as a dense (N-1)^3 matrix solved by LU (tiny grids only)."""
    n = N - 1
    A = np.zeros((n ** 3, n ** 3))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                r = (k * n + j) * n + i
                A[r, r] = -6.0 / (h * h) - kappa2
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    i2, j2, k2 = i + di, j + dj, k + dk
                    if 0 <= i2 < n and 0 <= j2 < n and 0 <= k2 < n:
                        A[r, (k2 * n + j2) * n + i2] = 1.0 / (h * h)
    v = np.zeros((N + 1,) * 3)
    v[1:N, 1:N, 1:N] = np.linalg.solve(A, b[1:N, 1:N, 1:N].reshape(-1)).reshape(n, n, n)
    return v


# --------------------------------------------------------------------------- Alg. 3
def interpolate_plus(geom: Geometry3D, v, jumps):
    """v^+ at every point (S8) by solving each 10x10 quadratic fit."""
    J, G, H = jumps
    nodes = geom.interp_nodes                                     # (P, 10, 3) (i, j, k)
    X = geom.xs[nodes]                                            # node coordinates
    d = X - geom.pts[:, None, :]
    taylor = J[:, None] + np.einsum("pd,pkd->pk", G, d) + 0.5 * np.einsum("pkd,pde,pke->pk", d, H, d)
    ii, jj, kk = nodes[..., 0], nodes[..., 1], nodes[..., 2]
    vals = v[kk, jj, ii] + np.where(geom.inside[kk, jj, ii], 0.0, taylor)
    x, y, z = d[..., 0] / geom.h, d[..., 1] / geom.h, d[..., 2] / geom.h
    V = np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, x * z, y * z], axis=2)
    coef = np.linalg.solve(V, vals[:, :, None])[:, :, 0]
    return coef[:, 0]


# ----------------------------------------------------------------- Sec. 2.2 / Alg. 1
def apply_interface(geom: Geometry3D, phi=None, psi=None, f_ctrl=None, F_grid=None,
                    solver=box_solve_dst, return_all=False):
    """Interface problem with [v] = phi, [d_n v] = psi, F = zero-extended F_grid and
    [F] = f on Gamma; v^+ at the points (and b, v)."""
    jm = geom.jumps(phi, psi, f_ctrl)
    b = correct_rhs(geom, jm, F_grid)
    v = solver(b, geom.N, geom.h, geom.kappa2)
    out = interpolate_plus(geom, v, jm)
    return (out, b, v) if return_all else out


def apply_double_layer(geom, phi, **kw):
    """K_D phi = (1/2 I + W) phi (Sec. 3.3): v^+ of the interface problem with the fitted
    density, plus half the difference between the point values and the fit (S10)."""
    phi = np.asarray(phi, dtype=np.float64)
    if kw.get("return_all"):
        out, b, v = apply_interface(geom, phi=phi, **kw)
        return out + 0.5 * (phi - geom.fitted(phi)), b, v
    return apply_interface(geom, phi=phi, **kw) + 0.5 * (phi - geom.fitted(phi))


def apply_volume(geom, f_grid, f_ctrl, **kw):
    """(Y f)^+ on Gamma (Sec. 2.2 table)."""
    return apply_interface(geom, f_ctrl=f_ctrl, F_grid=f_grid, **kw)


def solve_bvp(geom: Geometry3D, f_grid, f_ctrl, g_ctrl, tol=1e-10, m=50, max_restarts=20):
    """Dirichlet BVP through 1/2 phi + W phi + Y f = g (Sec. 2.1), GMRES (Alg. 5)."""
    ghat = np.asarray(g_ctrl, dtype=np.float64) - apply_volume(geom, f_grid, f_ctrl)
    phi, info = gmres(lambda p: apply_double_layer(geom, p), ghat, m=m, tol=tol,
                      max_restarts=max_restarts)
    _, _, v = apply_interface(geom, phi=phi, f_ctrl=f_ctrl, F_grid=f_grid, return_all=True)
    return np.where(geom.inside, v, 0.0), phi, info
