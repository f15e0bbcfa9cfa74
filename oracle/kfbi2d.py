"""FP64 CPU oracle of the 2-D KFBI method (TEST INFRASTRUCTURE ONLY; see package header).

What it computes (paper Sec. 2.1-2.2 and Alg. 1-5):
  * the interface problem  Lap v - kappa^2 v = F,  [v] = Phi,  [d_n v] = psi,  v = 0 on
    the box boundary (Sec. 2.2; the double-layer potential W phi is the case F = 0,
    Phi = phi, psi = 0 and the volume integral Y f the case F = zero-extended f, Phi = 0);
  * its second-order discretisation (Alg. 1): 5-point Laplacian, Taylor correction of
    the right-hand side at irregular nodes (Alg. 2), a sine-transform box solve (Alg. 4),
    corrected 6-point interpolation of v^+ at the control points (Alg. 3);
  * K_D phi = (1/2 I + W) phi as the one-sided limit v^+ (Sec. 3.3), the BIE
    1/2 phi + W phi + Y f = g (Sec. 2.1) solved by restarted GMRES with modified
    Gram-Schmidt and a least-squares solve (Alg. 5) or by Richardson iteration (Sec. 2.1);
  * the error norms of Sec. 5.

The paper defers the jump formulas, the interface interpolant and the stencils to its
CPU predecessor; the readings used here (derived from the interface conditions) are:
  R1  PDE written as Lap v - kappa^2 v (the paper prints an unsquared kappa);
  R2  [w] = w(inside) - w(outside); n is the outward normal; points are CCW;
      tau = (-n_y, n_x); curvature chi > 0 on convex parts (d tau/ds = -chi n);
  R3  the interface is the periodic degree-5 Lagrange interpolant of the control
      points in the uniform parameter t_k = 2 pi k / M: on [t_k, t_{k+1}) it passes
      through X_{k-2..k+3}; densities and f on Gamma are interpolated the same way;
  R4  crossings of Gamma with grid lines: 8 sub-samples per segment, a sub-interval
      [A, B] holds a crossing with line c iff (A >= c) != (B >= c), refined by bisection;
  R5  a crossing within 1e-10 h of a grid node is moved onto it; node (i, j) is inside
      iff an odd number of row-j crossings have x_q <= x_i (a node on Gamma joins the
      side to its right); on every grid line (row or column) the k-th crossing in
      increasing order belongs to the k-th arm whose end labels differ and must lie on
      that arm (1e-8 h slack), else GeometryError; two consecutive crossings strictly
      inside one arm whose end labels agree (a grid line grazing Gamma where its radius
      of curvature exceeds 2 h) are dropped first: they carry no correction; no node
      within two cells of the box boundary may be inside; the interface is rejected as
      under-resolved when |curvature| h > 4 at a control point (radius below h/4);
  R6  jumps in the local frame (xi = n, eta = tau):
        [v] = Phi, [v_xi] = psi, [v_eta] = Phi_s, [v_eta eta] = Phi_ss + chi psi,
        [v_xi eta] = psi_s - chi Phi_s, [v_xi xi] = [F] + kappa^2 Phi - Phi_ss - chi psi;
  R7  correction at irregular node p for the arm to nb crossing Gamma at q along axis a:
        b_p += sigma * ([v] + d [v_a] + d^2/2 [v_aa])(q) / h^2,  d = nb_a - q_a,
        sigma = -1 if p is inside, +1 if outside;
  R8  interpolation at z: nearest node c (round half up), stencil c, c +- e_x, c +- e_y,
      c + s_x e_x + s_y e_y with s = +1 where z >= c; values at outside nodes get the
      second-order Taylor expansion of the jump about z added; v^+(z) is the value at z
      of the quadratic through the 6 corrected values (6x6 solve);
  R9  box solve: sine transform in y, tridiagonal (Thomas) solve in x per mode, inverse
      sine transform (Alg. 4), dense sine matrix from a table sin(pi m / N);
  R10 Neumann data d_n u (Procedure 2): n . grad of the same 6-point quadratic as R8 at z;
      the Neumann BVP uses the single-layer density psi ([v] = 0, [d_n v] = psi).
"""
from __future__ import annotations

import numpy as np

SUBSAMPLES = 8           # R4
BISECTION_STEPS = 64     # bracket shrinks to 2^-67 of a segment: below FP64 resolution
SNAP = 1e-10             # a crossing this close (in units of h) to a node lies on it (R5)
ARM_TOL = 1e-8           # slack (units of h) when matching crossings to arms (R5)
GRAZE_CURV = 0.5         # a grazing pair is accepted where |curvature| h <= this (R5)
MAX_CURV_H = 4.0         # |curvature| h above this at a control point: under-resolved (R5)


class GeometryError(ValueError):
    """Interface under-resolved by the grid, or too close to the box boundary (R5)."""


# ----------------------------------------------------------------------------- R3
_NODES = np.arange(-2.0, 4.0)  # local parameter of X_{k-2..k+3} on segment k


def _basis_polys():
    polys = []
    for r in range(6):
        others = np.delete(_NODES, r)
        num = np.poly(others)                       # prod_{s != r} (tau - tau_s)
        den = np.prod(_NODES[r] - others)
        polys.append(num / den)
    return polys


_BASIS = _basis_polys()
_BASIS_D1 = [np.polyder(p) for p in _BASIS]
_BASIS_D2 = [np.polyder(p, 2) for p in _BASIS]


def lagrange_basis(tau):
    """Values and first/second tau-derivatives of the 6 Lagrange basis polynomials of
    the degree-5 interpolant (R3) at local parameters tau in [0, 1].  Each (K, 6)."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    L0 = np.stack([np.polyval(p, tau) for p in _BASIS], axis=1)
    L1 = np.stack([np.polyval(p, tau) for p in _BASIS_D1], axis=1)
    L2 = np.stack([np.polyval(p, tau) for p in _BASIS_D2], axis=1)
    return L0, L1, L2


def jumps_cartesian(phi, phi_s, phi_ss, psi, psi_s, Fj, n, tau, chi, kappa2):
    """Jumps [v], grad[v], Hess[v] in Cartesian axes from the interface data (R6).

    Arrays of shape (K,) except n, tau (K, 2).  Returns J (K,), G (K, 2), H (K, 2, 2)."""
    j_xi = psi
    j_eta = phi_s
    j_ee = phi_ss + chi * psi
    j_xe = psi_s - chi * phi_s
    j_xx = Fj + kappa2 * phi - phi_ss - chi * psi
    G = j_xi[:, None] * n + j_eta[:, None] * tau
    nn = n[:, :, None] * n[:, None, :]
    tt = tau[:, :, None] * tau[:, None, :]
    nt = n[:, :, None] * tau[:, None, :]
    H = j_xx[:, None, None] * nn + j_xe[:, None, None] * (nt + np.transpose(nt, (0, 2, 1))) \
        + j_ee[:, None, None] * tt
    return np.asarray(phi, dtype=np.float64).copy(), G, H


class Geometry2D:
    """Grid, interface interpolant, crossings, node labels and irregular-node arms.

    pts, normals: (M, 2) CCW control points and outward normals; curv: (M,) signed
    curvature; N cells per side of the box [lo, hi]^2; kappa >= 0 (R1)."""

    def __init__(self, pts, normals, curv, N, kappa, lo=-1.0, hi=1.0):
        self.pts = np.ascontiguousarray(pts, dtype=np.float64)
        self.normals = np.ascontiguousarray(normals, dtype=np.float64)
        self.curv = np.ascontiguousarray(curv, dtype=np.float64)
        self.M = int(self.pts.shape[0])
        self.N = int(N)
        self.kappa = float(kappa)
        self.kappa2 = self.kappa * self.kappa
        self.lo, self.hi = float(lo), float(hi)
        self.h = (self.hi - self.lo) / self.N
        self.xs = self.lo + np.arange(self.N + 1, dtype=np.float64) * self.h
        self.dt = 2.0 * np.pi / self.M
        self._stencil_idx = (np.arange(self.M)[:, None] + np.arange(-2, 4)[None, :]) % self.M
        if np.max(np.abs(self.curv)) * self.h > MAX_CURV_H:
            raise GeometryError("radius of curvature below a quarter cell (under-resolved interface)")
        self._find_crossings()
        self._classify()
        self._arms()
        self._controls()

    # ------------------------------------------------------------ interpolant (R3)
    def curve_derivs(self, seg, tau):
        """X, X', X'' (d/dt) of the interpolant on segments seg at local tau."""
        L0, L1, L2 = lagrange_basis(tau)
        P = self.pts[self._stencil_idx[seg]]            # (K, 6, 2)
        X = np.einsum("kr,krd->kd", L0, P)
        X1 = np.einsum("kr,krd->kd", L1, P) / self.dt
        X2 = np.einsum("kr,krd->kd", L2, P) / self.dt ** 2
        return X, X1, X2

    def _eval_coord(self, seg, tau, axis):
        L0, _, _ = lagrange_basis(tau)
        P = self.pts[self._stencil_idx[seg], axis]
        return np.sum(L0 * P, axis=1)

    # ------------------------------------------------------------ crossings (R4)
    def _find_crossings(self):
        M, S = self.M, SUBSAMPLES
        taus = np.arange(S + 1, dtype=np.float64) / S
        L0, _, _ = lagrange_basis(taus)
        P = self.pts[self._stencil_idx]                  # (M, 6, 2)
        samp = np.einsum("sr,mrd->msd", L0, P)           # (M, S+1, 2)
        samp[:, 0, :] = self.pts
        samp[:, S, :] = self.pts[(np.arange(M) + 1) % M]
        self.crossings = {}
        for axis in (0, 1):
            A = samp[:, :-1, axis].reshape(-1)
            B = samp[:, 1:, axis].reshape(-1)
            lo_v = np.minimum(A, B)
            i0 = np.floor((lo_v - self.lo) / self.h).astype(np.int64) - 1
            span = int(np.max(np.ceil((np.abs(B - A)) / self.h))) + 3
            cand = i0[:, None] + np.arange(span)[None, :]
            valid = (cand >= 0) & (cand <= self.N)
            c = self.xs[np.clip(cand, 0, self.N)]
            hit = valid & ((A[:, None] >= c) != (B[:, None] >= c))
            sub_id, which = np.nonzero(hit)
            line = cand[sub_id, which]
            seg = sub_id // S
            s = sub_id % S
            ta = s / S
            tb = (s + 1) / S
            cval = self.xs[line]
            fa_pos = A[sub_id] >= cval                   # sign state at the left end
            # bisection keeping (f(ta) >= 0) != (f(tb) >= 0)
            for _ in range(BISECTION_STEPS):
                tm = 0.5 * (ta + tb)
                fm_pos = self._eval_coord(seg, tm, axis) >= cval
                left = fm_pos == fa_pos
                ta = np.where(left, tm, ta)
                tb = np.where(left, tb, tm)
            tq = 0.5 * (ta + tb)
            X, X1, X2 = self.curve_derivs(seg, tq)
            pos = X.copy()
            pos[:, axis] = cval                          # the crossing lies on the line
            other = 1 - axis                             # snap onto a node if within SNAP*h
            k = np.floor((pos[:, other] - self.lo) / self.h + 0.5).astype(np.int64)
            near = self.xs[np.clip(k, 0, self.N)]
            pos[:, other] = np.where(np.abs(pos[:, other] - near) <= SNAP * self.h, near, pos[:, other])
            self.crossings[axis] = dict(line=line, seg=seg, tau=tq, pos=pos, X1=X1, X2=X2)
        # per-line sorted lists: axis 1 crossings lie on rows y = y_j (sorted by x),
        # axis 0 crossings lie on columns x = x_i (sorted by y)
        self.row_lists = self._per_line(1, 0)
        self.col_lists = self._per_line(0, 1)

    def _per_line(self, axis, along):
        cr = self.crossings[axis]
        order = np.lexsort((cr["pos"][:, along], cr["line"]))
        lists = [np.zeros(0, dtype=np.int64) for _ in range(self.N + 1)]
        line_sorted = cr["line"][order]
        starts = np.searchsorted(line_sorted, np.arange(self.N + 2))
        for L in range(self.N + 1):
            lists[L] = order[starts[L]:starts[L + 1]]
        return lists

    # ------------------------------------------------------------ labels (R5)
    def _classify(self):
        N = self.N
        inside = np.zeros((N + 1, N + 1), dtype=bool)       # [j, i]
        xq_rows = self.crossings[1]["pos"][:, 0]
        for j in range(N + 1):
            xq = np.sort(xq_rows[self.row_lists[j]])
            cnt = np.searchsorted(xq, self.xs, side="right")    # #{x_q <= x_i}
            inside[j] = (cnt % 2) == 1
        edge = np.zeros_like(inside)
        edge[:2, :] = edge[-2:, :] = edge[:, :2] = edge[:, -2:] = True
        if np.any(inside & edge):
            raise GeometryError("interface within two cells of the box boundary")
        self.inside = inside

    # ------------------------------------------------------------ arms (R5, R7)
    def _match_line(self, labels, lst, coord, curv):
        """k-th crossing (sorted) on a grid line <-> k-th arm whose end labels differ, after
        dropping grazing pairs: two consecutive crossings strictly inside one arm (more
        than ARM_TOL h from its nodes) whose end labels agree, where the curve is resolved
        (|curvature| h <= GRAZE_CURV at both), carry no correction (R5)."""
        flips = np.nonzero(labels[1:] != labels[:-1])[0]
        order = lst[np.argsort(coord[lst], kind="stable")]
        tol = ARM_TOL * self.h
        keep, q = [], 0
        while q < order.size:
            if q + 1 < order.size:
                a0, a1 = coord[order[q]], coord[order[q + 1]]
                t = int(np.floor((a0 - self.lo) / self.h))
                if (0 <= t < self.N and a0 > self.xs[t] + tol and a1 < self.xs[t + 1] - tol
                        and labels[t] == labels[t + 1]
                        and curv[order[q]] * self.h <= GRAZE_CURV
                        and curv[order[q + 1]] * self.h <= GRAZE_CURV):
                    q += 2
                    continue
            keep.append(order[q])
            q += 1
        order = np.asarray(keep, dtype=np.int64)
        if flips.size != order.size:
            raise GeometryError("a grid line meets the interface at a point where the "
                                "node labels do not change (tangency or under-resolution)")
        tol = ARM_TOL * self.h
        c = coord[order]
        if np.any(c < self.xs[flips] - tol) or np.any(c > self.xs[flips + 1] + tol):
            raise GeometryError("a grid arm is crossed more than once (under-resolved interface)")
        return dict(zip(flips.tolist(), order.tolist()))

    def _arms(self):
        N, ins = self.N, self.inside
        xq_rows = self.crossings[1]["pos"][:, 0]
        yq_cols = self.crossings[0]["pos"][:, 1]
        def abs_curv(cr):
            X1, X2 = cr["X1"], cr["X2"]
            return np.abs(X1[:, 0] * X2[:, 1] - X1[:, 1] * X2[:, 0]) / np.hypot(X1[:, 0], X1[:, 1]) ** 3
        kr, kc = abs_curv(self.crossings[1]), abs_curv(self.crossings[0])
        harm = [self._match_line(ins[j, :], self.row_lists[j], xq_rows, kr) for j in range(N + 1)]
        varm = [self._match_line(ins[:, i], self.col_lists[i], yq_cols, kc) for i in range(N + 1)]
        h_diff = ins[:, 1:] != ins[:, :-1]
        v_diff = ins[1:, :] != ins[:-1, :]
        irr = np.zeros_like(ins)
        irr[1:N, 1:N] = (h_diff[1:N, 1:N] | h_diff[1:N, 0:N - 1] |
                         v_diff[1:N, 1:N] | v_diff[0:N - 1, 1:N])
        self.irregular = irr
        arms = []   # (j, i, arm_axis, crossing_axis, crossing_id, delta, sigma)
        jj, ii = np.nonzero(irr)
        for j, i in zip(jj.tolist(), ii.tolist()):
            sigma = -1.0 if ins[j, i] else 1.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                i2, j2 = i + di, j + dj
                if ins[j2, i2] == ins[j, i]:
                    continue
                if dj == 0:      # horizontal arm of row j
                    q = harm[j][min(i, i2)]
                    arms.append((j, i, 0, 1, q, self.xs[i2] - xq_rows[q], sigma))
                else:            # vertical arm of column i
                    q = varm[i][min(j, j2)]
                    arms.append((j, i, 1, 0, q, self.xs[j2] - yq_cols[q], sigma))
        self.arms = arms

    # ------------------------------------------------------------ controls (R8)
    def _controls(self):
        M = self.M
        seg = np.arange(M)
        _, X1, X2 = self.curve_derivs(seg, np.zeros(M))
        self.ctrl_X1, self.ctrl_X2 = X1, X2
        z = self.pts
        ci = np.floor((z[:, 0] - self.lo) / self.h + 0.5).astype(np.int64)
        cj = np.floor((z[:, 1] - self.lo) / self.h + 0.5).astype(np.int64)
        sx = np.where(z[:, 0] >= self.xs[ci], 1, -1)
        sy = np.where(z[:, 1] >= self.xs[cj], 1, -1)
        offs = np.stack([np.zeros((M, 2), np.int64),
                         np.stack([np.ones(M, np.int64), np.zeros(M, np.int64)], 1),
                         np.stack([-np.ones(M, np.int64), np.zeros(M, np.int64)], 1),
                         np.stack([np.zeros(M, np.int64), np.ones(M, np.int64)], 1),
                         np.stack([np.zeros(M, np.int64), -np.ones(M, np.int64)], 1),
                         np.stack([sx, sy], 1)], axis=1)     # (M, 6, 2) as (di, dj)
        self.ctrl_nodes_i = ci[:, None] + offs[:, :, 0]
        self.ctrl_nodes_j = cj[:, None] + offs[:, :, 1]

    # ------------------------------------------------------------ density on Gamma
    def _surface_derivs(self, dens, seg, L0, L1, L2, X1, X2):
        """value, d/ds and d^2/ds^2 of a control-point function at interpolant points."""
        vals = dens[self._stencil_idx[seg]]
        f = np.sum(L0 * vals, axis=1)
        ft = np.sum(L1 * vals, axis=1) / self.dt
        ftt = np.sum(L2 * vals, axis=1) / self.dt ** 2
        sp = np.sqrt(np.sum(X1 * X1, axis=1))
        spp = np.sum(X1 * X2, axis=1) / sp
        fs = ft / sp
        fss = (ftt - fs * spp) / (sp * sp)
        return f, fs, fss

    def jumps_at_crossings(self, phi=None, psi=None, f_ctrl=None):
        """Cartesian jumps (J, G, H) at every crossing of each axis from the data."""
        out = {}
        for axis in (0, 1):
            cr = self.crossings[axis]
            K = cr["seg"].shape[0]
            L0, L1, L2 = lagrange_basis(cr["tau"])
            X1, X2 = cr["X1"], cr["X2"]
            sp = np.sqrt(np.sum(X1 * X1, axis=1))
            tau = X1 / sp[:, None]
            n = np.stack([tau[:, 1], -tau[:, 0]], axis=1)
            chi = (X1[:, 0] * X2[:, 1] - X1[:, 1] * X2[:, 0]) / sp ** 3
            zero = np.zeros(self.M)
            p, ps, pss = self._surface_derivs(zero if phi is None else phi, cr["seg"], L0, L1, L2, X1, X2)
            q, qs, _ = self._surface_derivs(zero if psi is None else psi, cr["seg"], L0, L1, L2, X1, X2)
            fj, _, _ = self._surface_derivs(zero if f_ctrl is None else f_ctrl, cr["seg"], L0, L1, L2, X1, X2)
            out[axis] = jumps_cartesian(p, ps, pss, q, qs, fj, n, tau, chi, self.kappa2) if K else \
                (np.zeros(0), np.zeros((0, 2)), np.zeros((0, 2, 2)))
        return out

    def jumps_at_controls(self, phi=None, psi=None, f_ctrl=None):
        M = self.M
        seg = np.arange(M)
        L0, L1, L2 = lagrange_basis(np.zeros(M))
        n = self.normals
        tau = np.stack([-n[:, 1], n[:, 0]], axis=1)
        zero = np.zeros(M)
        p, ps, pss = self._surface_derivs(zero if phi is None else phi, seg, L0, L1, L2, self.ctrl_X1, self.ctrl_X2)
        q, qs, _ = self._surface_derivs(zero if psi is None else psi, seg, L0, L1, L2, self.ctrl_X1, self.ctrl_X2)
        fj = zero if f_ctrl is None else np.asarray(f_ctrl, dtype=np.float64)
        return jumps_cartesian(p, ps, pss, q, qs, fj, n, tau, self.curv, self.kappa2)


# --------------------------------------------------------------------------- Alg. 2
def correct_rhs(geom: Geometry2D, jumps_cross, F_grid=None):
    """Corrected right-hand side on the (N+1)^2 grid (R7).  F_grid values at outside
    nodes are ignored (zero extension, Sec. 2.2 table); boundary entries are zero."""
    N, h = geom.N, geom.h
    b = np.zeros((N + 1, N + 1))
    if F_grid is not None:
        b[1:N, 1:N] = np.where(geom.inside[1:N, 1:N], np.asarray(F_grid)[1:N, 1:N], 0.0)
    for (j, i, arm_axis, cr_axis, q, delta, sigma) in geom.arms:
        J, G, H = jumps_cross[cr_axis]
        T = J[q] + delta * G[q, arm_axis] + 0.5 * delta * delta * H[q, arm_axis, arm_axis]
        b[j, i] += sigma * T / (h * h)
    return b


# --------------------------------------------------------------------------- Alg. 4
def sine_matrix(N):
    """S[j-1, l-1] = sin(pi j l / N), j, l = 1..N-1, from the table sin(pi m / N)."""
    table = np.sin(np.pi * np.arange(2 * N, dtype=np.float64) / N)
    jl = np.outer(np.arange(1, N), np.arange(1, N)) % (2 * N)
    return table[jl]


def box_solve_dst(b, N, h, kappa2):
    """Solve (Lap_h - kappa^2) v = b on interior nodes, v = 0 on the box boundary:
    sine transform along y, Thomas solve along x for each y-mode, inverse transform
    (scaled by 2/N).  b and the result are (N+1)^2 grids indexed [j, i]."""
    S = sine_matrix(N)
    n = N - 1
    Bh = S @ b[1:N, 1:N]                                  # [l, i]
    lam = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, N) / (2.0 * N)) ** 2
    off = 1.0 / (h * h)
    diag = -2.0 / (h * h) + lam - kappa2                  # per y-mode l
    cp = np.zeros((n, n))
    dp = np.zeros((n, n))
    cp[:, 0] = off / diag
    dp[:, 0] = Bh[:, 0] / diag
    for i in range(1, n):
        den = diag - off * cp[:, i - 1]
        cp[:, i] = off / den
        dp[:, i] = (Bh[:, i] - off * dp[:, i - 1]) / den
    Vh = np.zeros((n, n))
    Vh[:, n - 1] = dp[:, n - 1]
    for i in range(n - 2, -1, -1):
        Vh[:, i] = dp[:, i] - cp[:, i] * Vh[:, i + 1]
    v = np.zeros((N + 1, N + 1))
    v[1:N, 1:N] = (2.0 / N) * (S @ Vh)
    return v


def box_solve_dense(b, N, h, kappa2):
    """Same system assembled as a dense (N-1)^2 matrix and solved by LU with partial
    pivoting (tiny grids only)."""
    n = N - 1
    A = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            r = j * n + i
            A[r, r] = -4.0 / (h * h) - kappa2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                i2, j2 = i + di, j + dj
                if 0 <= i2 < n and 0 <= j2 < n:
                    A[r, j2 * n + i2] = 1.0 / (h * h)
    v = np.zeros((N + 1, N + 1))
    v[1:N, 1:N] = np.linalg.solve(A, b[1:N, 1:N].reshape(-1)).reshape(n, n)
    return v


# --------------------------------------------------------------------------- Alg. 3
def interpolate_plus(geom: Geometry2D, v, jumps_ctrl):
    """v^+ at every control point (R8), by solving each 6x6 quadratic fit."""
    J, G, H = jumps_ctrl
    z = geom.pts
    I, Jn = geom.ctrl_nodes_i, geom.ctrl_nodes_j                # (M, 6)
    px, py = geom.xs[I], geom.xs[Jn]
    d = np.stack([px - z[:, 0:1], py - z[:, 1:2]], axis=2)      # (M, 6, 2)
    taylor = J[:, None] + np.einsum("md,mkd->mk", G, d) + 0.5 * np.einsum("mkd,mde,mke->mk", d, H, d)
    vals = v[Jn, I] + np.where(geom.inside[Jn, I], 0.0, taylor)
    xi, eta = d[:, :, 0] / geom.h, d[:, :, 1] / geom.h
    V = np.stack([np.ones_like(xi), xi, eta, xi * xi, xi * eta, eta * eta], axis=2)
    coef = np.linalg.solve(V, vals[:, :, None])[:, :, 0]
    return coef[:, 0]


def interpolate_plus_grad(geom: Geometry2D, v, jumps_ctrl):
    """v^+ and grad v^+ at every control point (R8 with R10): the quadratic fitted to the
    same 6 corrected values as interpolate_plus, and its gradient at z.  Returns the
    values (M,) and the gradients (M, 2)."""
    J, G, H = jumps_ctrl
    z = geom.pts
    I, Jn = geom.ctrl_nodes_i, geom.ctrl_nodes_j
    px, py = geom.xs[I], geom.xs[Jn]
    d = np.stack([px - z[:, 0:1], py - z[:, 1:2]], axis=2)
    taylor = J[:, None] + np.einsum("md,mkd->mk", G, d) + 0.5 * np.einsum("mkd,mde,mke->mk", d, H, d)
    vals = v[Jn, I] + np.where(geom.inside[Jn, I], 0.0, taylor)
    xi, eta = d[:, :, 0] / geom.h, d[:, :, 1] / geom.h
    V = np.stack([np.ones_like(xi), xi, eta, xi * xi, xi * eta, eta * eta], axis=2)
    coef = np.linalg.solve(V, vals[:, :, None])[:, :, 0]
    return coef[:, 0], coef[:, 1:3] / geom.h


# ----------------------------------------------------------------- Sec. 2.2 / Alg. 1
def apply_interface(geom: Geometry2D, phi=None, psi=None, f_ctrl=None, F_grid=None,
                    solver=box_solve_dst, return_all=False):
    """Solve the interface problem with [v] = phi, [d_n v] = psi, F = zero-extended
    F_grid and [F] = f on Gamma; return v^+ at the control points (and b, v)."""
    jc = geom.jumps_at_crossings(phi, psi, f_ctrl)
    b = correct_rhs(geom, jc, F_grid)
    v = solver(b, geom.N, geom.h, geom.kappa2)
    out = interpolate_plus(geom, v, geom.jumps_at_controls(phi, psi, f_ctrl))
    if return_all:
        return out, b, v
    return out


def apply_interface_dn(geom: Geometry2D, phi=None, psi=None, f_ctrl=None, F_grid=None,
                       solver=box_solve_dst):
    """d_n v^+ = n . grad v^+ at the control points of the interface problem (the Neumann
    data of Procedure 2, reading R10)."""
    jc = geom.jumps_at_crossings(phi, psi, f_ctrl)
    b = correct_rhs(geom, jc, F_grid)
    v = solver(b, geom.N, geom.h, geom.kappa2)
    _, grad = interpolate_plus_grad(geom, v, geom.jumps_at_controls(phi, psi, f_ctrl))
    return np.sum(grad * geom.normals, axis=1)


def apply_single_layer(geom, psi, **kw):
    """v^+ of the single layer (reading C18: [v] = 0, [d_n v] = psi, F = 0)."""
    return apply_interface(geom, psi=psi, **kw)


def apply_single_layer_dn(geom, psi, **kw):
    """K_N psi = d_n v^+ of the single layer: the operator of the Neumann BIE."""
    return apply_interface_dn(geom, psi=psi, **kw)


def apply_volume_dn(geom, f_grid, f_ctrl, **kw):
    """d_n (Y f)^+ on Gamma."""
    return apply_interface_dn(geom, f_ctrl=f_ctrl, F_grid=f_grid, **kw)


def solve_neumann_bvp(geom: Geometry2D, f_grid, f_ctrl, gn_ctrl, tol=1e-10, m=50,
                      max_restarts=20):
    """Neumann BVP d_n u = g_N on Gamma (Procedures 2-3 with the single-layer density):
    u = V psi + Y f in Omega, so d_n(V psi)^+ = g_N - d_n(Y f)^+ is solved for psi by GMRES,
    then u is the inside-node solution of the interface problem with [d_n v] = psi and
    F = zero-extended f.  Needs kappa > 0 (for kappa = 0 the interior Neumann problem
    determines u only up to a constant and K_N is singular)."""
    ghat = np.asarray(gn_ctrl, dtype=np.float64) - apply_volume_dn(geom, f_grid, f_ctrl)
    psi, info = gmres(lambda p: apply_single_layer_dn(geom, p), ghat, m=m, tol=tol,
                      max_restarts=max_restarts)
    _, _, v = apply_interface(geom, psi=psi, f_ctrl=f_ctrl, F_grid=f_grid, return_all=True)
    return np.where(geom.inside, v, 0.0), psi, info


def apply_double_layer(geom, phi, **kw):
    """K_D phi = (1/2 I + W) phi on Gamma (Sec. 3.3): F = 0, Phi = phi."""
    return apply_interface(geom, phi=phi, **kw)


def apply_volume(geom, f_grid, f_ctrl, **kw):
    """(Y f)^+ on Gamma: F = zero extension of f, Phi = 0 (Sec. 2.2 table)."""
    return apply_interface(geom, f_ctrl=f_ctrl, F_grid=f_grid, **kw)


def combined_grid_solution(geom, phi, f_grid, f_ctrl, solver=box_solve_dst):
    """Grid solution of the interface problem with Phi = phi and F = zero-extended f:
    inside Omega it is u = W phi + Y f (Sec. 2.1)."""
    _, _, v = apply_interface(geom, phi=phi, f_ctrl=f_ctrl, F_grid=f_grid,
                              solver=solver, return_all=True)
    return v


# --------------------------------------------------------------------------- Alg. 5
def gmres(apply, rhs, m=50, tol=1e-10, max_restarts=20, x0=None):
    """Restarted GMRES(m): modified Gram-Schmidt Arnoldi, Givens rotations for the
    least-squares problem, true residual at every restart (Alg. 5).  Stops when
    ||rhs - A x|| <= tol ||rhs||.  Returns x and an info dict."""
    rhs = np.asarray(rhs, dtype=np.float64)
    n = rhs.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(rhs)
    applies = 0
    if bnorm == 0.0:
        return x, dict(iterations=0, applies=0, rel_residual=0.0, converged=True, history=[])
    r = rhs - apply(x) if x0 is not None else rhs.copy()
    applies += x0 is not None
    history = []
    iters = 0
    converged = False
    for _ in range(max_restarts + 1):
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= tol * bnorm:
            converged = True
            break
        V = np.zeros((m + 1, n))
        Hm = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply(V[j])
            applies += 1
            iters += 1
            for i in range(j + 1):
                Hm[i, j] = np.dot(w, V[i])
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            breakdown = np.linalg.norm(w) <= 1e-14 * beta
            if not breakdown:
                V[j + 1] = w / np.linalg.norm(w)
            if abs(g[j + 1]) <= tol * bnorm or breakdown:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(Hm[i, i + 1:k], y[i + 1:k])) / Hm[i, i]
        x = x + V[:k].T @ y
        r = rhs - apply(x)
        applies += 1
    else:
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        converged = beta <= tol * bnorm
    return x, dict(iterations=iters, applies=applies, rel_residual=history[-1],
                   converged=converged, history=history)


def richardson(apply, rhs, gamma=1.0, tol=1e-10, max_iter=500):
    """phi <- phi + gamma (rhs - K phi), gamma in (0, 1] (Sec. 2.1)."""
    x = np.zeros_like(rhs)
    bnorm = np.linalg.norm(rhs)
    for it in range(max_iter):
        r = rhs - apply(x)
        if np.linalg.norm(r) <= tol * bnorm:
            return x, dict(iterations=it, converged=True)
        x = x + gamma * r
    return x, dict(iterations=max_iter, converged=False)


def solve_bvp(geom: Geometry2D, f_grid, f_ctrl, g_ctrl, tol=1e-10, m=50, max_restarts=20,
              method="gmres"):
    """Dirichlet BVP by the BIE 1/2 phi + W phi + Y f = g (Sec. 2.1): g_hat = g - (Yf)^+,
    phi from K_D phi = g_hat, then u = W phi + Y f on inside nodes (0 elsewhere)."""
    yf = apply_volume(geom, f_grid, f_ctrl)
    ghat = np.asarray(g_ctrl, dtype=np.float64) - yf
    K = lambda p: apply_double_layer(geom, p)
    if method == "gmres":
        phi, info = gmres(K, ghat, m=m, tol=tol, max_restarts=max_restarts)
    else:
        phi, info = richardson(K, ghat, tol=tol)
    v = combined_grid_solution(geom, phi, f_grid, f_ctrl)
    u = np.where(geom.inside, v, 0.0)
    return u, phi, info


def error_norms(u_h, u_exact, inside):
    """Max norm and scaled l2 norm of the error over grid nodes inside Omega (Sec. 5)."""
    e = (np.asarray(u_h) - np.asarray(u_exact))[inside]
    return float(np.max(np.abs(e))), float(np.sqrt(np.sum(e * e) / e.size))
