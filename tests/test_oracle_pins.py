"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

P1 box solve vs dense LU and single modes; P2 double layer of a constant (kappa = 0)
is the indicator of Omega; P3 linearity / superposition; P4 closed-form box
double-layer potential on a circle, second order; P5 manufactured BVPs, second order;
P6 GMRES vs a dense solve of the assembled K_D; P7 Richardson (gamma in (0,1], Sec. 2.1)
reaches the same density; P8 90-degree grid symmetry; P9 jump formulas vs an analytic
jump field; P10 the corrected 5-point scheme is exact for piecewise quadratics with a
quadratic jump; P11 corrected interpolation reproduces piecewise quadratics; P13 the Lagrange basis and
the sine matrix on their own (nodal, polynomial reproduction; DST-I orthogonality).
The paper prints no intermediate values for a worked example, so no pin compares
against printed numbers (there are none).
"""
import numpy as np
import pytest

import kfbi_workloads as W
import oracle as O
from closed_forms import circle_double_layer_plus

C0 = (0.0123, -0.0071)   # off-centre circle: no grid node lies on it


def geom_of(iface, N, kappa):
    return O.Geometry2D(iface.pts, iface.normals, iface.curv, N, kappa)


# ------------------------------------------------------------------ P1
@pytest.mark.parametrize("N", [4, 6, 8, 12, 16])
@pytest.mark.parametrize("kappa", [0.0, 1.0, 10.0])
def test_p1_box_solve_matches_dense_lu(N, kappa):
    rng = np.random.default_rng(N * 100 + int(kappa))
    b = np.zeros((N + 1, N + 1))
    b[1:N, 1:N] = rng.standard_normal((N - 1, N - 1))
    h = 2.0 / N
    v1 = O.box_solve_dst(b, N, h, kappa * kappa)
    v2 = O.box_solve_dense(b, N, h, kappa * kappa)
    assert np.max(np.abs(v1 - v2)) <= 1e-13 * np.max(np.abs(v2))
    assert np.all(v1[0] == 0) and np.all(v1[-1] == 0) and np.all(v1[:, 0] == 0) and np.all(v1[:, -1] == 0)


@pytest.mark.parametrize("N,k,l", [(8, 1, 1), (8, 3, 5), (16, 15, 2), (32, 7, 31)])
def test_p1_single_mode_is_eigenvector(N, k, l):
    h = 2.0 / N
    i = np.arange(N + 1)
    b = np.outer(np.sin(np.pi * i * l / N), np.sin(np.pi * i * k / N))   # [j, i]
    lam = lambda m: -(4.0 / h ** 2) * np.sin(np.pi * m / (2 * N)) ** 2
    for kappa2 in (0.0, 4.0):
        v = O.box_solve_dst(b, N, h, kappa2)
        expect = b / (lam(k) + lam(l) - kappa2)
        assert np.max(np.abs(v - expect)) <= 1e-13 * np.max(np.abs(expect))


# ------------------------------------------------------------------ P2
@pytest.mark.parametrize("shape", ["flower", "ellipse"])
@pytest.mark.parametrize("N", [32, 128])
def test_p2_double_layer_of_constant_is_indicator(shape, N):
    iface = W.flower(2 * N) if shape == "flower" else W.ellipse(2 * N)
    g = geom_of(iface, N, 0.0)
    out, b, v = O.apply_interface(g, phi=np.ones(iface.M), return_all=True)
    assert np.max(np.abs(v - g.inside)) <= 1e-12
    assert np.max(np.abs(out - 1.0)) <= 1e-12


# ------------------------------------------------------------------ P3
def test_p3_linearity_and_superposition():
    N, kappa = 64, 1.0
    iface = W.ellipse(2 * N)
    g = geom_of(iface, N, kappa)
    a = W.random_density(iface.M, seed=1)
    c = W.random_density(iface.M, seed=2)
    Ka, Kc = O.apply_double_layer(g, a), O.apply_double_layer(g, c)
    K = O.apply_double_layer(g, 2.5 * a - 0.75 * c)
    assert np.max(np.abs(K - (2.5 * Ka - 0.75 * Kc))) <= 1e-11 * np.max(np.abs(K))
    prob = W.config_helmholtz(N, kappa, "ellipse")
    fg, fc = prob.f_grid(), prob.f_ctrl()
    vw = O.apply_interface(g, phi=a, return_all=True)[2]
    vy = O.apply_interface(g, f_ctrl=fc, F_grid=fg, return_all=True)[2]
    vc = O.combined_grid_solution(g, a, fg, fc)
    assert np.max(np.abs(vc - (vw + vy))) <= 1e-11 * np.max(np.abs(vc))


# ------------------------------------------------------------------ P4
@pytest.mark.parametrize("kappa", [0.0, 1.0, 10.0])
@pytest.mark.parametrize("k", [1, 3])
def test_p4_circle_closed_form_second_order(kappa, k):
    R = 0.5
    errs = []
    for N in (64, 128, 256):
        iface = W.circle(2 * N, R, C0)
        th = 2 * np.pi * np.arange(iface.M) / iface.M
        out = O.apply_double_layer(geom_of(iface, N, kappa), np.cos(k * th))
        errs.append(np.max(np.abs(out - circle_double_layer_plus(k, R, C0, kappa, th))))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[-1] < 1e-4
    assert min(ratios) > 3.0 and np.sqrt(ratios[0] * ratios[1]) > 3.5, (errs, ratios)


def test_p4_constant_density_kappa0_is_exact():
    iface = W.circle(128, 0.5, C0)
    out = O.apply_double_layer(geom_of(iface, 64, 0.0), np.ones(128))
    th = 2 * np.pi * np.arange(128) / 128
    assert np.max(np.abs(out - circle_double_layer_plus(0, 0.5, C0, 0.0, th))) < 1e-12


def _grazing_circle(N, R=0.5):
    """A circle whose top lies 0.04 h^2 / R above the grid row y_j nearest 0.4, centred
    0.4 h to the right of the node x = 0: the row meets it in two points 0.28 h either side
    of the centre, strictly inside the arm (x_i, x_i+1), whose end labels both say
    outside (a grid line grazing the interface)."""
    h = 2.0 / N
    j = int(round(1.4 / h))
    c0 = (-1.0 + (N // 2) * h + 0.4 * h, -1.0 + j * h - R + 0.04 * h * h / R)
    return W.circle(2 * N, R, c0), c0, j


@pytest.mark.parametrize("kappa,k", [(0.0, 1), (0.0, 3), (10.0, 3)])
def test_p4_grazing_row_keeps_second_order(kappa, k):
    """Reading R5 (grazing pairs): on a circle that grazes a grid row at every N, the row's
    two crossings are dropped (no label changes there, no correction) and the closed-form
    double-layer potential (P4) still converges at second order with P4's bounds."""
    R = 0.5
    errs = []
    for N in (64, 128, 256):
        iface, c0, j = _grazing_circle(N, R)
        g = geom_of(iface, N, kappa)
        assert len(g.row_lists[j]) == 2 and not g.inside[j].any()   # the grazing pair
        th = 2 * np.pi * np.arange(iface.M) / iface.M
        out = O.apply_double_layer(g, np.cos(k * th))
        errs.append(np.max(np.abs(out - circle_double_layer_plus(k, R, c0, kappa, th))))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[-1] < 1e-4
    assert min(ratios) > 3.0 and np.sqrt(ratios[0] * ratios[1]) > 3.5, (errs, ratios)


@pytest.mark.parametrize("mistake", ["pair_kept", "one_dropped"])
def test_planted_grazing_slips_are_caught(monkeypatch, mistake):
    """Keeping a grazing pair, or dropping only one of its crossings, leaves crossings that
    match no label change on the row: the geometry is rejected instead of silently
    corrected."""
    import oracle.kfbi2d as K
    iface, _, _ = _grazing_circle(128)
    geom_of(iface, 128, 0.0)                          # the correct rule accepts it
    if mistake == "pair_kept":
        monkeypatch.setattr(K, "GRAZE_CURV", -1.0)
    else:
        orig = K.Geometry2D._match_line

        def drop_one(self, labels, lst, coord, curv):
            order = lst[np.argsort(coord[lst], kind="stable")]
            flips = np.nonzero(labels[1:] != labels[:-1])[0]
            if order.size == flips.size + 2:         # a grazing pair is present: keep one
                for q in range(order.size - 1):
                    a0, a1 = coord[order[q]], coord[order[q + 1]]
                    t = int(np.floor((a0 - self.lo) / self.h))
                    if a1 < self.xs[t + 1] and labels[t] == labels[t + 1]:
                        lst = np.delete(order, q + 1)
                        break
            return orig(self, labels, lst, coord, curv)
        monkeypatch.setattr(K.Geometry2D, "_match_line", drop_one)
    with pytest.raises(O.GeometryError):
        geom_of(iface, 128, 0.0)


# ------------------------------------------------------------------ P5
@pytest.mark.parametrize("case", ["poisson_flower", "helmholtz_ellipse"])
def test_p5_manufactured_bvp_second_order(case):
    errs = []
    for N in (64, 128, 256):
        prob = W.config_poisson_flower(N, 2 * N) if case == "poisson_flower" else \
            W.config_helmholtz(N, 10.0, "ellipse")
        g = geom_of(prob.iface, N, prob.kappa)
        u, phi, info = O.solve_bvp(g, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-11)
        assert info["converged"]
        errs.append(O.error_norms(u, prob.u_grid(), g.inside)[1])
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert min(ratios) > 3.0 and np.sqrt(ratios[0] * ratios[1]) > 3.5, (errs, ratios)


# ------------------------------------------------------------------ P6, P7
def _tiny():
    N, M = 16, 32
    iface = W.circle(M, 0.45, C0)
    prob = W.Problem(iface, N, 1.0, W.manufactured_exp_sin2y(1.0))
    return prob, geom_of(iface, N, 1.0)


def test_p6_gmres_matches_dense_solve():
    prob, g = _tiny()
    M = prob.iface.M
    K = np.stack([O.apply_double_layer(g, e) for e in np.eye(M)], axis=1)
    ghat = prob.g_ctrl() - O.apply_volume(g, prob.f_grid(), prob.f_ctrl())
    phi_lu = np.linalg.solve(K, ghat)
    phi_g, info = O.gmres(lambda p: O.apply_double_layer(g, p), ghat, m=50, tol=1e-14)
    assert np.max(np.abs(phi_g - phi_lu)) <= 1e-12 * np.max(np.abs(phi_lu))
    # a restart length below the Krylov dimension still converges to the same density
    phi_r, info_r = O.gmres(lambda p: O.apply_double_layer(g, p), ghat, m=5, tol=1e-13, max_restarts=50)
    assert info_r["converged"] and np.max(np.abs(phi_r - phi_lu)) <= 1e-11 * np.max(np.abs(phi_lu))


def test_p7_richardson_reaches_gmres_density():
    prob, g = _tiny()
    ghat = prob.g_ctrl() - O.apply_volume(g, prob.f_grid(), prob.f_ctrl())
    Kf = lambda p: O.apply_double_layer(g, p)
    phi_g, _ = O.gmres(Kf, ghat, tol=1e-12)
    tol = 1e-11
    phi_r, info = O.richardson(Kf, ghat, gamma=1.0, tol=tol)
    assert info["converged"]
    assert np.max(np.abs(phi_r - phi_g)) <= 10 * tol * np.max(np.abs(phi_g))


# ------------------------------------------------------------------ P8
def test_p8_quarter_turn_symmetry():
    N, M = 64, 128
    iface = W.circle(M, 0.4567, (0.0, 0.0))
    g = geom_of(iface, N, 2.0)
    th = 2 * np.pi * np.arange(M) / M
    out = O.apply_double_layer(g, np.cos(4 * th) + 0.3)
    assert np.max(np.abs(np.roll(out, -M // 4) - out)) <= 1e-12 * np.max(np.abs(out))
    # grid field rotates with it: v(x, y) = v(-y, x)
    _, _, v = O.apply_interface(g, phi=np.cos(4 * th) + 0.3, return_all=True)
    assert np.max(np.abs(np.rot90(v) - v)) <= 1e-12 * np.max(np.abs(v))


# ------------------------------------------------------------------ P9
def test_p9_jump_formulas_match_analytic_jump_field():
    """Take a smooth J(x, y); feed Phi = J|Gamma, psi = d_n J, [F] = Lap J - k^2 J; the
    Cartesian jumps at every crossing must reproduce J, grad J and Hess J."""
    kappa = 1.5
    J = lambda x, y: np.exp(0.7 * x) * np.cos(1.3 * y) + x * y * y
    Jx = lambda x, y: 0.7 * np.exp(0.7 * x) * np.cos(1.3 * y) + y * y
    Jy = lambda x, y: -1.3 * np.exp(0.7 * x) * np.sin(1.3 * y) + 2 * x * y
    Jxx = lambda x, y: 0.49 * np.exp(0.7 * x) * np.cos(1.3 * y)
    Jxy = lambda x, y: -0.91 * np.exp(0.7 * x) * np.sin(1.3 * y) + 2 * y
    Jyy = lambda x, y: -1.69 * np.exp(0.7 * x) * np.cos(1.3 * y) + 2 * x
    errs = []
    for N in (64, 128, 256):
        iface = W.flower(2 * N)
        g = geom_of(iface, N, kappa)
        p = iface.pts
        phi = J(p[:, 0], p[:, 1])
        psi = Jx(p[:, 0], p[:, 1]) * iface.normals[:, 0] + Jy(p[:, 0], p[:, 1]) * iface.normals[:, 1]
        Fj = Jxx(p[:, 0], p[:, 1]) + Jyy(p[:, 0], p[:, 1]) - kappa ** 2 * phi
        jc = g.jumps_at_crossings(phi, psi, Fj)
        e = 0.0
        for axis in (0, 1):
            Jc, G, H = jc[axis]
            q = g.crossings[axis]["pos"]
            x, y = q[:, 0], q[:, 1]
            e = max(e, np.max(np.abs(Jc - J(x, y))), np.max(np.abs(G[:, 0] - Jx(x, y))),
                    np.max(np.abs(G[:, 1] - Jy(x, y))), np.max(np.abs(H[:, 0, 0] - Jxx(x, y))),
                    np.max(np.abs(H[:, 0, 1] - Jxy(x, y))), np.max(np.abs(H[:, 1, 1] - Jyy(x, y))))
        jz, Gz, Hz = g.jumps_at_controls(phi, psi, Fj)
        x, y = p[:, 0], p[:, 1]
        e = max(e, np.max(np.abs(Gz[:, 0] - Jx(x, y))), np.max(np.abs(Hz[:, 1, 1] - Jyy(x, y))),
                np.max(np.abs(Hz[:, 0, 1] - Jxy(x, y))))
        errs.append(e)
    # second derivatives of the degree-5 interpolant converge like dt^4
    assert errs[2] < 1e-2 and errs[0] / errs[1] > 8.0 and errs[1] / errs[2] > 8.0, errs


# ------------------------------------------------------------------ P10, P11
def _piecewise_quadratic(g):
    """v+ and v- quadratics, J = v+ - v- quadratic, exact jumps at crossings/controls."""
    vp = lambda x, y: 1.0 + 0.3 * x - 0.2 * y + 0.5 * x * x + 0.25 * x * y - 0.4 * y * y
    Jf = lambda x, y: 0.7 - 0.1 * x + 0.6 * y + 0.2 * x * x - 0.3 * x * y + 0.15 * y * y
    grad = lambda x, y: np.stack([-0.1 + 0.4 * x - 0.3 * y, 0.6 - 0.3 * x + 0.3 * y], 1)
    Hc = np.array([[0.4, -0.3], [-0.3, 0.3]])

    def jumps(pts):
        x, y = pts[:, 0], pts[:, 1]
        return Jf(x, y), grad(x, y), np.broadcast_to(Hc, (x.size, 2, 2)).copy()
    vm = lambda x, y: vp(x, y) - Jf(x, y)
    return vp, vm, jumps


def test_p10_correction_exact_for_piecewise_quadratics():
    N, kappa = 48, 2.0
    iface = W.ellipse(2 * N)
    g = geom_of(iface, N, kappa)
    vp, vm, jumps = _piecewise_quadratic(g)
    _, X, Y = W.grid_nodes(N)
    v = np.where(g.inside, vp(X, Y), vm(X, Y))
    jc = {a: jumps(g.crossings[a]["pos"]) for a in (0, 1)}
    b = O.correct_rhs(g, jc)                                     # corrections only (F = 0)
    lap_p = 0.5 * 2 - 0.4 * 2                                    # Lap v+ (constant)
    lap_m = lap_p - (0.2 * 2 + 0.15 * 2)                         # Lap v-
    F = np.where(g.inside, lap_p - kappa ** 2 * vp(X, Y), lap_m - kappa ** 2 * vm(X, Y))
    h = g.h
    Lv = (v[1:-1, 2:] + v[1:-1, :-2] + v[2:, 1:-1] + v[:-2, 1:-1] - 4 * v[1:-1, 1:-1]) / h ** 2 \
        - kappa ** 2 * v[1:-1, 1:-1]
    resid = Lv - (b[1:-1, 1:-1] + F[1:-1, 1:-1])
    assert np.max(np.abs(resid)) <= 1e-8 * (1.0 / h ** 2), np.max(np.abs(resid))


def test_p11_interpolation_reproduces_piecewise_quadratics():
    N = 64
    iface = W.flower(2 * N)
    g = geom_of(iface, N, 0.0)
    vp, vm, jumps = _piecewise_quadratic(g)
    _, X, Y = W.grid_nodes(N)
    v = np.where(g.inside, vp(X, Y), vm(X, Y))
    out = O.interpolate_plus(g, v, jumps(g.pts))
    assert np.max(np.abs(out - vp(g.pts[:, 0], g.pts[:, 1]))) <= 1e-12


# ------------------------------------------------------------------ planted mistakes
def _circle_error(K, kappa, k=3, N=128, R=0.5):
    iface = W.circle(2 * N, R, C0)
    th = 2 * np.pi * np.arange(iface.M) / iface.M
    out = K.apply_double_layer(geom_of(iface, N, kappa), np.cos(k * th))
    return np.max(np.abs(out - circle_double_layer_plus(k, R, C0, kappa, th)))


@pytest.mark.parametrize("mistake", ["curvature_sign", "dropped_kappa_term", "sigma_sign"])
def test_planted_mistakes_break_the_closed_form_pin(monkeypatch, mistake):
    """A plausible slip in the jump formulas (R6) or the correction sign (R7) must make
    the closed-form pin P4 at least 5x worse than the correct oracle."""
    import oracle.kfbi2d as K
    kappa, k = (1.0, 1) if mistake == "curvature_sign" else (10.0, 3)
    good = _circle_error(K, kappa, k)
    orig = K.jumps_cartesian
    if mistake == "curvature_sign":
        monkeypatch.setattr(K, "jumps_cartesian", lambda p, ps, pss, q, qs, F, n, t, chi, k2:
                            orig(p, ps, pss, q, qs, F, n, t, -chi, k2))
    elif mistake == "dropped_kappa_term":
        monkeypatch.setattr(K, "jumps_cartesian", lambda p, ps, pss, q, qs, F, n, t, chi, k2:
                            orig(p, ps, pss, q, qs, F, n, t, chi, 0.0))
    else:
        orig_arms = K.Geometry2D._arms

        def flipped(self):
            orig_arms(self)
            self.arms = [(j, i, a, c, q, d, -s) for (j, i, a, c, q, d, s) in self.arms]
        monkeypatch.setattr(K.Geometry2D, "_arms", flipped)
    assert _circle_error(K, kappa, k) > 5 * good


def test_planted_transposed_grid_is_caught():
    """Handing the interpolation a transposed grid ([i, j] for [j, i]) breaks P11."""
    N = 64
    iface = W.flower(2 * N)
    g = geom_of(iface, N, 0.0)
    vp, vm, jumps = _piecewise_quadratic(g)
    _, X, Y = W.grid_nodes(N)
    v = np.where(g.inside, vp(X, Y), vm(X, Y))
    out = O.interpolate_plus(g, v.T, jumps(g.pts))
    assert np.max(np.abs(out - vp(g.pts[:, 0], g.pts[:, 1]))) > 1e-3


# ------------------------------------------------------------------ geometry errors
def test_geometry_error_near_box_boundary():
    iface = W.circle(64, 0.95, (0.0, 0.0))
    with pytest.raises(O.GeometryError):
        geom_of(iface, 32, 0.0)


def test_geometry_error_under_resolved():
    iface = W.flower(64, r0=0.5, a=0.3, k=12)     # petals thinner than a cell
    with pytest.raises(O.GeometryError):
        geom_of(iface, 16, 0.0)


def test_node_on_interface_tie_is_consistent():
    """The flower at N = 128 passes through grid nodes (0, +-0.5): labels still come out
    consistent (designed tie case)."""
    prob = W.config_poisson_flower(128, 256)
    g = geom_of(prob.iface, 128, 0.0)
    out = O.apply_double_layer(g, np.ones(256))
    assert np.max(np.abs(out - 1.0)) < 1e-12


# ------------------------------------------------------------------ error norms (Sec. 5)
def test_error_norms_by_hand():
    """Max norm and l2 norm over the nodes inside Omega (reading C14: N in the l2 norm is the
    number of nodes inside Omega): a unit error at one inside node of 9 gives 1 and 1/3;
    errors at outside nodes are ignored."""
    inside = np.zeros((5, 5), dtype=bool)
    inside[1:4, 1:4] = True
    u = np.zeros((5, 5))
    u[2, 2] = 1.0
    u[0, 0] = 7.0                                   # outside Omega: not counted
    e_inf, e_l2 = O.error_norms(u, np.zeros((5, 5)), inside)
    assert e_inf == 1.0
    assert e_l2 == pytest.approx(1.0 / 3.0, rel=1e-15)
    u[1, 3] = -2.0                                  # two inside errors: sqrt((1 + 4) / 9)
    e_inf, e_l2 = O.error_norms(u, np.zeros((5, 5)), inside)
    assert e_inf == 2.0 and e_l2 == pytest.approx(np.sqrt(5.0 / 9.0), rel=1e-15)


# ------------------------------------------------------------------ single layer, Neumann BVP
@pytest.mark.parametrize("kappa,k", [(0.0, 1), (0.0, 3), (1.0, 2), (10.0, 3)])
def test_p4_single_layer_circle_closed_form(kappa, k):
    """Reading C18 (single layer by the interface problem [v] = 0, [d_n v] = psi) and R10
    (Neumann data from the gradient of the interpolating quadratic) against the closed-form
    box single-layer potential of cos(k theta) on a circle: v^+ converges at second order,
    d_n v^+ at order 1.5 or better."""
    from closed_forms import circle_single_layer_plus
    R = 0.5
    ev, ed = [], []
    for N in (64, 128, 256):
        iface = W.circle(2 * N, R, C0)
        g = geom_of(iface, N, kappa)
        th = 2 * np.pi * np.arange(iface.M) / iface.M
        psi = np.cos(k * th)
        v_ex, dn_ex = circle_single_layer_plus(k, R, C0, kappa, th)
        ev.append(np.max(np.abs(O.apply_single_layer(g, psi) - v_ex)))
        ed.append(np.max(np.abs(O.apply_single_layer_dn(g, psi) - dn_ex)))
    rv = [ev[i] / ev[i + 1] for i in range(2)]
    rd = [ed[i] / ed[i + 1] for i in range(2)]
    assert ev[-1] < 2e-5 and min(rv) > 2.2 and np.sqrt(rv[0] * rv[1]) > 3.5, (ev, rv)
    assert ed[-1] < 1e-3 and min(rd) > 2.8, (ed, rd)


def test_p11_gradient_reproduces_piecewise_quadratics():
    """R10: the gradient of the corrected interpolating quadratic at z is grad v^+ exactly
    for quadratic v+ and v- with their exact jumps."""
    N = 64
    iface = W.flower(2 * N)
    g = geom_of(iface, N, 0.0)
    vp, vm, jumps = _piecewise_quadratic(g)
    _, X, Y = W.grid_nodes(N)
    v = np.where(g.inside, vp(X, Y), vm(X, Y))
    val, grad = O.interpolate_plus_grad(g, v, jumps(g.pts))
    x, y = g.pts[:, 0], g.pts[:, 1]
    assert np.max(np.abs(val - vp(x, y))) <= 1e-12
    assert np.max(np.abs(grad[:, 0] - (0.3 + x + 0.25 * y))) <= 1e-10
    assert np.max(np.abs(grad[:, 1] - (-0.2 + 0.25 * x - 0.8 * y))) <= 1e-10


@pytest.mark.parametrize("shape,kappa", [("ellipse", 1.0), ("flower", 10.0)])
def test_p5_neumann_bvp_second_order(shape, kappa):
    """Neumann BVP (Procedures 2-3 with the single-layer density): u = exp(x) sin(2y),
    d_n u given at the control points; max and l2 errors of u fall about 4x per doubling."""
    errs = []
    for N in (64, 128, 256):
        prob = W.config_helmholtz(N, kappa, shape)
        g = geom_of(prob.iface, N, kappa)
        u, psi, info = O.solve_neumann_bvp(g, prob.f_grid(), prob.f_ctrl(), prob.gn_ctrl(), tol=1e-10)
        assert info["converged"]
        errs.append(O.error_norms(u, prob.u_grid(), g.inside))
    for q in (0, 1):
        r = [errs[i][q] / errs[i + 1][q] for i in range(2)]
        assert min(r) > 3.0 and np.sqrt(r[0] * r[1]) > 3.5, (errs, r)


def test_p6_neumann_gmres_matches_dense_solve():
    """GMRES on the single-layer Neumann operator K_N against LU of the assembled K_N."""
    N, M, kappa = 16, 32, 2.0
    prob = W.Problem(W.circle(M, 0.45, C0), N, kappa, W.manufactured_exp_sin2y(kappa))
    g = geom_of(prob.iface, N, kappa)
    K = np.stack([O.apply_single_layer_dn(g, e) for e in np.eye(M)], axis=1)
    ghat = prob.gn_ctrl() - O.apply_volume_dn(g, prob.f_grid(), prob.f_ctrl())
    psi_lu = np.linalg.solve(K, ghat)
    _, psi, info = O.solve_neumann_bvp(g, prob.f_grid(), prob.f_ctrl(), prob.gn_ctrl(), tol=1e-13)
    assert info["converged"] and np.max(np.abs(psi - psi_lu)) <= 1e-11 * np.max(np.abs(psi_lu))


def test_planted_normal_sign_breaks_the_single_layer_pin(monkeypatch):
    """Extracting the Neumann data along the inward normal fails the closed-form d_n pin."""
    from closed_forms import circle_single_layer_plus
    import oracle.kfbi2d as K
    N, R, k, kappa = 128, 0.5, 2, 1.0
    iface = W.circle(2 * N, R, C0)
    th = 2 * np.pi * np.arange(iface.M) / iface.M
    _, dn_ex = circle_single_layer_plus(k, R, C0, kappa, th)
    good = np.max(np.abs(K.apply_single_layer_dn(geom_of(iface, N, kappa), np.cos(k * th)) - dn_ex))
    orig = K.interpolate_plus_grad
    monkeypatch.setattr(K, "interpolate_plus_grad", lambda g, v, j: (lambda r: (r[0], -r[1]))(orig(g, v, j)))
    bad = np.max(np.abs(K.apply_single_layer_dn(geom_of(iface, N, kappa), np.cos(k * th)) - dn_ex))
    assert bad > 50 * good


# ------------------------------------------------------------------ P13 helpers
def test_p13_lagrange_basis_reproduces_quintics_and_their_derivatives():
    """The six basis polynomials of the degree-5 interpolant (R3) on the local nodes
    tau = -2..3: nodal (L_r(tau_s) = delta_rs), and any polynomial of degree <= 5 is
    reproduced with its first and second tau-derivatives from its node values."""
    nodes = np.arange(-2.0, 4.0)
    L0, _, _ = O.lagrange_basis(nodes)
    assert np.max(np.abs(L0 - np.eye(6))) <= 1e-13
    p = lambda t: 3 * t**5 - 2 * t**4 + t**3 - 5 * t + 0.25
    dp = lambda t: 15 * t**4 - 8 * t**3 + 3 * t**2 - 5
    d2p = lambda t: 60 * t**3 - 24 * t**2 + 6 * t
    tau = np.linspace(0.0, 1.0, 17)
    L0, L1, L2 = O.lagrange_basis(tau)
    pv = p(nodes)
    assert np.max(np.abs(L0 @ pv - p(tau))) <= 1e-11
    assert np.max(np.abs(L1 @ pv - dp(tau))) <= 1e-10
    assert np.max(np.abs(L2 @ pv - d2p(tau))) <= 1e-9
    # a degree-6 term is not reproduced (the interpolant really is of degree 5)
    assert np.max(np.abs(L0 @ nodes**6 - tau**6)) > 1e-3


@pytest.mark.parametrize("N", [2, 3, 8, 12, 17])
def test_p13_sine_matrix_is_the_orthogonal_dst1(N):
    """DST-I: S[j-1, l-1] = sin(pi j l / N) is symmetric with S S = (N / 2) I, and its
    first row is sin(pi l / N)."""
    from oracle.kfbi2d import sine_matrix
    S = sine_matrix(N)
    assert S.shape == (N - 1, N - 1)
    assert np.array_equal(S, S.T)
    assert np.max(np.abs(S @ S - 0.5 * N * np.eye(N - 1))) <= 1e-13 * N
    assert np.max(np.abs(S[0] - np.sin(np.pi * np.arange(1, N) / N))) <= 1e-15
