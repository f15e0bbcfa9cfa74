"""Pins of the 3-D FP64 oracle (oracle/kfbi3d.py) to facts outside itself.

P1   box solve: sine-transform/Thomas solver against dense LU on tiny grids, and the
     discrete eigen-pairs of the 7-point operator (textbook);
P2   constant density, kappa = 0: the grid solution is the indicator of Omega and
     K_D 1 = 1 at every point, to round-off (the correction is exact for constants);
P3   linearity of the apply;
P4   interface solver against a two-sided manufactured field (v- vanishing on the box,
     v+ arbitrary, [v], [d_n v] and [F] from the closed forms): second order on the grid
     and at the points, with psi != 0 so every curvature term of the jumps is exercised;
P5   Dirichlet BVP on a sphere and an ellipsoid: second-order convergence;
P6   GMRES against a dense LU solve of the assembled discrete BIE on a tiny grid;
P9   least-squares surface derivatives of a linear function on a sphere against the
     closed forms grad_G = (I - n n^T) a, Hess_G = -(a . n)/R I;
P10  local truncation: quadratic v+ and v- with their exact jumps make the corrected
     7-point system exact at every interior node;
P11  interpolation reproduces v+ exactly for quadratic v+ and v-;
P4s  the double-layer apply (reading S10 included) converges at second order to the
     closed-form box double-layer potential of a harmonic-polynomial density on a sphere
     (free-space Y_l field with coefficients (l+1)/(2l+1) inside, -l/(2l+1) outside, or
     the modified spherical Bessel pair for kappa > 0, plus the cube's double sine series);
S10  spectrum of the assembled discrete K_D on a sphere: the continuous operator 1/2 I + W
     has its spectrum in (1/2, 1] accumulating only at 1/2 (W compact), so every
     eigenvalue must have real part in [0.4, 1.05] and most must lie near 1/2;
P13  the shape-operator unpacking (its quadratic form) and the tangent frame
     (orthonormal, right-handed);
plus planted mistakes that these pins must catch, and the geometry errors."""
import numpy as np
import pytest

import kfbi_workloads.surfaces3d as S3
from closed_forms import sphere_double_layer_plus
from oracle import GeometryError
from oracle import kfbi3d as O3


def geom(surface, N, kappa=0.0):
    I = S3.intersect(surface, N)
    return O3.Geometry3D(I.pts, I.normals, I.shape, N, kappa), I


# ------------------------------------------------------------------------------- P1
@pytest.mark.parametrize("N", [4, 6, 8])
@pytest.mark.parametrize("kappa", [0.0, 1.0, 10.0])
def test_p1_box_solve_matches_dense_lu(N, kappa):
    rng = np.random.default_rng(100 + N)
    b = np.zeros((N + 1,) * 3)
    b[1:N, 1:N, 1:N] = rng.standard_normal((N - 1,) * 3)
    h = 2.0 / N
    a = O3.box_solve_dst(b, N, h, kappa * kappa)
    d = O3.box_solve_dense(b, N, h, kappa * kappa)
    assert np.abs(a - d).max() <= 1e-13 * np.abs(d).max()


def test_p1_single_mode_eigenpair():
    N, h, k2 = 12, 2.0 / 12, 4.0
    idx = np.arange(N + 1)
    l, m, p = 3, 7, 10
    mode = (np.sin(np.pi * p * idx / N)[None, None, :] * np.sin(np.pi * m * idx / N)[None, :, None]
            * np.sin(np.pi * l * idx / N)[:, None, None])
    lam = lambda q: -(4.0 / (h * h)) * np.sin(np.pi * q / (2.0 * N)) ** 2
    v = O3.box_solve_dst(mode, N, h, k2)
    assert np.abs(v - mode / (lam(l) + lam(m) + lam(p) - k2)).max() <= 1e-14


# ------------------------------------------------------------------------------- P2
@pytest.mark.parametrize("shape,N", [("sphere", 16), ("ellipsoid", 24)])
def test_p2_constant_density_gives_indicator(shape, N):
    g, _ = geom(S3.sphere() if shape == "sphere" else S3.ellipsoid(), N)
    out, b, v = O3.apply_double_layer(g, np.ones(g.P), return_all=True)
    assert np.abs(v - g.inside).max() <= 1e-12
    assert np.abs(out - 1.0).max() <= 1e-12


# ------------------------------------------------------------------------------- P3
def test_p3_linearity():
    g, I = geom(S3.ellipsoid(), 16, kappa=1.0)
    a, b = S3.random_density3(g.P, I.pts, seed=1), S3.random_density3(g.P, I.pts, seed=2)
    lhs = O3.apply_double_layer(g, 2.0 * a - 3.0 * b)
    rhs = 2.0 * O3.apply_double_layer(g, a) - 3.0 * O3.apply_double_layer(g, b)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


# ------------------------------------------------------------------------------- P4
def _two_sided(kappa):
    vm = lambda x, y, z: (np.sin(np.pi * (x + 1) / 2) * np.sin(np.pi * (y + 1) / 2)
                          * np.sin(np.pi * (z + 1) / 2))
    gm = lambda x, y, z: (np.pi / 2) * np.stack([
        np.cos(np.pi * (x + 1) / 2) * np.sin(np.pi * (y + 1) / 2) * np.sin(np.pi * (z + 1) / 2),
        np.sin(np.pi * (x + 1) / 2) * np.cos(np.pi * (y + 1) / 2) * np.sin(np.pi * (z + 1) / 2),
        np.sin(np.pi * (x + 1) / 2) * np.sin(np.pi * (y + 1) / 2) * np.cos(np.pi * (z + 1) / 2)], -1)
    Fm = lambda x, y, z: (-3 * (np.pi / 2) ** 2 - kappa ** 2) * vm(x, y, z)
    vp = lambda x, y, z: np.exp(0.5 * x) * np.cos(y) + z * z
    gp = lambda x, y, z: np.stack([0.5 * np.exp(0.5 * x) * np.cos(y),
                                   -np.exp(0.5 * x) * np.sin(y), 2 * z], -1)
    Fp = lambda x, y, z: -0.75 * np.exp(0.5 * x) * np.cos(y) + 2.0 - kappa ** 2 * vp(x, y, z)
    return vm, gm, Fm, vp, gp, Fp


def _interface_errors(N, kappa, jump_fn=None):
    vm, gm, Fm, vp, gp, Fp = _two_sided(kappa)
    g, I = geom(S3.ellipsoid(), N, kappa)
    x, y, z = I.pts.T
    phi = vp(x, y, z) - vm(x, y, z)
    psi = np.sum((gp(x, y, z) - gm(x, y, z)) * I.normals, axis=1)
    jm = g.jumps(phi, psi, Fp(x, y, z) - Fm(x, y, z)) if jump_fn is None else jump_fn(g, phi, psi)
    _, X, Y, Z = S3.grid_nodes3(N)
    b = O3.correct_rhs(g, jm, None)
    b[1:N, 1:N, 1:N] += np.where(g.inside, Fp(X, Y, Z), Fm(X, Y, Z))[1:N, 1:N, 1:N]
    v = O3.box_solve_dst(b, N, g.h, g.kappa2)
    exact = np.where(g.inside, vp(X, Y, Z), vm(X, Y, Z))
    e_grid = np.abs(v - exact)[1:N, 1:N, 1:N].max()
    e_pts = np.abs(O3.interpolate_plus(g, v, jm) - vp(x, y, z)).max()
    return e_grid, e_pts


@pytest.mark.parametrize("kappa", [0.0, 2.0])
def test_p4_interface_solver_second_order(kappa):
    e16 = _interface_errors(16, kappa)
    e32 = _interface_errors(32, kappa)
    assert e16[0] / e32[0] > 3.0 and e16[1] / e32[1] > 3.0, (e16, e32)
    assert e32[0] < 2e-3 and e32[1] < 3e-3


# ------------------------------------------------------------------------------- P5
@pytest.mark.parametrize("shape", ["sphere", "ellipsoid"])
def test_p5_dirichlet_bvp_second_order(shape):
    errs, iters = [], []
    for N in (24, 48):
        surf = S3.sphere() if shape == "sphere" else S3.ellipsoid()
        g, I = geom(surf, N)
        prob = S3.Problem3D(I, 0.0, S3.manufactured_sin3(0.0))
        u, phi, info = O3.solve_bvp(g, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-10)
        assert info["converged"]
        errs.append(np.abs(u - prob.u_grid())[g.inside].max())
        iters.append(info["iterations"])
    assert errs[0] / errs[1] > 3.5, errs
    assert max(iters) <= 30, iters          # a second-kind equation: few iterations


# ------------------------------------------------------------------------------- P6
def test_p6_gmres_matches_dense_solve():
    g, I = geom(S3.sphere(), 12, kappa=1.0)
    P = g.P
    K = np.stack([O3.apply_double_layer(g, e) for e in np.eye(P)], axis=1)
    rhs = S3.random_density3(P, I.pts, seed=5)
    phi, info = O3.gmres(lambda p: O3.apply_double_layer(g, p), rhs, tol=1e-14, m=50)
    ref = np.linalg.solve(K, rhs)
    assert np.abs(phi - ref).max() <= 1e-11 * np.abs(ref).max()


# ------------------------------------------------------------------------------- P9
def test_p9_surface_derivatives_on_sphere():
    a = np.array([0.3, -1.1, 0.7])
    errs = []
    for N in (16, 32):
        g, I = geom(S3.sphere(), N)
        R = 0.5
        f, grad, H = g.surface_derivs(I.pts @ a)
        n = I.normals
        g_exact = a[None, :] - (n @ a)[:, None] * n
        T = np.stack([g.t1, g.t2], axis=1)
        g_t = np.einsum("pai,pi->pa", T, g_exact)
        H_exact = -(n @ a)[:, None, None] / R * np.eye(2)[None]
        assert np.abs(f - I.pts @ a).max() <= 1e-2 * g.h ** 2 * 100
        errs.append((np.abs(grad - g_t).max(), np.abs(H - H_exact).max()))
    assert errs[1][0] < 1e-3 and errs[0][0] / errs[1][0] > 3.0, errs
    assert errs[1][1] < 0.1 and errs[0][1] / errs[1][1] > 3.0, errs


# ------------------------------------------------------------------------------ P10/P11
def _quadratic_pair(seed, kappa):
    rng = np.random.default_rng(seed)
    cp, cm = rng.standard_normal(10), rng.standard_normal(10)

    def q(c):
        f = lambda x, y, z: (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y
                             + c[6] * z * z + c[7] * x * y + c[8] * x * z + c[9] * y * z)
        g = lambda x, y, z: np.stack([c[1] + 2 * c[4] * x + c[7] * y + c[8] * z,
                                      c[2] + 2 * c[5] * y + c[7] * x + c[9] * z,
                                      c[3] + 2 * c[6] * z + c[8] * x + c[9] * y], -1)
        H = np.array([[2 * c[4], c[7], c[8]], [c[7], 2 * c[5], c[9]], [c[8], c[9], 2 * c[6]]])
        lap = 2 * (c[4] + c[5] + c[6])
        F = lambda x, y, z: lap - kappa * kappa * f(x, y, z)
        return f, g, H, F
    return q(cp), q(cm)


def _exact_jumps(I, plus, minus):
    x, y, z = I.pts.T
    J = plus[0](x, y, z) - minus[0](x, y, z)
    G = plus[1](x, y, z) - minus[1](x, y, z)
    H = np.broadcast_to(plus[2] - minus[2], (I.P, 3, 3)).copy()
    return J, G, H


@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_p10_corrected_system_exact_for_quadratics(kappa):
    N = 16
    g, I = geom(S3.ellipsoid(), N, kappa)
    plus, minus = _quadratic_pair(7, kappa)
    _, X, Y, Z = S3.grid_nodes3(N)
    v = np.where(g.inside, plus[0](X, Y, Z), minus[0](X, Y, Z))
    b = O3.correct_rhs(g, _exact_jumps(I, plus, minus), None)
    b += np.where(g.inside, plus[3](X, Y, Z), minus[3](X, Y, Z))
    h = g.h
    c = v[1:N, 1:N, 1:N]
    Lv = ((v[2:, 1:N, 1:N] + v[:-2, 1:N, 1:N] + v[1:N, 2:, 1:N] + v[1:N, :-2, 1:N]
           + v[1:N, 1:N, 2:] + v[1:N, 1:N, :-2] - 6 * c) / (h * h) - kappa * kappa * c)
    assert np.abs(Lv - b[1:N, 1:N, 1:N]).max() <= 1e-9 * np.abs(b).max()


def test_p11_interpolation_reproduces_quadratics():
    N = 16
    g, I = geom(S3.ellipsoid(), N)
    plus, minus = _quadratic_pair(9, 0.0)
    _, X, Y, Z = S3.grid_nodes3(N)
    v = np.where(g.inside, plus[0](X, Y, Z), minus[0](X, Y, Z))
    out = O3.interpolate_plus(g, v, _exact_jumps(I, plus, minus))
    x, y, z = I.pts.T
    assert np.abs(out - plus[0](x, y, z)).max() <= 1e-12 * np.abs(out).max()


# ---------------------------------------------------------------------- planted mistakes
def test_planted_curvature_sign_fails_p4(monkeypatch):
    real = O3.jumps_from_surface

    def wrong(phi, g_phi, H_phi, psi, g_psi, n, t1, t2, S, Fj, kappa2):
        return real(phi, g_phi, H_phi, psi, g_psi, n, t1, t2, -S, Fj, kappa2)
    monkeypatch.setattr(O3, "jumps_from_surface", wrong)
    e16 = _interface_errors(16, 0.0)
    e32 = _interface_errors(32, 0.0)
    assert not (e16[0] / e32[0] > 3.0 and e16[1] / e32[1] > 3.0)


def test_planted_delta_sign_fails_p10():
    N = 16
    g, I = geom(S3.ellipsoid(), N)
    plus, minus = _quadratic_pair(7, 0.0)
    g.arm_delta = -g.arm_delta
    _, X, Y, Z = S3.grid_nodes3(N)
    v = np.where(g.inside, plus[0](X, Y, Z), minus[0](X, Y, Z))
    b = O3.correct_rhs(g, _exact_jumps(I, plus, minus), None)
    b += np.where(g.inside, plus[3](X, Y, Z), minus[3](X, Y, Z))
    h = g.h
    c = v[1:N, 1:N, 1:N]
    Lv = (v[2:, 1:N, 1:N] + v[:-2, 1:N, 1:N] + v[1:N, 2:, 1:N] + v[1:N, :-2, 1:N]
          + v[1:N, 1:N, 2:] + v[1:N, 1:N, :-2] - 6 * c) / (h * h)
    assert np.abs(Lv - b[1:N, 1:N, 1:N]).max() > 1e-3 * np.abs(b).max()


# ------------------------------------------------------------------------ geometry errors
def test_point_off_the_grid_lines_is_rejected():
    I = S3.intersect(S3.sphere(), 16)
    pts = I.pts.copy()
    pts[3] += 0.01
    with pytest.raises(GeometryError):
        O3.Geometry3D(pts, I.normals, I.shape, 16, 0.0)


def test_missing_point_is_rejected():
    I = S3.intersect(S3.sphere(), 16)
    keep = np.ones(I.P, dtype=bool)
    keep[5] = False
    with pytest.raises(GeometryError):
        O3.Geometry3D(I.pts[keep], I.normals[keep], I.shape[keep], 16, 0.0)


def test_surface_near_the_box_boundary_is_rejected():
    I = S3.intersect(S3.sphere(0.9), 16)
    with pytest.raises(GeometryError):
        O3.Geometry3D(I.pts, I.normals, I.shape, 16, 0.0)


# ------------------------------------------------------------------------------- P4s
SPHERE_POLYS = {   # homogeneous harmonic polynomials of degree l in the offset d = x - c
    1: lambda d: d[..., 2],
    2: lambda d: d[..., 0] * d[..., 1],
    3: lambda d: d[..., 2] * (2 * d[..., 2] ** 2 - 3 * d[..., 0] ** 2 - 3 * d[..., 1] ** 2),
}


@pytest.mark.parametrize("kappa,l", [(0.0, 1), (0.0, 3), (2.0, 2)])
def test_p4_sphere_closed_form_second_order(kappa, l):
    """K_D p through apply_double_layer (jumps of the fitted density plus half the fit's
    residual, reading S10) against the exact box double-layer potential on the sphere
    R = 0.5: relative max error ratio about 4 (or better) per grid doubling."""
    R, c0 = 0.5, np.asarray(S3.CENTER)
    errs = []
    for N in (16, 32, 64):
        g, I = geom(S3.sphere(R), N, kappa)
        out = O3.apply_double_layer(g, SPHERE_POLYS[l](I.pts - c0))
        ex = sphere_double_layer_plus(l, SPHERE_POLYS[l], R, c0, kappa, I.pts)
        errs.append(np.abs(out - ex).max() / np.abs(ex).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert min(ratios) > 3.5 and errs[2] < 5e-3, (errs, ratios)


# ------------------------------------------------------------------------------- S10
def _sphere_spectrum(variant="correct", N=16):
    g, I = geom(S3.sphere(), N)
    if variant == "correct":
        apply = lambda p: O3.apply_double_layer(g, p)
    elif variant == "factor_one":          # the whole fit residual instead of half of it
        apply = lambda p: O3.apply_interface(g, phi=p) + (p - g.fitted(p))
    else:                                  # raw point values in the jumps, no identity part
        orig = g.surface_derivs

        def raw(dens):
            _, gr, H = orig(dens)
            return np.asarray(dens, dtype=np.float64), gr, H
        g.surface_derivs = raw
        apply = lambda p: O3.apply_interface(g, phi=p)
    K = np.stack([apply(e) for e in np.eye(g.P)], axis=1)
    return np.linalg.eigvals(K)


def _spectrum_pin(ev):
    re = ev.real
    near_half = np.mean(np.abs(re - 0.5) < 0.05)
    return (re.min() >= 0.4 and re.max() <= 1.05 and np.abs(ev.imag).max() <= 0.05
            and near_half >= 0.8 and abs(np.median(re) - 0.5) <= 0.02), (re.min(), re.max(),
                                                                          near_half, np.median(re))


def test_s10_spectrum_of_the_discrete_operator_on_a_sphere():
    """Reading S10 pinned by the operator it discretises: on a sphere (kappa = 0, N = 16)
    the eigenvalues of the assembled K_D lie in [0.4, 1.05] with small imaginary parts,
    1 is one of them (the constant density), and they accumulate at 1/2."""
    ev = _sphere_spectrum("correct")
    ok, stats = _spectrum_pin(ev)
    assert ok, stats
    assert np.min(np.abs(ev - 1.0)) <= 1e-10


@pytest.mark.parametrize("variant", ["factor_one", "raw_values"])
def test_planted_s10_slips_fail_the_spectrum_pin(variant):
    """Adding the whole fit residual (eigenvalues pile up at 1, not 1/2) or putting the raw
    point values into the jumps (spurious eigenvalues near 0) fails the spectral pin."""
    ok, stats = _spectrum_pin(_sphere_spectrum(variant))
    assert not ok, stats


# ------------------------------------------------------------------------------ P13
def test_p13_unpack_shape_gives_the_packed_quadratic_form():
    """Packed shape operators (Sxx, Syy, Szz, Sxy, Sxz, Syz) unpack to the symmetric
    matrix whose quadratic form is Sxx x^2 + Syy y^2 + Szz z^2 + 2 (Sxy xy + Sxz xz + Syz yz)."""
    rng = np.random.default_rng(12)
    p = rng.standard_normal((40, 6))
    S = O3.unpack_shape(p)
    assert np.array_equal(S, np.transpose(S, (0, 2, 1)))
    x = rng.standard_normal((40, 3))
    q = np.einsum("pi,pij,pj->p", x, S, x)
    qf = (p[:, 0] * x[:, 0] ** 2 + p[:, 1] * x[:, 1] ** 2 + p[:, 2] * x[:, 2] ** 2
          + 2 * (p[:, 3] * x[:, 0] * x[:, 1] + p[:, 4] * x[:, 0] * x[:, 2] + p[:, 5] * x[:, 1] * x[:, 2]))
    assert np.max(np.abs(q - qf)) <= 1e-12 * np.max(np.abs(qf))
    # the shape operator of a sphere of radius R, (I - n n^T) / R, maps n to 0
    n = rng.standard_normal((40, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    A = (np.eye(3)[None] - n[:, :, None] * n[:, None, :]) / 0.7
    packed = np.stack([A[:, 0, 0], A[:, 1, 1], A[:, 2, 2], A[:, 0, 1], A[:, 0, 2], A[:, 1, 2]], axis=1)
    assert np.max(np.abs(np.einsum("pij,pj->pi", O3.unpack_shape(packed), n))) <= 1e-14


def test_p13_tangent_frame_is_a_right_handed_orthonormal_frame():
    """(t1, t2, n) is orthonormal and right-handed (t1 x t2 = n) for unit normals,
    including the axis directions and normals with equal components, and t1 is
    orthogonal to the axis least aligned with n."""
    rng = np.random.default_rng(5)
    n = np.concatenate([rng.standard_normal((200, 3)), np.eye(3), -np.eye(3),
                        np.array([[1.0, 1.0, 1.0], [1.0, -1.0, 0.0], [0.0, 1e-9, -1.0]])])
    n /= np.linalg.norm(n, axis=1)[:, None]
    t1, t2 = O3.tangent_frame(n)
    F = np.stack([t1, t2, n], axis=1)                                # rows t1, t2, n
    assert np.max(np.abs(F @ np.transpose(F, (0, 2, 1)) - np.eye(3)[None])) <= 1e-14
    assert np.max(np.abs(np.cross(t1, t2) - n)) <= 1e-14
    e = np.argmin(np.abs(n), axis=1)
    assert np.max(np.abs(t1[np.arange(len(n)), e])) <= 1e-15
