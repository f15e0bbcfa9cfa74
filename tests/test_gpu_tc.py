"""GPU parity of the tensor-core box solve (KFBI_TF32X3: the dense sine-matrix form of the
DST-I diagonalisation of Alg. 4 as four tcgen05 GEMMs, TF32 with a three-term split)
against the FP64 CPU oracle, through the C ABI.

Tolerances: FP32-class, as for the FFT FP32 path (2e-5 relative for one box solve and a
double-layer apply, 1e-4 for an interface solve with a volume source and for an apply at
the largest grid); the mixed-precision solver with tensor-core applies as
its lowest tier converges to the FP64 density within 1e-6 relative."""
import numpy as np
import pytest

import kfbi_workloads as W
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2404_15249_gb300 as K


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make(prob, **kw):
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa, **kw)
    geom = O.Geometry2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa)
    return ctx, geom


@pytest.mark.parametrize("N", [128, 256, 384])
@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_tc_box_solve_parity(N, kappa):
    """Several 128 x 64 tiles and K chunks; N = 384 is not a power of two."""
    prob = W.Problem(W.circle(64, 0.4, (0.01, 0.02)), N, kappa, W.manufactured_sinpi(kappa))
    ctx, geom = make(prob)
    rng = np.random.default_rng(N + 7)
    b = np.zeros((N + 1, N + 1))
    b[1:N, 1:N] = rng.standard_normal((N - 1, N - 1))
    ref = O.box_solve_dst(b, N, geom.h, kappa * kappa)
    v = ctx.box_solve(b, K.KFBI_TF32X3).cpu().numpy()
    assert rel(v, ref) < 2e-5
    assert np.all(v[0] == 0) and np.all(v[-1] == 0) and np.all(v[:, 0] == 0) and np.all(v[:, -1] == 0)
    again = ctx.box_solve(b, K.KFBI_TF32X3).cpu().numpy()
    assert np.array_equal(v, again)
    ctx.close()


def test_tc_box_solve_single_mode():
    """A single sine mode is an eigenvector: the solve divides it by its eigenvalue."""
    N, kappa = 256, 2.0
    prob = W.Problem(W.circle(64, 0.4), N, kappa, W.manufactured_sinpi(kappa))
    ctx, geom = make(prob)
    h = geom.h
    i = np.arange(N + 1)
    l, m = 37, 5
    mode = np.outer(np.sin(np.pi * l * i / N), np.sin(np.pi * m * i / N))
    mode[:, -1] = 0.0
    mode[-1, :] = 0.0
    lam = -(4.0 / h**2) * (np.sin(np.pi * l / (2 * N))**2 + np.sin(np.pi * m / (2 * N))**2) - kappa**2
    v = ctx.box_solve(mode, K.KFBI_TF32X3).cpu().numpy()
    assert rel(v, mode / lam) < 2e-5
    ctx.close()


@pytest.mark.parametrize("case", ["flower256_k10", "ellipse512_k1"])
def test_tc_apply_and_interface_parity(case):
    prob = {"flower256_k10": lambda: W.config_helmholtz(256, 10.0, "flower"),
            "ellipse512_k1": lambda: W.config_helmholtz(512, 1.0, "ellipse")}[case]()
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=13)
    ref = O.apply_double_layer(geom, phi)
    got = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_TF32X3).cpu().numpy()
    assert rel(got, ref) < 2e-5
    fg, fc = prob.f_grid(), prob.f_ctrl()
    out_ref, b_ref, v_ref = O.apply_interface(geom, phi=phi, f_ctrl=fc, F_grid=fg, return_all=True)
    rhs, v, out = ctx.interface_solve(phi, fg, fc, K.KFBI_TF32X3)
    assert rel(rhs.cpu().numpy(), b_ref) < 1e-6
    # the volume source enters through corrections of size 1/h^2 next to v: FP32 rounding
    # of the right-hand side alone is about 1e-5 of v at N = 512
    assert rel(v.cpu().numpy(), v_ref) < 1e-4
    assert rel(out.cpu().numpy(), out_ref) < 1e-4
    ctx.close()


def test_tc_full_size_apply_parity():
    """N = 4096 (the largest tensor-core grid), flower, kappa = 10, M = 2N: every control
    point against the oracle."""
    prob = W.config_helmholtz(4096, 10.0, "flower")
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=21)
    ref = O.apply_double_layer(geom, phi)
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_TF32X3).cpu().numpy(), ref) < 1e-4
    ctx.close()


def test_tc_mixed_solver_converges():
    prob = W.config_helmholtz(256, 10.0, "ellipse")
    ctx, geom = make(prob, precision=K.KFBI_TF32X3, tol=1e-10, inner_tol=1e-5)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), allow_not_converged=True)
    u_o, phi_o, _ = O.solve_bvp(geom, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-12)
    assert info["converged"], info
    assert info["applies_low"] > 0, info
    assert rel(phi.cpu().numpy(), phi_o) < 1e-6
    disc = np.max(np.abs(u_o - prob.u_grid())[geom.inside])
    assert np.max(np.abs(u.cpu().numpy() - u_o)[geom.inside]) < disc
    ctx.close()


def test_tc_unsupported_sizes_are_refused():
    prob = W.Problem(W.circle(64, 0.4), 96, 0.0, W.manufactured_sinpi(0.0))   # 96 % 128 != 0
    ctx, geom = make(prob)
    with pytest.raises(K.KfbiError) as e:
        ctx.box_solve(np.zeros((97, 97)), K.KFBI_TF32X3)
    assert e.value.status == 8
    with pytest.raises(K.KfbiError) as e:
        ctx.apply_layer_potential(np.ones(prob.iface.M), 0, K.KFBI_TF32X3)
    assert e.value.status == 8
    ctx.close()
    with pytest.raises(K.KfbiError) as e:
        make(prob, precision=K.KFBI_TF32X3)
    assert e.value.status == 8


# ------------------------------------------------------------------ 3-D (six GEMMs)
def make3(prob, **kw):
    import kfbi_workloads.surfaces3d as S3  # noqa: F401
    from oracle import kfbi3d as O3
    I = prob.iface
    ctx = K.Kfbi3D(I.pts, I.normals, I.shape, I.N, prob.kappa, **kw)
    geom = O3.Geometry3D(I.pts, I.normals, I.shape, I.N, prob.kappa)
    return ctx, geom


@pytest.mark.parametrize("kappa", [0.0, 2.0])
def test_tc_box_solve_parity_3d(kappa):
    """N = 128: the N^2 x N GEMMs span 128 row tiles; every unknown against the oracle."""
    import kfbi_workloads.surfaces3d as S3
    from oracle import kfbi3d as O3
    N = 128
    prob = S3.Problem3D(S3.intersect(S3.sphere(), N), kappa, S3.manufactured_sin3(kappa))
    ctx, geom = make3(prob)
    rng = np.random.default_rng(5)
    b = np.zeros((N + 1,) * 3)
    b[1:N, 1:N, 1:N] = rng.standard_normal((N - 1,) * 3)
    ref = O3.box_solve_dst(b, N, geom.h, kappa * kappa)
    v = ctx.box_solve(b, K.KFBI_TF32X3).cpu().numpy()
    assert rel(v, ref) < 2e-5
    assert np.all(v[0] == 0) and np.all(v[-1] == 0) and np.all(v[:, :, 0] == 0)
    ctx.close()


def test_tc_apply_parity_and_mixed_solve_3d():
    import kfbi_workloads.surfaces3d as S3
    from oracle import kfbi3d as O3
    prob = S3.Problem3D(S3.intersect(S3.ellipsoid(), 128), 1.0, S3.manufactured_sin3(1.0))
    ctx, geom = make3(prob, tol=1e-10)
    phi = S3.random_density3(geom.P, prob.iface.pts, seed=8)
    ref = O3.apply_double_layer(geom, phi)
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_TF32X3).cpu().numpy(), ref) < 1e-4
    u64, phi64, _ = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    ctx.set_solver(K.KFBI_TF32X3, 50, 20, 1e-10, 1e-5)
    u, phi_tc, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info["converged"] and info["applies_low"] > 0, info
    assert rel(phi_tc.cpu().numpy(), phi64.cpu().numpy()) < 1e-6
    exact = prob.u_grid()
    e64 = np.abs(u64.cpu().numpy() - exact)[geom.inside].max()
    assert np.abs(u.cpu().numpy() - exact)[geom.inside].max() < 1.1 * e64
    ctx.close()


def test_tc_largest_2d_grid_box_solve_manufactured():
    """N = 8192 (S tables of 2 x 268 MB): a discrete solution v, b = (Lap_h - kappa^2) v in
    FP64, the tensor-core solve must give v back.  A random v is the hardest case: b is
    dominated by the highest modes (|lambda| ~ 8/h^2) and every error in the sums of the low
    modes is amplified by up to lambda_max / lambda_min ~ N^2.  The dense sums run over
    K = 8192 terms with the tensor core's FP32 accumulation (two partial accumulators per
    tile at this width), against log2 N rounding stages of the FFT: measured 2.8e-3 here
    against < 1e-3 for the FFT FP32 path."""
    N, kappa = 8192, 2.0
    iface = W.circle(2 * N, 0.45)
    ctx = K.Kfbi2D(iface.pts, iface.normals, iface.curv, N, kappa)
    h = 2.0 / N
    g = torch.Generator(device="cuda").manual_seed(N)
    v = torch.zeros((N + 1, N + 1), dtype=torch.float64, device="cuda")
    v[1:N, 1:N] = torch.rand((N - 1, N - 1), generator=g, device="cuda", dtype=torch.float64) - 0.5
    b = torch.zeros_like(v)
    b[1:N, 1:N] = ((v[2:, 1:N] + v[:-2, 1:N] + v[1:N, 2:] + v[1:N, :-2] - 4.0 * v[1:N, 1:N]) / (h * h)
                   - kappa * kappa * v[1:N, 1:N])
    out = ctx.box_solve(b, K.KFBI_TF32X3)
    assert float((out - v).abs().max()) / float(v.abs().max()) < 5e-3
    ctx.close()
