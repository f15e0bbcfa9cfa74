"""GPU parity of the 3-D path (through the C ABI) against the 3-D FP64 CPU oracle on the
same seeded inputs (grid-line intersections of an ellipsoid, a sphere and the star surface
rho = 0.5 + 0.1 sin 3 theta cos 4 phi).

Tolerances as in 2-D: FP64 GPU path within 1e-11 relative of the oracle; FP32 box
solves within 2e-5 relative for one transform and 1e-4 for an apply; node labels and
counts bit-exact; the mixed-precision BVP density within 1e-6 of the FP64 one and its
grid error below the discretisation error."""
import numpy as np
import pytest

import kfbi_workloads.surfaces3d as S3
from oracle import kfbi3d as O3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2404_15249_gb300 as K


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = {
    "ellipsoid32_k0": lambda: S3.Problem3D(S3.intersect(S3.ellipsoid(), 32), 0.0, S3.manufactured_sin3(0.0)),
    "sphere48_k2": lambda: S3.Problem3D(S3.intersect(S3.sphere(), 48), 2.0, S3.manufactured_sin3(2.0)),
    "ellipsoid64_k1": lambda: S3.Problem3D(S3.intersect(S3.ellipsoid(), 64), 1.0, S3.manufactured_sin3(1.0)),
    "star64_k0": lambda: S3.Problem3D(S3.intersect(S3.star(), 64), 0.0, S3.manufactured_sin3(0.0)),
}


def make(prob, **kw):
    I = prob.iface
    ctx = K.Kfbi3D(I.pts, I.normals, I.shape, I.N, prob.kappa, **kw)
    geom = O3.Geometry3D(I.pts, I.normals, I.shape, I.N, prob.kappa)
    return ctx, geom


@pytest.mark.parametrize("case", list(CASES))
def test_geometry_labels_and_counts_bit_exact(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    mask = ctx.inside_mask().cpu().numpy().astype(bool)
    assert np.array_equal(mask, geom.inside)
    info = ctx.info()
    assert info["dim"] == 3
    assert info["n_irregular"] == int(geom.irregular.sum())
    assert info["n_inside"] == int(geom.inside.sum())
    counts = [int((geom.axis == a).sum()) for a in range(3)]
    assert [info["n_crossings_x"], info["n_crossings_y"], info["n_crossings_z"]] == counts
    ctx.close()


@pytest.mark.parametrize("N", [32, 48])
@pytest.mark.parametrize("kappa", [0.0, 2.0])
def test_box_solve_parity(N, kappa):
    prob = S3.Problem3D(S3.intersect(S3.sphere(), N), kappa, S3.manufactured_sin3(kappa))
    ctx, geom = make(prob)
    rng = np.random.default_rng(N)
    b = np.zeros((N + 1,) * 3)
    b[1:N, 1:N, 1:N] = rng.standard_normal((N - 1,) * 3)
    ref = O3.box_solve_dst(b, N, geom.h, kappa * kappa)
    v64 = ctx.box_solve(b, K.KFBI_FP64).cpu().numpy()
    v32 = ctx.box_solve(b, K.KFBI_MIXED_FP32).cpu().numpy()
    vr = ctx.box_solve(b, K.KFBI_FP32_REFINED).cpu().numpy()
    assert rel(v64, ref) < 1e-12
    assert rel(v32, ref) < 2e-5
    assert rel(vr, ref) < 1e-11
    assert np.all(v64[-1] == 0) and np.all(v64[:, -1] == 0) and np.all(v64[:, :, 0] == 0)
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_double_layer_apply_parity(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = S3.random_density3(geom.P, prob.iface.pts, seed=11)
    ref = O3.apply_double_layer(geom, phi)
    a64 = ctx.apply_layer_potential(phi, 0, K.KFBI_FP64).cpu().numpy()
    a32 = ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy()
    ar = ctx.apply_layer_potential(phi, 0, K.KFBI_FP32_REFINED).cpu().numpy()
    a1 = ctx.apply_layer_potential(phi, 0, K.KFBI_FP32_REFINED_ONCE).cpu().numpy()
    assert rel(a64, ref) < 1e-11
    assert rel(a32, ref) < 1e-4
    assert rel(ar, ref) < 1e-11
    assert rel(a1, ref) < 1e-9
    again = ctx.apply_layer_potential(phi, 0, K.KFBI_FP64).cpu().numpy()
    assert np.array_equal(a64, again)
    ctx.close()


@pytest.mark.parametrize("case", ["ellipsoid32_k0", "sphere48_k2"])
def test_interface_solve_stages_fp64(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = S3.random_density3(geom.P, prob.iface.pts, seed=3)
    f, fc = prob.f_grid(), prob.f_ctrl()
    out_ref, b_ref, v_ref = O3.apply_interface(geom, phi=phi, f_ctrl=fc, F_grid=f, return_all=True)
    rhs, v, out = ctx.interface_solve(phi, f, fc, K.KFBI_FP64)
    assert rel(rhs.cpu().numpy(), b_ref) < 1e-11
    assert rel(v.cpu().numpy(), v_ref) < 1e-11
    assert rel(out.cpu().numpy(), out_ref) < 1e-11
    ctx.close()


def test_volume_potential_parity():
    prob = CASES["sphere48_k2"]()
    ctx, geom = make(prob)
    ref = O3.apply_volume(geom, prob.f_grid(), prob.f_ctrl())
    out = ctx.apply_volume(prob.f_grid(), prob.f_ctrl(), K.KFBI_FP64).cpu().numpy()
    assert rel(out, ref) < 1e-11
    ctx.close()


def test_constant_density_indicator_kappa0():
    prob = CASES["ellipsoid32_k0"]()
    ctx, geom = make(prob)
    out = ctx.apply_layer_potential(np.ones(geom.P), 0, K.KFBI_FP64).cpu().numpy()
    assert np.abs(out - 1.0).max() < 1e-12
    _, v, _ = ctx.interface_solve(np.ones(geom.P), None, None, K.KFBI_FP64)
    assert np.abs(v.cpu().numpy() - geom.inside).max() < 1e-12
    ctx.close()


@pytest.mark.parametrize("case", ["ellipsoid32_k0", "sphere48_k2"])
def test_interface_solve_refined_fp32(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = S3.random_density3(geom.P, prob.iface.pts, seed=4)
    f, fc = prob.f_grid(), prob.f_ctrl()
    out_ref, _, v_ref = O3.apply_interface(geom, phi=phi, f_ctrl=fc, F_grid=f, return_all=True)
    _, v, out = ctx.interface_solve(phi, f, fc, K.KFBI_FP32_REFINED)
    assert rel(v.cpu().numpy(), v_ref) < 1e-11
    assert rel(out.cpu().numpy(), out_ref) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", ["ellipsoid32_k0", "sphere48_k2"])
def test_solve_bvp_fp64_matches_oracle(case):
    prob = CASES[case]()
    ctx, geom = make(prob, tol=1e-13)
    u_ref, phi_ref, _ = O3.solve_bvp(geom, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-13)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info["converged"]
    assert rel(phi.cpu().numpy(), phi_ref) < 1e-10
    assert rel(u.cpu().numpy(), u_ref) < 1e-10
    ctx.close()


@pytest.mark.parametrize("case", ["ellipsoid64_k1", "star64_k0"])
def test_solve_bvp_mixed_precision(case):
    prob = CASES[case]()
    ctx64, geom = make(prob, tol=1e-10)
    u64, phi64, _ = ctx64.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    ctx64.close()
    I = prob.iface
    ctx = K.Kfbi3D(I.pts, I.normals, I.shape, I.N, prob.kappa, precision=K.KFBI_MIXED_FP32,
                   tol=1e-10)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info["converged"] and info["applies_low"] > 0
    assert rel(phi.cpu().numpy(), phi64.cpu().numpy()) < 1e-6
    exact = prob.u_grid()
    e_mixed = np.abs(u.cpu().numpy() - exact)[geom.inside].max()
    e64 = np.abs(u64.cpu().numpy() - exact)[geom.inside].max()
    diff = np.abs(u.cpu().numpy() - u64.cpu().numpy())[geom.inside].max()
    assert diff < e64 and e_mixed < 1.1 * e64
    ctx.close()


def test_missing_point_is_a_geometry_error():
    I = S3.intersect(S3.sphere(), 32)
    keep = np.ones(I.P, dtype=bool)
    keep[17] = False
    with pytest.raises(K.KfbiError) as e:
        K.Kfbi3D(I.pts[keep], I.normals[keep], I.shape[keep], 32, 0.0)
    assert e.value.status == 2


@pytest.mark.parametrize("case", ["ellipsoid32_k0", "sphere48_k2", "star64_k0"])
def test_single_layer_apply_parity(case):
    """3-D single layer ([v] = 0, [d_n v] = psi; jumps of the fitted psi): v^+ at the points
    against the oracle's interface problem with psi, FP64 and refined FP32 within 1e-11,
    plain FP32 within 1e-4."""
    prob = CASES[case]()
    ctx, geom = make(prob)
    psi = S3.random_density3(geom.P, prob.iface.pts, seed=17)
    ref = O3.apply_interface(geom, psi=psi)
    assert rel(ctx.apply_layer_potential(psi, K.KFBI_SINGLE_LAYER, K.KFBI_FP64).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential(psi, K.KFBI_SINGLE_LAYER, K.KFBI_FP32_REFINED).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential(psi, K.KFBI_SINGLE_LAYER, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 1e-4
    ctx.close()


def test_neumann_data_is_unsupported_in_3d():
    prob = CASES["ellipsoid32_k0"]()
    ctx, geom = make(prob)
    with pytest.raises(K.KfbiError) as e:
        ctx.apply_layer_potential_dn(np.ones(geom.P), K.KFBI_SINGLE_LAYER, K.KFBI_FP64)
    assert e.value.status == 8
    ctx.close()


@pytest.mark.parametrize("N", [128])
def test_larger_grid_apply_parity(N):
    """Ellipsoid at N = 128 (2.1e4 points): one FP64 and one FP32 apply against the
    oracle at every point."""
    prob = S3.Problem3D(S3.intersect(S3.ellipsoid(), N), 0.0, S3.manufactured_sin3(0.0))
    ctx, geom = make(prob)
    phi = S3.random_density3(geom.P, prob.iface.pts, seed=21)
    ref = O3.apply_double_layer(geom, phi)
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_FP64).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 1e-4
    ctx.close()
