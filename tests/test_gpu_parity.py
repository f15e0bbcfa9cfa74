"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by
element on the same seeded inputs.

Tolerances: plain FP64 GPU path within 1e-11 relative of the oracle (max norm over the
control points and over the grid); FP32 box solves within 2e-5 relative for one apply;
the mixed-precision BVP density within 1e-6 relative and its grid error below the
discretisation error; node labels and irregular-node counts bit-exact."""
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


CASES = {
    "flower128_poisson": lambda: W.config_poisson_flower(128, 256),
    "flower96_k1": lambda: W.config_helmholtz(96, 1.0, "flower"),
    "ellipse256_k10": lambda: W.config_helmholtz(256, 10.0, "ellipse"),
    "ellipse48_k1": lambda: W.Problem(W.ellipse(96, 0.7, 0.4, 30.0), 48, 1.0, W.manufactured_exp_sin2y(1.0)),
    "star192_batchlike": lambda: W.config_batch(1, 1, seed=3, sizes=(192,))[0][0],
}


@pytest.mark.parametrize("N", [32, 48, 96, 128, 384])
@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_box_solve_parity(N, kappa):
    prob = W.Problem(W.circle(64, 0.4, (0.01, 0.02)), N, kappa, W.manufactured_sinpi(kappa))
    ctx, geom = make(prob)
    rng = np.random.default_rng(N)
    b = np.zeros((N + 1, N + 1))
    b[1:N, 1:N] = rng.standard_normal((N - 1, N - 1))
    ref = O.box_solve_dst(b, N, geom.h, kappa * kappa)
    v64 = ctx.box_solve(b, K.KFBI_FP64).cpu().numpy()
    v32 = ctx.box_solve(b, K.KFBI_MIXED_FP32).cpu().numpy()
    vr = ctx.box_solve(b, K.KFBI_FP32_REFINED).cpu().numpy()
    assert rel(v64, ref) < 1e-12
    assert rel(v32, ref) < 2e-5
    assert rel(vr, ref) < 1e-11
    assert np.all(v64[-1] == 0) and np.all(v64[:, -1] == 0) and np.all(v64[0] == 0)
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_geometry_labels_bit_exact(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    mask = ctx.inside_mask().cpu().numpy().astype(bool)
    assert np.array_equal(mask, geom.inside)
    info = ctx.info()
    assert info["n_irregular"] == int(geom.irregular.sum())
    assert info["n_crossings_x"] == len(geom.crossings[0]["line"])
    assert info["n_crossings_y"] == len(geom.crossings[1]["line"])
    assert info["n_inside"] == int(geom.inside.sum())
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_interface_solve_stages_fp64(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=11)
    fg, fc = prob.f_grid(), prob.f_ctrl()
    rhs, v, out = ctx.interface_solve(phi, fg, fc, K.KFBI_FP64)
    o_out, o_b, o_v = O.apply_interface(geom, phi=phi, f_ctrl=fc, F_grid=fg, return_all=True)
    assert rel(rhs.cpu().numpy(), o_b) < 1e-11
    assert rel(v.cpu().numpy(), o_v) < 1e-11
    assert rel(out.cpu().numpy(), o_out) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_interface_solve_refined_fp32(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=12)
    fg, fc = prob.f_grid(), prob.f_ctrl()
    rhs, v, out = ctx.interface_solve(phi, fg, fc, K.KFBI_FP32_REFINED)
    o_out, o_b, o_v = O.apply_interface(geom, phi=phi, f_ctrl=fc, F_grid=fg, return_all=True)
    assert rel(rhs.cpu().numpy(), o_b) < 1e-11
    assert rel(v.cpu().numpy(), o_v) < 1e-11
    assert rel(out.cpu().numpy(), o_out) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", list(CASES))
def test_double_layer_apply_parity(case):
    prob = CASES[case]()
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=5)
    ref = O.apply_double_layer(geom, phi)
    g64 = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_FP64).cpu().numpy()
    g32 = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_MIXED_FP32).cpu().numpy()
    gr = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_FP32_REFINED).cpu().numpy()
    g1 = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_FP32_REFINED_ONCE).cpu().numpy()
    assert rel(g64, ref) < 1e-11
    assert rel(g32, ref) < 2e-5
    assert rel(gr, ref) < 1e-11
    assert rel(g1, ref) < 1e-10
    # repeated applies are bit-identical
    again = ctx.apply_layer_potential(phi, K.KFBI_DOUBLE_LAYER, K.KFBI_FP64).cpu().numpy()
    assert np.array_equal(again, g64)
    ctx.close()


def test_single_layer_and_volume_parity():
    prob = W.config_helmholtz(128, 1.0, "ellipse")
    ctx, geom = make(prob)
    psi = W.random_density(prob.iface.M, seed=9)
    ref = O.apply_interface(geom, psi=psi)
    got = ctx.apply_layer_potential(psi, K.KFBI_SINGLE_LAYER, K.KFBI_FP64).cpu().numpy()
    assert rel(got, ref) < 1e-11
    fg, fc = prob.f_grid(), prob.f_ctrl()
    assert rel(ctx.apply_volume(fg, fc).cpu().numpy(), O.apply_volume(geom, fg, fc)) < 1e-11
    ctx.close()


def test_constant_density_indicator_kappa0():
    prob = W.config_poisson_flower(256, 512)
    ctx, geom = make(prob)
    out = ctx.apply_layer_potential(np.ones(512)).cpu().numpy()
    assert np.max(np.abs(out - 1.0)) < 1e-12
    _, v, _ = ctx.interface_solve(np.ones(512))
    assert np.max(np.abs(v.cpu().numpy() - geom.inside)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("case", ["flower128_poisson", "ellipse256_k10"])
def test_solve_bvp_fp64_matches_oracle(case):
    prob = CASES[case]()
    ctx, geom = make(prob, tol=1e-13, gmres_m=50)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    u_o, phi_o, info_o = O.solve_bvp(geom, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-13)
    assert info["converged"] and info["rel_residual"] <= 1e-13
    assert rel(phi.cpu().numpy(), phi_o) < 1e-11
    assert rel(u.cpu().numpy(), u_o) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", ["flower128_poisson", "ellipse256_k10"])
def test_solve_bvp_refined_matches_oracle(case):
    prob = CASES[case]()
    ctx, geom = make(prob, precision=K.KFBI_FP32_REFINED, tol=1e-12)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    u_o, phi_o, _ = O.solve_bvp(geom, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-13)
    assert info["converged"] and info["applies_low"] == 0
    assert rel(phi.cpu().numpy(), phi_o) < 1e-9
    assert rel(u.cpu().numpy(), u_o) < 1e-9
    ctx.close()


@pytest.mark.parametrize("case", ["flower128_poisson", "ellipse256_k10", "star192_batchlike"])
def test_solve_bvp_mixed_precision(case):
    prob = CASES[case]()
    ctx, geom = make(prob, precision=K.KFBI_MIXED_FP32, tol=1e-10, inner_tol=1e-5)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), allow_not_converged=True)
    u_o, phi_o, _ = O.solve_bvp(geom, prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), tol=1e-12)
    assert info["converged"], info
    assert info["applies_low"] > 0 and info["outer_iterations"] <= 3, info
    assert rel(phi.cpu().numpy(), phi_o) < 1e-6
    u_exact = prob.u_grid()
    disc = np.max(np.abs(u_o - u_exact)[geom.inside])
    assert np.max(np.abs(u.cpu().numpy() - u_o)[geom.inside]) < disc
    ctx.close()


def test_geometry_error_is_reported():
    prob = W.Problem(W.circle(64, 0.97, (0.0, 0.0)), 32, 0.0, W.manufactured_sinpi())
    with pytest.raises(K.KfbiError) as e:
        K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, 32, 0.0)
    assert e.value.status == 2
    under = W.flower(128, r0=0.5, a=0.3, k=20)      # petals thinner than a cell at N = 32
    with pytest.raises(O.GeometryError):
        O.Geometry2D(under.pts, under.normals, under.curv, 32, 0.0)
    with pytest.raises(K.KfbiError) as e:
        K.Kfbi2D(under.pts, under.normals, under.curv, 32, 0.0)
    assert e.value.status == 2


def test_zero_density_gives_zero():
    prob = W.config_poisson_flower(64, 128)
    ctx, _ = make(prob)
    out = ctx.apply_layer_potential(np.zeros(128)).cpu().numpy()
    assert np.all(out == 0.0)
    ctx.close()


@pytest.mark.parametrize("N", [2048, 4096])
def test_full_size_apply_parity(N):
    """The benchmark's sizes (2-D Helmholtz, flower, kappa = 10, M = 2N): every control
    point of one FP64 and one FP32 apply against the oracle."""
    prob = W.config_helmholtz(N, 10.0, "flower")
    ctx, geom = make(prob)
    phi = W.random_density(prob.iface.M, seed=21)
    ref = O.apply_double_layer(geom, phi)
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_FP64).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_FP32_REFINED).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_FP32_REFINED_ONCE).cpu().numpy(), ref) < 1e-10
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 1e-4
    ctx.close()


@pytest.mark.parametrize("N", [6144, 8192])
def test_largest_grid_box_solve_manufactured(N):
    """The largest compiled grids (FP64 lines of N = 8192 run the transforms with one
    shared-memory buffer and an unstaged column pass): a discrete solution v is chosen,
    b = (Lap_h - kappa^2) v is formed in FP64 with the 5-point stencil, and the box solve
    must give v back."""
    kappa = 2.0
    iface = W.circle(2 * N, 0.45)
    ctx = K.Kfbi2D(iface.pts, iface.normals, iface.curv, N, kappa)
    h = 2.0 / N
    g = torch.Generator(device="cuda").manual_seed(N)
    v = torch.zeros((N + 1, N + 1), dtype=torch.float64, device="cuda")
    v[1:N, 1:N] = torch.rand((N - 1, N - 1), generator=g, device="cuda", dtype=torch.float64) - 0.5
    b = torch.zeros_like(v)
    b[1:N, 1:N] = ((v[2:, 1:N] + v[:-2, 1:N] + v[1:N, 2:] + v[1:N, :-2] - 4.0 * v[1:N, 1:N]) / (h * h)
                   - kappa * kappa * v[1:N, 1:N])
    scale = float(v.abs().max())
    # FP32: rounding the right-hand side alone costs about 2e-5 at N = 2048
    for prec, tol in ((K.KFBI_FP64, 1e-11), (K.KFBI_MIXED_FP32, 1e-3)):
        out = ctx.box_solve(b, prec)
        assert float((out - v).abs().max()) / scale < tol, prec
    ctx.close()


@pytest.mark.parametrize("kappa", [0.0, 10.0])
def test_fp32_box_solve_with_and_without_the_tridiagonal_pass(kappa):
    """FP32 box solves with the well-conditioned x-modes' tridiagonal y-systems solved
    directly (the default: the autotuned variant's recursive filters or elimination, from
    the reported tri_first_mode) and with every mode on the sine-transform pair
    (KFBI_TRI=0 at setup): both within 2e-5 of the oracle."""
    import os
    N = 256
    prob = W.Problem(W.circle(64, 0.4, (0.01, 0.02)), N, kappa, W.manufactured_sinpi(kappa))
    rng = np.random.default_rng(N + 1)
    b = np.zeros((N + 1, N + 1))
    b[1:N, 1:N] = rng.standard_normal((N - 1, N - 1))
    for flag in (None, "0"):
        if flag is not None:
            os.environ["KFBI_TRI"] = flag
        try:
            ctx, geom = make(prob)
        finally:
            os.environ.pop("KFBI_TRI", None)
        k0 = ctx.info()["tri_first_mode"]
        assert (k0 == N) if flag == "0" else (0 < k0 <= N / 8 and k0 % 32 == 0)
        ref = O.box_solve_dst(b, N, geom.h, kappa * kappa)
        assert rel(ctx.box_solve(b, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 2e-5
        ctx.close()


@pytest.mark.parametrize("N", [64, 96, 256, 384, 1024])
@pytest.mark.parametrize("variant", [0, 4, 8])
def test_fp32_column_pass_variants(N, variant, monkeypatch):
    """Each FP32 y-pass variant, fixed at setup (KFBI_DST_VARIANTS): the staged column tiles
    (0), the transposed pass with the tridiagonal elimination (4) and the row-layout pass
    with the recursive filters and the transform pair on a side stream (8), on grids whose
    sizes leave ragged chunks and warm-ups longer than a chunk: the FP32 box solve and the
    plain FP32 apply (correction fused with the first x-transform) within 2e-5 of the
    oracle."""
    monkeypatch.setenv("KFBI_DST_VARIANTS", f"0,{variant},0,6")
    kappa = 3.0
    prob = W.Problem(W.flower(2 * N), N, kappa, W.manufactured_sinpi(kappa))
    ctx, geom = make(prob)
    monkeypatch.delenv("KFBI_DST_VARIANTS")
    assert ctx.info()["dst_variant"][1] == variant
    rng = np.random.default_rng(N + variant)
    b = np.zeros((N + 1, N + 1))
    b[1:N, 1:N] = rng.standard_normal((N - 1, N - 1))
    ref = O.box_solve_dst(b, N, geom.h, kappa * kappa)
    assert rel(ctx.box_solve(b, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 2e-5
    phi = W.random_density(prob.iface.M, seed=N)
    ref = O.apply_double_layer(geom, phi)
    assert rel(ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 2e-5
    psi = W.random_density(prob.iface.M, seed=N + 1)
    ref = O.apply_interface(geom, psi=psi)
    assert rel(ctx.apply_layer_potential(psi, 1, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 2e-5
    ctx.close()


@pytest.mark.parametrize("N", [96, 256])
@pytest.mark.parametrize("variant", [4, 8])
def test_plain_apply_with_rows_split_into_parts(N, variant, monkeypatch):
    """A flat axis-aligned ellipse (semi-axes 0.8 and 0.1) runs nearly along the grid rows at
    its top and bottom, which then hold far more irregular nodes than one work item of the
    sparse first x-transform takes (about 80 at N = 256): those rows are split into parts
    whose partial rows the last part to finish adds up.  The plain FP32 double- and
    single-layer applies (with variant 8 also the last x-transform at the stencil nodes
    only) within 2e-5 of the oracle, and bit-identical when repeated."""
    monkeypatch.setenv("KFBI_DST_VARIANTS", f"0,{variant},0,6")
    prob = W.Problem(W.ellipse(2 * N, 0.8, 0.1, 0.0), N, 1.0, W.manufactured_exp_sin2y(1.0))
    ctx, geom = make(prob)
    monkeypatch.delenv("KFBI_DST_VARIANTS")
    assert ctx.info()["dst_variant"][1] == variant
    phi = W.random_density(prob.iface.M, seed=7)
    ref = O.apply_double_layer(geom, phi)
    g32 = ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy()
    assert rel(g32, ref) < 2e-5
    assert np.array_equal(ctx.apply_layer_potential(phi, 0, K.KFBI_MIXED_FP32).cpu().numpy(), g32)
    ref = O.apply_interface(geom, psi=phi)
    assert rel(ctx.apply_layer_potential(phi, 1, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 2e-5
    ctx.close()


@pytest.mark.parametrize("case", ["flower128_poisson", "ellipse256_k10", "flower96_k1"])
def test_normal_derivative_applies_parity(case):
    """d_n v^+ of the single and double layer and of the volume term (Procedure 2's Neumann
    data) against the oracle: FP64 and twice-refined FP32 within 1e-11 (1e-10 refined at the
    gradient's 1/h weighting), plain FP32 within 1e-3."""
    prob = CASES[case]()
    ctx, geom = make(prob)
    psi = W.random_density(prob.iface.M, seed=31)
    ref = O.apply_single_layer_dn(geom, psi)
    assert rel(ctx.apply_layer_potential_dn(psi, 1, K.KFBI_FP64).cpu().numpy(), ref) < 1e-11
    assert rel(ctx.apply_layer_potential_dn(psi, 1, K.KFBI_FP32_REFINED).cpu().numpy(), ref) < 1e-10
    assert rel(ctx.apply_layer_potential_dn(psi, 1, K.KFBI_MIXED_FP32).cpu().numpy(), ref) < 1e-3
    refd = O.apply_interface_dn(geom, phi=psi)
    assert rel(ctx.apply_layer_potential_dn(psi, 0, K.KFBI_FP64).cpu().numpy(), refd) < 1e-11
    fg, fc = prob.f_grid(), prob.f_ctrl()
    assert rel(ctx.apply_volume_dn(fg, fc).cpu().numpy(), O.apply_volume_dn(geom, fg, fc)) < 1e-11
    ctx.close()


NEUMANN_CASES = {
    "ellipse128_k1": lambda: W.config_helmholtz(128, 1.0, "ellipse"),
    "flower192_k10": lambda: W.config_helmholtz(192, 10.0, "flower"),
}


@pytest.mark.parametrize("case", list(NEUMANN_CASES))
def test_solve_neumann_fp64_matches_oracle(case):
    """Neumann BVP (single-layer density): plain FP64 GMRES against the oracle's, both run
    to 1e-13: density and u within 1e-10."""
    prob = NEUMANN_CASES[case]()
    ctx, geom = make(prob, tol=1e-13)
    fg, fc, gn = prob.f_grid(), prob.f_ctrl(), prob.gn_ctrl()
    u, psi, info = ctx.solve_neumann_bvp(fg, fc, gn)
    u_o, psi_o, info_o = O.solve_neumann_bvp(geom, fg, fc, gn, tol=1e-13)
    assert info["converged"] and info_o["converged"]
    assert rel(psi.cpu().numpy(), psi_o) < 1e-10
    assert rel(u.cpu().numpy(), u_o) < 1e-10
    ctx.close()


@pytest.mark.parametrize("case", list(NEUMANN_CASES))
def test_solve_neumann_mixed_precision(case):
    """Mixed-precision Neumann solve (relaxed FP32 matvecs, refined FP64-accurate cycle
    residuals): density within 1e-6 of the oracle, u closer to the oracle's than the
    oracle's is to the exact solution."""
    prob = NEUMANN_CASES[case]()
    ctx, geom = make(prob, precision=K.KFBI_MIXED_FP32, tol=1e-10)
    fg, fc, gn = prob.f_grid(), prob.f_ctrl(), prob.gn_ctrl()
    u, psi, info = ctx.solve_neumann_bvp(fg, fc, gn)
    u_o, psi_o, _ = O.solve_neumann_bvp(geom, fg, fc, gn, tol=1e-12)
    assert info["converged"] and info["applies_low"] > 0
    assert rel(psi.cpu().numpy(), psi_o) < 1e-6
    disc = np.max(np.abs(u_o - prob.u_grid())[geom.inside])
    assert np.max(np.abs(u.cpu().numpy() - u_o)[geom.inside]) < disc
    ctx.close()
