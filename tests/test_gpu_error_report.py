"""Each FP64-on-GPU quantity against the FP64 oracle, reported (printed in the test output)
and bounded: geometry (labels, crossing and irregular-node counts), the jump Taylor terms
(the corrected right-hand side of the double-layer and of the volume interface problems),
the box solve (FP64, and FP32 refined twice against the double-single residual), the
corrected interpolation (v+ at the control points), and the Arnoldi process (the density
of the plain FP64 solve and of the mixed solve)."""
import numpy as np
import pytest

import kfbi_workloads as W
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2404_15249_gb300 as K


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("case", ["flower128_poisson", "ellipse256_k10"])
def test_per_quantity_errors_against_the_oracle(case, capsys):
    prob = (W.config_poisson_flower(128, 256) if case == "flower128_poisson"
            else W.config_helmholtz(256, 10.0, "ellipse"))
    geom = O.Geometry2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa)
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa,
                   tol=1e-13)
    rep = {}
    info = ctx.info()
    mask = ctx.inside_mask().cpu().numpy().astype(bool)
    rep["geometry: node labels differing"] = int(np.sum(mask != geom.inside))
    rep["geometry: crossing / irregular count differences"] = int(
        abs(info["n_crossings_x"] - len(geom.crossings[0]["line"]))
        + abs(info["n_crossings_y"] - len(geom.crossings[1]["line"]))
        + abs(info["n_irregular"] - int(geom.irregular.sum())))
    phi = W.random_density(prob.iface.M, seed=21)
    fg, fc = prob.f_grid(), prob.f_ctrl()
    rhs, v, out = ctx.interface_solve(phi, None, None, K.KFBI_FP64)
    o_out, o_b, o_v = O.apply_interface(geom, phi=phi, return_all=True)
    rep["jump terms: corrected RHS, double layer"] = rel(rhs.cpu().numpy(), o_b)
    rep["interpolation: v+ at the control points"] = rel(out.cpu().numpy(), o_out)
    rhs_f, _, _ = ctx.interface_solve(None, fg, fc, K.KFBI_FP64)
    _, o_bf, _ = O.apply_interface(geom, f_ctrl=fc, F_grid=fg, return_all=True)
    rep["jump terms: corrected RHS, volume term"] = rel(rhs_f.cpu().numpy(), o_bf)
    rng = np.random.default_rng(3)
    b = np.zeros((prob.N + 1,) * 2)
    b[1:-1, 1:-1] = rng.standard_normal((prob.N - 1,) * 2)
    ref = O.box_solve_dst(b, prob.N, geom.h, prob.kappa ** 2)
    rep["box solve: FP64"] = rel(ctx.box_solve(b, K.KFBI_FP64).cpu().numpy(), ref)
    rep["box solve: FP32 refined twice (double-single residual)"] = rel(
        ctx.box_solve(b, K.KFBI_FP32_REFINED).cpu().numpy(), ref)
    rep["box solve: FP32 (no refinement)"] = rel(ctx.box_solve(b, K.KFBI_MIXED_FP32).cpu().numpy(), ref)
    gc = prob.g_ctrl()
    _, phi_o, _ = O.solve_bvp(geom, fg, fc, gc, tol=1e-13)
    _, phi64, _ = ctx.solve_bvp(fg, fc, gc)
    rep["Arnoldi/GMRES: FP64 density (both to 1e-13)"] = rel(phi64.cpu().numpy(), phi_o)
    ctx.set_solver(K.KFBI_MIXED_FP32, 50, 20, 1e-10, 1e-5)
    _, phim, _ = ctx.solve_bvp(fg, fc, gc)
    rep["Arnoldi/GMRES: mixed density (GPU to 1e-10)"] = rel(phim.cpu().numpy(), phi_o)
    ctx.close()
    with capsys.disabled():
        print(f"\n[{case}] error of each GPU quantity against the FP64 oracle (max-norm relative)")
        for k, val in rep.items():
            print(f"  {k:58s} {val:.3e}" if isinstance(val, float) else f"  {k:58s} {val}")
    assert rep["geometry: node labels differing"] == 0
    assert rep["geometry: crossing / irregular count differences"] == 0
    for k in ("jump terms: corrected RHS, double layer", "jump terms: corrected RHS, volume term",
              "interpolation: v+ at the control points", "box solve: FP64",
              "box solve: FP32 refined twice (double-single residual)",
              "Arnoldi/GMRES: FP64 density (both to 1e-13)"):
        assert rep[k] < 1e-11, (k, rep[k])
    assert rep["box solve: FP32 (no refinement)"] < 2e-5
    assert rep["Arnoldi/GMRES: mixed density (GPU to 1e-10)"] < 1e-6
