"""Failure paths of the solver, driven from the host without faulting the GPU: a NaN in the
boundary data (KFBI_ERR_NUMERIC), an unreachable tolerance within one restart cycle
(KFBI_ERR_NOT_CONVERGED with the last iterate), and a bounded device-side wait made to
give up at once by a test-only poll limit read at setup (KFBI_ERR_TIMEOUT; the wait then
drains its own copy, so the context stays usable and the numbers stay right)."""
import os

import numpy as np
import pytest

import kfbi_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2404_15249_gb300 as K


def _ctx(precision, **kw):
    prob = W.config_poisson_flower(128, 256)
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, 128, 0.0,
                   precision=precision, **kw)
    return ctx, prob


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_the_boundary_data_is_a_numeric_error(precision):
    ctx, prob = _ctx(precision)
    g = prob.g_ctrl().copy()
    g[17] = np.nan
    with pytest.raises(K.KfbiError) as e:
        ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), g)
    assert e.value.status == 7                       # KFBI_ERR_NUMERIC
    # the context is still usable afterwards
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info["converged"] and torch.isfinite(phi).all()
    ctx.close()


def test_nan_in_one_batched_problem_stops_the_batch_with_numeric_error():
    ctx, prob = _ctx(1)
    dev = torch.device("cuda")
    g = prob.g_ctrl().copy()
    g[3] = np.inf
    fg = [torch.as_tensor(prob.f_grid(), device=dev)] * 2
    fc = [torch.as_tensor(prob.f_ctrl(), device=dev)] * 2
    gc = [torch.as_tensor(prob.g_ctrl(), device=dev), torch.as_tensor(g, device=dev)]
    ub = [torch.empty((129, 129), dtype=torch.float64, device=dev) for _ in range(2)]
    with pytest.raises(K.KfbiError) as e:
        K.batch_solve([ctx], fg, fc, gc, ub, 2)
    assert e.value.status == 7
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_unreachable_tolerance_returns_not_converged_with_the_last_iterate(precision):
    ctx, prob = _ctx(precision, gmres_m=10, max_restarts=0, tol=1e-16)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(),
                                 allow_not_converged=True)
    assert info["converged"] == 0 and info["outer_iterations"] == 1
    assert info["iterations"] == 10
    assert 1e-16 < info["rel_residual"] < 1e-2
    assert torch.isfinite(phi).all() and torch.isfinite(u).all()
    with pytest.raises(K.KfbiError) as e:                 # the status itself
        ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert e.value.status == 5                           # KFBI_ERR_NOT_CONVERGED
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_expired_bounded_wait_is_reported_as_timeout(precision, monkeypatch):
    ref, prob = _ctx(precision)
    _, phi_ref, _ = ref.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    ref.close()
    monkeypatch.setenv("KFBI_TEST_POLL_LIMIT", "0")    # every staged-copy wait gives up
    ctx, _ = _ctx(precision)
    monkeypatch.delenv("KFBI_TEST_POLL_LIMIT")
    phi = torch.full_like(phi_ref, float("nan"))
    with pytest.raises(K.KfbiError) as e:
        ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl(), dens_out=phi)
    assert e.value.status == 6                           # KFBI_ERR_TIMEOUT
    # each wait drained its own copy before going on: the numbers are still right (the
    # two contexts may run different autotuned kernel variants, hence a tolerance)
    scale = float(phi_ref.abs().max())
    assert float((phi - phi_ref).abs().max()) <= 1e-8 * scale
    ctx.close()
    # a context made without the test limit is unaffected
    ok, _ = _ctx(precision)
    _, phi2, info2 = ok.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info2["converged"]
    assert float((phi2 - phi_ref).abs().max()) <= 1e-8 * scale
    ok.close()


def test_neumann_solve_with_kappa_zero_is_refused():
    """kappa = 0: the interior Neumann problem fixes u only up to a constant (K_N is
    singular), so the solve is refused with KFBI_ERR_ARG before any device work and the
    context stays usable."""
    ctx, prob = _ctx(0)
    with pytest.raises(K.KfbiError) as e:
        ctx.solve_neumann_bvp(prob.f_grid(), prob.f_ctrl(), prob.gn_ctrl())
    assert e.value.status == 1                           # KFBI_ERR_ARG
    assert "kappa" in str(e.value)
    u, phi, info = ctx.solve_bvp(prob.f_grid(), prob.f_ctrl(), prob.g_ctrl())
    assert info["converged"]
    ctx.close()
