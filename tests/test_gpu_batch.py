"""Batched BVPs through kfbi_batch_solve: problems of uneven size (2-D random stars of the
batched configuration and one 3-D sphere) with several right-hand sides, solved
concurrently by the worker pool, must give bit-for-bit the results of the same contexts
solved one at a time (each solve is deterministic and problems share nothing)."""
import numpy as np
import pytest

import kfbi_workloads as W
import kfbi_workloads.surfaces3d as S3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2404_15249_gb300 as K


def _problems(nrhs):
    out = []
    for prob, sols in W.config_batch(11, nrhs, seed=5, sizes=(64, 96, 128, 192)):
        ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa,
                       precision=K.KFBI_MIXED_FP32)
        rhs = []
        for sol in sols:
            p = W.Problem(prob.iface, prob.N, prob.kappa, sol)
            rhs.append((p.f_grid(), p.f_ctrl(), p.g_ctrl(), p.u_grid()))
        out.append((ctx, rhs, (prob.N + 1,) * 2))
    I = S3.intersect(S3.sphere(), 32)
    ctx = K.Kfbi3D(I.pts, I.normals, I.shape, 32, 1.0, precision=K.KFBI_MIXED_FP32)
    rhs = []
    for r in range(nrhs):
        p = S3.Problem3D(I, 1.0, S3.manufactured_sin3(1.0))
        rhs.append((p.f_grid() * (1 + r), p.f_ctrl() * (1 + r), p.g_ctrl() * (1 + r), p.u_grid() * (1 + r)))
    out.append((ctx, rhs, (33,) * 3))
    return out


def test_batch_matches_one_at_a_time():
    nrhs = 2
    probs = _problems(nrhs)
    dev = torch.device("cuda")
    fg, fc, gc, ub = [], [], [], []
    for ctx, rhs, shape in probs:
        for f, f_c, g_c, _ in rhs:
            fg.append(torch.as_tensor(f, device=dev))
            fc.append(torch.as_tensor(f_c, device=dev))
            gc.append(torch.as_tensor(g_c, device=dev))
            ub.append(torch.empty(shape, dtype=torch.float64, device=dev))
    infos = K.batch_solve([p[0] for p in probs], fg, fc, gc, ub, nrhs)
    assert all(i["converged"] for i in infos)
    q = 0
    for ctx, rhs, shape in probs:
        for f, f_c, g_c, u_exact in rhs:
            u1, _, _ = ctx.solve_bvp(fg[q], fc[q], gc[q])
            assert torch.equal(u1, ub[q]), q
            inside = ctx.inside_mask().cpu().numpy().astype(bool)
            err = np.abs(ub[q].cpu().numpy() - u_exact)[inside].max()
            assert err < 1e-2 * np.abs(u_exact).max(), (q, err)
            q += 1
    for ctx, _, _ in probs:
        ctx.close()
