"""kfbi_box_solve_static, the allocation-free box solve, against the context box solve
kfbi_box_solve (Alg. 4) on the same right-hand sides, through the C ABI.

Collected last on purpose: it must also pass after every other test has run in the same
process (other contexts created and destroyed, kernels already loaded)."""
import ctypes
import os

import numpy as np
import pytest

import kfbi_workloads as W
import paper_2404_15249_gb300 as K


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(K.LIB_PATH):
        from paper_2404_15249_gb300 import build
        build.build()
    return K.lib()


def test_oversize_and_bad_arguments_rejected_before_device_work(lib):
    dummy = ctypes.c_void_p(256)
    st = lib.kfbi_box_solve_static(2 * K.KFBI_STATIC_MAX_N, -1.0, 1.0, 0.0, K.KFBI_FP64, dummy,
                                   dummy, None)
    assert st == 1
    msg = lib.kfbi_last_error()
    assert b"exceeds" in msg and str(K.KFBI_STATIC_MAX_N).encode() in msg
    assert lib.kfbi_box_solve_static(100, -1.0, 1.0, 0.0, K.KFBI_FP64, dummy, dummy, None) == 1
    assert lib.kfbi_box_solve_static(64, -1.0, 1.0, 0.0, K.KFBI_FP32_REFINED, dummy, dummy, None) == 1
    assert lib.kfbi_box_solve_static(64, 1.0, -1.0, 0.0, K.KFBI_FP64, dummy, dummy, None) == 1
    assert lib.kfbi_box_solve_static(64, -1.0, 1.0, 0.0, K.KFBI_FP64, None, dummy, None) == 1


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.gpu
@pytest.mark.parametrize("N,kappa,precision,tol", [
    (256, 3.0, K.KFBI_FP64, 1e-12),
    (256, 3.0, K.KFBI_MIXED_FP32, 2e-5),
    (K.KFBI_STATIC_MAX_N, 1.0, K.KFBI_FP64, 1e-12),
    (96, 0.0, K.KFBI_MIXED_FP32, 2e-5),
])
def test_static_box_solve_matches_context_twice_in_a_row(lib, N, kappa, precision, tol):
    import torch
    iface = W.flower(2 * N)
    ctx = K.Kfbi2D(iface.pts, iface.normals, iface.curv, N, kappa=kappa)
    try:
        rng = np.random.default_rng(W.SEED + N)
        bs = [torch.as_tensor(rng.standard_normal((N + 1, N + 1)), dtype=torch.float64).cuda()
              for _ in range(2)]
        refs = [ctx.box_solve(b, precision) for b in bs]
        outs = [torch.full_like(b, float("nan")) for b in bs]
        # two calls in a row on one stream, no synchronisation in between
        for b, o in zip(bs, outs):
            K.box_solve_static(N, b, kappa=kappa, precision=precision, out=o)
        torch.cuda.synchronize()
        K.box_solve_static_check()          # no bounded wait of either call gave up
        for o, r in zip(outs, refs):
            assert torch.isfinite(o).all()
            assert _rel(o, r) <= tol
            assert float(o[0].abs().max()) == 0.0 and float(o[:, N].abs().max()) == 0.0
    finally:
        ctx.close()


@pytest.mark.gpu
def test_static_box_solve_sizes_alternate_and_allocate_nothing(lib):
    """Back-to-back calls of different N (the scratch is re-laid-out per call), and device
    free memory unchanged across a second round of calls (the first round loads the
    kernels and the scratch array)."""
    import torch
    rng = np.random.default_rng(W.SEED)
    cases = []
    for N in (K.KFBI_STATIC_MAX_N, 48, 512):
        iface = W.flower(2 * N)
        ctx = K.Kfbi2D(iface.pts, iface.normals, iface.curv, N, kappa=2.0)
        b = torch.as_tensor(rng.standard_normal((N + 1, N + 1)), dtype=torch.float64).cuda()
        cases.append((N, ctx, b, ctx.box_solve(b, K.KFBI_FP64), torch.empty_like(b)))
    try:
        for N, _, b, _, out in cases:            # first calls: kernels and scratch loaded
            out.fill_(float("nan"))
            K.box_solve_static(N, b, kappa=2.0, out=out)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for N, _, b, _, out in cases:
            out.fill_(float("nan"))
            K.box_solve_static(N, b, kappa=2.0, out=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for N, _, _, ref, out in cases:
            assert _rel(out, ref) <= 1e-12, N
    finally:
        for c in cases:
            c[1].close()
