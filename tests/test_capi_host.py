"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads,
exports every function include/kfbi.h declares, and rejects bad arguments before any
device work."""
import ctypes
import os

import pytest

import paper_2404_15249_gb300 as K


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(K.LIB_PATH):
        from paper_2404_15249_gb300 import build
        build.build()
    return K.lib()


def test_every_declared_symbol_is_exported(lib):
    names = K.header_symbols()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    for code in range(9):
        assert lib.kfbi_status_string(code)
    o = K.default_options()
    assert (o.dim, o.N, o.lo, o.hi, o.kappa, o.gmres_m, o.max_restarts) == (2, 128, -1.0, 1.0, 0.0, 50, 20)
    assert o.tol == 1e-10 and o.precision == K.KFBI_FP64


def test_bad_arguments_are_rejected_on_the_host(lib):
    o = K.default_options()
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    # null interface pointers
    assert lib.kfbi_setup(ctypes.byref(o), 64, None, None, None, None, ctypes.byref(h)) == 1
    # unsupported grid size (not 2^a or 3 * 2^a)
    o.N = 100
    assert lib.kfbi_setup(ctypes.byref(o), 64, dummy, dummy, dummy, None, ctypes.byref(h)) == 1
    assert b"N = 100" in lib.kfbi_last_error()
    o.N = 128
    o.dim = 4
    assert lib.kfbi_setup(ctypes.byref(o), 64, dummy, dummy, dummy, None, ctypes.byref(h)) == 8
    assert not h.value
    # 3-D grids stop at N = 512
    o.dim, o.N = 3, 1024
    assert lib.kfbi_setup(ctypes.byref(o), 64, dummy, dummy, dummy, None, ctypes.byref(h)) == 1
    assert b"512" in lib.kfbi_last_error()
    assert not h.value
    # unknown solver precision
    o.dim, o.N, o.precision = 2, 128, 99
    assert lib.kfbi_setup(ctypes.byref(o), 64, dummy, dummy, dummy, None, ctypes.byref(h)) == 1
    assert not h.value
    assert lib.kfbi_apply_layer_potential(None, 0, 0, dummy, dummy, None) == 1
    assert lib.kfbi_batch_create(None, 0, ctypes.byref(h)) == 1
    # batches hold handles without touching them: stand-in handles test the list checks
    fake = (ctypes.c_void_p * 3)(64, 128, 64)
    assert lib.kfbi_batch_create(fake, 3, ctypes.byref(h)) == 1 and not h.value
    assert b"more than once" in lib.kfbi_last_error()
    assert lib.kfbi_batch_create(fake, 2, ctypes.byref(h)) == 0 and h.value
    assert lib.kfbi_batch_destroy(h) == 0
    # null handles: KFBI_ERR_ARG with a message naming the entry point
    info, times = K.CtxInfo(), K.StageTimes()
    for name, call in (("kfbi_destroy", lambda: lib.kfbi_destroy(None)),
                       ("kfbi_get_info", lambda: lib.kfbi_get_info(None, ctypes.byref(info))),
                       ("kfbi_get_inside_mask", lambda: lib.kfbi_get_inside_mask(None, dummy, None)),
                       ("kfbi_profile", lambda: lib.kfbi_profile(None, 1)),
                       ("kfbi_profile_read", lambda: lib.kfbi_profile_read(None, ctypes.byref(times))),
                       ("kfbi_batch_destroy", lambda: lib.kfbi_batch_destroy(None)),
                       ("kfbi_solve_neumann_bvp",
                        lambda: lib.kfbi_solve_neumann_bvp(None, dummy, dummy, dummy, dummy, None,
                                                           None, None))):
        assert call() == 1, name
        assert lib.kfbi_last_error().decode().startswith(name), name


def test_product_path_does_not_import_the_oracle():
    """The binding, build script and CUDA sources never reach into oracle/."""
    pkg = os.path.dirname(K.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_binding_constants_match_the_header():
    """Every enum value the binding defines is the one include/kfbi.h declares."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "kfbi.h")).read()
    declared = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(KFBI_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    bound = {k: v for k, v in vars(K).items() if k.startswith("KFBI_") and isinstance(v, int)
             and k in declared}
    assert {"KFBI_FP64", "KFBI_MIXED_FP32", "KFBI_TF32X3", "KFBI_DOUBLE_LAYER"} <= set(bound)
    for k, v in bound.items():
        assert declared[k] == v, k


def test_batch_solve_checks_its_tensor_lists_before_the_library():
    """The binding's batch_solve refuses lists of the wrong length, dtype or size before any
    library call (the library reads one pointer per (problem, rhs) from each list)."""
    import types
    import torch

    class Stand:
        dim, dev = 2, "cpu"

        def __init__(self, N, M):
            self.N, self.M, self.torch = N, M, torch
            self._out = types.MethodType(K.Kfbi2D._out, self)

    ctxs = [Stand(32, 64), Stand(64, 128)]
    g = lambda c: torch.zeros((c.N + 1) ** 2, dtype=torch.float64)
    v = lambda c: torch.zeros(c.M, dtype=torch.float64)
    fg = [g(c) for c in ctxs for _ in range(2)]
    fc = [v(c) for c in ctxs for _ in range(2)]
    with pytest.raises(ValueError, match="g_ctrls must hold 4"):
        K.batch_solve(ctxs, fg, fc, fc[:3], fg, 2)
    bad = list(fc)
    bad[3] = torch.zeros(64, dtype=torch.float64)            # problem 1 has M = 128
    with pytest.raises(ValueError, match=r"g_ctrls\[3\]"):
        K.batch_solve(ctxs, fg, fc, bad, fg, 2)
    bad = list(fg)
    bad[0] = bad[0].float()
    with pytest.raises(ValueError, match=r"u_grids\[0\]"):
        K.batch_solve(ctxs, fg, fc, fc, bad, 2)


def test_binding_checks_input_and_output_sizes_before_the_library():
    """Each context method refuses an input or a caller-supplied output whose size is not
    the one the library reads or writes (grid (N+1)^dim, M values at the points), before
    any library call; stand-in contexts carry only the sizes."""
    import types
    import torch

    class Stand:
        dev = "cpu"

        def __init__(self, N, M, dim):
            self.N, self.M, self.dim, self.torch = N, M, dim, torch
            for f in ("_vec", "_out", "_grid", "_new"):
                setattr(self, f, types.MethodType(getattr(K.Kfbi2D, f), self))

    z = lambda n: torch.zeros(n, dtype=torch.float64)
    for N, M, dim in ((32, 64, 2), (16, 300, 3)):
        c = Stand(N, M, dim)
        G = (N + 1) ** dim
        calls = {
            "density": lambda: K.Kfbi2D.apply_layer_potential(c, z(M - 1)),
            "f_grid": lambda: K.Kfbi2D.apply_volume(c, z(G + 1), z(M)),
            "f_ctrl": lambda: K.Kfbi2D.solve_bvp(c, z(G), z(M + 1), z(M)),
            "g_ctrl": lambda: K.Kfbi2D.solve_bvp(c, z(G), z(M), z(1)),
            "u_out": lambda: K.Kfbi2D.solve_bvp(c, z(G), z(M), z(M), u_out=z(G - 1)),
            "dens_out": lambda: K.Kfbi2D.solve_bvp(c, z(G), z(M), z(M), u_out=z(G),
                                                   dens_out=z(M).float()),
            "gn_ctrl": lambda: K.Kfbi2D.solve_neumann_bvp(c, z(G), z(M), z(2 * M)),
            "b_grid": lambda: K.Kfbi2D.box_solve(c, z(N)),
        }
        for what, call in calls.items():
            with pytest.raises(ValueError, match=what):
                call()
    with pytest.raises(ValueError, match="b_grid"):
        K.box_solve_static(64, z(65 * 65))                  # a host tensor


def test_contexts_check_the_interface_shapes_before_any_device_work():
    import numpy as np
    with pytest.raises(ValueError, match=r"\(M, 2\)"):
        K.Kfbi2D(np.zeros((10, 2)), np.zeros((10, 3)), np.zeros(10), 32)
    with pytest.raises(ValueError, match="M x 1"):
        K.Kfbi2D(np.zeros((10, 2)), np.zeros((10, 2)), np.zeros(9), 32)
    with pytest.raises(ValueError, match="M x 6"):
        K.Kfbi3D(np.zeros((10, 3)), np.zeros((10, 3)), np.zeros((10, 3)), 32)
