"""Python binding of libkfbi (include/kfbi.h): GB300 kernel-free boundary integral method.

Argument marshalling only: every step of the method runs in the CUDA library.  PyTorch
provides device memory and streams.  If the library has not been built the binding
raises instead of falling back to anything else.

Low-level functions carry the C names (kfbi_setup, kfbi_apply_layer_potential, ...) and
take raw device pointers; `Kfbi2D` wraps one context with torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkfbi.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "kfbi.h")

KFBI_OK = 0
KFBI_ERR_NOT_CONVERGED = 5
KFBI_FP64 = 0
KFBI_MIXED_FP32 = 1
KFBI_FP32_REFINED = 2
KFBI_FP32_REFINED_ONCE = 3
KFBI_TF32X3 = 4
KFBI_STATIC_MAX_N = 1024                  # limits of kfbi_box_solve_static (kfbi.h)
KFBI_STATIC_SCRATCH_BYTES = 9 << 20
KFBI_DOUBLE_LAYER = 0
KFBI_SINGLE_LAYER = 1
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_GEOMETRY", 3: "ERR_NOMEM", 4: "ERR_CUDA",
          5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_NUMERIC", 8: "ERR_UNSUPPORTED"}


class KfbiError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}".strip())


class Options(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("kappa", ctypes.c_double), ("precision", ctypes.c_int),
                ("gmres_m", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("applies_fp64", ctypes.c_int), ("applies_low", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CtxInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("n_crossings_x", ctypes.c_int),
                ("n_crossings_y", ctypes.c_int), ("n_irregular", ctypes.c_int),
                ("n_inside", ctypes.c_int), ("device_bytes", ctypes.c_int64),
                ("dst_variant", ctypes.c_int * 4), ("dim", ctypes.c_int),
                ("n_crossings_z", ctypes.c_int), ("tri_first_mode", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["dst_variant"] = list(self.dst_variant)
        return d


NSTAGES = 16


class StageTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NSTAGES), ("launches", ctypes.c_longlong * NSTAGES),
                ("nstages", ctypes.c_int)]


_LIB = None
P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
_SIGS = {
    "kfbi_default_options": (None, [ctypes.POINTER(Options)]),
    "kfbi_setup": (I, [ctypes.POINTER(Options), ctypes.c_int64, P, P, P, P, ctypes.POINTER(P)]),
    "kfbi_apply_layer_potential": (I, [P, I, I, P, P, P]),
    "kfbi_apply_volume": (I, [P, I, P, P, P, P]),
    "kfbi_interface_solve": (I, [P, I, P, P, P, P, P, P, P]),
    "kfbi_box_solve": (I, [P, I, P, P, P]),
    "kfbi_box_solve_static": (I, [I, D, D, D, I, P, P, P]),
    "kfbi_box_solve_static_check": (I, [P]),
    "kfbi_solve_bvp": (I, [P, P, P, P, P, P, ctypes.POINTER(SolveInfo), P]),
    "kfbi_solve_neumann_bvp": (I, [P, P, P, P, P, P, ctypes.POINTER(SolveInfo), P]),
    "kfbi_apply_layer_potential_dn": (I, [P, I, I, P, P, P]),
    "kfbi_apply_volume_dn": (I, [P, I, P, P, P, P]),
    "kfbi_get_inside_mask": (I, [P, P, P]),
    "kfbi_get_info": (I, [P, ctypes.POINTER(CtxInfo)]),
    "kfbi_set_solver": (I, [P, I, I, I, D, D]),
    "kfbi_destroy": (I, [P]),
    "kfbi_status_string": (ctypes.c_char_p, [I]),
    "kfbi_last_error": (ctypes.c_char_p, []),
    "kfbi_batch_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P)]),
    "kfbi_batch_solve": (I, [P, I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                             ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(SolveInfo), P]),
    "kfbi_batch_destroy": (I, [P]),
    "kfbi_measure_fma_peak": (I, [I, ctypes.POINTER(D), P]),
    "kfbi_profile": (I, [P, I]),
    "kfbi_profile_read": (I, [P, ctypes.POINTER(StageTimes)]),
    "kfbi_stage_name": (ctypes.c_char_p, [I]),
}


def header_symbols(path: str = HEADER):
    """Names of the functions include/kfbi.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kfbi_[a-z_0-9]+)\s*\(", txt)))


def lib():
    """The loaded libkfbi.so (raises if it has not been built: no fallback exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str):
    if status != KFBI_OK:
        raise KfbiError(status, where, lib().kfbi_last_error().decode(errors="replace"))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def default_options() -> Options:
    o = Options()
    lib().kfbi_default_options(ctypes.byref(o))
    return o


class Kfbi2D:
    """One 2-D KFBI context: interface + grid, device-resident setup.

    pts, normals: (M, 2) and curv: (M,) arrays (numpy or torch); they are copied to the
    device, then kfbi_setup builds the geometry on the GPU."""

    dim = 2

    def __init__(self, pts, normals, curv, N, kappa=0.0, lo=-1.0, hi=1.0, precision=KFBI_FP64,
                 gmres_m=50, max_restarts=20, tol=1e-10, inner_tol=1e-5, stream=None):
        import torch
        self.torch = torch
        # kfbi_setup copies M x dim points and normals and M x (1 or 6) curvature values
        P, Nr, C = (torch.as_tensor(a, dtype=torch.float64) for a in (pts, normals, curv))
        ncurv = 1 if self.dim == 2 else 6
        if (P.dim() != 2 or P.shape[1] != self.dim or tuple(Nr.shape) != tuple(P.shape)
                or C.numel() != P.shape[0] * ncurv):
            raise ValueError(f"pts and normals must be (M, {self.dim}) and the curvature data "
                             f"M x {ncurv} values; got {tuple(P.shape)}, {tuple(Nr.shape)}, "
                             f"{tuple(C.shape)}")
        self.dev = torch.device("cuda", torch.cuda.current_device())
        t = lambda a: a.contiguous().to(self.dev)
        self.pts, self.nrm, self.curv = t(P), t(Nr), t(C)
        self.M = int(self.pts.shape[0])
        self.N = int(N)
        self.stream = stream
        o = default_options()
        o.dim = self.dim
        o.N, o.lo, o.hi, o.kappa = int(N), float(lo), float(hi), float(kappa)
        o.precision, o.gmres_m, o.max_restarts = int(precision), int(gmres_m), int(max_restarts)
        o.tol, o.inner_tol = float(tol), float(inner_tol)
        self.opt = o
        h = ctypes.c_void_p()
        _check(lib().kfbi_setup(ctypes.byref(o), self.M, _ptr(self.pts), _ptr(self.nrm),
                                _ptr(self.curv), _stream_ptr(stream), ctypes.byref(h)), "kfbi_setup")
        self.handle = h

    # ------------------------------------------------------------------ helpers
    def _vec(self, a, numel, what):
        """An input as a contiguous float64 tensor on this context's device, of numel values
        (the library reads exactly that many)."""
        v = self.torch.as_tensor(a, dtype=self.torch.float64).contiguous().to(self.dev)
        if v.numel() != numel:
            raise ValueError(f"{what} must have {numel} values, got {v.numel()}")
        return v

    def _grid(self, dtype=None):
        return self.torch.empty((self.N + 1,) * self.dim, dtype=dtype or self.torch.float64,
                                device=self.dev)

    def _new(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.dev)

    def _out(self, out, numel, what="out"):
        """A caller-supplied buffer: contiguous float64 on this context's device."""
        t = self.torch
        if not (isinstance(out, t.Tensor) and out.dtype == t.float64 and out.is_contiguous()
                and out.device == t.device(self.dev) and out.numel() == numel):
            raise ValueError(f"{what} must be a contiguous float64 tensor of {numel} elements "
                             f"on {self.dev}")
        return out

    # ------------------------------------------------------------------ API
    def apply_layer_potential(self, density, layer=KFBI_DOUBLE_LAYER, precision=KFBI_FP64, out=None):
        d = self._vec(density, self.M, "density")
        out = self._new(self.M) if out is None else self._out(out, self.M)
        _check(lib().kfbi_apply_layer_potential(self.handle, int(layer), int(precision), _ptr(d),
                                                _ptr(out), _stream_ptr(self.stream)),
               "kfbi_apply_layer_potential")
        return out

    def apply_layer_potential_dn(self, density, layer=KFBI_SINGLE_LAYER, precision=KFBI_FP64,
                                 out=None):
        """kfbi_apply_layer_potential_dn: d_n v^+ at the control points (2-D)."""
        d = self._vec(density, self.M, "density")
        out = self._new(self.M) if out is None else self._out(out, self.M)
        _check(lib().kfbi_apply_layer_potential_dn(self.handle, int(layer), int(precision), _ptr(d),
                                                   _ptr(out), _stream_ptr(self.stream)),
               "kfbi_apply_layer_potential_dn")
        return out

    def apply_volume_dn(self, f_grid, f_ctrl, precision=KFBI_FP64):
        """kfbi_apply_volume_dn: d_n (Y f)^+ at the control points (2-D)."""
        fg, fc = self._vec(f_grid, (self.N + 1) ** self.dim, "f_grid"), self._vec(f_ctrl, self.M, "f_ctrl")
        out = self._new(self.M)
        _check(lib().kfbi_apply_volume_dn(self.handle, int(precision), _ptr(fg), _ptr(fc),
                                          _ptr(out), _stream_ptr(self.stream)), "kfbi_apply_volume_dn")
        return out

    def solve_neumann_bvp(self, f_grid, f_ctrl, gn_ctrl, u_out=None, dens_out=None,
                          allow_not_converged=False):
        """kfbi_solve_neumann_bvp: (u grid, single-layer density psi, info) (2-D)."""
        fg, fc = self._vec(f_grid, (self.N + 1) ** self.dim, "f_grid"), self._vec(f_ctrl, self.M, "f_ctrl")
        gc = self._vec(gn_ctrl, self.M, "gn_ctrl")
        u = self._grid() if u_out is None else self._out(u_out, (self.N + 1) ** self.dim, "u_out")
        psi = self._new(self.M) if dens_out is None else self._out(dens_out, self.M, "dens_out")
        info = SolveInfo()
        st = lib().kfbi_solve_neumann_bvp(self.handle, _ptr(fg), _ptr(fc), _ptr(gc), _ptr(u),
                                          _ptr(psi), ctypes.byref(info), _stream_ptr(self.stream))
        if not (allow_not_converged and st == KFBI_ERR_NOT_CONVERGED):
            _check(st, "kfbi_solve_neumann_bvp")
        return u, psi, info.as_dict()

    def apply_volume(self, f_grid, f_ctrl, precision=KFBI_FP64):
        fg, fc = self._vec(f_grid, (self.N + 1) ** self.dim, "f_grid"), self._vec(f_ctrl, self.M, "f_ctrl")
        out = self._new(self.M)
        _check(lib().kfbi_apply_volume(self.handle, int(precision), _ptr(fg), _ptr(fc), _ptr(out),
                                       _stream_ptr(self.stream)), "kfbi_apply_volume")
        return out

    def interface_solve(self, density=None, f_grid=None, f_ctrl=None, precision=KFBI_FP64):
        d = None if density is None else self._vec(density, self.M, "density")
        fg = None if f_grid is None else self._vec(f_grid, (self.N + 1) ** self.dim, "f_grid")
        fc = None if f_ctrl is None else self._vec(f_ctrl, self.M, "f_ctrl")
        rhs, v, out = self._grid(), self._grid(), self._new(self.M)
        _check(lib().kfbi_interface_solve(self.handle, int(precision), _ptr(d), _ptr(fg), _ptr(fc),
                                          _ptr(rhs), _ptr(v), _ptr(out), _stream_ptr(self.stream)),
               "kfbi_interface_solve")
        return rhs, v, out

    def box_solve(self, b_grid, precision=KFBI_FP64, out=None):
        b = self._vec(b_grid, (self.N + 1) ** self.dim, "b_grid")
        v = self._grid() if out is None else self._out(out, (self.N + 1) ** self.dim)
        _check(lib().kfbi_box_solve(self.handle, int(precision), _ptr(b), _ptr(v),
                                    _stream_ptr(self.stream)), "kfbi_box_solve")
        return v

    def set_solver(self, precision=KFBI_FP64, gmres_m=50, max_restarts=20, tol=1e-10, inner_tol=1e-5):
        _check(lib().kfbi_set_solver(self.handle, int(precision), int(gmres_m), int(max_restarts),
                                     float(tol), float(inner_tol)), "kfbi_set_solver")

    def solve_bvp(self, f_grid, f_ctrl, g_ctrl, u_out=None, dens_out=None, allow_not_converged=False):
        fg, fc = self._vec(f_grid, (self.N + 1) ** self.dim, "f_grid"), self._vec(f_ctrl, self.M, "f_ctrl")
        gc = self._vec(g_ctrl, self.M, "g_ctrl")
        u = self._grid() if u_out is None else self._out(u_out, (self.N + 1) ** self.dim, "u_out")
        phi = self._new(self.M) if dens_out is None else self._out(dens_out, self.M, "dens_out")
        info = SolveInfo()
        st = lib().kfbi_solve_bvp(self.handle, _ptr(fg), _ptr(fc), _ptr(gc), _ptr(u), _ptr(phi),
                                  ctypes.byref(info), _stream_ptr(self.stream))
        if not (allow_not_converged and st == KFBI_ERR_NOT_CONVERGED):
            _check(st, "kfbi_solve_bvp")
        return u, phi, info.as_dict()

    def inside_mask(self):
        m = self._grid(self.torch.uint8)
        _check(lib().kfbi_get_inside_mask(self.handle, _ptr(m), _stream_ptr(self.stream)),
               "kfbi_get_inside_mask")
        return m

    def info(self):
        i = CtxInfo()
        _check(lib().kfbi_get_info(self.handle, ctypes.byref(i)), "kfbi_get_info")
        return i.as_dict()

    def profile(self, enable=True):
        """Start (clearing the totals) or stop per-stage event timing."""
        _check(lib().kfbi_profile(self.handle, 1 if enable else 0), "kfbi_profile")

    def profile_read(self):
        """{stage name: (ms, launches)} since the last profile(True)."""
        t = StageTimes()
        _check(lib().kfbi_profile_read(self.handle, ctypes.byref(t)), "kfbi_profile_read")
        return {lib().kfbi_stage_name(i).decode(): (t.ms[i], t.launches[i]) for i in range(t.nstages)}

    def close(self):
        if getattr(self, "handle", None):
            lib().kfbi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Kfbi3D(Kfbi2D):
    """One 3-D KFBI context: the interface is given by its intersections with the grid lines
    of the box [lo, hi]^3 (pts, normals: (P, 3); shape: (P, 6) packed symmetric shape
    operators Sxx, Syy, Szz, Sxy, Sxz, Syz with dn = S dx), which are also the control
    points; grids are (N+1)^3 indexed [k, j, i].  Same methods as Kfbi2D (double layer
    and volume potentials, interface/box solves, the Dirichlet BVP)."""

    dim = 3

    def __init__(self, pts, normals, shape, N, kappa=0.0, **kw):
        super().__init__(pts, normals, shape, N, kappa, **kw)


def box_solve_static(N, b_grid, kappa=0.0, lo=-1.0, hi=1.0, precision=KFBI_FP64, out=None,
                     stream=None):
    """kfbi_box_solve_static: the box solve without a context, its workspace in the
    library's static device array (nothing allocated by the library).  b_grid and out
    are (N+1, N+1) float64 CUDA tensors (out is created here when None)."""
    import torch

    def grid_ok(t):
        return (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == (int(N) + 1) ** 2)

    if not grid_ok(b_grid):
        raise ValueError(f"b_grid must be a contiguous float64 CUDA tensor of (N+1)^2 = "
                         f"{(int(N) + 1) ** 2} values")
    out = torch.empty_like(b_grid) if out is None else out
    if not (grid_ok(out) and out.device == b_grid.device):
        raise ValueError("out must be a contiguous float64 tensor of b_grid's size on its device")
    _check(lib().kfbi_box_solve_static(int(N), float(lo), float(hi), float(kappa), int(precision),
                                       _ptr(b_grid), _ptr(out), _stream_ptr(stream)),
           "kfbi_box_solve_static")
    return out


def measure_fma_peak(fp64: bool, stream=None) -> float:
    """kfbi_measure_fma_peak: measured FMA throughput of the current device in TFLOP/s."""
    out = ctypes.c_double()
    _check(lib().kfbi_measure_fma_peak(1 if fp64 else 0, ctypes.byref(out), _stream_ptr(stream)),
           "kfbi_measure_fma_peak")
    return out.value


def box_solve_static_check(stream=None):
    """kfbi_box_solve_static_check: synchronises the stream and raises KfbiError
    (ERR_TIMEOUT) if a bounded wait of an earlier static box solve gave up."""
    _check(lib().kfbi_box_solve_static_check(_stream_ptr(stream)), "kfbi_box_solve_static_check")


def batch_solve(ctxs, f_grids, f_ctrls, g_ctrls, u_grids, nrhs, stream=None, dens_out=None):
    """kfbi_batch_create / kfbi_batch_solve / kfbi_batch_destroy over Kfbi2D contexts.
    The per-(problem, rhs) lists hold device tensors, problem-major; dens_out (optional)
    is a list of the same length of float64 tensors of M_p values for the densities.  The
    lists are checked (length, dtype, layout, device, size per problem) before the call: the
    library reads one pointer per (problem, rhs) from each."""
    n = len(ctxs)
    lists = {"f_grids": f_grids, "f_ctrls": f_ctrls, "g_ctrls": g_ctrls, "u_grids": u_grids}
    if dens_out is not None:
        lists["dens_out"] = dens_out
    for name, ts in lists.items():
        if len(ts) != n * nrhs:
            raise ValueError(f"{name} must hold {n * nrhs} tensors (problem-major), got {len(ts)}")
    for p, c in enumerate(ctxs):
        size = {"f_grids": (c.N + 1) ** c.dim, "u_grids": (c.N + 1) ** c.dim,
                "f_ctrls": c.M, "g_ctrls": c.M, "dens_out": c.M}
        for r in range(nrhs):
            for name, ts in lists.items():
                c._out(ts[p * nrhs + r], size[name], f"{name}[{p * nrhs + r}]")
    arr = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    b = ctypes.c_void_p()
    _check(lib().kfbi_batch_create(arr, n, ctypes.byref(b)), "kfbi_batch_create")
    try:
        mk = lambda ts: (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
        infos = (SolveInfo * (n * nrhs))()
        st = lib().kfbi_batch_solve(b, int(nrhs), mk(f_grids), mk(f_ctrls), mk(g_ctrls),
                                    mk(u_grids), None if dens_out is None else mk(dens_out),
                                    infos, _stream_ptr(stream))
        if st not in (KFBI_OK, KFBI_ERR_NOT_CONVERGED):
            _check(st, "kfbi_batch_solve")
        return [i.as_dict() for i in infos]
    finally:
        lib().kfbi_batch_destroy(b)
