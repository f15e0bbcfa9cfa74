#!/usr/bin/env python
"""Benchmark of the KFBI Dirichlet BVP solve on one GB300 (or N independent replicas).

Metric: KFBI full-solve ms & grid-pts/s per potential apply, mixed precision vs FP64 at
the same error.  One step = one full BVP solve of the 2-D modified Helmholtz problem
(flower r = 0.5 + 0.15 cos 5t, N = 4096 cells per side, M = 8192 control points,
kappa = 1, manufactured u = exp(x) sin(2y), GMRES(50) to 1e-10): volume term, GMRES with
the layer-potential apply as its operator, final grid solution.  The geometry setup is
timed separately (setup_ms).

value = (N+1)^2 * (layer-potential applies per solve) / (solve time), summed over ranks
(grid points per second per apply); ms_per_step is the full-solve time.

--impl reference times the FP64 CPU oracle on the host cores on the same workload: each
step is one oracle layer-potential apply (the oracle's full solve at N = 4096 would take
minutes), reported in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KFBI full-solve ms & grid-pts/s per potential apply: mixed vs FP64, same error"
UNIT = "grid-pts/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_FP64_GFLOPS = 1250.0
NOMINAL_TF32_PER_BF16 = 1.1 / 2.25     # dense tensor rates, TF32 : BF16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfbi", choices=["kfbi", "reference"])
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--kappa", type=float, default=1.0)
    ap.add_argument("--shape", default="flower", choices=["flower", "ellipse"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--n3d", default="128,256,512",
                    help="grid sizes of the 3-D companion measurement, comma separated (0: skip)")
    ap.add_argument("--ntc", type=int, default=1024,
                    help="grid size of the tensor-core box-solve measurement (0: skip)")
    ap.add_argument("--batch", type=int, default=256,
                    help="problems in the batched companion measurement (0: skip)")
    ap.add_argument("--nneu", type=int, default=2048,
                    help="grid size of the Neumann BVP companion measurement (0: skip)")
    return ap.parse_args()


def workload_name(a):
    return (f"2-D modified Helmholtz Dirichlet BVP (Lap u - kappa^2 u = f), {a.shape} interface, "
            f"N={a.N} ({a.N + 1}^2 nodes), M={2 * a.N}, kappa={a.kappa:g}, u=exp(x)sin(2y), "
            f"double-layer BIE by GMRES(50) to 1e-10")


# ------------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# the CUDA sources that define each kernel (the y-pass span: the filter kernel in
# dst_ycol.cu and the low-mode column kernel in dst_impl.cuh)
YPASS = "ycol_filter_kernel+ycol_lines_kernel"
KERNEL_SOURCE = {"rows_kernel": ("dst_impl.cuh",), "yline_kernel": ("dst_impl.cuh",),
                 "cols_kernel": ("dst_impl.cuh",), "transpose_vec_kernel": ("dst_impl.cuh",),
                 "ytri_kernel": ("dst_tri.cu",), "sparse_rows_kernel": ("apply2d.cu",),
                 "sparse_out_kernel": ("apply2d.cu",), "ds_residual4_kernel": ("apply2d.cu",),
                 YPASS: ("dst_ycol.cu", "dst_impl.cuh")}


def kernel_source_hash(kernel):
    """First 12 hex digits of the SHA-256 of the CUDA sources that define `kernel`."""
    h = hashlib.sha256()
    for src in KERNEL_SOURCE.get(kernel.split("<")[0], ("dst_impl.cuh",)):
        h.update(open(os.path.join(ROOT, "paper_2404_15249_gb300", "csrc", src), "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel, N):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash(kernel)
    for line in open(p):
        f = line.split()
        if len(f) >= 5 and not line.startswith("#") and f[0] == kernel and f[1] == src:
            n_cap, bytes_cap = int(f[2]), float(f[3])
            return bytes_cap * (N * N) / (n_cap * n_cap)      # scale by grid units
    return None


STAGE_KERNEL = {"dst_rows_f32": ("rows_kernel<float>", 4), "dst_cols_f32": ("cols_kernel<float>", 4),
                "dst_rows_f64": ("rows_kernel<double>", 8), "dst_cols_f64": ("cols_kernel<double>", 8),
                "transpose": ("transpose_vec_kernel<float>", 4),
                "dst_tri_f32": ("ytri_kernel<float>", 4)}


def roofline(stage_ms, N, variants, tri_k0):
    """Dominant stage of the timed region -> roofline entry for its kernel.  The column
    stage is yline_kernel when the autotuner chose the transposed column pass (variant bit
    2; the transposes are then their own stage), else cols_kernel.  In FP32 the y-line
    transform pair runs on the x-modes below tri_k0 and the tridiagonal y-solve on the
    rest, so their algorithmic bytes cover tri_k0 and N - tri_k0 lines."""
    kernels = dict(STAGE_KERNEL)
    lines = {k: N for k in kernels}
    if variants[1] & 4:
        kernels["dst_cols_f32"] = ("yline_kernel<float>", 4)
        lines["dst_cols_f32"] = tri_k0
    lines["dst_tri_f32"] = N - tri_k0
    if variants[1] & 8:
        # the row-layout y-pass, timed as one span over its two streams: the filters of the
        # modes from tri_k0 up and the transform pair of the modes below, every unknown of
        # the grid read and written once
        kernels["dst_tri_f32"] = (YPASS, 4)
        lines["dst_tri_f32"] = N
    if variants[3] & 4:
        kernels["dst_cols_f64"] = ("yline_kernel<double>", 8)
    cand = {k: v for k, v in stage_ms.items() if k in kernels and v[1] > 0 and v[0] > 0}
    if not cand:
        return None
    name = max(cand, key=lambda k: cand[k][0])
    ms, launches = cand[name]
    avg_s = ms / launches / 1e3
    kernel, esize = kernels[name]
    if name.endswith("f64"):
        # FP64 transforms are bound by the FP64 ALU: 5 N log2 N flops per complex FFT of
        # length N per line (rows: 1 FFT per line, columns: 2)
        ffts = 1 if "rows" in name else 2
        flops = ffts * N * 5.0 * N * math.log2(N)
        return {"bound": "alu", "kernel": kernel, "achieved": flops / avg_s / 1e12,
                "peak": NOMINAL_FP64_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": flops / avg_s / 1e12 / (NOMINAL_FP64_GFLOPS / 1e3),
                "peak_source": "nominal FP64", "traffic": None, "launches": launches,
                "avg_launch_us": avg_s * 1e6}
    peak, src = peaks()
    nbytes = 2.0 * N * lines[name] * esize   # every unknown of its lines read and written once
    ach = nbytes / avg_s / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_source": src, "traffic": traffic_for(kernel, N),
            "algorithmic_bytes": nbytes, "launches": launches, "avg_launch_us": avg_s * 1e6}


def fp64_roofline(stage_ms, N, alu):
    """Dominant FP64 transform stage of the plain FP64 solve against the measured FP64 FMA
    throughput: 5 N log2 N flops per complex FFT of length N (the conventional count), one
    FFT per line for the row pass and two for the y-transform pair, N lines per launch."""
    cand = {k: v for k, v in stage_ms.items()
            if k in ("dst_rows_f64", "dst_cols_f64") and v[1] > 0 and v[0] > 0}
    if not cand or not alu:
        return None
    name = max(cand, key=lambda k: cand[k][0])
    ms, launches = cand[name]
    avg_s = ms / launches / 1e3
    ffts = 1 if "rows" in name else 2
    flops = ffts * N * 5.0 * N * math.log2(N)
    ach = flops / avg_s / 1e12
    return {"bound": "alu", "kernel": "rows_kernel<double>" if "rows" in name else "yline_kernel<double>",
            "achieved": ach, "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
            "frac": ach / alu["fp64_tflops"], "peak_source": "measured (kfbi_measure_fma_peak, FP64)",
            "launches": launches, "avg_launch_us": avg_s * 1e6,
            "stage_share": ms / sum(v[0] for v in stage_ms.values() if v[1])}


# stages whose kernels carry the box solve's sine transforms and y-solves (Alg. 4)
DST_STAGES = ("dst_rows_f32", "dst_cols_f32", "dst_tri_f32", "sparse_x_f32", "transpose")


def dst_bytes(stage_ms, N):
    """Algorithmic bytes of the box solves behind the launch counts in stage_ms: 24 B per
    interior unknown per dense-right-hand-side box solve and 16 B per plain apply's
    sparse one (a plain apply runs one sparse x-transform and one row pass, a dense box
    solve two row passes); returns (bytes, dense solves, sparse solves)."""
    sparse = stage_ms.get("sparse_x_f32", (0.0, 0))[1]
    rows = stage_ms.get("dst_rows_f32", (0.0, 0))[1]
    dense = max(rows - sparse, 0) / 2.0
    return (24.0 * dense + 16.0 * sparse) * float(N - 1) ** 2, dense, sparse


def batch_dst_roofline(per_ctx, wall_ms):
    """The box-solve bytes of a whole batch against the HBM roofline: per_ctx holds
    (N, stage_ms) of every context over one batch (launch counts), wall_ms the batch's
    wall time without stage events; concurrent problems overlap, so this is the whole
    job's rate, not one kernel's."""
    total = sum(dst_bytes(st, n)[0] for n, st in per_ctx)
    if wall_ms <= 0 or total <= 0:
        return None
    peak, src = peaks()
    ach = total / (wall_ms / 1e3) / 1e9
    return {"bound": "hbm", "algorithmic_bytes": total, "wall_ms": wall_ms, "achieved": ach,
            "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_source": src}


def dst_stage_roofline(stage_ms, N, solves):
    """The box-solve (DST) stage of the mixed solve as a whole against the HBM roofline:
    algorithmic bytes 24 B per interior unknown for a box solve of a dense right-hand side
    (three passes, each reading and writing the FP32 grid once) and 16 B for a plain
    double-layer apply (its first x-transform reads only the irregular nodes and writes
    the grid, the y-pass reads and writes it, the last x-transform reads it and writes
    only the stencil nodes), over the summed device time of the stage's kernels.  The
    y-pass runs two streams at once and is timed as one wall-clock span, so no interval
    is counted twice.  A plain apply runs one sparse x-transform and one row pass, a dense
    box solve two row passes, so the counts follow from the launches of the two kernels."""
    ms = sum(stage_ms[k][0] for k in DST_STAGES if k in stage_ms)
    if ms <= 0 or solves <= 0:
        return None
    nbytes, dense, sparse = dst_bytes(stage_ms, N)
    nbytes, dense, sparse = nbytes / solves, dense / solves, sparse / solves
    peak, src = peaks()
    ach = nbytes / (ms / solves / 1e3) / 1e9
    return {"bound": "hbm", "stage": "box solves of one mixed BVP solve (" + ", ".join(
                k for k in DST_STAGES if k in stage_ms and stage_ms[k][1]) + ")",
            "dense_box_solves": dense, "sparse_box_solves": sparse,
            "algorithmic_bytes": nbytes, "ms": ms / solves, "achieved": ach, "peak": peak,
            "unit": "GB/s", "frac": ach / peak, "peak_source": src}


# ------------------------------------------------------------------------ arms
def pipelined_e2e_ms(ctx, torch, st, flush, steps, h_in, h_out):
    """Milliseconds per step of `steps` BVP solves through the API from and to pinned host
    buffers, timed as one region: step k+1's inputs are copied in and step k's results
    copied out on a copy stream while the solves run on `st` (two device buffers of each,
    events ordering every copy against the solve that produces or consumes it)."""
    cp = torch.cuda.Stream()
    d_in = [[torch.empty(x.shape, dtype=x.dtype, device=st.device) for x in h_in] for _ in range(2)]
    d_out = [[torch.empty(x.shape, dtype=x.dtype, device=st.device) for x in h_out] for _ in range(2)]
    h_res = [[torch.empty_like(x).pin_memory() for x in h_out] for _ in range(2)]
    loaded = [torch.cuda.Event() for _ in range(2)]      # inputs of buffer b on the device
    used = [torch.cuda.Event() for _ in range(2)]        # solve of buffer b done
    saved = [torch.cuda.Event() for _ in range(2)]       # results of buffer b on the host

    def load(b):
        cp.wait_event(used[b])
        with torch.cuda.stream(cp):
            for d, h in zip(d_in[b], h_in):
                d.copy_(h, non_blocking=True)
        loaded[b].record(cp)

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    cp.wait_stream(st)
    load(0)
    for k in range(steps):
        b = k % 2
        if k + 1 < steps:
            load(1 - b)                                  # next step's inputs, concurrently
        st.wait_event(loaded[b])
        st.wait_event(saved[b])                          # this buffer's last results are out
        flush.fill_(1.0)
        fg, fc, gc = d_in[b]
        ctx.solve_bvp(fg, fc, gc, u_out=d_out[b][0], dens_out=d_out[b][1])
        used[b].record(st)
        cp.wait_event(used[b])
        with torch.cuda.stream(cp):
            for h, d in zip(h_res[b], d_out[b]):
                h.copy_(d, non_blocking=True)
        saved[b].record(cp)
    st.wait_stream(cp)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself on one rank): the job's step time is that of
    its slowest replica."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, grid_points, applies, ms):
    """Grid points per second per apply summed over the world's replicas, each of which
    runs the same solve in ms milliseconds (the slowest rank's time)."""
    return world * grid_points * applies / (ms / 1e3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_applies(prob, budget_s=12.0, max_applies=4):
    """Time FP64 oracle double-layer applies on the host cores (bounded sample)."""
    import numpy as np
    import kfbi_workloads as W
    import oracle as O
    g = O.Geometry2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa)
    phi = W.random_density(prob.iface.M, seed=5)
    n, t0 = 0, time.perf_counter()
    while n < max_applies and (n == 0 or time.perf_counter() - t0 < budget_s):
        O.apply_double_layer(g, phi)
        n += 1
    dt = time.perf_counter() - t0
    return n, dt


def run_reference(a):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import kfbi_workloads as W
    import oracle as O
    prob = W.config_helmholtz(a.N, a.kappa, a.shape)
    g = O.Geometry2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, prob.N, prob.kappa)
    phi = W.random_density(prob.iface.M, seed=5)
    for _ in range(a.warmup):
        O.apply_double_layer(g, phi)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        O.apply_double_layer(g, phi)
    dt = (time.perf_counter() - t0) / a.steps
    value = (a.N + 1) ** 2 / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "N": a.N, "M": 2 * a.N, "kappa": a.kappa,
                       "step": "one FP64 oracle double-layer apply (numpy, host cores)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{a.steps} timed oracle applies at N={a.N}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_kfbi(a):
    import numpy as np
    import torch
    import kfbi_workloads as W
    import paper_2404_15249_gb300 as K

    rank, world, local = dist_info()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    N, M = a.N, 2 * a.N
    prob = W.config_helmholtz(N, a.kappa, a.shape)
    fg = torch.as_tensor(prob.f_grid(), device=dev)
    fc = torch.as_tensor(prob.f_ctrl(), device=dev)
    gc = torch.as_tensor(prob.g_ctrl(), device=dev)
    u = torch.empty((N + 1, N + 1), dtype=torch.float64, device=dev)
    phi = torch.empty(M, dtype=torch.float64, device=dev)
    u_exact = prob.u_grid()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, N, a.kappa,
                   precision=K.KFBI_MIXED_FP32, gmres_m=50, max_restarts=20, tol=1e-10)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    inside = ctx.inside_mask().cpu().numpy().astype(bool)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def err_inf(ut):
        return float(np.max(np.abs(ut.cpu().numpy() - u_exact)[inside]))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- mixed-precision solve (the timed path)
    for _ in range(a.warmup):
        ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
    st = torch.cuda.current_stream()
    ctx.profile(True)                 # clears the launch counters ...
    ctx.profile(False)                # ... which keep counting without per-launch events
    clocks = Clocks(local)
    clocks.start()
    barrier()
    step_ms, infos = [], []
    for _ in range(a.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _, _, info = ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
        e1.record(st)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    counted = ctx.profile_read()      # launches of the timed steps (no device times)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), dist, dev)
    applies = infos[-1]["applies_fp64"] + infos[-1]["applies_low"]
    err_mixed = err_inf(u)
    value = whole_job_rate(world, (N + 1) ** 2, applies, ms)

    # ---------------- the same solves again with CUDA events around every launch (on the
    # library's stream): per-stage device time and the dominant kernel's launch duration
    nprof = min(a.steps, 5)
    ctx.profile(True)
    for _ in range(nprof):
        flush.fill_(1.0)
        ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
    stages = ctx.profile_read()
    ctx.profile(False)

    # measured FMA throughput of this GPU (FP64 and FP32), the denominators of the ALU
    # rooflines of the FP64 transforms and of the FP32 transforms' arithmetic
    alu_peaks = {"fp64_tflops": K.measure_fma_peak(True), "fp32_tflops": K.measure_fma_peak(False),
                 "how": "kfbi_measure_fma_peak: 8 independent FMA chains per thread, every SM "
                        "full, best of 3 launches (2 flops per FMA)"}

    # ---------------- FP64 path on the same inputs (same error check, speedup)
    fp64 = {}
    if not a.no_fp64:
        ctx.set_solver(K.KFBI_FP64, 50, 20, 1e-10, 1e-5)
        ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
        t64 = []
        for _ in range(2):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, _, i64 = ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
            e1.record(st)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        ctx.profile(True)
        flush.fill_(1.0)
        ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
        st64 = ctx.profile_read()
        ctx.profile(False)
        fp64 = {"fp64_solve_ms": statistics.mean(t64), "err_inf_fp64": err_inf(u),
                "fp64_iterations": i64["iterations"],
                "speedup_vs_fp64": statistics.mean(t64) / ms,
                "fp64_stage_ms": {k: round(v[0], 4) for k, v in st64.items() if v[1]},
                "fp64_roofline": fp64_roofline(st64, N, alu_peaks)}
        ctx.set_solver(K.KFBI_MIXED_FP32, 50, 20, 1e-10, 1e-5)

    # ---------------- end to end through the API with host buffers
    e2e = None
    if not a.no_e2e:
        h_fg = torch.as_tensor(prob.f_grid()).pin_memory()
        h_fc = torch.as_tensor(prob.f_ctrl()).pin_memory()
        h_gc = torch.as_tensor(prob.g_ctrl()).pin_memory()
        h_u = torch.empty((N + 1, N + 1), dtype=torch.float64).pin_memory()
        h_phi = torch.empty(M, dtype=torch.float64).pin_memory()
        d_fg, d_fc, d_gc = torch.empty_like(fg), torch.empty_like(fc), torch.empty_like(gc)
        e2e_ms = []
        barrier()
        for _ in range(a.steps):             # one step at a time: copy in, solve, copy out
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            d_fg.copy_(h_fg, non_blocking=True)
            d_fc.copy_(h_fc, non_blocking=True)
            d_gc.copy_(h_gc, non_blocking=True)
            ctx.solve_bvp(d_fg, d_fc, d_gc, u_out=u, dens_out=phi)
            h_u.copy_(u, non_blocking=True)
            h_phi.copy_(phi, non_blocking=True)
            e1.record(st)
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
        serial = max_over_ranks(statistics.mean(e2e_ms), dist, dev)
        em = max_over_ranks(pipelined_e2e_ms(ctx, torch, st, flush, a.steps, (h_fg, h_fc, h_gc),
                                             (h_u, h_phi)), dist, dev)
        e2e = {"value": whole_job_rate(world, (N + 1) ** 2, applies, em), "unit": UNIT,
               "ms_per_step": em,
               "h2d_bytes_per_step": (h_fg.numel() + h_fc.numel() + h_gc.numel()) * 8,
               "d2h_bytes_per_step": (h_u.numel() + h_phi.numel()) * 8,
               "mode": "pipelined: step k+1's inputs are copied in while step k solves and "
                       "step k's results copied out while step k+1 solves (a copy stream, "
                       "double buffers); every step's copies and an L2 flush before every "
                       "solve inside the timed region of all steps",
               "serial_ms_per_step": serial}

    # ---------------- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        n, dt = cpu_oracle_applies(prob)
        cpu = {"value": (N + 1) ** 2 * n / dt, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{n} FP64 oracle double-layer applies of this N={N} problem "
                         f"({dt:.1f} s, numpy on the host cores); unit as value"}

    companion = None
    n3d = [int(x) for x in str(a.n3d).split(",") if int(x) > 0]
    if rank == 0 and n3d:
        companion = [run_3d_companion(n, dev, flush) for n in n3d]
    batch = None
    if rank == 0 and a.batch > 0:
        batch = run_batch_companion(a, dev)
    neu = None
    if rank == 0 and a.nneu > 0:
        neu = run_neumann_companion(a.nneu, dev, flush)
    tc = None
    if rank == 0 and a.ntc > 0:
        tc = run_tc_companion(a, dev, flush, ctx, N) if N % 128 == 0 and N <= 8192 else None

    launches = int(sum(v[1] for v in counted.values()))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "N": N, "M": M, "kappa": a.kappa,
                       "precision": "FP32 box solves, FP64 geometry/Krylov/refinement",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "replicas": world},
            "roofline": roofline(stages, N, ctx.info()["dst_variant"], ctx.info()["tri_first_mode"]),
            "dst_stage_roofline": dst_stage_roofline(stages, N, nprof),
            "alu_peaks": alu_peaks,
            "dst_variant": ctx.info()["dst_variant"],
            "cpu_baseline": cpu,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "setup_ms": setup_ms,
            "applies_per_solve": applies,
            "iterations": infos[-1]["iterations"],
            "outer_iterations": infos[-1]["outer_iterations"],
            "rel_residual": infos[-1]["rel_residual"],
            "err_inf_mixed": err_mixed,
            "stage_ms": {k: round(v[0] / nprof, 4) for k, v in stages.items() if v[1]},
            "stage_launches": {k: int(v[1]) for k, v in counted.items() if v[1]},
            "stage_note": (f"stage_ms: per solve, from {nprof} further solves with CUDA events "
                           "around every launch (the headline steps run without them); "
                           "stage_launches: over the timed steps"),
            **fp64,
            "companion_3d": companion,
            "companion_batch": batch,
            "companion_neumann": neu,
            "companion_tc": tc}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_3d_companion(N, dev, flush):
    """The 3-D configuration (ellipsoid 0.7 x 0.5 x 0.4, u = sin x sin y sin z, kappa = 0)
    at one grid size: setup, mixed and FP64 Dirichlet solves timed with CUDA events
    (L2 flushed before each), errors against the exact solution.  Reported beside the
    2-D line, not folded into its value."""
    import numpy as np
    import torch
    import kfbi_workloads.surfaces3d as S3
    import paper_2404_15249_gb300 as K

    prob = S3.config_poisson3d(N, "ellipsoid")
    I = prob.iface
    fg = torch.as_tensor(prob.f_grid(), device=dev)
    fc = torch.as_tensor(prob.f_ctrl(), device=dev)
    gc = torch.as_tensor(prob.g_ctrl(), device=dev)
    u = torch.empty((N + 1,) * 3, dtype=torch.float64, device=dev)
    phi = torch.empty(I.P, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = K.Kfbi3D(I.pts, I.normals, I.shape, N, 0.0, precision=K.KFBI_MIXED_FP32, tol=1e-10)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    inside = ctx.inside_mask().cpu().numpy().astype(bool)
    u_exact = prob.u_grid()
    st = torch.cuda.current_stream()

    def timed(n):
        out, info = [], None
        for _ in range(n):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, _, info = ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
            e1.record(st)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        err = float(np.max(np.abs(u.cpu().numpy() - u_exact)[inside]))
        return statistics.mean(out), info, err

    ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
    ms_mixed, info, err_mixed = timed(3)
    applies = info["applies_fp64"] + info["applies_low"]
    ctx.set_solver(K.KFBI_FP64, 50, 20, 1e-10, 1e-5)
    ctx.solve_bvp(fg, fc, gc, u_out=u, dens_out=phi)
    ms64, info64, err64 = timed(2)
    # box solve alone: FFT FP32 form against the tensor-core dense form (36 N^4 flops)
    tc = None
    if N % 128 == 0:
        b = torch.randn((N + 1,) * 3, dtype=torch.float64, device=dev)
        vb = torch.empty_like(b)

        def box_ms(prec, n=5):
            for _ in range(2):
                ctx.box_solve(b, prec, out=vb)
            out = []
            for _ in range(n):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ctx.box_solve(b, prec, out=vb)
                e1.record(st)
                e1.synchronize()
                out.append(e0.elapsed_time(e1))
            return statistics.median(out)

        ms_fft, ms_tc = box_ms(K.KFBI_MIXED_FP32), box_ms(K.KFBI_TF32X3)
        flops = 36.0 * N ** 4
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        bf16 = float(json.load(open(pk))["bf16_tflops"]) if os.path.exists(pk) else 1900.0
        peak = bf16 * NOMINAL_TF32_PER_BF16
        tc = {"fft_fp32_box_solve_ms": ms_fft, "tc_box_solve_ms": ms_tc,
              "note": "box solves of a random right-hand side, including the conversions "
                      "between the user grid and the work grid",
              "tensor_tflops": flops / (ms_tc / 1e3) / 1e12,
              "tensor_frac": flops / (ms_tc / 1e3) / 1e12 / peak,
              "peak_source": "measured BF16 burst x nominal TF32/BF16 ratio"}
    ctx.close()
    return {"workload": f"3-D Dirichlet Poisson, ellipsoid (0.7, 0.5, 0.4), N={N} "
                        f"({N + 1}^3 nodes), {I.P} grid-line intersection points, "
                        f"u = sin x sin y sin z, GMRES(50) to 1e-10",
            "N": N, "points": I.P, "setup_ms": setup_ms,
            "mixed_solve_ms": ms_mixed, "grid_pts_per_s_per_apply": (N + 1) ** 3 * applies / (ms_mixed / 1e3),
            "applies_per_solve": applies, "iterations": info["iterations"],
            "err_inf_mixed": err_mixed, "fp64_solve_ms": ms64, "err_inf_fp64": err64,
            "fp64_iterations": info64["iterations"], "speedup_vs_fp64": ms64 / ms_mixed,
            "box_solve_fft_vs_tc": tc}


def run_neumann_companion(N, dev, flush):
    """The Neumann BVP (d_n u given on Gamma, single-layer density) on the 2-D Helmholtz
    configuration's ellipse (kappa = 1, u = exp(x) sin(2y), M = 2N): mixed-precision and
    plain FP64 solves timed with CUDA events (L2 flushed before each), errors against the
    exact solution.  Reported beside the 2-D line."""
    import numpy as np
    import torch
    import kfbi_workloads as W
    import paper_2404_15249_gb300 as K

    prob = W.config_helmholtz(N, 1.0, "ellipse")
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, N, 1.0,
                   precision=K.KFBI_MIXED_FP32, tol=1e-10)
    fg = torch.as_tensor(prob.f_grid(), device=dev)
    fc = torch.as_tensor(prob.f_ctrl(), device=dev)
    gn = torch.as_tensor(prob.gn_ctrl(), device=dev)
    u = torch.empty((N + 1, N + 1), dtype=torch.float64, device=dev)
    inside = ctx.inside_mask().cpu().numpy().astype(bool)
    st = torch.cuda.current_stream()

    def timed(n):
        out, info = [], None
        for _ in range(n):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, _, info = ctx.solve_neumann_bvp(fg, fc, gn, u_out=u)
            e1.record(st)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        err = float(np.max(np.abs(u.cpu().numpy() - prob.u_grid())[inside]))
        return statistics.mean(out), info, err

    ctx.solve_neumann_bvp(fg, fc, gn, u_out=u)
    ms_mixed, info, err_mixed = timed(3)
    ctx.set_solver(K.KFBI_FP64, 50, 20, 1e-10, 1e-5)
    ctx.solve_neumann_bvp(fg, fc, gn, u_out=u)
    ms64, info64, err64 = timed(2)
    ctx.close()
    applies = info["applies_fp64"] + info["applies_low"]
    return {"workload": f"2-D modified Helmholtz Neumann BVP, ellipse (0.7, 0.4, 30 deg), "
                        f"N={N}, M={2 * N}, kappa=1, u = exp(x) sin(2y), single-layer density, "
                        f"GMRES(50) to 1e-10",
            "N": N, "mixed_solve_ms": ms_mixed,
            "grid_pts_per_s_per_apply": (N + 1) ** 2 * applies / (ms_mixed / 1e3),
            "iterations": info["iterations"], "applies_low": info["applies_low"],
            "err_inf_mixed": err_mixed, "fp64_solve_ms": ms64, "err_inf_fp64": err64,
            "fp64_iterations": info64["iterations"], "speedup_vs_fp64": ms64 / ms_mixed}


def run_tc_companion(a, dev, flush, main_ctx, main_N):
    """The tensor-core box solve (dense sine-matrix form, four tcgen05 TF32 GEMMs with a
    three-term split, operands loaded by TMA) against the FFT FP32 box solve: median of 10
    solves each (L2 flushed before each) on the headline context (N = main_N) and on a
    flower context at N = --ntc, plus one mixed-precision BVP solve there with the
    tensor-core apply as its lowest tier.  Tensor roofline (at main_N): 24 N^3 flops per
    solve (4 GEMMs x 3 products x 2 N^3) against the TF32 peak taken as the measured BF16
    burst peak times the nominal TF32/BF16 ratio."""
    import numpy as np
    import torch
    import kfbi_workloads as W
    import paper_2404_15249_gb300 as K

    st = torch.cuda.current_stream()
    rng = np.random.default_rng(W.SEED)

    def med(ctx, n_grid, prec, n=10):
        b = torch.as_tensor(rng.standard_normal((n_grid + 1, n_grid + 1)), device=dev)
        v = torch.empty_like(b)
        for _ in range(3):
            ctx.box_solve(b, prec, out=v)
        out = []
        for _ in range(n):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.box_solve(b, prec, out=v)
            e1.record(st)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    big_tc = med(main_ctx, main_N, K.KFBI_TF32X3)
    big_fft = med(main_ctx, main_N, K.KFBI_MIXED_FP32)
    N = a.ntc
    prob = W.config_helmholtz(N, a.kappa, "flower")
    ctx = K.Kfbi2D(prob.iface.pts, prob.iface.normals, prob.iface.curv, N, a.kappa,
                   precision=K.KFBI_TF32X3, tol=1e-10)
    ms_tc, ms_fft = med(ctx, N, K.KFBI_TF32X3), med(ctx, N, K.KFBI_MIXED_FP32)
    fg = torch.as_tensor(prob.f_grid(), device=dev)
    fc = torch.as_tensor(prob.f_ctrl(), device=dev)
    gc = torch.as_tensor(prob.g_ctrl(), device=dev)
    u = torch.empty((N + 1, N + 1), dtype=torch.float64, device=dev)
    ctx.solve_bvp(fg, fc, gc, u_out=u)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    _, _, info = ctx.solve_bvp(fg, fc, gc, u_out=u)
    e1.record(st)
    e1.synchronize()
    inside = ctx.inside_mask().cpu().numpy().astype(bool)
    err = float(np.max(np.abs(u.cpu().numpy() - prob.u_grid())[inside]))
    ctx.close()
    flops = 24.0 * main_N ** 3
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = float(json.load(open(pk))["bf16_tflops"]) if os.path.exists(pk) else 1900.0
    peak = bf16 * NOMINAL_TF32_PER_BF16
    return {"workload": f"box solves (Alg. 4, dense form on the tensor cores vs FFT FP32) of a "
                        f"random right-hand side at N={main_N} (headline context) and N={N} "
                        f"(flower, kappa={a.kappa}); mixed BVP solve at N={N} with tensor-core "
                        f"applies as the lowest tier",
            "N": main_N, "tc_box_solve_ms": big_tc, "fft_fp32_box_solve_ms": big_fft,
            "roofline": {"bound": "tensor", "kernel": "dst_gemm_kernel (tcgen05 kind::tf32, TMA)",
                         "achieved": flops / (big_tc / 1e3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": flops / (big_tc / 1e3) / 1e12 / peak,
                         "peak_source": "measured BF16 burst x nominal TF32/BF16 ratio",
                         "flops_per_solve": flops},
            "small": {"N": N, "tc_box_solve_ms": ms_tc, "fft_fp32_box_solve_ms": ms_fft,
                      "tensor_tflops": 24.0 * N ** 3 / (ms_tc / 1e3) / 1e12},
            "mixed_tc_solve_ms": e0.elapsed_time(e1), "mixed_tc_iterations": info["iterations"],
            "mixed_tc_applies_low": info["applies_low"], "mixed_tc_err_inf": err}


def run_batch_companion(a, dev):
    """The batched configuration (random star curves, N from {64, ..., 1024}, kappa ~ U(0,5),
    4 right-hand sides per problem, M = 2N, GMRES(50) to 1e-10) through kfbi_batch_solve:
    setup of all contexts; the whole batch in mixed precision and then in plain FP64,
    each timed with CUDA events after a warm-up batch; errors against the exact solutions;
    and one more mixed batch with CUDA events around every launch of every context, whose
    summed device time against the batch's wall time tells how busy the GPU was.
    Reported beside the 2-D line."""
    import numpy as np
    import torch
    import kfbi_workloads as W
    import paper_2404_15249_gb300 as K

    nrhs, m, restarts = 4, 50, 20
    cfg = W.config_batch(a.batch, nrhs)
    t0 = time.perf_counter()
    ctxs = [K.Kfbi2D(p.iface.pts, p.iface.normals, p.iface.curv, p.N, p.kappa,
                     precision=K.KFBI_MIXED_FP32, gmres_m=m, max_restarts=restarts, tol=1e-10)
            for p, _ in cfg]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    fg, fc, gc, ub, exact = [], [], [], [], []
    for p, sols in cfg:
        for sol in sols:
            q = W.Problem(p.iface, p.N, p.kappa, sol)
            fg.append(torch.as_tensor(q.f_grid(), device=dev))
            fc.append(torch.as_tensor(q.f_ctrl(), device=dev))
            gc.append(torch.as_tensor(q.g_ctrl(), device=dev))
            ub.append(torch.empty((p.N + 1, p.N + 1), dtype=torch.float64, device=dev))
            exact.append(q.u_grid())
    st = torch.cuda.current_stream()
    insides = [c.inside_mask().cpu().numpy().astype(bool) for c in ctxs]

    def timed_batch():
        K.batch_solve(ctxs, fg, fc, gc, ub, nrhs)          # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        infos = K.batch_solve(ctxs, fg, fc, gc, ub, nrhs)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        pts_applies, err = 0.0, 0.0
        for k, (p, _) in enumerate(cfg):
            for r in range(nrhs):
                q = k * nrhs + r
                i = infos[q]
                pts_applies += (p.N + 1) ** 2 * (i["applies_fp64"] + i["applies_low"])
                err = max(err, float(np.abs(ub[q].cpu().numpy() - exact[q])[insides[k]].max()))
        bad = [(q // nrhs, q % nrhs, i["rel_residual"]) for q, i in enumerate(infos)
               if not i["converged"]]
        return ms, infos, pts_applies, err, bad

    ms, infos, pts_applies, err, bad = timed_batch()
    # device busy time: every launch of every context timed with events (one more batch)
    for c in ctxs:
        c.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    K.batch_solve(ctxs, fg, fc, gc, ub, nrhs)
    e1.record(st)
    e1.synchronize()
    wall_prof = e0.elapsed_time(e1)
    busy = 0.0
    launches = 0
    per_ctx = []
    for c, (p, _) in zip(ctxs, cfg):
        t = c.profile_read()
        busy += sum(v[0] for v in t.values())
        launches += sum(v[1] for v in t.values())
        per_ctx.append((p.N, t))
        c.profile(False)
    # the same batch in plain FP64
    for c in ctxs:
        c.set_solver(K.KFBI_FP64, m, restarts, 1e-10, 1e-5)
    ms64, infos64, _, err64, bad64 = timed_batch()
    for c in ctxs:
        c.close()
    return {"workload": f"batched 2-D Poisson/Helmholtz: {a.batch} random star curves, "
                        f"N from {{64..1024}}, M = 2N, kappa ~ U(0,5), {nrhs} right-hand sides "
                        f"each, GMRES({m}) with {restarts} restarts to 1e-10; mixed precision "
                        f"(timed) and plain FP64 (timed) on the same inputs",
            "problems": a.batch, "rhs": nrhs, "setup_s": setup_s, "batch_ms": ms,
            "solves_per_s": a.batch * nrhs / (ms / 1e3),
            "grid_pts_per_s_per_apply": pts_applies / (ms / 1e3),
            "converged": sum(1 for i in infos if i["converged"]), "not_converged": bad[:16],
            "max_rel_residual": max(i["rel_residual"] for i in infos),
            "total_iterations": sum(i["iterations"] for i in infos), "max_err_inf": err,
            "fp64_batch_ms": ms64, "speedup_vs_fp64": ms64 / ms,
            "fp64_converged": sum(1 for i in infos64 if i["converged"]),
            "fp64_not_converged": bad64[:16],
            "fp64_total_iterations": sum(i["iterations"] for i in infos64),
            "fp64_max_err_inf": err64,
            "dst_roofline": batch_dst_roofline(per_ctx, ms),
            "device_busy": {"kernel_ms_sum": busy, "wall_ms": wall_prof, "launches": launches,
                            "note": "summed device time of every launch of every context "
                                    "(events around each launch) over the wall time of the "
                                    "same mixed batch; concurrent streams can make the sum "
                                    "exceed the wall time"}}


def main():
    a = parse()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        return run_reference(a)
    return run_kfbi(a)


if __name__ == "__main__":
    sys.exit(main())
