"""Box-solve micro-benchmark: kfbi_box_solve (Alg. 4) alone (or, with --apply, one
double-layer apply), on a flower context.

    python boxbench.py --N 8192 --precision 1 --reps 5

Sets up one context (flower r = 0.5 + 0.15 cos 5t, M = 2N), then times `--reps` box
solves of a seeded random right-hand side with CUDA events on the default stream, after
`--warmup` untimed ones, flushing L2 (a 256 MiB write) before each timed solve.  Prints
one JSON line: the median time per solve, the kernel variants the setup-time autotuner
chose, and the throughput on the algorithmic bytes of the three transform passes (each
reads and writes the N x N work grid once).  Used to profile the transform kernels on
grids larger than L2.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--precision", type=int, default=1, help="0 FP64, 1 FP32, 2/3 refined FP32, 4 tensor-core TF32x3")
    ap.add_argument("--kappa", type=float, default=1.0)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--apply", action="store_true",
                    help="time kfbi_apply_layer_potential (double layer) instead of the box solve")
    a = ap.parse_args(argv)

    import torch
    import kfbi_workloads as W
    from paper_2404_15249_gb300 import Kfbi2D, lib, _ptr

    N = a.N
    iface = W.flower(2 * N)
    ctx = Kfbi2D(iface.pts, iface.normals, iface.curv, N, kappa=a.kappa)
    rng = np.random.default_rng(W.SEED)
    b = torch.as_tensor(rng.standard_normal((N + 1, N + 1)), dtype=torch.float64).cuda()
    v = torch.empty_like(b)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=b.device)

    dens = torch.as_tensor(W.random_density(iface.M), dtype=torch.float64).cuda()
    out = torch.empty_like(dens)

    def solve():
        if a.apply:
            st = lib().kfbi_apply_layer_potential(ctx.handle, 0, a.precision, _ptr(dens), _ptr(out), None)
        else:
            st = lib().kfbi_box_solve(ctx.handle, a.precision, _ptr(b), _ptr(v), None)
        if st != 0:
            raise RuntimeError(f"kfbi call failed with status {st}")

    for _ in range(a.warmup):
        solve()
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.reps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0.record()
        solve()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    info = ctx.info()
    ms = statistics.median(times)
    # plain solves only: a refined solve runs several transforms plus residual passes
    nbytes = 3 * 2.0 * N * N * (8 if a.precision == 0 else 4) if a.precision in (0, 1) else None
    # tensor-core solve: four N x N x N GEMMs, three TF32 products each
    flops = 4 * 3 * 2.0 * N**3 if a.precision == 4 else None
    if a.apply:
        nbytes = flops = None
    print(json.dumps({"N": N, "precision": a.precision, "apply": a.apply, "ms_per_solve": ms,
                      "times_ms": times, "dst_variant": list(info["dst_variant"]),
                      "transform_bytes": nbytes,
                      "transform_GBps": nbytes / ms / 1e6 if nbytes else None,
                      "tensor_TFLOPs": flops / ms / 1e9 if flops else None}))
    ctx.close()


if __name__ == "__main__":
    main()
