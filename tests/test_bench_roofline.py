"""The bench's roofline bookkeeping on synthetic stage timings (no GPU): the dominant stage
is picked by total time, its algorithmic bytes cover the lines its kernel owns, and the
committed DRAM traffic is used only while the kernel's source hash matches."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N = 4096


def test_dominant_stage_and_bytes():
    stages = {"dst_rows_f32": (5.6, 98), "dst_cols_f32": (1.0, 70), "dst_tri_f32": (2.3, 70),
              "transpose": (2.1, 98), "krylov": (9.9, 1000)}
    r = bench.roofline(stages, N, [0, 4, 1, 6], 252)
    assert r["kernel"] == "rows_kernel<float>"          # krylov is not a transform stage
    assert r["algorithmic_bytes"] == 2 * N * N * 4
    assert r["achieved"] == pytest.approx(2 * N * N * 4 / (5.6 / 98 / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_split_y_pass_bytes():
    stages = {"dst_cols_f32": (9.0, 70), "dst_tri_f32": (2.3, 70)}
    r = bench.roofline(stages, N, [0, 4, 1, 6], 252)
    assert r["kernel"] == "yline_kernel<float>"
    assert r["algorithmic_bytes"] == 2 * N * 252 * 4      # only the low x-modes
    stages = {"dst_cols_f32": (1.0, 70), "dst_tri_f32": (2.3, 70)}
    r = bench.roofline(stages, N, [0, 4, 1, 6], 252)
    assert r["kernel"] == "ytri_kernel<float>"
    assert r["algorithmic_bytes"] == 2 * N * (N - 252) * 4


def test_row_layout_y_pass_is_one_span_over_the_whole_grid():
    # variant 8: the y-pass (filters on one stream, low-mode transform pair on another) is
    # timed as one span per launch of the filter kernel, covering every unknown
    stages = {"dst_rows_f32": (3.5, 170), "dst_tri_f32": (3.8, 70), "sparse_x_f32": (1.7, 51)}
    r = bench.roofline(stages, N, [0, 8, 1, 6], 256)
    assert r["kernel"] == bench.YPASS
    assert r["algorithmic_bytes"] == 2 * N * N * 4
    assert r["achieved"] == pytest.approx(2 * N * N * 4 / (3.8 / 70 / 1e3) / 1e9)
    assert len(bench.kernel_source_hash(bench.YPASS)) == 12


def test_traffic_only_for_the_current_source():
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    lines = [l.split() for l in open(p) if l.strip() and not l.startswith("#")]
    rows = [f for f in lines if f[0] == "rows_kernel<float>"]
    assert rows, "the dominant kernel has a committed traffic line"
    current = bench.kernel_source_hash("rows_kernel<float>")
    got = bench.traffic_for("rows_kernel<float>", N)
    if rows[0][1] == current:
        assert got == pytest.approx(float(rows[0][3]))
    else:
        assert got is None
    assert bench.traffic_for("no_such_kernel", N) is None


def test_dst_stage_roofline_counts_dense_and_sparse_box_solves():
    # per solve: 42 plain applies (sparse right-hand side: one sparse x-transform and one
    # row pass each) and 28 dense box solves (two row passes each), over 5 profiled solves
    solves = 5
    stages = {"dst_rows_f32": (28.0, solves * (42 + 2 * 28)), "sparse_x_f32": (11.0, solves * 42),
              "dst_tri_f32": (11.5, solves * 70), "dst_cols_f32": (5.0, solves * 70),
              "transpose": (10.7, solves * 98), "krylov": (11.0, solves * 300)}
    r = bench.dst_stage_roofline(stages, N, solves)
    assert r["sparse_box_solves"] == pytest.approx(42)
    assert r["dense_box_solves"] == pytest.approx(28)
    nbytes = (24 * 28 + 16 * 42) * (N - 1) ** 2
    assert r["algorithmic_bytes"] == pytest.approx(nbytes)
    ms = (28.0 + 11.0 + 11.5 + 5.0 + 10.7) / solves          # krylov is not a DST stage
    assert r["ms"] == pytest.approx(ms)
    assert r["frac"] == pytest.approx(nbytes / (ms / 1e3) / 1e9 / r["peak"])


def test_fp64_roofline_uses_the_measured_peak():
    stages = {"dst_rows_f64": (100.0, 200), "dst_cols_f64": (50.0, 100), "krylov": (10.0, 50)}
    r = bench.fp64_roofline(stages, N, {"fp64_tflops": 1.2, "fp32_tflops": 70.0})
    flops = N * 5.0 * N * 12
    assert r["kernel"] == "rows_kernel<double>"
    assert r["achieved"] == pytest.approx(flops / (100.0 / 200 / 1e3) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.2)
    assert bench.fp64_roofline(stages, N, None) is None


def test_batch_dst_roofline_sums_the_box_solve_bytes_of_every_context():
    # two contexts: one plain apply (1 sparse x-transform + 1 row pass) at N = 64 and one
    # dense box solve (2 row passes) at N = 128, over a 2 ms batch
    per_ctx = [(64, {"sparse_x_f32": (0.1, 1), "dst_rows_f32": (0.1, 1)}),
               (128, {"dst_rows_f32": (0.2, 2)})]
    r = bench.batch_dst_roofline(per_ctx, 2.0)
    want = 16.0 * 63 ** 2 + 24.0 * 127 ** 2
    assert r["algorithmic_bytes"] == pytest.approx(want)
    assert r["achieved"] == pytest.approx(want / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.batch_dst_roofline([], 2.0) is None
