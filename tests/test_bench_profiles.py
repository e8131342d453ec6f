"""bench.py's use of the committed ncu summaries: a summary's DRAM traffic
is reported only while the hash it records matches the current code of its
kernel's sources, and a comment edit leaves that hash unchanged."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2401_09792_gb300 import synth  # noqa: E402


def test_code_only_ignores_comments_and_blank_lines():
    a = "int x;  // one\n/* two\n   three */ int y;\n\n   \n"
    b = "int x;\n int y;"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only("int x;") != bench._code_only("int z;")


def test_recorded_traffic_requires_the_current_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_sinr_link_blk_w.md").write_text(
        "kernel_source_hash: abc\ndram_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "abc")
    assert bench.recorded_traffic("k_sinr_link_blk", "w") == 1234.0
    assert bench.recorded_traffic("k_sinr_link_blk", "other") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "def")
    assert bench.recorded_traffic("k_sinr_link_blk", "w") is None


def test_paper64_traffic_scales_the_eight_cell_capture(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_sinr_link_wide_paper64_j8.md").write_text(
        "kernel_source_hash: abc\ndram_bytes_per_launch: 1000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "abc")
    bench.select_workload("paper64_u5")
    try:
        t, basis = bench.wide_link_traffic(bench.WORKLOAD)
        # 21 cells: 420 interfering links per launch against 56 at 8 cells
        assert t == 1000 * 420 / 56 and "paper64_j8" in basis
        assert synth.WORKLOADS["paper64_j8"].J == 8
    finally:
        bench.select_workload("mid")


def test_launch_counts_follow_the_measured_kernel_sequences():
    """gpu_launches in the bench line: the kernels of one SVD-precoded call,
    as the ncu launch lists of the differentiation and mid steps show them
    (phase steps, [core operand, projections, serving projections, serving
    pass,] eigensolve, precoder rest, close pairs, [precoder tiles,] link
    pass, finalize, refine)."""
    from paper_2401_09792_gb300 import tuckersinr as ts
    diff, mid = synth.WORKLOADS["diff"], synth.WORKLOADS["mid"]
    # the two-kernel precoder, the tensor-core serving pass and link pass
    assert bench.svd_launches(diff, ts.TS_PREC_TF32X3) == 12
    # FP32: the serving pass of the link kernel, one link launch
    assert bench.svd_launches(diff, ts.TS_PREC_FP32) == 8
    # TF32 keeps the FP32 serving pass
    assert bench.svd_launches(diff, ts.TS_PREC_TF32) == 11
    # mid: the precoder forms the serving channels itself (one kernel)
    assert mid.m * mid.n * mid.p <= 8192
    assert bench.svd_launches(mid, ts.TS_PREC_TF32X3) == 9
    assert bench.svd_launches(mid, ts.TS_PREC_FP32) == 6
