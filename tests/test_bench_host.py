"""Host logic of bench.py's roofline fields (no GPU): the algorithmic bytes of
each pencil pass, the lookup of ncu DRAM traffic keyed by the kernel sources'
hash, and the peak denominators' fallback."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_pass_bytes_of_the_two_workloads():
    """U = N^d complex elements.  2D with 3 fields: the fused pass reads the
    N x 2N half spectrum (2U) and three (N+1)^2 multiplier octants and writes
    three N x 2N fields (3 x 2U).  3D: the fused pass reads the N x 2N x 2N
    input (4U) and writes 4U per field; the strided pass reads 2U and writes 4U."""
    U2, oct2 = 1024 ** 2 * 8, 1025 ** 2 * 8
    b2 = bench.pass_bytes(2, 1024, 3, 8)
    assert b2["fused_axis0"] == 2 * U2 + 3 * oct2 + 3 * 2 * U2 == 92323864
    assert b2["fwd_rows"] == 3 * U2 and b2["inv_rows"] == 9 * U2
    U3, oct3 = 256 ** 3 * 8, 257 ** 3 * 8
    b3 = bench.pass_bytes(3, 256, 1, 8)
    assert b3["fused_axis0"] == 4 * U3 + oct3 + 4 * U3
    assert b3["fwd_axis1"] == 2 * U3 + 4 * U3 and b3["inv_axis1"] == 6 * U3
    assert sum(b3.values()) == 3 * U3 + 6 * U3 + 8 * U3 + oct3 + 6 * U3 + 3 * U3


def _copy_sources(tmp_path):
    csrc = tmp_path / "paper_1604_03155_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench.APPLY_KERNEL_SOURCES + ("tc_fused.cu",):
        shutil.copy(os.path.join(ROOT, "paper_1604_03155_gb300", "csrc", fn), csrc / fn)
    (tmp_path / "profiles").mkdir()


def test_traffic_rows_are_used_only_for_the_sources_they_were_taken_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _copy_sources(tmp_path)
    h = bench.kernel_source_hash()
    htc = bench.kernel_source_hash(("tc_fused.cu",))
    assert h != htc and len(h) == 16
    with open(tmp_path / "profiles" / "dram_traffic.md", "w") as fh:
        fh.write("| pass | workload | bytes | source hash |\n|---|---|---|---|\n")
        fh.write(f"| fused_axis0 | w2d | 53499136 | {h} |\n")
        fh.write("| inv_rows | w2d | 50379008 | 0000000000000000 |\n")
        fh.write(f"| fused_axis0[tc_bf16x2] | w3d | 1283440640 | {htc} |\n")
    assert bench.ncu_traffic("fused_axis0", "w2d") == 53499136.0
    assert bench.ncu_traffic("inv_rows", "w2d") is None  # taken on other sources
    assert bench.ncu_traffic("fused_axis0", "w3d") is None  # no row
    assert bench.ncu_traffic("fused_axis0[tc_bf16x2]", "w3d") == 1283440640.0
    # one changed byte of a kernel source invalidates the row
    with open(tmp_path / "paper_1604_03155_gb300" / "csrc" / "apply_f32.cu", "a") as fh:
        fh.write("\n")
    assert bench.kernel_source_hash() != h
    assert bench.ncu_traffic("fused_axis0", "w2d") is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_hbm() == (bench.FALLBACK_HBM_GBS, "fallback")
    assert bench.measured_peak_bf16(False) == (bench.FALLBACK_BF16_TFLOPS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, '
                                                  '"bf16_tflops_sustained": 1700.0}')
    assert bench.measured_peak_hbm() == (7000.0, "measured")
    assert bench.measured_peak_bf16(True) == (1700.0, "measured")
