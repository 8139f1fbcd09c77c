"""Host-side pieces of bench.py on the CPU: the kernel-code fingerprint that
keys the measured DRAM traffic, the algorithmic byte and flop counts per bin
(closed forms on config 3), launch-shape names and the job value."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2003_02845_gb300 import workloads as W  # noqa: E402

CODE = """// header comment
template <typename T>
__device__ T twice(T x) {   // trailing comment
  /* block
     comment */
  return x + x;
}
"""


def _fp(tmp_path, text, name):
    p = tmp_path / name
    p.write_text(text)
    return bench.kernel_fingerprint(str(p))


def test_fingerprint_ignores_comments_and_blank_lines(tmp_path):
    a = _fp(tmp_path, CODE, "a.cu")
    b = _fp(tmp_path, "\n// another comment\n" + CODE.replace("// trailing comment", "// reworded") + "\n\n", "b.cu")
    assert a == b


def test_fingerprint_sees_code_changes(tmp_path):
    a = _fp(tmp_path, CODE, "a.cu")
    b = _fp(tmp_path, CODE.replace("x + x", "x * 2"), "b.cu")
    assert a != b


def test_traffic_only_for_known_captures():
    assert bench.measured_traffic("no such workload", "mixed", "split/256") is None
    rec = bench.TRAFFIC[("config3_cc2d_256x64x12x80x3", "mixed", "split/256")]
    got = bench.measured_traffic("config3_cc2d_256x64x12x80x3", "mixed", "split/256")
    # either the capture matches the kernel code, or the figure is withheld
    assert got in (rec[0], None)
    assert (got is not None) == (bench.kernel_fingerprint() == rec[1])


def test_algorithmic_counts_on_config3():
    p = W.config3()
    # f read and written once (float32), opacities over 80 angles, the
    # background over 80 angles x 12 groups x 3 species
    assert bench.algorithmic_bytes_per_bin(p, True) == pytest.approx(8 + 24 / 80 + 56 / (80 * 12 * 3))
    assert bench.algorithmic_bytes_per_bin(p, False) == pytest.approx(16 + 24 / 80 + 56 / (80 * 12 * 3))
    # three unique faces per zone: six trilinear remaps (12 flops each), 28
    # for the half step and flux, the weight chains shared by 36 rows; 20
    # for the collision
    assert bench.algorithmic_flops_per_bin(p) == pytest.approx(3 * (6 * 12 + 28 + 6 * 150 / 36) + 20)


def test_launch_shape_names():
    from paper_2003_02845_gb300 import bt
    assert bench.parse_shape("fused/256") == 256
    assert bench.parse_shape("split/512") == bt.SHAPE_SPLIT | 512
    assert "k_flux_faces<float>" in bench.kernel_name(True, True)
    assert bench.kernel_name(False, False) == "k_flux_collide<double>"


def test_job_value_counts_every_rank():
    assert bench.job_value(1000.0, 1, 10.0) == pytest.approx(1000.0 / 10e-3)
    assert bench.job_value(1000.0, 4, 10.0) == pytest.approx(4 * 1000.0 / 10e-3)


def test_hbm_peak_reads_the_measured_figure():
    assert bench.hbm_peak({"hbm_gbs": 6793.4}) == 6793.4
    assert bench.hbm_peak({"hbm_gbs": {"value": 7000.0}}) == 7000.0
    assert bench.hbm_peak({}) == 6800.0
