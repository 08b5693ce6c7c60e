"""Host logic of bench.py that needs no GPU: the clock sampler's parsing, the
source digest and the rule by which a committed ncu summary's figures are used
(only on the sources it was taken on, or on later sources it lists as leaving
the kernel unchanged), the measured-peak lookup and the algorithmic flop count."""
import os

import pytest

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_give_median_and_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2000, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(0)
    c.proc, c.path = _Proc(), str(path)
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not path.exists()


def test_clock_sampler_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _tree(root, source):
    csrc = root / "paper_2311_12818_gb300" / "csrc"
    csrc.mkdir(parents=True, exist_ok=True)
    (csrc / "a.cu").write_text(source)
    (root / "paper_2311_12818_gb300" / "build.py").write_text("FLAGS = []\n")
    (root / "profiles").mkdir(exist_ok=True)


def test_profile_figures_follow_the_source_digest(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, "kernel v1")
    d1 = bench.kernel_digest()
    assert len(d1) == 64 and d1 == bench.kernel_digest()
    (tmp_path / "profiles" / "k.md").write_text(
        "Kernel source digest (CUDA sources and build script): %s.\n"
        "dram_bytes_per_launch: 123456\n"
        "executed FP32 = 0.077 of the derived 80.5 TFLOP/s\n" % d1)
    assert bench.profiled_traffic("k.md") == 123456
    assert bench.profiled_fraction("k.md") == pytest.approx(0.077)
    assert bench.profiled_traffic("missing.md") is None
    # another source: the figures no longer apply
    _tree(tmp_path, "kernel v2")
    d2 = bench.kernel_digest()
    assert d2 != d1
    assert bench.profiled_traffic("k.md") is None and bench.profiled_fraction("k.md") is None
    # until the summary lists the new digest as leaving its kernel unchanged
    with open(tmp_path / "profiles" / "k.md", "a") as f:
        f.write("Kernel unchanged at digest: %s (another kernel changed).\n" % d2)
    assert bench.profiled_traffic("k.md") == 123456
    # the file name enters the digest as well as the contents
    os.rename(tmp_path / "paper_2311_12818_gb300" / "csrc" / "a.cu", tmp_path / "paper_2311_12818_gb300" / "csrc" / "b.cu")
    assert bench.kernel_digest() not in (d1, d2)


def test_measured_peak_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6797.6}')
    assert bench.measured_hbm() == (6797.6, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"bf16_tflops": 1900}')
    assert bench.measured_hbm() == (6800.0, "fallback")


def test_algorithmic_flops_is_the_counter_weighted_sum():
    F = {"frame_sphere": 3, "normal_sphere": 5, "vertex_blocks": 7, "vertex_constraint": 11,
         "thomas_first_row": 13, "thomas_row": 17, "ggt_row": 19, "ray_sphere": 23, "ray_rect": 29,
         "ray_triangle": 31, "ray_box": 37}
    st = {"full_evals": 2, "c_evals": 3, "newton_steps": 4, "thomas_rows": 10, "ggt_rows": 5, "sphere_tests": 6,
          "plane_tests": 7, "tri_tests": 8, "node_tests": 9}
    want = (2 * (3 + 7) + 3 * (5 + 11) + 4 * 13 + (10 - 4) * 17 + 5 * 19 + 6 * 23 + 7 * 29 + 8 * 31 + 9 * 37)
    assert bench.algorithmic_flops(st, F) == want
    # the per-unit figures come from the committed table
    F = bench.unit_flops()
    assert all(F[k] > 0 for k in ("vertex_blocks", "vertex_constraint", "thomas_row", "ray_sphere"))
