"""Host-side pieces of bench.py, on CPU: the committed ncu figures it quotes
(traffic of the headline collide, instruction mix of the FP64 collide) are
read back, tied to the kernel sources by hash, and the roofline arithmetic
they feed is consistent."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _field(path, key):
    for line in open(path):
        if line.startswith(key + ":"):
            return line.split(":", 1)[1].strip()
    return None


def test_committed_profiles_parse():
    p = os.path.join(bench.PROFILE_DIR, "k_collide_f32_channel_256.txt")
    assert len(_field(p, "source_sha")) == 16
    t = float(_field(p, "dram_bytes_per_launch_full_size"))
    # the full-size launch moves close to the algorithmic 152 B per site of
    # 256^3 (writes still in L2 at the end of the capture make it a little less)
    assert 0.85 * 152 * 256 ** 3 < t < 1.05 * 152 * 256 ** 3
    p = os.path.join(bench.PROFILE_DIR, "k_collide_f64_160.txt")
    assert len(_field(p, "source_sha")) == 16
    inst, flop = float(_field(p, "fp64_inst_per_site")), float(_field(p, "fp64_flop_per_site"))
    assert inst <= flop <= 2 * inst


def test_quoted_figures_follow_the_source_hash(tmp_path, monkeypatch):
    # a summary whose hash differs from the sources is not quoted
    src = os.path.join(bench.PROFILE_DIR, "k_collide_f32_channel_256.txt")
    text = open(src).read()
    sha = _field(src, "source_sha")
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    (tmp_path / "k_collide_f32_channel_256.txt").write_text(text)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    assert bench.committed_traffic("k_collide_f32_channel_256") == float(_field(src, "dram_bytes_per_launch_full_size"))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.committed_traffic("k_collide_f32_channel_256") is None


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2.07 GHz x 2 FP64 lanes x 2 flops = the nominal 1.25 TFLOP/s
    peak = bench.SM_COUNT * bench.SM_MAX_HZ * bench.FP64_LANES_PER_SM_CLK * 2
    assert abs(peak / 1.25e12 - 1) < 0.01


def test_algorithmic_bytes_of_the_headline():
    # 512^3 FP32 with 1e5 colloids: 152 B a site, plus 64 nodes x 3 components
    # x 4 B per colloid twice for the collide (force in, velocity out) and
    # five times for the whole step (spread read + write, collide, interpolation)
    V, n = 512 ** 3, 100000
    assert bench.collide_bytes("f32", V, n) == 152 * V + 2 * 768 * n
    assert bench.step_bytes("f32", V, n) == 152 * V + 5 * 768 * n
    assert bench.step_bytes("bf16s", V, n) == 76 * V + 5 * 768 * n
    assert bench.default_colloids(512) == 100000 and bench.default_colloids(128) == 1562


def test_cpu_sample_runs_the_cropped_recipe():
    r = bench.cpu_sample(16, 0.2, max_steps=3)
    assert r["value"] > 0 and r["cores"] >= 1 and "16^3" in r["sample"]
