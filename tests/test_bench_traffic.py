"""bench.py's roofline traffic: read from the committed ncu summary only while the
K1 sources hash to the value recorded there; per-RHS bytes scale with the launch
group's right-hand sides, per-group bytes (spectrum octants) are added once."""
import os

import bench


def _write(tmp_path, source_hash, per_rhs="1000", per_group=None):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    lines = ["# summary", "", f"- dram_bytes_per_rhs: {per_rhs}"]
    if per_group is not None:
        lines.append(f"- dram_bytes_per_group: {per_group}")
    lines.append(f"- source_hash: `{source_hash}`")
    (d / "fft_conv_1mm_grid.md").write_text("\n".join(lines) + "\n")


def test_traffic_scales_with_rhs_and_adds_group_bytes(tmp_path, monkeypatch):
    h = bench._conv_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_conv_source_hash", lambda: h)
    _write(tmp_path, h, per_rhs="1000", per_group="300")
    assert bench._traffic_per_launch(8) == 8 * 1000 + 300
    _write(tmp_path, h, per_rhs="1000")
    assert bench._traffic_per_launch(4) == 4000


def test_traffic_is_null_when_the_kernels_changed(tmp_path, monkeypatch):
    h = bench._conv_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_conv_source_hash", lambda: h)
    _write(tmp_path, "0" * 16)
    assert bench._traffic_per_launch(8) is None
    os.remove(tmp_path / "profiles" / "fft_conv_1mm_grid.md")
    assert bench._traffic_per_launch(8) is None
