"""bench.py's use of the committed ncu summary (host logic, CPU): a figure
is read only while the sha256 of the kernel's sources matches the hash the
summary records, so a changed kernel reports null traffic and issue rate
instead of stale ones."""
import hashlib

import bench


def _setup(tmp_path, monkeypatch, record_hash):
    srcs = []
    for i, text in enumerate(("kernel one\n", "kernel two\n")):
        f = tmp_path / f"k{i}.cu"
        f.write_text(text)
        srcs.append(str(f))
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(f, "rb").read())
    sha = h.hexdigest()[:16] if record_hash else "0" * 16
    prof = tmp_path / "summary.md"
    prof.write_text(f"`kernel_source_sha: {sha}`\n- `traffic_bytes_per_launch: 123456`\n"
                    "| mix | (`fp32_lane_ops_per_ray_step: 150.5`) |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", srcs)
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    return srcs


def test_figures_are_read_while_the_sources_match(tmp_path, monkeypatch):
    _setup(tmp_path, monkeypatch, True)
    assert bench.profiled_traffic() == 123456
    r = bench.fp32_issue(1e11)
    assert r["fp32_lane_ops_per_ray_step"] == 150.5
    assert abs(r["frac"] - 150.5e11 / bench.FP32_ISSUE_PEAK) < 1e-12


def test_a_changed_kernel_gives_null_figures(tmp_path, monkeypatch):
    srcs = _setup(tmp_path, monkeypatch, True)
    with open(srcs[1], "a") as f:
        f.write("// edited\n")
    assert bench.profiled_traffic() is None
    assert bench.fp32_issue(1e11) is None


def test_a_wrong_recorded_hash_gives_null_figures(tmp_path, monkeypatch):
    _setup(tmp_path, monkeypatch, False)
    assert bench.profiled_traffic() is None
