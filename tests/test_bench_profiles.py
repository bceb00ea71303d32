"""Host logic of bench.py's roofline inputs: the ncu summaries under
profiles/ are read per window (a flow launch holds many windows), ignored
once the kernel sources have changed since the capture, and every committed
summary parses with the counters the roofline needs."""
import glob
import os

import pytest

import bench


def _write(tmp_path, name, text):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / (name + "_traffic.txt")).write_text(text)


def test_flow_capture_is_read_per_window(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "abcd")
    _write(tmp_path, "flow512_kernel_config2",
           "kernel_sources_sha256_16: abcd\nbytes_per_launch: 9800\nread_bytes: 4900\nwrite_bytes: 4900\n"
           "warp_instructions_per_launch: 98000\nunits_per_launch: 7\nwindows_per_launch: 98\n")
    tr = bench.profile_traffic("flow512_kernel_config2")
    assert tr["bytes_per_launch"] == 100 and tr["warp_instructions_per_launch"] == 1000
    assert tr["read_bytes"] == 50 and tr["units_per_launch"] == 7
    # a window launch's capture is taken as it is
    _write(tmp_path, "step_kernel_dendrite",
           "kernel_sources_sha256_16: abcd\nbytes_per_launch: 9800\nwarp_instructions_per_launch: 98000\n"
           "units_per_launch: 7\n")
    tr = bench.profile_traffic("step_kernel_dendrite")
    assert tr["bytes_per_launch"] == 9800 and tr["warp_instructions_per_launch"] == 98000


def test_stale_or_missing_capture_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "new")
    _write(tmp_path, "flow256_kernel_config2", "kernel_sources_sha256_16: old\nbytes_per_launch: 1\n")
    assert bench.profile_traffic("flow256_kernel_config2") is None
    assert bench.profile_traffic("no_such_profile") is None


def test_roofline_per_window():
    """Issue roofline from per-window counts: achieved = instructions per
    window / time per window; HBM on 8S + 52 and 8S + 36 bytes."""
    tr = {"bytes_per_launch": 1000, "warp_instructions_per_launch": 33_000_000}
    r = bench.roofline(10, False, 294_780, 44e-6, 6693.5, "measured", tr, 2070.0, issue_bound=True,
                       sms=152)
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(33e6 / 44e-6)
    assert r["peak"] == pytest.approx(152 * 4 * 2070e6)
    assert r["hbm"]["achieved"] == pytest.approx(294_780 * 132 / 44e-6 / 1e9)
    assert r["hbm"]["achieved_fixed_point"] == pytest.approx(294_780 * 116 / 44e-6 / 1e9)
    assert r["traffic"] == 1000


def test_committed_summaries_parse():
    files = glob.glob(os.path.join(bench.ROOT, "profiles", "*_traffic.txt"))
    assert files
    for f in files:
        kv = dict(line.split(":", 1) for line in open(f) if ":" in line)
        assert "kernel_sources_sha256_16" in kv and "bytes_per_launch" in kv and "units_per_launch" in kv, f
        assert int(kv["bytes_per_launch"]) > 0 and int(kv["units_per_launch"]) > 0
        md = f.replace("_traffic.txt", ".md")
        assert os.path.exists(md) and "ncu" in open(md).read(), md
