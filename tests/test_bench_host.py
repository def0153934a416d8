"""Host logic of bench.py on CPU: the clock record (with a stand-in
nvidia-smi) and the per-launch DRAM traffic taken from the committed ncu
summaries only while the kernel sources are the profiled ones.

The stand-in prints one CSV line per period in the query's column order
(index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap); the SM clock counts
up by one per line, so a test can tell which lines were kept.
"""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _fake_smi(tmp_path, reason_from=None):
    script = tmp_path / "nvidia-smi"
    reason = "-1" if reason_from is None else str(reason_from)
    script.write_text(f"""#!{sys.executable}
import sys, time
period = 0.05
for a in sys.argv:
    if a.isdigit():
        period = int(a) / 1000.0
k = 0
while True:
    slow = "Active" if {reason} >= 0 and k >= {reason} else "Not Active"
    print(f"0, {{1000 + k}}, 2070, 500.0, 0x0, Not Active, {{slow}}, Not Active, Not Active", flush=True)
    k += 1
    time.sleep(period)
""")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


@pytest.fixture
def bench_mod(monkeypatch):
    import importlib
    import bench
    return importlib.reload(bench)


def test_samples_only_from_the_timed_region(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path) + os.pathsep + os.environ["PATH"])
    with bench_mod.ClockSampler(0) as clocks:
        first_line_seen = len(clocks.lines) >= 1   # the region starts after the first sample
        time.sleep(0.4)
    s = clocks.summary()
    assert first_line_seen
    assert s["in_region"] and s["samples"] >= 4
    assert s["sm_max_mhz"] == 2070.0 and s["reasons"] == []
    # lines stamped before the region began are not in the median: the first
    # line (1000 MHz) came before the region, so the median is above it
    assert s["sm_mhz"] > 1000.0
    assert 350.0 <= s["region_ms"] <= 1000.0


def test_throttle_reason_seen_inside_the_region(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, reason_from=3) + os.pathsep + os.environ["PATH"])
    with bench_mod.ClockSampler(0) as clocks:
        time.sleep(0.5)
    s = clocks.summary()
    assert "hw_thermal_slowdown" in s["reasons"]


def test_short_region_falls_back_to_the_next_sample(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path) + os.pathsep + os.environ["PATH"])
    monkeypatch.setattr(bench_mod.ClockSampler, "PERIOD_MS", 300)
    with bench_mod.ClockSampler(0) as clocks:
        pass
    # stop the stand-in's reader from adding lines after the region
    s = clocks.summary()
    assert s is not None and s["samples"] >= 1


def test_no_nvidia_smi_gives_no_record(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory: no nvidia-smi at all
    with bench_mod.ClockSampler(0) as clocks:
        pass
    assert clocks.summary() is None


def test_default_steps_per_workload(bench_mod):
    assert bench_mod.DEFAULT_STEPS["mutated"] * 2.4e-3 >= 0.3   # about half a second of pair steps
    assert all(v >= 10 for v in bench_mod.DEFAULT_STEPS.values())


def test_profiled_traffic_only_while_the_kernel_source_is_unchanged(tmp_path, monkeypatch, bench_mod):
    """roofline.traffic comes from a committed ncu summary only while the
    kernel's sources hash to the ones that were profiled; any edit of them
    turns it into null."""
    import shutil
    root = tmp_path / "tree"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2011_01441_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("pair_kernels.cu", "bp_device.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_2011_01441_gb300", "csrc", f), csrc / f)
    import hashlib
    h = hashlib.sha256()
    for f in ("pair_kernels.cu", "bp_device.cuh"):
        h.update((csrc / f).read_bytes())
    (root / "profiles" / "k_pair_bp_pair131072_launches.md").write_text(
        f"# a summary\n\nsource_sha256: {h.hexdigest()}\ntraffic_bytes_per_launch: 4753408\n")
    monkeypatch.setattr(bench_mod, "ROOT", str(root))
    srcs = ["pair_kernels.cu", "bp_device.cuh"]
    committed = bench_mod._profiled_traffic("k_pair_bp_pair131072_launches.md", srcs)
    assert committed == 4753408
    with open(csrc / "bp_device.cuh", "a") as f:
        f.write("\n// an edit after the capture\n")
    assert bench_mod._profiled_traffic("k_pair_bp_pair131072_launches.md", srcs) is None
    assert bench_mod._profiled_traffic("no_such_summary.md", srcs) is None


def test_every_committed_summary_matches_its_kernel_source(bench_mod):
    """Each ncu summary that carries a traffic figure was taken on the kernel
    source as committed (so the bench reports it, not null)."""
    cases = {"k_pair_bp_pair131072_launches.md": ["pair_kernels.cu", "bp_device.cuh"],
             "k_batch_batch4096_full.md": ["batch.cu", "bp_device.cuh"],
             "k_affine_batch4096_full.md": ["affine.cu", "bp_device.cuh"],
             "k_affine_pair131072_launches.md": ["affine.cu", "bp_device.cuh"],
             "k_lws_n131072_full.md": ["lws.cu", "bp_device.cuh"]}
    for prof, srcs in cases.items():
        assert bench_mod._profiled_traffic(prof, srcs) is not None, prof


def test_profile_commands_run_committed_files_only():
    """Every ncu summary under profiles/ gives the command that made it, and
    the scripts those commands run are files of this repository (bench.py,
    or inline `python -c` code that imports the package)."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pdir = os.path.join(root, "profiles")
    for name in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, name)).read()
        assert "ncu " in text and "--clock-control none" in text, name
        for script in re.findall(r"python ([\w./-]+\.py)", text):
            assert os.path.isfile(os.path.join(root, script)), (name, script)
            assert not script.startswith("_work"), (name, script)
