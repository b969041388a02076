"""Host logic of the benchmark's measurement contract, on the CPU: the clock
samplers (NVML through a fake library object, the nvidia-smi CSV fallback
through a fake process), the staleness check of the committed event-kernel
traffic figure, the algorithmic byte count and the launch statistics."""
import os
import shutil
import time

import numpy as np
import pytest

import bench


class _FakeNvml:
    """Stands in for the read-only NVML wrapper: a fixed SM clock and a
    throttle-reason word that alternates between two values."""
    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL = (bench._Nvml.SW_POWER_CAP, bench._Nvml.HW_SLOWDOWN,
                                                          bench._Nvml.SW_THERMAL, bench._Nvml.HW_THERMAL)

    def __init__(self, gpu, words=(0, 0)):
        self.words = words
        self.k = 0

    def clock(self, maximum=False):
        return 2032.0 if maximum else 1980.0

    def reasons(self):
        self.k += 1
        return self.words[self.k % len(self.words)]


def _sample(monkeypatch, words):
    monkeypatch.setattr(bench, "_Nvml", lambda gpu: _FakeNvml(gpu, words))
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.03)
    return c.stop()


def test_nvml_sampler_clean_run(monkeypatch):
    r = _sample(monkeypatch, (0,))
    assert r["source"] == "nvml" and r["samples"] > 0
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == []


def test_nvml_sampler_reports_every_reason_seen(monkeypatch):
    r = _sample(monkeypatch, (_FakeNvml.SW_POWER_CAP, _FakeNvml.HW_SLOWDOWN | _FakeNvml.SW_THERMAL))
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_nvml_sampler_maps_the_thermal_bit(monkeypatch):
    r = _sample(monkeypatch, (_FakeNvml.HW_THERMAL,))
    assert r["reasons"] == ["hw_thermal_slowdown"]


class _FakeSmi:
    """Stands in for `nvidia-smi --query-gpu=... -lms 200`: writes its rows to
    the file it is given as stdout."""
    rows = ""

    def __init__(self, argv, stdout=None, stderr=None):
        assert argv[0] == "nvidia-smi" and "--format=csv,noheader,nounits" in argv
        stdout.write(self.rows)
        stdout.flush()

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_smi_fallback_parses_rows(monkeypatch):
    def no_nvml(gpu):
        raise OSError("no NVML")
    monkeypatch.setattr(bench, "_Nvml", no_nvml)
    _FakeSmi.rows = ("0, 2032, 2032, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                     "0, 1900, 2032, 1100.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                     "0, 2010, 2032, 1010.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                     "garbled line\n")
    monkeypatch.setattr(bench.subprocess, "Popen", _FakeSmi)
    c = bench.Clocks(0)
    c.start()
    r = c.stop()
    os.unlink(c.f.name)
    assert r["source"] == "nvidia-smi" and r["samples"] == 3
    assert r["sm_mhz"] == 2010.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == ["sw_power_cap"]


def test_smi_fallback_without_samples(monkeypatch):
    def no_nvml(gpu):
        raise OSError("no NVML")
    monkeypatch.setattr(bench, "_Nvml", no_nvml)
    _FakeSmi.rows = ""
    monkeypatch.setattr(bench.subprocess, "Popen", _FakeSmi)
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
    os.unlink(c.f.name)


def _profile_value(root):
    for line in open(os.path.join(root, "profiles", "event_mixed_o5_c2.txt")):
        if line.startswith("traffic_bytes_per_launch_full_size:"):
            return float(line.split(":", 1)[1])
    raise AssertionError("no traffic line")


def _copy_tree(tmp_path):
    root = tmp_path / "r"
    (root / "paper_2504_02034_b300" / "csrc").mkdir(parents=True)
    (root / "profiles").mkdir()
    for n in ("event.cu", "internal.cuh", "mass.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2504_02034_b300", "csrc", n),
                    root / "paper_2504_02034_b300" / "csrc" / n)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "event_mixed_o5_c2.txt"), root / "profiles")
    return root


def test_traffic_figure_follows_the_kernel_source(monkeypatch, tmp_path):
    """The committed DRAM traffic is reported only while the kernel sources
    hash to the value recorded beside it."""
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    live = bench.traffic_from_profiles()
    # the committed summary matches the committed sources, or reports none
    assert live is None or live == _profile_value(str(root))
    # a summary whose hash line names these sources is read back
    import hashlib
    h = hashlib.sha256()
    for n in ("event.cu", "internal.cuh", "mass.cuh"):
        h.update(open(root / "paper_2504_02034_b300" / "csrc" / n, "rb").read())
    prof = root / "profiles" / "event_mixed_o5_c2.txt"
    lines = [("kernel_source_sha256_16: " + h.hexdigest()[:16] + "\n")
             if l.startswith("kernel_source_sha256_16:") else l for l in open(prof)]
    prof.write_text("".join(lines))
    assert bench.traffic_from_profiles() == _profile_value(str(root))
    # any change to one of the hashed sources makes the figure stale
    with open(root / "paper_2504_02034_b300" / "csrc" / "mass.cuh", "a") as f:
        f.write("\n")
    assert bench.traffic_from_profiles() is None
    # no summary at all
    os.unlink(prof)
    assert bench.traffic_from_profiles() is None


def test_algorithmic_bytes():
    cat = {"sample_off": np.array([0, 10, 25]), "pix_off": np.array([0, 3, 7]), "n_z": 50}
    # 25 samples x 16 B + 7 pixel rows x 50 points x 4 B + 50 points x 4 B x H
    assert bench.algorithmic_bytes(cat, 4) == 25 * 16 + 7 * 50 * 4 + 50 * 4 * 4


def test_launch_stats():
    t = [3.0, 1.0, 2.0, 4.0, 100.0]
    s = bench.launch_stats(t)
    assert s["launches"] == 5
    assert s["p50_ms"] == 3.0
    assert s["mean_ms"] == pytest.approx(22.0)
    assert 4.0 < s["p99_ms"] <= 100.0
