"""Host logic of bench.py (no GPU): the clock record taken over the timed
region, the DRAM-traffic lookup's source-hash check, the FP64 roofline
arithmetic and the split of independent meshes over ranks."""
import json

import numpy as np

import bench


class _Proc:
    """Stands in for the nvidia-smi process of a ClockSampler."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _line(sm, smax=2070, power=150.0, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, {power}, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def _sampler(samples, t0, t1):
    s = bench.ClockSampler()
    s.proc = _Proc()
    s.lines = list(samples)
    s.t0, s.t1 = t0, t1
    return s


def test_clock_record_takes_the_timed_region_only():
    samples = [(0.0, _line(1200)), (0.5, _line(1300, power=90.0)),  # before the region
               (1.0, _line(2070)), (1.2, _line(2055, cap="Active")), (1.4, _line(2070, power=310.0)),
               (3.0, _line(900, hw="Active"))]  # after it
    out = _sampler(samples, 1.0, 1.5).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0  # median of 2070, 2055, 2070
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the region
    assert out["power_w_max"] == 310.0
    assert "note" not in out


def test_clock_record_of_a_short_region_uses_the_nearest_samples():
    samples = [(0.0, _line(2000)), (1.0, _line(2010)), (2.0, _line(2020)), (3.0, _line(2030)),
               (4.0, _line(2040)), (9.0, _line(500, hw="Active"))]
    out = _sampler(samples, 2.01, 2.02).stop()  # no sample inside the region
    assert out["samples"] == 4 and "note" in out
    assert out["sm_mhz"] == np.median([2010, 2020, 2030, 2040])  # the samples at 1, 2, 3, 4 s
    assert out["reasons"] == []


def test_clock_record_skips_malformed_lines_and_reports_throttles():
    samples = [(1.0, "garbage"), (1.1, _line("[N/A]")), (1.2, _line(1800, hwt="Active")),
               (1.3, _line(1810, swt="Active"))]
    out = _sampler(samples, 1.0, 1.4).stop()
    assert out["samples"] == 2
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler()
    s.proc = None
    out = s.stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None and "unavailable" in out["note"]


def test_traffic_figures_only_for_the_source_they_were_taken_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    rec = {"gather_persistent_kernel|cube100|mixed64": {"dram_bytes_per_launch": 123, "csrc_hash": "aaaa"},
           "stab_star_kernel|cube100|mixed64": {"dram_bytes_per_launch": 456, "csrc_hash": "bbbb"}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_hash", lambda: "aaaa")
    assert bench.read_traffic("gather_persistent_kernel", "cube100", "mixed64") == 123
    assert bench.read_traffic("stab_star_kernel", "cube100", "mixed64") is None  # other source
    assert bench.read_traffic("step_kernel", "cube100", "mixed64") is None  # never taken
    (tmp_path / "profiles" / "traffic.json").write_text("{not json")
    assert bench.read_traffic("gather_persistent_kernel", "cube100", "mixed64") is None


def test_source_hash_covers_every_kernel_source():
    h = bench.csrc_hash()
    assert len(h) == 16 and int(h, 16) >= 0


def test_fp64_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "fp64_peak", lambda: (1.25, "test peak"))
    r = bench.fp64_roofline(6_000_000, 3.0, flops_per_tet=400)
    assert np.isclose(r["achieved"], 400 * 6e6 / 3e-3 / 1e12)  # 0.8 TFLOP/s
    assert np.isclose(r["frac"], 0.8 / 1.25)
    assert r["bound"] == "fp64" and r["unit"] == "TFLOP/s" and r["peak_source"] == "test peak"


def test_meshes_split_over_ranks_each_once_and_balanced():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 4, 8):
        sizes = [int(x) for x in rng.integers(1_000, 1_300_000, size=64)]
        parts = bench.shard_meshes(sizes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)  # greedy largest-first bound
    assert bench.shard_meshes([5, 5], 4) == [[0], [1], [], []]
