"""CPU checks of the bench's host logic: the DRAM-traffic figure tied to the
source it was captured on, the clock summary of the timed region, and the
FP64 view of the merge wires."""
import datetime
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _traffic_tree(tmp_path, src_text):
    """A copy of the repository layout that ncu_traffic reads: one summary
    line naming a source file and the sha256 it had at capture time."""
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2505_03307_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_text(src_text)
    sha = hashlib.sha256(b"captured source\n").hexdigest()
    (tmp_path / "profiles" / "ncu_traffic_wl.txt").write_text(
        "# comment line\ntraffic_per_launch emit 12345 k.cuh " + sha + "\n")


def test_traffic_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    _traffic_tree(tmp_path, "captured source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("emit", "wl") == 12345.0
    assert bench.ncu_traffic("other", "wl") is None
    assert bench.ncu_traffic("emit", "missing") is None
    (tmp_path / "paper_2505_03307_gb300" / "csrc" / "k.cuh").write_text("changed\n")
    assert bench.ncu_traffic("emit", "wl") is None


def test_committed_traffic_summaries_parse():
    """Every committed traffic summary has a well-formed kernel line whose
    source file exists."""
    prof = os.path.join(ROOT, "profiles")
    found = 0
    for name in os.listdir(prof):
        if not name.startswith("ncu_traffic_"):
            continue
        for ln in open(os.path.join(prof, name)):
            parts = ln.split()
            if parts and parts[0] == "traffic_per_launch":
                assert len(parts) == 5
                assert float(parts[2]) > 0
                assert os.path.exists(os.path.join(ROOT, "paper_2505_03307_gb300", "csrc",
                                                   parts[3]))
                assert len(parts[4]) == 64
                found += 1
    assert found >= 1


def _line(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), "2070", "900.00", "0x0"] + list(reasons))


class _Proc:  # stands in for the nvidia-smi process once it has ended
    pass


def _sampler(lines, window):
    s = bench.ClockSampler(0)
    s.proc = _Proc()
    s.out = "\n".join(lines) + "\n"
    s.mark(*window)
    return s


def test_clock_summary_keeps_the_timed_region():
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 1.0, 900),                                 # before the region
             _line(t0 + 0.1, 2070), _line(t0 + 0.2, 2055), _line(t0 + 0.3, 2070),
             _line(t0 + 0.4, 1980, ("Not Active", "Not Active", "Not Active", "Active")),
             _line(t0 + 5.0, 600, ("Active", "Not Active", "Not Active", "Not Active")),
             "garbled line", ""]
    s = _sampler(lines, (t0, t0 + 1.0)).summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == pytest.approx(2062.5)
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]   # the hw_slowdown sample lies outside


def test_clock_summary_widens_a_short_region():
    """A region shorter than the sampling interval takes the samples within
    50 ms on each side."""
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 0.03, 2070, ("Active", "Not Active", "Not Active", "Not Active")),
             _line(t0 + 0.2, 1500)]
    s = _sampler(lines, (t0, t0 + 0.001)).summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown"]


def test_clock_summary_without_samples():
    assert bench.ClockSampler(0).summary() is None
    t0 = 1_700_000_000.0
    assert _sampler([_line(t0 - 9.0, 2070)], (t0, t0 + 1.0)).summary() is None


def test_fp64_view():
    d = {"ms": 2.0, "launches": 16}
    v = bench.fp64_view("merge_blocks", d, 1_000_000, 1.25)
    # 4 flops per term per launch over 0.125 ms
    assert v["achieved_tflops"] == pytest.approx(4e6 / 0.125e-3 / 1e12)
    assert v["frac"] == pytest.approx(v["achieved_tflops"] / 1.25)
    assert bench.fp64_view("expand_emit", d, 1_000_000, 1.25) is None
    assert bench.fp64_view("merge_blocks", {"ms": 0.0, "launches": 1}, 10, 1.25) is None
    assert bench.fp64_view("merge_blocks", d, 10, None) is None


def test_operator_bounds():
    instrs = [("H", 0, -1, 0.0), ("S", 1, -1, 0.0), ("CX", 0, 1, 0.0), ("CZ", 1, 2, 0.0),
              ("T", 2, -1, 0.0)]
    assert bench.operator_bounds(instrs) == [(0, 2), (2, 4), (4, 5)]
    assert bench.operator_bounds([]) == []
