import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running check")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Worst weight error of every parity test that compared weights with the
    oracle (or with another path), so the log shows the margin to the bound."""
    gpu_util = sys.modules.get("gpu_util")
    if gpu_util is None or not gpu_util.WORST:
        return
    tr = terminalreporter
    tr.section("parity: worst weight error per test")
    tr.write_line(f"{'max |dw|':>10} {'max rel':>10} {'weights':>10}  test")
    for key in sorted(gpu_util.WORST):
        a, r, c = gpu_util.WORST[key]
        tr.write_line(f"{a:10.2e} {r:10.2e} {c:10d}  {key}")
