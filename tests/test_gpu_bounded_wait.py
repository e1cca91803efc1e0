"""Bounded device-side waits end in an error status, not a hang.

The wait that the general merge uses for a group leader's publish is the same
bounded loop as the one exercised here: a flag that nothing sets makes it give
up after about timeout_ms, the call returns QX_ETIMEOUT, and the device stays
usable (a propagation right after it matches the oracle).
"""
import time

import pytest

from gpu_util import compare_result
from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def test_published_flag_ends_the_wait():
    qx.wait_selftest(timeout_ms=1000, publish=True)


def test_missing_publish_times_out_and_device_stays_usable():
    t0 = time.perf_counter()
    with pytest.raises(qx.QxError) as e:
        qx.wait_selftest(timeout_ms=50, publish=False)
    assert e.value.name == "QX_ETIMEOUT"
    assert time.perf_counter() - t0 < 30.0
    n, instrs = W.random_layers(2)
    res = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)))
    compare_result(res, O.propagate(n, instrs, mode="plan"))
