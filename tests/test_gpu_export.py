"""Raw export of a result into device buffers and into pinned host buffers
(written by the export kernel across the host link): the same terms, and the
same terms as the oracle."""
import numpy as np
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


@pytest.mark.parametrize("n", [20, 100])
def test_raw_into_pinned_host_equals_device(n):
    import torch
    if n == 20:
        _, instrs = W.fan_in_heavy(5, n=20, n_s=8, total=500, tail=80)
    else:
        _, instrs = W.random_clifford(n, n, 4 * n)
        instrs = list(instrs) + [("T", q, -1, 0.0) for q in range(0, n, 7)]
    res = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)))
    k = res.nterms
    dev = res.raw_device()
    host = [torch.empty((k + 3, res.W), dtype=torch.int64, pin_memory=True),
            torch.empty((k + 3, res.W), dtype=torch.int64, pin_memory=True),
            torch.empty(k + 3, dtype=torch.float64, pin_memory=True),
            torch.empty(k + 3, dtype=torch.int32, pin_memory=True)]
    assert res.raw_into(*host) == k
    for d, h in zip(dev, host):
        assert np.array_equal(d.cpu().numpy(), h[:k].numpy())
    with pytest.raises(ValueError):
        res.raw_into(host[0][:0], host[1], host[2], host[3])
    with pytest.raises(ValueError):  # pageable host memory is refused
        res.raw_into(torch.empty((k, res.W), dtype=torch.int64), host[1], host[2], host[3])
    if n == 20:
        compare_result(res, O.propagate(n, instrs, mode="plan", threads=8))
