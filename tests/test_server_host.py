"""Host-side behaviour of the request loop (no GPU needed).

Without a usable device every request must come back through
qx_server_wait with the library's error, the statistics must count it, and
shutting the server down must not hang.
"""
import pytest

from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_server_rejects_bad_options():
    with pytest.raises(qx.QxError):
        qx.Server(slots=0)
    with pytest.raises(qx.QxError):
        qx.Server(precision=16)


def test_server_queue_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    srv = qx.Server(slots=3, max_queue=100)
    tickets = [srv.submit(*W.random_layers(s)) for s in range(7)]
    for t in tickets:
        with pytest.raises(qx.QxError) as e:
            srv.wait(t)
        assert e.value.name in ("QX_EUNSUPPORTED", "QX_ECUDA")
    st = srv.stats()
    assert st["failed"] == 7 and st["completed"] == 0 and st["queued"] == 0
    with pytest.raises(qx.QxError):
        srv.wait(tickets[0])  # a ticket is waited for once
    srv.close()


def test_server_queue_limit():
    srv = qx.Server(slots=1, max_queue=2)
    n, instrs = W.random_layers(1)
    accepted, rejected = 0, 0
    for _ in range(50):
        try:
            srv.submit(n, instrs)
            accepted += 1
        except qx.QxError as e:
            assert e.name == "QX_ECAP"
            rejected += 1
    assert accepted >= 2
    srv.close()


def test_server_rejects_an_invalid_circuit_in_the_planner():
    """A request with a bad instruction fails in its planner with the error
    of qx_load_circuit (QX_EINVAL, naming the first bad instruction); the
    valid requests around it are planned as usual."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    n, instrs = W.random_layers(3)
    bad = list(instrs)
    bad[17] = ("CX", 2, 2, 0.0)
    bad[40] = ("H", 99, -1, 0.0)
    srv = qx.Server(slots=1, max_queue=10)
    t_ok = srv.submit(n, instrs)
    t_bad = srv.submit(n, bad)
    with pytest.raises(qx.QxError) as e:
        srv.wait(t_bad)
    assert e.value.name == "QX_EINVAL" and "instruction 17: bad second wire" in str(e.value)
    with pytest.raises(qx.QxError) as e:
        srv.wait(t_ok)
    assert e.value.name in ("QX_EUNSUPPORTED", "QX_ECUDA")  # planned, then no GPU
    srv.close()
