"""Host logic of the continuous-batching server, without a GPU: admission against the
device-memory budget (a request that cannot fit even alone is rejected; a batch stops where the
next request would push the bytes in flight over the budget), the work bound per batch, and the
exact workspace bytes a batch is charged (rox_jobs_workspace_size of its jobs plus its outputs).
The server object is assembled by hand around a stand-in for the prepared line lists, so no
device memory, stream or kernel is involved."""
import pytest

from paper_2510_20870_gb300 import _binding as rb
from paper_2510_20870_gb300 import serve
from paper_2510_20870_gb300.partition import PartitionFunction


class _Prepared:
    """Stand-in for a prepared list: line_range as if 400 lines reached every cm^-1 of window."""
    def line_range(self, first, n):
        return first, 4 * n + 20_000


def _server(budget, batch_evals=6e10, max_wait_s=None):
    s = object.__new__(serve.Server)
    s.prepared = [_Prepared()]
    s.lattice = (300.0, 0.01, 2970001)
    s.cutoff = 25.0
    s.win_pts = 5001
    s.mass = 16.0
    s.Q = PartitionFunction(("analytic", 0.05))
    s.Q_ref = s.Q(296.0)
    s.streams = [None, None, None]
    s.max_batch = 32
    s.mem_budget = int(budget)
    s.batch_evals = float(batch_evals)
    s.max_wait_s = max_wait_s
    s.promote_s = 0.25
    s.evals = s.launches = 0
    s.rejected = []
    s.max_inflight_seen = s.max_batch_seen = s.max_bytes_seen = s.max_queue_seen = 0
    return s


def _req(rid, n, t=0.0):
    return serve.Request(rid, t, 0, 1.0, 1000.0, 1000 + 10 * rid, n)


def test_batch_bytes_are_the_jobs_workspace_plus_outputs():
    s = _server(1 << 40)
    reqs = [_req(0, 5000), _req(1, 300)]
    jobs = [s._job(r, 0) for r in reqs]
    assert s.batch_bytes(reqs) == int(rb.rox_jobs_workspace_size(jobs)) + 4 * (5000 + 300)
    # the workspace holds 12 bytes of strengths per line of each job, and the split-item scratch
    assert s.batch_bytes(reqs) > 12 * (4 * 5300 + 40_000)


def test_a_request_over_the_budget_is_rejected_without_launching():
    r = _req(0, 500_001)
    s = _server(_server(1 << 40).batch_bytes([r]) - 1)        # one byte short of what it needs alone
    assert s.run([r], realtime=False) == []
    assert s.rejected == [r] and s.launches == 0


def test_batches_stop_at_the_memory_budget_and_the_work_bound():
    reqs = [_req(k, 1000) for k in range(6)]
    probe = _server(1 << 40)
    work = {id(r): probe.work(r) for r in reqs}
    three = probe.batch_bytes(reqs[:3])
    s = _server(three + 1000)
    assert s._form_batch(reqs, 0, 32, work) == reqs[:3]            # the 4th would exceed the budget
    assert s._form_batch(reqs, three, 32, work) == []              # nothing fits next to 3 in flight
    s = _server(1 << 40, batch_evals=2.5 * work[id(reqs[0])])
    assert s._form_batch(reqs, 0, 32, work) == reqs[:2]            # the work bound
    s = _server(1 << 40, batch_evals=1.0)
    assert s._form_batch(reqs, 0, 32, work) == reqs[:1]            # a larger request still runs alone
    assert _server(1 << 40)._form_batch(reqs, 0, 4, work) == reqs[:4]   # max_batch


def test_work_estimate():
    s = _server(1 << 40)
    assert s.work(_req(0, 100)) == (4 * 100 + 20_000) * 100
    assert s.work(_req(0, 100_000)) == (4 * 100_000 + 20_000) * 5001


@pytest.mark.parametrize("wait", [0.0])
def test_requests_waiting_too_long_are_rejected(wait):
    s = _server(1 << 40, max_wait_s=wait)
    s.streams = []                                              # no slot ever frees: every request waits
    reqs = [_req(k, 100, t=0.0) for k in range(3)]
    import time
    t0 = time.perf_counter()
    assert s.run(reqs, realtime=False) == []
    assert len(s.rejected) == 3 and time.perf_counter() - t0 < 5.0
