"""Scheduling logic of the continuous-batching server, on CPU with a fake
executor: every job completes with its own result, jobs are admitted in
arrival order as slots and memory free up (not batch by batch), the device
memory in use never exceeds the budget, oversized jobs are refused."""
import threading
import time

import pytest

from paper_2604_09221_gb300.serve import Job, Server, percentile


class FakeExecutor:
    """Job (tri, n, base) 'runs' for n microseconds; its result is a function of
    the job only."""

    def __init__(self):
        self.t_end = {}
        self.order = []
        self.lock = threading.Lock()

    def start(self, slot, job):
        with self.lock:
            self.order.append((job.tri, job.base))
            self.t_end[slot] = time.perf_counter() + job.n * 1e-6

    def done(self, slot):
        return time.perf_counter() >= self.t_end[slot]

    def result(self, slot, job):
        return {job.tri * 1000 + job.base % 97: job.n}, None


def test_every_job_completes_with_its_own_result():
    ex = FakeExecutor()
    srv = Server(ex, slots=4, mem_budget=1 << 20)
    jobs = [Job(tri=i % 5, n=200 + 37 * i, base=1000 + i) for i in range(60)]
    futs = [srv.submit(j) for j in jobs]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    for j, r in zip(jobs, res):
        assert r.hist == {j.tri * 1000 + j.base % 97: j.n}
        assert r.latency >= r.queued >= 0
    assert srv.peak_running == 4
    assert [(j.tri, j.base) for j in jobs] == ex.order  # FIFO admission


def test_admission_respects_the_memory_budget():
    ex = FakeExecutor()
    budget = 16 * 5000
    srv = Server(ex, slots=8, mem_budget=budget)
    jobs = [Job(tri=0, n=2000 + 100 * (i % 7), base=i, want_codes=True) for i in range(30)]
    futs = [srv.submit(j) for j in jobs]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    assert srv.peak_mem <= budget
    assert srv.peak_running <= 2      # 2 x 2000 x 16 bytes fit, 3 do not
    with pytest.raises(ValueError):
        Server(FakeExecutor(), 1, 100).submit(Job(tri=0, n=10, base=0, want_codes=True))


def test_continuous_admission_fills_a_freed_slot_before_the_batch_drains():
    ex = FakeExecutor()
    srv = Server(ex, slots=2, mem_budget=1 << 20)
    long = srv.submit(Job(tri=0, n=1000000, base=0))     # 1 s
    short = [srv.submit(Job(tri=1, n=1000, base=i)) for i in range(1, 6)]
    for f in short:
        r = f.result(timeout=30)
        assert r.latency < 0.8    # served while the long job still runs
    assert not long.done()
    long.result(timeout=30)
    srv.close()


def test_percentile():
    xs = list(range(101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99


class FlakyExecutor(FakeExecutor):
    """Fails to launch the job with base 7 and to read the job with base 13."""

    def start(self, slot, job):
        if job.base == 7:
            raise RuntimeError("launch failed")
        super().start(slot, job)

    def result(self, slot, job):
        if job.base == 13:
            raise RuntimeError("3 instances failed")
        return super().result(slot, job)


def test_a_failing_job_fails_alone():
    ex = FlakyExecutor()
    srv = Server(ex, slots=3, mem_budget=16 * 4000)
    jobs = [Job(tri=i % 3, n=300 + 11 * i, base=i, want_codes=i % 2 == 0) for i in range(24)]
    futs = [srv.submit(j) for j in jobs]
    for j, f in zip(jobs, futs):
        if j.base in (7, 13):
            with pytest.raises(RuntimeError):
                f.result(timeout=30)
        else:
            assert f.result(timeout=30).hist == {j.tri * 1000 + j.base % 97: j.n}
    # the server keeps serving, and every slot and byte came back
    assert srv.submit(Job(tri=1, n=50, base=99)).result(timeout=30).hist == {1000 + 99 % 97: 50}
    srv.close()
    assert sorted(j.base for j in srv.failed) == [7, 13]
    assert len(srv.completed) == 23 and srv.mem_used == 0 and sorted(srv.free) == [0, 1, 2]
