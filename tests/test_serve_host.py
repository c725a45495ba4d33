"""Scheduling logic of the continuous-batching server, on CPU with a fake
executor: every job completes with its own result, jobs are admitted in
arrival order as slots and memory free up (not batch by batch), the device
memory in use never exceeds the budget, oversized jobs are refused."""
import collections
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


def test_job_kinds_and_their_memory():
    import numpy as np

    from paper_2604_09221_gb300.serve import Job
    q = Job(tri=0, kind="query", signs=np.zeros((300, 2), dtype=np.uint64), words=5)
    assert q.n == 300 and q.mem_bytes() == 8 * 5 * 300        # signs and codes on the device
    e = Job(tri=0, kind="enum", lo=1000, hi=5096, flags=1)
    assert e.n == 4096 and e.mem_bytes() == 0                 # histogram only
    s = Job(tri=0, n=100, base=0, want_codes=True, words=3)
    assert s.mem_bytes() == 8 * 3 * 100
    s.hist_bytes = 12345
    assert s.mem_bytes() == 8 * 3 * 100 + 12345
    with pytest.raises(ValueError):
        Job(tri=0, kind="query")
    with pytest.raises(ValueError):
        Job(tri=0, kind="enum", lo=5, hi=4)
    with pytest.raises(ValueError):
        Job(tri=0, kind="bogus")


class ResidentExecutor(FakeExecutor):
    def __init__(self, resident):
        super().__init__()
        self.resident = resident

    def resident_bytes(self):
        return self.resident


def test_resident_memory_counts_against_the_budget():
    ex = ResidentExecutor(16 * 3000)
    srv = Server(ex, slots=8, mem_budget=16 * 3000 + 16 * 4500)
    jobs = [Job(tri=0, n=2000, base=i, want_codes=True) for i in range(12)]
    for f in [srv.submit(j) for j in jobs]:
        f.result(timeout=30)
    srv.close()
    assert srv.peak_running <= 2 and srv.peak_mem <= 16 * 4500   # 2 jobs of 32000 bytes fit, 3 do not
    with pytest.raises(ValueError):
        Server(ResidentExecutor(1000), slots=1, mem_budget=999)


class OverflowExecutor(FakeExecutor):
    """Jobs with n > 500 overflow the resident histogram; with a histogram of
    their own (hist_bytes set by the server) they succeed."""

    def __init__(self):
        super().__init__()
        self.runs = collections.Counter()

    def code_words(self, job):
        return 1

    def start(self, slot, job):
        self.runs[job.base] += 1
        super().start(slot, job)

    def result(self, slot, job):
        from paper_2604_09221_gb300.serve import HistogramOverflow
        if job.n > 500 and not job.hist_bytes:
            raise HistogramOverflow()
        return super().result(slot, job)


def test_an_overflowing_job_reruns_with_its_own_histogram():
    from paper_2604_09221_gb300.serve import hist_bytes
    ex = OverflowExecutor()
    srv = Server(ex, slots=3, mem_budget=1 << 20)
    jobs = [Job(tri=0, n=100 + 97 * i, base=i) for i in range(10)]
    for j, f in zip(jobs, [srv.submit(j) for j in jobs]):
        assert f.result(timeout=30).hist == {j.base % 97: j.n}
    srv.close()
    big = [j for j in jobs if j.n > 500]
    assert sorted(j.base for j in srv.requeued) == sorted(j.base for j in big)
    assert all(ex.runs[j.base] == (2 if j.n > 500 else 1) for j in jobs)
    assert all(j.hist_bytes == hist_bytes(j.n, 1) for j in big)
    assert srv.mem_used == 0 and sorted(srv.free) == [0, 1, 2]
    # a job whose own histogram exceeds the budget fails alone
    srv = Server(OverflowExecutor(), slots=1, mem_budget=hist_bytes(600, 1) - 1)
    with pytest.raises(ValueError):
        srv.submit(Job(tri=0, n=600, base=1)).result(timeout=30)
    assert srv.submit(Job(tri=0, n=50, base=2)).result(timeout=30).hist == {2: 50}
    srv.close()


class SlowReadExecutor(FakeExecutor):
    """Reading the result of the job with base 0 waits for an event."""

    def __init__(self):
        super().__init__()
        self.release = threading.Event()

    def result(self, slot, job):
        if job.base == 0:
            assert self.release.wait(timeout=30)
        return super().result(slot, job)


def test_reading_a_result_does_not_stop_admission():
    ex = SlowReadExecutor()
    srv = Server(ex, slots=2, mem_budget=1 << 20, result_workers=2)
    slow = srv.submit(Job(tri=0, n=10, base=0))
    quick = [srv.submit(Job(tri=1, n=1000, base=i)) for i in range(1, 9)]
    for f in quick:   # admitted, run and read while the slow read still waits
        f.result(timeout=30)
    assert not slow.done()
    ex.release.set()
    assert slow.result(timeout=30).hist == {0: 10}
    srv.close()
    assert srv.mem_used == 0 and sorted(srv.free) == [0, 1]
