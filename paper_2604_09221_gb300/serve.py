"""Continuous-batching job server on one GPU.

A job asks for the real schemes of a set of sign vectors of one resident
triangulation.  Three kinds:

* ``sample``: the sign vectors of the splitmix64 counters base, base + 1, ...,
  base + n - 1 (word w of counter k is splitmix64(k * W + w), cut to |A|
  bits); the result is the job's histogram of schemes and, if the job asks
  for it, the code of every sign vector.
* ``query``: the caller's own sign vectors (an (n, W) uint64 host array, or
  an int64 CUDA tensor of n * W words); the result is the code of every sign
  vector and their histogram.
* ``enum``: an exhaustive range of the sweep, the masks m(k) for k in
  [lo, hi) under ts_enumerate's flags (0, TS_ENUM_FLIP or TS_ENUM_REDUCED);
  the result is the histogram.

Jobs queue in arrival order.  The scheduler keeps up to ``slots`` jobs on the
GPU at once, each on its own CUDA stream, so their kernels overlap on the
device.  A waiting job is admitted as soon as a slot is free and the device
memory it needs fits in what the running jobs leave of the budget; jobs that
finish free their slot and memory at once, so admission is continuous rather
than batch by batch.  The budget is ``mem_budget`` minus what the executor
keeps resident for the server's life (triangulations with their kernels, and
each slot's histograms, one per code width and size class); a job's own
memory is its sign-vector and code buffers, plus a dedicated histogram when
it needs one: a job whose schemes overflow its slot's largest resident
histogram goes back to the front of the queue with a histogram of its own,
sized for all its sign vectors and counted in its memory.

Reading a finished job's histogram and copying its codes to the host happen
on a worker thread, not on the scheduler thread, so admission goes on
meanwhile; the job's slot and memory return when its result is complete.  A
job whose launch or result raises (a CUDA error, failed instances) fails its
own future only; its slot and memory return to the pool and the server goes
on.

The scheduling logic talks to the device through an executor; the GPU
executor drives the C ABI, and tests can pass a fake one to check admission on
the CPU.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Dict, List, Optional

KINDS = ("sample", "query", "enum")


class HistogramOverflow(Exception):
    """The job has more distinct schemes than the histogram it ran with."""


@dataclass
class Job:
    tri: int                 # index of a resident triangulation
    n: int = 0               # sample: sign vectors
    base: int = 0            # sample: splitmix64 counter of the first sign vector
    want_codes: bool = False  # sample: also return every code (query always does)
    kind: str = "sample"     # "sample", "query" or "enum"
    signs: object = None     # query: (n, W) uint64 host array or int64 CUDA tensor
    lo: int = 0              # enum: the range [lo, hi) of the sweep ...
    hi: int = 0
    flags: int = 0           # ... under ts_enumerate's flags
    words: int = 2           # sign words + code words per sign vector (set by the server)
    hist_bytes: int = 0      # a dedicated histogram (set after an overflow)
    submitted: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    future: Future = field(default_factory=Future)

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown job kind {self.kind!r}")
        if self.kind == "query":
            if self.signs is None:
                raise ValueError("a query job needs its sign vectors")
            self.n = len(self.signs) if hasattr(self.signs, "__len__") else 0
        if self.kind == "enum":
            if self.hi < self.lo:
                raise ValueError("enum job: hi < lo")
            self.n = self.hi - self.lo

    def mem_bytes(self) -> int:
        """Device memory the job holds while it runs."""
        buffers = self.kind == "query" or (self.kind == "sample" and self.want_codes)
        return (8 * self.words * self.n if buffers else 0) + self.hist_bytes


@dataclass
class Result:
    hist: Dict[int, int]
    codes: Optional[object]  # numpy uint64 array for query jobs and sample jobs that want codes
    latency: float            # seconds from submission to completion
    queued: float             # seconds spent waiting for admission
    kind: str = "sample"


def hist_bytes(capacity: int, code_words: int) -> int:
    """Device bytes of a ts_hist of the given capacity (ts_hist_create: slots
    = the power of two >= 2 x capacity, at least 16; keys and counts, their
    packed copies for ts_hist_read, and four counter words)."""
    s = 16
    while s < 2 * capacity:
        s <<= 1
    return 2 * s * 8 * (code_words + 1) + 32


class GpuExecutor:
    """Runs jobs through the engine: ts_enumerate with TS_ENUM_SPLITMIX (sample)
    or the job's flags (enum) into a histogram, ts_real_schemes on device sign
    vectors (query, and sample jobs that want codes: ts_splitmix_masks
    first)."""

    # histogram size classes kept resident per slot and code width: a job of
    # n sign vectors has at most n distinct schemes, and its class is the
    # smallest >= n, capped (random sign vectors of degree <= 16 give some
    # 10^4 schemes per 2^22 vectors); a job that still overflows is re-run
    # with a histogram of its own
    CLASSES = (1 << 10, 1 << 14, 1 << 18)

    def __init__(self, tris, slots: int, kernel: Optional[int] = None, classes=None):
        import torch

        from . import Histogram
        if classes is not None:
            self.CLASSES = tuple(sorted(classes))
        self.torch = torch
        self.tris = list(tris)
        if kernel is not None:
            for t in self.tris:
                t.set_kernel(kernel)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        cws = sorted({t.code_words for t in self.tris})
        # resident histograms: every slot, code width and size class, made now
        self.hists = [{(cw, c): Histogram(c, cw) for cw in cws for c in self.CLASSES}
                      for _ in range(slots)]
        self.resident = slots * sum(hist_bytes(c, cw) for cw in cws for c in self.CLASSES)
        self.cur: List[object] = [None] * slots
        self.own: List[object] = [None] * slots      # a job's dedicated histogram
        self.buffers: List[Optional[tuple]] = [None] * slots
        self.events = [torch.cuda.Event() for _ in range(slots)]

    def resident_bytes(self) -> int:
        return self.resident

    def words(self, job: Job) -> int:
        t = self.tris[job.tri]
        return t.sign_words + t.code_words

    def code_words(self, job: Job) -> int:
        return self.tris[job.tri].code_words

    def _hist(self, slot: int, job: Job):
        from . import Histogram
        cw = self.tris[job.tri].code_words
        if job.hist_bytes:   # sized for all the job's sign vectors
            self.own[slot] = Histogram(max(job.n, 1), cw)
            return self.own[slot]
        cap = next((c for c in self.CLASSES if c >= job.n), self.CLASSES[-1])
        return self.hists[slot][(cw, cap)]

    def start(self, slot: int, job: Job):
        from . import TS_ENUM_SPLITMIX, enumerate_schemes, splitmix_masks
        torch = self.torch
        st = self.streams[slot]
        tri = self.tris[job.tri]
        self.buffers[slot] = None
        with torch.cuda.stream(st):
            if job.kind == "query":
                codes = torch.empty((job.n, tri.code_words), dtype=torch.int64, device="cuda")
                signs = job.signs
                if not (hasattr(signs, "is_cuda") and signs.is_cuda):
                    host = signs if hasattr(signs, "is_pinned") else torch.from_numpy(
                        signs.reshape(job.n, tri.sign_words).view("int64"))
                    signs = torch.empty(host.shape, dtype=torch.int64, device="cuda")
                    signs.copy_(host, non_blocking=True)
                tri.real_schemes(signs, out=codes, stream=st, sync=False)
                self.buffers[slot] = (signs, codes)
                self.cur[slot] = None
            else:
                h = self.cur[slot] = self._hist(slot, job)
                h.clear(st)
                if job.kind == "enum":
                    enumerate_schemes(tri, job.lo, job.hi, h, job.flags, stream=st)
                else:
                    enumerate_schemes(tri, job.base, job.base + job.n, h, TS_ENUM_SPLITMIX, stream=st)
                    if job.want_codes:
                        masks = torch.empty((job.n, tri.sign_words), dtype=torch.int64, device="cuda")
                        codes = torch.empty((job.n, tri.code_words), dtype=torch.int64, device="cuda")
                        splitmix_masks(tri.d, job.base, job.n, masks, stream=st)
                        tri.real_schemes(masks, out=codes, stream=st, sync=False)
                        self.buffers[slot] = (masks, codes)
            self.events[slot].record(st)

    def done(self, slot: int) -> bool:
        return self.events[slot].query()

    def result(self, slot: int, job: Job):
        """(hist, codes) of a finished job; raises HistogramOverflow if its
        schemes did not fit the histogram it ran with."""
        import numpy as np

        from . import TSError, code_to_int
        st = self.streams[slot]
        tri = self.tris[job.tri]
        try:
            hist = None
            if self.cur[slot] is not None:
                try:
                    codes, counts, failed = self.cur[slot].read(st)
                except TSError as e:
                    if e.status == 5:  # TS_EOVERFLOW: more schemes than the table holds
                        raise HistogramOverflow() from e
                    raise
                if failed:
                    raise RuntimeError(f"{failed} instances failed")
                hist = {code_to_int(c): int(k) for c, k in zip(codes, counts)}
            out = None
            if self.buffers[slot] is not None:
                _, cbuf = self.buffers[slot]
                tri.sync(st)
                out = cbuf.cpu().numpy().view("uint64").copy()
                if out.shape[1] == 1:
                    out = out[:, 0]
                if hist is None:   # a query job: the histogram of its codes
                    if out.ndim == 1:
                        u, c = np.unique(out, return_counts=True)
                        hist = {int(a): int(b) for a, b in zip(u, c)}
                    else:
                        hist = dict(collections.Counter(code_to_int(r) for r in out))
            return hist, out
        finally:
            self.buffers[slot] = None
            if self.own[slot] is not None:
                self.own[slot].close()
                self.own[slot] = None


class Server:
    def __init__(self, executor, slots: int, mem_budget: int, result_workers: int = 2):
        self.ex = executor
        self.slots = slots
        resident = executor.resident_bytes() if hasattr(executor, "resident_bytes") else 0
        if resident > mem_budget:
            raise ValueError("the executor's resident memory exceeds the server's budget")
        self.resident = resident
        self.mem_budget = mem_budget - resident  # what jobs may hold
        self.queue: collections.deque = collections.deque()
        self.running: Dict[int, Job] = {}
        self.finishing: Dict[int, Job] = {}      # results being read on a worker thread
        self.free: List[int] = list(range(slots))
        self.mem_used = 0
        self.peak_mem = 0
        self.peak_running = 0
        self.completed: List[Job] = []
        self.failed: List[Job] = []     # jobs whose start or result raised
        self.requeued: List[Job] = []   # jobs re-run with a histogram of their own
        self.cv = threading.Condition()
        self.stop_flag = False
        self.error: Optional[BaseException] = None
        self.workers = ThreadPoolExecutor(max_workers=result_workers)
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def submit(self, job: Job) -> Future:
        if hasattr(self.ex, "words"):
            job.words = self.ex.words(job)
        if job.kind == "query" and not (hasattr(job.signs, "is_cuda") and job.signs.is_cuda):
            job.signs = self._pinned(job)
        if job.mem_bytes() > self.mem_budget:
            raise ValueError("job needs more device memory than the server's budget")
        job.submitted = time.perf_counter()
        with self.cv:
            self.queue.append(job)
            self.cv.notify()
        return job.future

    def _pinned(self, job: Job):
        """A query job's host sign vectors in page-locked memory (copied on the
        caller's thread), so that the slot's stream copies them to the device
        asynchronously."""
        try:
            import torch
        except ImportError:
            return job.signs
        if not torch.cuda.is_available() or not hasattr(job.signs, "view"):
            return job.signs
        host = torch.from_numpy(job.signs.reshape(job.n, -1).view("int64"))
        return host.pin_memory()

    def close(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify()
        self.thread.join()
        self.workers.shutdown(wait=True)
        if self.error:
            raise self.error

    def _loop(self):
        try:
            while True:
                with self.cv:
                    if (self.stop_flag and not self.queue and not self.running
                            and not self.finishing):
                        return
                    # continuous admission: FIFO, while a slot and the memory allow
                    while (self.queue and self.free and
                           self.mem_used + self.queue[0].mem_bytes() <= self.mem_budget):
                        job = self.queue.popleft()
                        slot = self.free.pop()
                        if not job.admitted:
                            job.admitted = time.perf_counter()
                        try:
                            self.ex.start(slot, job)
                        except Exception as e:  # this job fails; the slot stays free
                            self.free.append(slot)
                            self._fail(job, e)
                            continue
                        self.running[slot] = job
                        self.mem_used += job.mem_bytes()
                        self.peak_mem = max(self.peak_mem, self.mem_used)
                        self.peak_running = max(self.peak_running, len(self.running))
                    running = list(self.running.items())
                finished = [(s, j) for s, j in running if self.ex.done(s)]
                for slot, job in finished:
                    with self.cv:
                        del self.running[slot]
                        self.finishing[slot] = job
                    self.workers.submit(self._finish, slot, job)
                if not finished:
                    with self.cv:
                        if not self.queue or not self.free:
                            self.cv.wait(timeout=0.0002)
        except BaseException as e:  # a failure of the scheduler itself ends it
            self.error = e
            with self.cv:
                for j in (list(self.queue) + list(self.running.values())
                          + list(self.finishing.values())):
                    if not j.future.done():
                        j.future.set_exception(e)

    def _finish(self, slot: int, job: Job):
        """On a worker thread: read the job's result, then return its slot and
        memory (an overflowed job goes back to the front of the queue with a
        histogram of its own)."""
        overflow = False
        try:
            hist, codes = self.ex.result(slot, job)
            err = None
        except HistogramOverflow as e:
            overflow, err = not job.hist_bytes, e
        except Exception as e:  # this job fails; the others keep running
            err = e
        with self.cv:
            del self.finishing[slot]
            self.free.append(slot)
            self.mem_used -= job.mem_bytes()
            if overflow:
                cw = self.ex.code_words(job) if hasattr(self.ex, "code_words") else 1
                job.hist_bytes = hist_bytes(max(job.n, 1), cw)
                if job.mem_bytes() <= self.mem_budget:
                    self.requeued.append(job)
                    self.queue.appendleft(job)
                    self.cv.notify()
                    return
                err = ValueError("the job's own histogram exceeds the server's budget")
            job.finished = time.perf_counter()
            if err is None:
                self.completed.append(job)
            self.cv.notify()
        if err is not None:
            self._fail(job, err)
            return
        job.future.set_result(Result(hist, codes, job.finished - job.submitted,
                                     job.admitted - job.submitted, job.kind))

    def _fail(self, job: Job, err: BaseException):
        job.finished = time.perf_counter()
        with self.cv:
            self.failed.append(job)
        job.future.set_exception(err)

    def latencies(self, kind: Optional[str] = None) -> List[float]:
        return [j.finished - j.submitted for j in self.completed if kind in (None, j.kind)]


def percentile(xs, q: float) -> float:
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]
