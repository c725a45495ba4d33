"""Continuous-batching job server on one GPU.

A job asks for the real schemes of n sign vectors of one resident
triangulation: the sign vectors of the splitmix64 counters base, base + 1, ...
(word w of counter k is splitmix64(k * W + w), cut to |A| bits).  The result is the job's histogram of schemes and, if the
job asks for it, the code of every sign vector.

Jobs queue in arrival order.  The scheduler keeps up to ``slots`` jobs on the
GPU at once, each on its own CUDA stream with its own resident device
histogram, so their kernels overlap on the device.  A waiting job is admitted
as soon as a slot is free and the device memory it needs (its sign-vector and
code buffers when it wants codes; nothing else, the histograms are resident)
fits in what the running jobs leave of ``mem_budget``; jobs that finish free
their slot and memory at once, so admission is continuous rather than batch by
batch.  Triangulations (with their kernels prepared) and histograms stay
resident for the server's life.  A job whose launch or result raises (a CUDA
error, failed instances, an overflow that cannot be recovered) fails its own
future only; its slot and memory return to the pool and the server goes on.

The scheduling logic talks to the device through an executor; the GPU
executor drives the C ABI, and tests can pass a fake one to check admission on
the CPU.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Dict, List, Optional


@dataclass
class Job:
    tri: int                 # index of a resident triangulation
    n: int                   # sign vectors
    base: int                # splitmix64 counter of the first sign vector
    want_codes: bool = False
    words: int = 2           # sign words + code words per sign vector (set by the server)
    submitted: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    future: Future = field(default_factory=Future)

    def mem_bytes(self) -> int:
        return 8 * self.words * self.n if self.want_codes else 0   # masks + codes


@dataclass
class Result:
    hist: Dict[int, int]
    codes: Optional[object]  # numpy uint64 array when requested
    latency: float            # seconds from submission to completion
    queued: float             # seconds spent waiting for admission


class GpuExecutor:
    """Runs jobs through the engine: ts_enumerate with TS_ENUM_SPLITMIX into
    the slot's resident histogram, plus ts_splitmix_masks and ts_real_schemes
    when the job wants codes."""

    # histogram size classes: a job of n sign vectors has at most n distinct
    # schemes; the class is the smallest >= n, capped (random sign vectors of
    # degree <= 16 give some 10^4 schemes per 2^22 vectors; a job that still
    # overflows is re-run with a table of its own size)
    CLASSES = (1 << 10, 1 << 14, 1 << 18)

    def __init__(self, tris, slots: int, kernel: Optional[int] = None):
        import torch
        self.torch = torch
        self.tris = list(tris)
        if kernel is not None:
            for t in self.tris:
                t.set_kernel(kernel)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        # resident histograms per slot, by (code words, size class), made on first use
        self.hists: List[Dict[tuple, object]] = [{} for _ in range(slots)]
        self.cur: Dict[int, object] = {}
        self.events = [torch.cuda.Event() for _ in range(slots)]
        self.buffers: Dict[int, tuple] = {}

    def _hist(self, slot: int, cw: int, n: int):
        from . import Histogram
        cap = next((c for c in self.CLASSES if c >= n), self.CLASSES[-1])
        h = self.hists[slot].get((cw, cap))
        if h is None:
            h = self.hists[slot][(cw, cap)] = Histogram(cap, cw)
        return h

    def start(self, slot: int, job: Job):
        from . import TS_ENUM_SPLITMIX, enumerate_schemes, splitmix_masks
        torch = self.torch
        st = self.streams[slot]
        tri = self.tris[job.tri]
        h = self.cur[slot] = self._hist(slot, tri.code_words, job.n)
        with torch.cuda.stream(st):
            h.clear(st)
            enumerate_schemes(tri, job.base, job.base + job.n, h, TS_ENUM_SPLITMIX, stream=st)
            if job.want_codes:
                masks = torch.empty((job.n, tri.sign_words), dtype=torch.int64, device="cuda")
                codes = torch.empty((job.n, tri.code_words), dtype=torch.int64, device="cuda")
                splitmix_masks(tri.d, job.base, job.n, masks, stream=st)
                tri.real_schemes(masks, out=codes, stream=st, sync=False)
                self.buffers[slot] = (masks, codes)
            self.events[slot].record(st)

    def words(self, job: Job) -> int:
        t = self.tris[job.tri]
        return t.sign_words + t.code_words

    def done(self, slot: int) -> bool:
        return self.events[slot].query()

    def result(self, slot: int, job: Job):
        from . import TS_ENUM_SPLITMIX, Histogram, TSError, code_to_int, enumerate_schemes
        st = self.streams[slot]
        tri = self.tris[job.tri]
        try:
            codes, counts, failed = self.cur[slot].read(st)
        except TSError as e:
            if e.status != 5:  # TS_EOVERFLOW: more schemes than the class holds
                raise
            big = Histogram(job.n, tri.code_words)
            enumerate_schemes(tri, job.base, job.base + job.n, big, TS_ENUM_SPLITMIX, stream=st)
            codes, counts, failed = big.read(st)
            big.close()
        if failed:
            raise RuntimeError(f"{failed} instances failed")
        hist = {code_to_int(c): int(k) for c, k in zip(codes, counts)}
        out = None
        if slot in self.buffers:
            masks, cbuf = self.buffers.pop(slot)
            self.tris[job.tri].sync(st)
            out = cbuf.cpu().numpy().view("uint64").copy()
            if out.shape[1] == 1:
                out = out[:, 0]
            del masks, cbuf
        return hist, out


class Server:
    def __init__(self, executor, slots: int, mem_budget: int):
        self.ex = executor
        self.slots = slots
        self.mem_budget = mem_budget
        self.queue: collections.deque = collections.deque()
        self.running: Dict[int, Job] = {}
        self.free: List[int] = list(range(slots))
        self.mem_used = 0
        self.peak_mem = 0
        self.peak_running = 0
        self.completed: List[Job] = []
        self.failed: List[Job] = []     # jobs whose start or result raised
        self.cv = threading.Condition()
        self.stop_flag = False
        self.error: Optional[BaseException] = None
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def submit(self, job: Job) -> Future:
        if hasattr(self.ex, "words"):
            job.words = self.ex.words(job)
        if job.mem_bytes() > self.mem_budget:
            raise ValueError("job needs more device memory than the server's budget")
        job.submitted = time.perf_counter()
        with self.cv:
            self.queue.append(job)
            self.cv.notify()
        return job.future

    def close(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify()
        self.thread.join()
        if self.error:
            raise self.error

    def _loop(self):
        try:
            while True:
                with self.cv:
                    if self.stop_flag and not self.queue and not self.running:
                        return
                    # continuous admission: FIFO, while a slot and the memory allow
                    while (self.queue and self.free and
                           self.mem_used + self.queue[0].mem_bytes() <= self.mem_budget):
                        job = self.queue.popleft()
                        slot = self.free.pop()
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
                    try:
                        hist, codes = self.ex.result(slot, job)
                        err = None
                    except Exception as e:  # this job fails; the others keep running
                        err = e
                    job.finished = time.perf_counter()
                    with self.cv:
                        del self.running[slot]
                        self.free.append(slot)
                        self.mem_used -= job.mem_bytes()
                        if err is None:
                            self.completed.append(job)
                    if err is not None:
                        self._fail(job, err)
                        continue
                    job.future.set_result(Result(hist, codes, job.finished - job.submitted,
                                                 job.admitted - job.submitted))
                if not finished:
                    with self.cv:
                        if not self.queue or not self.free:
                            self.cv.wait(timeout=0.0002)
        except BaseException as e:  # a failure of the scheduler itself ends it
            self.error = e
            with self.cv:
                for j in list(self.queue) + list(self.running.values()):
                    if not j.future.done():
                        j.future.set_exception(e)

    def _fail(self, job: Job, err: BaseException):
        job.finished = time.perf_counter()
        self.failed.append(job)
        job.future.set_exception(err)

    def latencies(self) -> List[float]:
        return [j.finished - j.submitted for j in self.completed]


def percentile(xs, q: float) -> float:
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]
