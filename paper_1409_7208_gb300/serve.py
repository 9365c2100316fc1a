"""Serving: a request loop over the C ABI with continuous batching.

Jobs (one read set, k, d) arrive at any time.  A fixed number of worker
slots, each with its own library context and CUDA stream, take jobs from
one FIFO queue; a job is admitted when a slot is free and its estimated
device memory fits the HBM budget next to the jobs in flight and the
results still held on the device.  Jobs that arrive while others run are
admitted as slots and memory free up, and their work overlaps on the device
(one stream per slot).  A job's result (solid and mercy tables, SdBG) stays
resident until the client releases it, and counts against the budget until
then.  Host logic only: every step of a job runs in libmh's kernels.
"""
from __future__ import annotations

import collections
import threading
import time


def key_words(k: int) -> int:
    return 1 if 2 * (k + 1) <= 64 else (2 if 2 * (k + 1) <= 128 else 4)


def estimate_bytes(n_bases: int, n_reads: int, k: int) -> int:
    """Peak device bytes of one job (measured: about 40 bytes per window and
    key word for counting, which dominates), plus a fixed 64 MB."""
    windows = max(0, n_bases - n_reads * k)
    return (64 << 20) + 48 * key_words(k) * windows + 2 * n_bases


class Job:
    """A count + mercy + build request."""

    def __init__(self, ascii, offs, k: int, d: int = 2, tag=None):
        self.ascii, self.offs, self.k, self.d, self.tag = ascii, offs, k, d, tag
        self.n_bases = int(len(ascii))
        self.n_reads = int(len(offs)) - 1
        self.est = estimate_bytes(self.n_bases, self.n_reads, k)
        self.submit_t = self.start_t = self.end_t = None
        self.result = None
        self.error = None
        self.slot = None
        self.done = threading.Event()
        self._server = None

    @property
    def latency(self) -> float:
        return self.end_t - self.submit_t

    def wait(self, timeout=None) -> "Job":
        if not self.done.wait(timeout):
            raise TimeoutError("job not finished")
        if self.error is not None:
            raise self.error
        return self

    def release(self):
        """Free the resident result and return its memory to the budget."""
        if self._server is not None:
            self._server._release(self)


class Server:
    """``slots`` workers under an HBM budget.  ``runner(job, slot)`` runs a
    job and returns its result (a dict of resident handles); the default
    runs the library on GPU ``device``.  ``auto_release`` frees each result
    as soon as its job completes."""

    def __init__(self, slots: int = 4, hbm_budget: int = 150 << 30, runner=None, device: int = 0,
                 auto_release: bool = False):
        self.slots = slots
        self.budget = hbm_budget
        self.auto_release = auto_release
        self.runner = runner if runner is not None else DeviceRunner(device, slots)
        self._q = collections.deque()
        self._cv = threading.Condition()
        self._held = 0          # bytes of admitted, unreleased jobs
        self.max_held = 0
        self._stop = False
        self._threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for t in self._threads:
            t.start()

    def submit(self, job: Job) -> Job:
        job.submit_t = time.perf_counter()
        job._server = self
        with self._cv:
            self._q.append(job)
            self._cv.notify_all()
        return job

    def _fits(self, job: Job) -> bool:
        # a job larger than the whole budget runs when nothing else is held
        return self._held + job.est <= self.budget or self._held == 0

    def _worker(self, slot: int):
        while True:
            with self._cv:
                while not self._stop and not (self._q and self._fits(self._q[0])):
                    self._cv.wait()
                if self._stop and not self._q:
                    return
                job = self._q.popleft()
                self._held += job.est
                self.max_held = max(self.max_held, self._held)
                self._cv.notify_all()
            job.slot = slot
            job.start_t = time.perf_counter()
            try:
                job.result = self.runner(job, slot)
            except Exception as e:  # the job fails; the server keeps serving
                job.error = e
            job.end_t = time.perf_counter()
            if self.auto_release or job.error is not None:
                self._release(job)
            job.done.set()

    def _release(self, job: Job):
        with self._cv:
            if job._server is None:
                return
            job._server = None
            if isinstance(job.result, dict):
                for h in job.result.values():
                    if hasattr(h, "free"):
                        h.free()
            job.result = None
            self._held -= job.est
            self._cv.notify_all()

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()


class DeviceRunner:
    """One library context and one CUDA stream per slot.  The contexts use
    the library's own stream-ordered pools (no Python in the allocation
    path, so the slots' host threads do not contend for the interpreter);
    a slot trims its pool after a job above ``trim_bytes``."""

    def __init__(self, device: int, slots: int, trim_bytes: int = 8 << 30):
        import torch

        from . import Context
        self.trim_bytes = trim_bytes
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.ctxs = [Context(device=device, stream=s, torch_allocator=False) for s in self.streams]

    def __call__(self, job: Job, slot: int) -> dict:
        import torch

        from . import mh_build_sdbg, mh_count_kmers, mh_mercy_kmers, mh_pack_reads
        ctx, s = self.ctxs[slot], self.streams[slot]
        with torch.cuda.stream(s):
            reads = mh_pack_reads(ctx, job.ascii, job.offs)
            solid = mh_count_kmers(ctx, reads, job.k, job.d)
            mercy = mh_mercy_kmers(ctx, reads, solid)
            sdbg = mh_build_sdbg(ctx, solid, mercy)
            reads.free()
        s.synchronize()
        if job.est > self.trim_bytes:
            ctx.trim()
        return {"solid": solid, "mercy": mercy, "sdbg": sdbg}

    def close(self):
        for c in self.ctxs:
            c.close()
