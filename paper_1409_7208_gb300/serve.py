"""Serving over the C ABI: a thin wrapper of the library's request server
(``mh_server_*``).

Jobs (one read set, k, d) arrive at any time.  The server's ``slots``
worker threads, each with a worker context of its own (stream and
stream-ordered pool), take jobs from one first-in first-out queue; a job is
admitted when a slot is free and its estimated device memory
(``mh_job_bytes``) fits the HBM budget next to the jobs running and the
results still held, or when nothing is held.  Jobs that arrive while others
run are admitted as slots and memory free up, and their work overlaps on the
device.  A job's result (solid and mercy tables, SdBG) stays resident until
the client releases it, and counts against the budget until then.  The
scheduling and every step of a job run in libmh; this module only marshals
arguments and converts the server's clock to ``time.perf_counter``.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import (MH_BATCH_BUILD, MH_BATCH_MERCY, MH_ETIMEOUT, MH_OK, MH_SERVE_AUTO_RELEASE, MH_SERVE_DRY_RUN,
               Context, JobInfo, Kmers, MhError, ReadSet, Sdbg, SetResult, _ptr_of, _strerror, load_library)


def _read_set(ascii, offs):
    """(ReadSet, kept arrays) for host numpy arrays or torch tensors."""
    if isinstance(ascii, np.ndarray):
        ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
    pa, da = _ptr_of(ascii)
    po, do = _ptr_of(offs)
    if da != do:
        raise ValueError("ascii and offs must both be on the host or both on the device")
    n_bases = int(ascii.shape[0])
    return ReadSet(pa if n_bases else None, n_bases, po, int(offs.shape[0]) - 1, da), (ascii, offs)


def estimate_bytes(ascii, offs, k: int) -> int:
    """The library's admission estimate for one job (``mh_job_bytes``)."""
    rs, _ = _read_set(ascii, offs)
    return int(load_library().mh_job_bytes(ctypes.byref(rs), int(k)))


class Job:
    """A count + mercy + build request.  Times (``submit_t``, ``start_t``,
    ``end_t``) are on ``time.perf_counter``'s clock."""

    def __init__(self, ascii, offs, k: int, d: int = 2, tag=None):
        self.ascii, self.offs, self.k, self.d, self.tag = ascii, offs, k, d, tag
        self.n_bases = int(len(ascii))
        self.n_reads = int(len(offs)) - 1
        self.est = estimate_bytes(ascii, offs, k)
        self.submit_t = self.start_t = self.end_t = None
        self.slot = None
        self.status = None
        self.result = None
        self.id = None
        self._server = None
        self._keep = None

    @property
    def latency(self) -> float:
        return self.end_t - self.submit_t

    def finished(self) -> bool:
        """True once the job has ended (without waiting)."""
        return self._server is not None and self._server._wait(self, 0.0)

    def wait(self, timeout=None) -> "Job":
        """Wait for the job to end; raises TimeoutError if it has not ended
        within ``timeout`` seconds, MhError if it failed."""
        if self._server is None:
            raise RuntimeError("job not submitted, or already released")
        if not self._server._wait(self, -1.0 if timeout is None else float(timeout)):
            raise TimeoutError("job not finished")
        if self.status != MH_OK:
            raise MhError(self.status, "job %r failed: %s" % (self.tag, _strerror(self.status)))
        return self

    def release(self):
        """Free the resident result and return its memory to the budget."""
        if self._server is not None:
            self._server._release(self)


class _WorkerContext(Context):
    """A server's worker context, owned by the server: its kernel statistics
    and the device its results live on."""

    def __init__(self, lib, h, device: int):
        import torch
        self._lib, self._h = lib, h
        self.device = torch.device("cuda", device)

    def close(self):
        self._h = None


class Server:
    """``slots`` workers under an HBM budget on GPU ``device``.
    ``auto_release`` frees each result as soon as its job ends.  ``dry_run``
    runs no device work (a job takes ``n_reads`` microseconds on the host):
    the scheduling alone, without a GPU."""

    def __init__(self, slots: int = 4, hbm_budget: int = 150 << 30, device: int = 0, auto_release: bool = False,
                 dry_run: bool = False):
        lib = load_library()
        self._lib = lib
        self.slots = slots
        self.budget = hbm_budget
        self.dry_run = dry_run
        self.ctx = None if dry_run else Context(device=device, torch_allocator=False)
        flags = MH_BATCH_MERCY | MH_BATCH_BUILD | (MH_SERVE_AUTO_RELEASE if auto_release else 0) | \
            (MH_SERVE_DRY_RUN if dry_run else 0)
        h = ctypes.c_void_p()
        self._t0 = time.perf_counter()  # the server's clock starts inside the call
        rc = lib.mh_server_create(self.ctx.handle if self.ctx else None, int(slots), int(hbm_budget), flags,
                                  ctypes.byref(h))
        if rc != MH_OK:
            raise MhError(rc, "mh_server_create failed")
        self._h = h
        self.contexts = [] if dry_run else [
            _WorkerContext(lib, lib.mh_server_context(h, i), device) for i in range(slots)]

    def submit(self, job: Job) -> Job:
        rs, job._keep = _read_set(job.ascii, job.offs)
        jid = ctypes.c_uint64()
        rc = self._lib.mh_server_submit(self._h, ctypes.byref(rs), int(job.k), int(job.d), ctypes.byref(jid))
        if rc != MH_OK:
            raise MhError(rc, "mh_server_submit failed")
        job.id = jid.value
        job._server = self
        return job

    def _wait(self, job: Job, timeout: float) -> bool:
        res, info = SetResult(), JobInfo()
        rc = self._lib.mh_server_wait(self._h, job.id, timeout, ctypes.byref(res), ctypes.byref(info))
        if rc == MH_ETIMEOUT:
            return False
        if rc != MH_OK:
            raise MhError(rc, "mh_server_wait failed")
        job.submit_t = self._t0 + info.submit_s
        job.start_t = self._t0 + info.start_s
        job.end_t = self._t0 + info.end_s
        job.slot = info.slot
        job.status = info.status
        if job.result is None and res.solid:
            wc = self.contexts[info.slot]
            job.result = {"solid": Kmers(wc, res.solid), "mercy": Kmers(wc, res.mercy) if res.mercy else None,
                          "sdbg": Sdbg(wc, res.sdbg) if res.sdbg else None}
            for v in job.result.values():
                if v is not None:
                    v.borrowed = True
        return True

    def _release(self, job: Job):
        if job._server is not self:
            return
        rc = self._lib.mh_server_release(self._h, job.id)
        if rc != MH_OK:
            raise MhError(rc, "mh_server_release: the job has not ended")
        if isinstance(job.result, dict):
            for v in job.result.values():
                if v is not None:
                    v._h = None
        job.result = None
        job._server = None
        job._keep = None

    def stats(self) -> dict:
        a, b, c, d = (ctypes.c_uint64() for _ in range(4))
        self._lib.mh_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
        return {"held": a.value, "max_held": b.value, "queued": c.value, "running": d.value}

    @property
    def max_held(self) -> int:
        return self.stats()["max_held"]

    def reset_max(self):
        self._lib.mh_server_reset_max(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mh_server_destroy(self._h)
            self._h = None
            for c in self.contexts:
                c.close()
            if self.ctx is not None:
                self.ctx.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
