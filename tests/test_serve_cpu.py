"""The serving loop's scheduling on CPU, with a runner that sleeps instead of
running kernels: FIFO admission, the HBM budget never exceeded by admitted
and resident jobs, overlap of jobs across slots, failures isolated, results
held until released.  No GPU."""
import threading
import time

import numpy as np
import pytest

from paper_1409_7208_gb300 import serve


def _job(n_reads, k=31, tag=None):
    L = 100
    ascii = np.zeros(n_reads * L, dtype=np.uint8)
    offs = np.arange(n_reads + 1, dtype=np.uint64) * L
    return serve.Job(ascii, offs, k, 2, tag)


class SleepRunner:
    def __init__(self, secs=0.02):
        self.secs = secs
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.order = []

    def __call__(self, job, slot):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.order.append(job.tag)
        time.sleep(self.secs)
        with self.lock:
            self.running -= 1
        if job.tag == "fail":
            raise RuntimeError("planted failure")
        return {"value": job.tag}


def test_overlap_fifo_and_budget():
    r = SleepRunner()
    jobs = [_job(1000 + i, tag=i) for i in range(40)]
    budget = int(3.5 * jobs[0].est)
    srv = serve.Server(slots=8, hbm_budget=budget, runner=r, auto_release=True)
    for j in jobs:
        srv.submit(j)
    for j in jobs:
        j.wait(10)
    srv.close()
    assert r.order == list(range(40)), "admission is FIFO"
    assert 2 <= r.max_running <= 3, "overlap, bounded by the budget"
    assert srv.max_held <= budget
    assert all(j.start_t >= j.submit_t and j.end_t > j.start_t for j in jobs)


def test_results_held_until_released():
    r = SleepRunner(0.005)
    a, b, c = _job(500, tag="a"), _job(500, tag="b"), _job(500, tag="c")
    srv = serve.Server(slots=4, hbm_budget=2 * a.est, runner=r)
    srv.submit(a)
    srv.submit(b)
    srv.submit(c)
    a.wait(5)
    b.wait(5)
    assert a.result == {"value": "a"}
    time.sleep(0.1)
    assert not c.done.is_set(), "c waits for memory held by a and b"
    a.release()
    c.wait(5)
    assert c.result == {"value": "c"}
    b.release()
    c.release()
    srv.close()


def test_failed_job_releases_and_others_run():
    r = SleepRunner(0.005)
    jobs = [_job(300, tag=t) for t in (0, "fail", 2, 3)]
    srv = serve.Server(slots=2, hbm_budget=10 * jobs[0].est, runner=r, auto_release=True)
    for j in jobs:
        srv.submit(j)
    with pytest.raises(RuntimeError):
        jobs[1].wait(5)
    for j in (jobs[0], jobs[2], jobs[3]):
        j.wait(5)
    srv.close()


def test_oversized_job_runs_alone():
    r = SleepRunner(0.01)
    small = [_job(200, tag=i) for i in range(3)]
    big = _job(100000, tag="big")
    srv = serve.Server(slots=4, hbm_budget=big.est // 2, runner=r, auto_release=True)
    srv.submit(small[0])
    srv.submit(big)
    srv.submit(small[1])
    for j in small[:2] + [big]:
        j.wait(5)
    srv.close()
    assert big.start_t >= small[0].end_t, "runs when nothing else is held"
    assert small[1].start_t >= big.end_t, "FIFO behind the big job"


def test_batch_read_counts_follow_the_batched_config():
    """64 read counts: lognormal around a median of 500k (the geometric mean
    of the bounds), clipped to [50k, 5M], even (pairs), reproducible."""
    import numpy as np

    import synth
    c = synth.batch_read_counts(5, 64)
    assert len(c) == 64 and np.array_equal(c, synth.batch_read_counts(5, 64))
    assert c.min() >= 50_000 - 1 and c.max() <= 5_000_000 and np.all(c % 2 == 0)
    big = synth.batch_read_counts(11, 20_000)
    assert 0.8 * 500_000 < np.median(big) < 1.2 * 500_000
    # sigma is a quarter of ln(5M / 50k): about 2.3% of the mass beyond each bound
    assert 0.01 < np.mean(big >= 5_000_000) < 0.04 and 0.01 < np.mean(big <= 50_000) < 0.04
