"""The request server's scheduling (``mh_server_*`` in libmh) on CPU, in its
dry-run mode: no device work, a job takes n_reads microseconds on the host.
FIFO admission, the HBM budget never exceeded by admitted and resident jobs
(by the library's own estimate), overlap of jobs across slots, results held
until released, a job larger than the budget alone.  No GPU."""
import time

import numpy as np
import pytest

from paper_1409_7208_gb300 import serve


def _job(n_reads, k=31, tag=None):
    L = 100
    ascii = np.zeros(n_reads * L, dtype=np.uint8)
    offs = np.arange(n_reads + 1, dtype=np.uint64) * L
    return serve.Job(ascii, offs, k, 2, tag)


def _max_overlap(jobs):
    ev = sorted([(j.start_t, 1) for j in jobs] + [(j.end_t, -1) for j in jobs], key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, e in ev:
        cur += e
        best = max(best, cur)
    return best


def test_estimate_is_the_library_formula():
    j = _job(1000, k=31)
    windows = j.n_bases - j.n_reads * 31
    assert j.est == (64 << 20) + 48 * windows + 2 * j.n_bases + (512 << 20)
    assert _job(1000, k=47).est - (64 << 20) - 2 * j.n_bases - (512 << 20) == 2 * 48 * (j.n_bases - 1000 * 47)


def test_overlap_fifo_and_budget():
    jobs = [_job(20000 + i, tag=i) for i in range(24)]
    budget = int(3.5 * jobs[-1].est)
    srv = serve.Server(slots=8, hbm_budget=budget, auto_release=True, dry_run=True)
    for j in jobs:
        srv.submit(j)
    for j in jobs:
        j.wait(30)
    assert srv.max_held <= budget
    srv.close()
    starts = [j.start_t for j in jobs]
    assert starts == sorted(starts), "admission is FIFO"
    assert 2 <= _max_overlap(jobs) <= 3, "overlap, bounded by the budget"
    assert all(j.start_t >= j.submit_t and j.end_t >= j.start_t + 0.019 for j in jobs)


def test_results_held_until_released():
    a, b, c = _job(5000, tag="a"), _job(5000, tag="b"), _job(5000, tag="c")
    srv = serve.Server(slots=4, hbm_budget=2 * a.est, dry_run=True)
    for j in (a, b, c):
        srv.submit(j)
    a.wait(5)
    b.wait(5)
    time.sleep(0.1)
    assert not c.finished(), "c waits for memory held by a and b"
    assert srv.stats()["held"] == a.est + b.est and srv.stats()["queued"] == 1
    a.release()
    c.wait(5)
    b.release()
    c.release()
    assert srv.stats()["held"] == 0
    with pytest.raises(RuntimeError):
        a.wait(1)  # released: no record any more
    srv.close()


def test_oversized_job_runs_alone():
    small = [_job(20000, tag=i) for i in range(3)]
    big = _job(100000, tag="big")
    srv = serve.Server(slots=4, hbm_budget=big.est // 2, auto_release=True, dry_run=True)
    srv.submit(small[0])
    srv.submit(big)
    srv.submit(small[1])
    for j in small[:2] + [big]:
        j.wait(5)
    srv.close()
    assert big.start_t >= small[0].end_t, "runs when nothing else is held"
    assert small[1].start_t >= big.end_t, "FIFO behind the big job"


def test_wait_times_out_and_bad_arguments_are_rejected():
    slow = _job(300000, tag="slow")  # 0.3 s
    srv = serve.Server(slots=1, dry_run=True)
    srv.submit(slow)
    with pytest.raises(TimeoutError):
        slow.wait(0.01)
    slow.wait(5)
    with pytest.raises(Exception):
        srv.submit(_job(10, k=1))
    srv.close()


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
