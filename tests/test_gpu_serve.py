"""Serving on the GPU: every job's result is the same alone and in the mix
(jobs of different sizes and k admitted while others run, on four streams),
bit for bit; and a mixed job agrees with the oracle."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _jobs():
    from paper_1409_7208_gb300 import serve
    jobs = []
    for i, (n_reads, L, k) in enumerate([(3000, 100, 21), (800, 150, 31), (5000, 120, 41), (1200, 100, 61),
                                         (2500, 140, 31), (400, 100, 21), (6000, 110, 31), (1500, 150, 41)]):
        ascii, offs = synth.uniform_genome_reads(40 + i, max(5000, n_reads * L // 20), n_reads, L, 0.01)
        jobs.append(serve.Job(ascii, offs, k, 2, tag=i))
    return jobs


def _fetch(job):
    r = job.result
    s, m, g = r["solid"].numpy(), r["mercy"].numpy(), r["sdbg"].numpy()
    return {"sk": s["keys"], "sc": s["counts"], "mk": m["keys"], "mc": m["counts"], "W": g["W"],
            "last": g["last"], "dummy": g["dummy"], "F": g["F"], "aux": g["aux"]}


def test_results_alone_equal_results_in_the_mix():
    from paper_1409_7208_gb300 import serve
    alone = {}
    srv = serve.Server(slots=1, hbm_budget=1 << 40)
    for j in _jobs():
        srv.submit(j).wait(120)
        alone[j.tag] = _fetch(j)
        j.release()
    srv.close()

    srv = serve.Server(slots=4, hbm_budget=1 << 40)
    jobs = _jobs()
    for i, j in enumerate(jobs):
        srv.submit(j)
        if i % 3 == 2:
            time.sleep(0.01)  # some arrive while others run
    for j in jobs:
        j.wait(120)
    assert len({j.slot for j in jobs}) > 1, "jobs ran on several slots"
    for j in jobs:
        got = _fetch(j)
        for key, want in alone[j.tag].items():
            assert np.array_equal(got[key], want), (j.tag, key)
    # one mixed job against the oracle
    j = jobs[1]
    w = oracle.count(j.ascii, j.offs, j.k, 2, mercy=True)
    got = _fetch(j)
    assert np.array_equal(got["sk"], w["solid_keys"]) and np.array_equal(got["mk"], w["mercy_keys"])
    for j in jobs:
        j.release()
    srv.close()
