"""Serving on the GPU through the library's request server: every job's
result is the same alone and in the mix (jobs of different sizes and k
admitted while others run, on four streams), bit for bit, and a mixed job
agrees with the oracle; a failing job is reported while the others finish;
the admission estimate covers each job's measured peak."""
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


def test_failed_job_is_reported_and_the_others_run():
    """A job whose read offsets run backwards fails in the packing step with
    its error; the jobs around it finish and match the oracle."""
    from paper_1409_7208_gb300 import MhError, serve
    good = _jobs()[:3]
    ascii, offs = synth.uniform_genome_reads(77, 5000, 200, 100, 0.01)
    bad_offs = offs.copy()
    bad_offs[5], bad_offs[6] = bad_offs[6], bad_offs[5]
    bad = serve.Job(ascii, bad_offs, 31, 2, tag="bad")
    srv = serve.Server(slots=2, hbm_budget=1 << 40)
    for j in (good[0], bad, good[1], good[2]):
        srv.submit(j)
    with pytest.raises(MhError):
        bad.wait(120)
    for j in good:
        j.wait(120)
    w = oracle.count(good[2].ascii, good[2].offs, good[2].k, 2, mercy=True)
    got = _fetch(good[2])
    assert np.array_equal(got["sk"], w["solid_keys"]) and np.array_equal(got["mk"], w["mercy_keys"])
    for j in good + [bad]:
        j.release()
    assert srv.stats()["held"] == 0
    srv.close()


def test_admission_estimate_covers_the_measured_peak():
    """mh_job_bytes, the estimate jobs are admitted by, is at least the
    device memory a job really holds at its peak (the library's own pool,
    host input, whole path), for every key width."""
    import paper_1409_7208_gb300 as mh
    from paper_1409_7208_gb300 import serve
    # sizes where the per-window term of the estimate outweighs its fixed part
    for seed, (n_reads, L, k) in enumerate([(200000, 150, 21), (200000, 150, 31), (150000, 150, 47),
                                            (80000, 150, 99), (300000, 100, 27)]):
        ascii, offs = synth.uniform_genome_reads(300 + seed, 2000000, n_reads, L, 0.01)
        ctx = mh.Context(device=0, torch_allocator=False)
        reads = mh.mh_pack_reads(ctx, ascii, offs)
        solid = mh.mh_count_kmers(ctx, reads, k, 2)
        mercy = mh.mh_mercy_kmers(ctx, reads, solid)
        g = mh.mh_build_sdbg(ctx, solid, mercy)
        peak = ctx.memory()[1]
        est = serve.estimate_bytes(ascii, offs, k)
        assert 0 < peak <= est, (k, peak, est)
        for h in (g, mercy, solid, reads):
            h.free()
        ctx.close()
