"""Failure detection on the GPU without a GPU fault: a bounded device wait
that runs out, and an allocation that fails, each made on the host side.

* MH_SPIN_LIMIT (a short look-back bound) with MH_TEST_WITHHOLD_TILE0=1 (the
  first scatter launch keeps its tile 0 from publishing its counts): the
  tiles after it give up waiting, the kernel still ends, and mh_count_kmers
  returns MH_ETIMEOUT with no handle and no memory held.  The next count on
  the same context succeeds and matches the oracle.
* MH_FAULT=alloc:N (the N-th device allocation of the process fails as if
  the device were out of memory): the call that met it returns MH_ENOMEM
  with no handle and no memory held; the calls after it succeed and match
  the oracle.

Each case runs in a child process, since the variables are read once."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, %r)
import oracle, synth, paper_1409_7208_gb300 as mh
want_code = int(sys.argv[1])
ascii, offs = synth.uniform_genome_reads(7, 60000, 8000, 150, 0.01)
k, d = 31, 2
ctx = mh.Context(device=0)


def path():
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    solid = mh.mh_count_kmers(ctx, reads, k, d)
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    g = mh.mh_build_sdbg(ctx, solid, mercy)
    return solid.numpy(), mercy.numpy(), g.numpy()


failed, got = None, None
for attempt in range(40):
    before = ctx.memory()[0]
    try:
        got = path()
        break
    except mh.MhError as e:
        assert e.code == want_code, "expected %%d, got %%d (%%s)" %% (want_code, e.code, e)
        failed = attempt
    assert ctx.memory()[0] == before, "memory held after the failed call"
assert failed is not None and got is not None, (failed, got is None)
w = oracle.count(ascii, offs, k, d, mercy=True)
s, m, g = got
assert np.array_equal(s["keys"], w["solid_keys"]) and np.array_equal(s["counts"], w["solid_cnt"])
assert np.array_equal(m["keys"], w["mercy_keys"]) and np.array_equal(m["counts"], w["mercy_cnt"])
wg = oracle.build_sdbg(k, w["solid_keys"], w["solid_cnt"], w["mercy_keys"], w["mercy_cnt"])
for key in ("W", "last", "dummy", "F", "aux"):
    assert np.array_equal(g[key], wg[key]), key
print("ok", failed)
""" % ROOT


def _run(env, code):
    full = dict(os.environ)
    full.update(env)
    p = subprocess.run([sys.executable, "-c", CHILD, str(code)], env=full, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.startswith("ok"), p.stdout
    return int(p.stdout.split()[1])


def test_look_back_wait_runs_out_and_reports_timeout():
    import paper_1409_7208_gb300 as mh

    # the first count fails, the second (same context) succeeds
    assert _run({"MH_SPIN_LIMIT": "20000", "MH_TEST_WITHHOLD_TILE0": "1"}, mh.MH_ETIMEOUT) == 0


@pytest.mark.parametrize("n", [1, 2, 7, 30])
def test_injected_allocation_failure_is_enomem(n):
    import paper_1409_7208_gb300 as mh

    _run({"MH_FAULT": "alloc:%d" % n}, mh.MH_ENOMEM)
