"""Sort paths that only large inputs reach, run on inputs small enough for
the oracle by a child process with a tuning variable set: the radix sort's
multi-chunk path (several look-back chains per pass, digit offsets carried
between chunks; 1 or 3 tiles per chunk), and the count sort's fix-up of
keys sharing their top bits (passes over the top 8, 16 or 24 bits only, so
that groups of every size occur: a few keys sorted by one thread, tens to
thousands by a warp or a CTA, and crowded groups by the segment fallback),
the key-value form of the spread order for solid tables (thread, warp and
segment sorts of groups), the out-of-core count (2 or 16 buckets of keys counted one at a time,
spectra concatenated, solid tables merged), and reads streamed from host
memory through staging pieces of 48 bytes or 4 KB (pieces that end inside a
read, reads that span several pieces, invalid bytes found mid-stream).

The unit counting (8-bit passes over the top bits, then each unit sorted
and counted by a warp; the inputs have k = 21 and 31, 47, 99: 1-, 2- and
4-word keys) is forced through its rarer paths the
same way: units too large for a warp's shared memory (counted from global
memory one distinct key a round, or, with too many distinct keys, set aside,
sorted by the general radix sort and counted from the sorted keys), one unit
holding every key, many nearly empty units under three passes, and runs of
one key thousands of windows long (a read repeated 7,000 times); and many
units set aside at once (gathered, sorted together, moved back).  The spread
route (passes over the top bits, a fix-up, a run pass) stays selectable and
is checked as well."""
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
ctx = mh.Context(device=0)
shifts = (30 - 2 * np.arange(16)).astype(np.uint32)
for a, o in (synth.random_reads(5, 400, 0, 300), synth.random_reads(6, 300, 0, 200, p_invalid=0.02),
             synth.random_reads(7, 50, 0, 40, p_lower=0.3)):
    bases, fo, fr = oracle.fragments(a, o)
    r = mh.mh_pack_reads(ctx, a, o).tensors()
    codes = np.zeros((len(bases) + 15) // 16 * 16, dtype=np.uint32)
    codes[: len(bases)] = np.frombuffer(bases, dtype=np.uint8) if isinstance(bases, bytes) else bases
    lut = np.zeros(256, dtype=np.uint32)
    lut[list(b"ACGT")] = np.arange(4, dtype=np.uint32)
    words = np.bitwise_or.reduce(lut[codes].reshape(-1, 16) << shifts, axis=1).astype(np.uint32)
    assert r["n_packed"] == len(bases) and r["n_frags"] == len(fr)
    assert np.array_equal(r["packed"].cpu().numpy().view(np.uint32), words)
    assert np.array_equal(r["frag_offs"].cpu().numpy().view(np.uint64), fo)
    assert np.array_equal(r["frag_read"].cpu().numpy().view(np.uint32), fr)
def repeated(seed):
    # one 40-base read 7,000 times among random reads: runs longer than a unit holds
    a, o = synth.uniform_genome_reads(seed, 4000, 800, 150, 0.01)
    rep = np.frombuffer(bytes(a[:40]), dtype=np.uint8)
    ascii = np.concatenate([np.tile(rep, 7000), a])
    offs = np.concatenate([np.arange(7000, dtype=np.uint64) * 40, o.astype(np.uint64) + 7000 * 40])
    return ascii, offs
for seed, k, n_reads in ((1, 21, 3000), (2, 31, 2500), (3, 47, 1500), (4, 99, 900), (5, 21, 0)):
    if n_reads:
        ascii, offs = synth.uniform_genome_reads(seed, 4000, n_reads, 150, 0.01)
    else:
        ascii, offs = repeated(seed)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    s = mh.mh_count_kmers(ctx, reads, k, 2)
    m = mh.mh_mercy_kmers(ctx, reads, s)
    g = mh.mh_build_sdbg(ctx, s, m)
    w = oracle.count(ascii, offs, k, 2, mercy=True)
    wg = oracle.build_sdbg(k, w["solid_keys"], w["solid_cnt"], w["mercy_keys"], w["mercy_cnt"])
    gs, gm, gg = s.numpy(), m.numpy(), g.numpy()
    assert np.array_equal(gs["keys"], w["solid_keys"]) and np.array_equal(gs["counts"], w["solid_cnt"])
    assert np.array_equal(gm["keys"], w["mercy_keys"]) and np.array_equal(gm["counts"], w["mercy_cnt"])
    for key in ("W", "last", "dummy", "F", "aux"):
        assert np.array_equal(gg[key], wg[key]), key
print("ok")
""" % ROOT


@pytest.mark.parametrize("env", [
    {"MH_SORT_CHUNK_TILES": "1"}, {"MH_SORT_CHUNK_TILES": "3"},
    {"MH_COUNT_PATH": "spread", "MH_SPREAD_BITS": "8"}, {"MH_COUNT_PATH": "spread", "MH_SPREAD_BITS": "16"},
    {"MH_COUNT_PATH": "spread", "MH_SPREAD_BITS": "24"}, {"MH_COUNT_PATH": "spread"},
    {"MH_GROUP_CAP": "16"}, {"MH_GROUP_CAP": "200"}, {"MH_GROUP_UNIT_BITS": "0"},
    {"MH_GROUP_UNIT_BITS": "6", "MH_GROUP_CAP": "64"},
    {"MH_GROUP_UNIT_BITS": "14"}, {"MH_GROUP_UNIT_BITS": "22", "MH_SORT_CHUNK_TILES": "3"},
    {"MH_COUNT_BUCKET_BITS": "1"}, {"MH_COUNT_BUCKET_BITS": "4"},
    {"MH_COUNT_BUCKET_BITS": "4", "MH_COUNT_PATH": "spread"}, {"MH_SPREAD_KV_MIN": "0"},
    {"MH_PACK_PIECE": "48"}, {"MH_PACK_PIECE": "4096"},
    {"MH_EXTRACT_SCATTER": "1"}, {"MH_EXTRACT_SCATTER": "1", "MH_SORT_CHUNK_TILES": "1"},
    {"MH_EXTRACT_SCATTER": "1", "MH_SORT_VARIANT": "1"},
    {"MH_EXTRACT_SCATTER": "1", "MH_SCATTER_CAP": "5000", "MH_GROUP_UNIT_BITS": "22", "MH_SORT_CHUNK_TILES": "3"}],
    ids=lambda e: ",".join("%s=%s" % kv for kv in e.items()))
def test_small_input_paths_match_oracle(env):
    # every run also sorts the small solid tables by the spread key-value path
    full = dict(os.environ, MH_SPREAD_KV_MIN="0")
    full.update(env)
    p = subprocess.run([sys.executable, "-c", CHILD], env=full, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "ok" in p.stdout


SET_ASIDE = r"""
import sys, numpy as np
sys.path.insert(0, %r)
import oracle, synth, paper_1409_7208_gb300 as mh
k, n_reads = int(sys.argv[1]), int(sys.argv[2])
ctx = mh.Context(device=0, profile=True)
# reads of independent random bases: nearly every key distinct, so a unit
# over the lowered cap has more distinct keys than the global-memory path
# takes, and is set aside
ascii, offs = synth.random_reads(11 + k, n_reads, 150, 150)
reads = mh.mh_pack_reads(ctx, ascii, offs)
s = mh.mh_count_kmers(ctx, reads, k, 1)
w = oracle.count(ascii, offs, k, 1, mercy=False)
gs = s.numpy()
assert np.array_equal(gs["keys"], w["solid_keys"]) and np.array_equal(gs["counts"], w["solid_cnt"])
prof = ctx.profile()
assert prof.get("move_units", (0,))[0] == 2, "the set-aside units were sorted together: %%r" %% sorted(prof)
print("ok")
""" % ROOT


@pytest.mark.parametrize("k,n_reads,bits,cap", [(31, 6000, 13, 110), (47, 5000, 12, 160), (99, 8000, 12, 130)])
def test_many_set_aside_units_sorted_together(k, n_reads, bits, cap):
    """A few per cent of the units over the cap, each with more than 64
    distinct keys: they are gathered, sorted by one spread sort and moved
    back (1-, 2- and 4-word keys), and the count equals the oracle's."""
    env = dict(os.environ, MH_GROUP_UNIT_BITS=str(bits), MH_GROUP_CAP=str(cap))
    p = subprocess.run([sys.executable, "-c", SET_ASIDE, str(k), str(n_reads)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "ok" in p.stdout


FUSED = r"""
import sys, numpy as np
sys.path.insert(0, %r)
import oracle, synth, paper_1409_7208_gb300 as mh
n_reads, expect = int(sys.argv[1]), sys.argv[2].split(",")
ctx = mh.Context(device=0, profile=True)
ascii, offs = synth.metagenome_reads(seed=9, n_genomes=20, median_len=2e5, n_pairs=n_reads // 2)
reads = mh.mh_pack_reads(ctx, ascii, offs)
s = mh.mh_count_kmers(ctx, reads, 31, 2)
w = oracle.count(ascii, offs, 31, 2, mercy=False)
gs = s.numpy()
assert np.array_equal(gs["keys"], w["solid_keys"]) and np.array_equal(gs["counts"], w["solid_cnt"])
prof = ctx.profile()
for name in expect:
    assert (name[1:] not in prof) if name.startswith("-") else (name in prof), (name, sorted(prof))
print("ok")
""" % ROOT


@pytest.mark.parametrize("n_reads,env,expect", [
    (4000, {"MH_EXTRACT_SCATTER": "1"}, "extract_scatter,-extract_canonical"),
    (12000, {"MH_EXTRACT_SCATTER": "1"}, "extract_scatter,-extract_canonical"),
    (12000, {"MH_EXTRACT_SCATTER": "1", "MH_SCATTER_CAP": "4096"}, "extract_scatter,extract_canonical"),
    (12000, {"MH_EXTRACT_SCATTER": "0"}, "-extract_scatter,extract_canonical")])
def test_extraction_fused_with_first_pass(n_reads, env, expect):
    """The extraction that makes the first 8-bit pass itself (keys written
    to fixed-size digit segments, then a pass that reads the segments):
    the count equals the oracle's, with the fused kernel in place of the
    plain extraction; with segments too small for their digits (more than
    4,096 keys a digit: 12,000 reads of 150 bp give 1.43 M keys) the
    overflow is caught and the unfused path gives the same count."""
    full = dict(os.environ)
    full.update(env)
    p = subprocess.run([sys.executable, "-c", FUSED, str(n_reads), expect], env=full, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "ok" in p.stdout
