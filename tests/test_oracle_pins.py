"""Pins of the CPU oracle against things other than itself: hand-worked
cases, brute force on tiny inputs, exhaustive enumeration, closed forms and
invariants (paper, Sec. 2).  CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute, check

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _as_dict(keys, cnt, n):
    return dict(zip(oracle.keys_to_strs(keys, n), [int(c) for c in cnt]))


def _golden_cases(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("case:"):
                yield [p.strip() for p in line[5:].split("|")]


# ------------------------------------------------------------------ counting

def test_count_hand_cases():
    for reads, k, want in _golden_cases("count_hand.txt"):
        ascii, offs = synth.reads_from_strings(reads.split(","))
        r = oracle.count(ascii, offs, int(k), 1, mercy=False)
        exp = {kv.split(":")[0]: int(kv.split(":")[1]) for kv in want.split()}
        assert _as_dict(r["solid_keys"], r["solid_cnt"], int(k) + 1) == exp


@pytest.mark.parametrize("seed", range(12))
def test_count_vs_brute_random(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 9))
    d = int(rng.integers(1, 4))
    ascii, offs = synth.random_reads(seed, int(rng.integers(1, 40)), 0, 30, p_invalid=0.05,
                                     p_lower=0.1, alphabet=b"ACGT" if seed % 3 else b"AC")
    reads = [bytes(ascii[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)]
    r = oracle.count(ascii, offs, k, d, mercy=True)
    assert _as_dict(r["solid_keys"], r["solid_cnt"], k + 1) == brute.solid(reads, k, d)
    assert _as_dict(r["mercy_keys"], r["mercy_cnt"], k + 1) == brute.mercy(reads, k, d)
    assert r["n_kmers"] == sum(brute.count(reads, k).values())


def test_count_exhaustive_single_reads():
    """Every read over {A,C,G,T}^L, L <= 6, k = 2, d in {1, 2}."""
    for L in range(0, 7):
        for tup in itertools.product("ACGT", repeat=L):
            read = "".join(tup)
            ascii, offs = synth.reads_from_strings([read])
            for d in (1, 2):
                r = oracle.count(ascii, offs, 2, d, mercy=False)
                assert _as_dict(r["solid_keys"], r["solid_cnt"], 3) == brute.solid([read], 2, d)


def test_count_sum_invariant():
    """With d = 1 every distinct (k+1)-mer is kept: counts sum to
    |K| = 2 * sum over fragments of max(0, L - k)."""
    ascii, offs = synth.random_reads(7, 300, 0, 60, p_invalid=0.02)
    for k in (3, 8, 21, 31, 32, 63, 64, 100):
        r = oracle.count(ascii, offs, k, 1, mercy=False)
        frags = brute.fragments([bytes(ascii[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)])
        n = 2 * sum(max(0, len(f) - k) for f in frags)
        assert r["n_kmers"] == n
        assert int(r["solid_cnt"].astype(np.uint64).sum()) == n
        check.check_kmers(r["solid_keys"], r["solid_cnt"], k, 1)


def test_key_width_boundaries():
    """31/32, 63/64 symbols: the word count changes exactly where 2(k+1)
    crosses 64 and 128 bits, and packed keys decode back to the strings."""
    assert [oracle.words_for(k) for k in (2, 31, 32, 63, 64, 127)] == [1, 1, 2, 2, 4, 4]
    read = "ACGTTGCAAGTCCATGGATCCAGTTGACGTAGCATGCAAGTCAGTCAGGCTTAGCAGTCGATCGATGCAGTCGATGCATGCATGCTAGCTAGGCTAGCTAGCTAGCTGACTGACTAGCTAGCATCGATCGATCGAT"
    for k in (31, 32, 63, 64, 127):
        ascii, offs = synth.reads_from_strings([read, read])
        r = oracle.count(ascii, offs, k, 1, mercy=False)
        got = _as_dict(r["solid_keys"], r["solid_cnt"], k + 1)
        assert got == brute.solid([read, read], k, 1)


def test_closed_form_single_genome():
    """Error-free high-coverage reads of one random genome: the solid set is
    every genome (k+1)-mer on both strands, there is no mercy edge, and the
    SdBG is two simple paths: t = 2 dummy edges, u = 2 '$' edges, no minus
    flag, m = 2 (G - k) + 4."""
    G, k = 3000, 21
    ascii, offs, genome = synth.genome_tiling_reads(5, G, 80, 3)
    g = genome.decode()
    kmers = [g[i:i + k + 1] for i in range(G - k)]
    kmers_rc = [brute.rc(x) for x in kmers]
    nodes = [g[i:i + k] for i in range(G - k + 1)]
    assert len(set(kmers + kmers_rc)) == 2 * len(kmers)          # no repeat (w.h.p.)
    assert len(set(nodes + [brute.rc(x) for x in nodes])) == 2 * len(nodes)
    r = oracle.count(ascii, offs, k, 2, mercy=True)
    assert set(oracle.keys_to_strs(r["solid_keys"], k + 1)) == set(kmers + kmers_rc)
    assert r["mercy_keys"].shape[0] == 0
    sd = oracle.build_sdbg(k, r["solid_keys"], r["solid_cnt"], r["mercy_keys"], r["mercy_cnt"])
    assert sd["t"] == 2 and sd["u"] == 2
    assert sd["m"] == 2 * (G - k) + 4
    assert not np.any(sd["W"] > 4)
    assert sorted(oracle.keys_to_strs(sd["aux"], k)) == sorted([g[:k], brute.rc(g[-k:])])
    check.check_sdbg(sd, k, r["solid_keys"], r["solid_cnt"])


# --------------------------------------------------------------------- mercy

def test_mercy_hand_cases():
    for reads, want in _golden_cases("mercy_hand.txt"):
        ascii, offs = synth.reads_from_strings(reads.split(","))
        r = oracle.count(ascii, offs, 2, 2, mercy=True)
        exp = {kv.split(":")[0]: int(kv.split(":")[1]) for kv in want.split()}
        assert _as_dict(r["mercy_keys"], r["mercy_cnt"], 3) == exp


@pytest.mark.parametrize("seed", range(8))
def test_mercy_flank_gap_flank(seed):
    """High-coverage left and right flanks of a random genome, one low-coverage
    read across the gap: mercy = the gap edges and their reverse complements
    (k = 9, d = 2), checked against the all-pairs brute force."""
    rng = np.random.default_rng(100 + seed)
    k = 9
    g = "".join(rng.choice(list("ACGT"), size=120))
    left, right = g[0:40], g[70:110]
    span = g[20:90]
    reads = [left] * 3 + [right] * 3 + [span]
    ascii, offs = synth.reads_from_strings(reads)
    r = oracle.count(ascii, offs, k, 2, mercy=True)
    got = _as_dict(r["mercy_keys"], r["mercy_cnt"], k + 1)
    assert got == brute.mercy(reads, k, 2)
    gap = {g[j:j + k + 1] for j in range(40 - k, 70)}
    want = gap | {brute.rc(x) for x in gap}
    solid = set(oracle.keys_to_strs(r["solid_keys"], k + 1))
    assert set(got) == want - solid
    check.check_kmers(r["mercy_keys"], r["mercy_cnt"], k, 1, 1)


# ---------------------------------------------------------------------- BOSS

def _golden_boss():
    vals = {}
    with open(os.path.join(GOLDEN, "boss_k2_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or ":" not in line:
                continue
            key, v = line.split(":", 1)
            vals[key.strip()] = v.split()
    return vals


def test_boss_hand_example():
    g = _golden_boss()
    k = int(g["k"][0])
    keys = oracle.strs_to_keys(g["edges"], oracle.words_for(k))
    sd = oracle.build_sdbg(k, keys)
    assert sd["W"].tolist() == [int(x) for x in g["W"]]
    assert sd["last"].tolist() == [int(x) for x in g["last"]]
    assert sd["dummy"].tolist() == [int(x) for x in g["dummy"]]
    assert sd["F"].tolist() == [int(x) for x in g["F"]]
    assert oracle.keys_to_strs(sd["aux"], k) == g["aux"]
    assert (sd["m"], sd["t"], sd["u"]) == (int(g["m"][0]), int(g["t"][0]), int(g["u"][0]))
    assert np.all(sd["valid"] == 1)
    check.check_sdbg(sd, k, keys)


@pytest.mark.parametrize("seed", range(10))
def test_boss_vs_brute_random_edges(seed):
    """Random edge sets (not closed under reverse complement), k = 2..6."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 7))
    n = int(rng.integers(1, 60))
    edges = sorted({"".join(rng.choice(list("ACG" if seed % 2 else "ACGT"), size=k + 1))
                    for _ in range(n)})
    keys = oracle.strs_to_keys(edges, oracle.words_for(k))
    sd = oracle.build_sdbg(k, keys)
    b = brute.boss(edges, k)
    assert sd["W"].tolist() == b["W"]
    assert sd["last"].tolist() == b["last"]
    assert sd["dummy"].tolist() == b["dummy"]
    assert sd["F"].tolist() == b["F"]
    assert oracle.keys_to_strs(sd["aux"], k) == b["aux"]
    check.check_sdbg(sd, k, keys)


@pytest.mark.parametrize("k", [2, 5, 21, 31, 32, 47, 63, 64, 99, 127])
def test_pipeline_invariants(k):
    """Random reads through count, mercy and SdBG; the decoded graph is the
    edge set and every invariant holds."""
    ascii, offs = synth.random_reads(k, 150, 0, k + 40, alphabet=b"ACGT" if k > 8 else b"ACG")
    # duplicate reads so that d = 2 keeps something
    ascii2 = np.concatenate([ascii, ascii[: int(offs[60])]])
    offs2 = np.concatenate([offs, offs[1:61] + offs[-1]])
    r = oracle.count(ascii2, offs2, k, 2, mercy=True)
    check.check_kmers(r["solid_keys"], r["solid_cnt"], k, 2)
    check.check_kmers(r["mercy_keys"], r["mercy_cnt"], k, 1, 1)
    edges = np.concatenate([r["solid_keys"], r["mercy_keys"]])
    mult = np.concatenate([r["solid_cnt"], r["mercy_cnt"]])
    sd = oracle.build_sdbg(k, r["solid_keys"], r["solid_cnt"], r["mercy_keys"], r["mercy_cnt"])
    check.check_sdbg(sd, k, edges, mult[np.lexsort([edges[:, w] for w in range(edges.shape[1])])])
    assert int(sd["last"].sum()) == sd["n_nodes"]


# ----------------------------------------------- the checks catch mistakes

def _corruptions(sd):
    """Plausible slips, planted in a copy of the oracle's output."""
    m = sd["m"]
    W = sd["W"]
    yield "drop minus", dict(sd, W=np.where(W > 4, W - 4, W))
    i = int(np.nonzero((W >= 1) & (W <= 4) & (sd["dummy"] == 0))[0][-1])
    W2 = W.copy(); W2[i] += 4
    yield "extra minus", dict(sd, W=W2)
    L2 = sd["last"].copy(); j = int(np.nonzero(L2 == 1)[0][0]); L2[j] = 0
    yield "merged nodes", dict(sd, last=L2)
    F2 = sd["F"].copy(); F2[3] += 1
    yield "F off by one", dict(sd, F=F2)
    if sd["t"] >= 2:
        yield "aux swapped", dict(sd, aux=sd["aux"][::-1].copy())
    perm = np.arange(m); a = int(np.nonzero(sd["last"][:-1] == 1)[0][len(perm) // 4]);
    perm[[a, a + 1]] = perm[[a + 1, a]]
    yield "two entries swapped", dict(sd, W=W[perm], last=sd["last"][perm], dummy=sd["dummy"][perm])


def test_check_sdbg_rejects_planted_mistakes():
    ascii, offs = synth.uniform_genome_reads(3, 2000, 300, 60, 0.01)
    k = 11
    r = oracle.count(ascii, offs, k, 2, mercy=True)
    edges = np.concatenate([r["solid_keys"], r["mercy_keys"]])
    sd = oracle.build_sdbg(k, r["solid_keys"], r["solid_cnt"], r["mercy_keys"], r["mercy_cnt"])
    assert np.any(sd["W"] > 4) and sd["t"] >= 2
    check.check_sdbg(sd, k, edges)
    for name, bad in _corruptions(sd):
        with pytest.raises(AssertionError):
            check.check_sdbg(bad, k, edges)
            raise RuntimeError("planted mistake not caught: " + name)


def test_lex_instead_of_colex_is_caught():
    """Sorting the edges lexicographically (the misreading of 'reverse
    lexicographic') must fail the decode check."""
    g = _golden_boss()
    k = int(g["k"][0])
    keys = oracle.strs_to_keys(g["edges"], 1)
    b = brute.boss(g["edges"], k)
    rows = sorted(b["rows"], key=lambda r: ("$ACGT".index(r[0][0]), r[0], r[1]))
    W = np.array(["$ACGT".index(r[1]) for r in rows], np.uint8)
    last = np.array([1 if i == len(rows) - 1 or rows[i + 1][0] != r[0] else 0
                     for i, r in enumerate(rows)], np.uint8)
    dummy = np.array([1 if r[2] else 0 for r in rows], np.uint8)
    aux = oracle.strs_to_keys([r[3] for r in rows if r[2]], 1)
    bad = {"W": W, "last": last, "dummy": dummy, "F": np.array(b["F"]), "aux": aux}
    with pytest.raises(AssertionError):
        check.check_sdbg(bad, k, keys)


def test_count_queries_matches_count():
    ascii, offs = synth.uniform_genome_reads(4, 5000, 500, 100, 0.01)
    for k in (21, 40):
        r = oracle.count(ascii, offs, k, 1, mercy=False)
        sel = np.arange(0, r["solid_keys"].shape[0], 7)
        q = r["solid_keys"][sel]
        got = oracle.count_queries(ascii, offs, k, q, n_threads=3)
        assert np.array_equal(got, r["solid_cnt"][sel].astype(np.uint64))
        absent = oracle.strs_to_keys(["A" * (k + 1)], oracle.words_for(k))
        assert oracle.count_queries(ascii, offs, k, absent)[0] == brute.count(
            [bytes(ascii[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)], k).get("A" * (k + 1), 0)


# --------------------------------------------------- fragments and windows

@pytest.mark.parametrize("seed", [11, 12, 13])
def test_fragments_match_brute(seed):
    """orc_fragments (the oracle behind the packing parity) against the
    brute-force split of each read into maximal ACGT runs, upper-cased:
    bases, fragment offsets and the read of every fragment, on random reads
    with N, lower case, empty reads and reads made only of N."""
    ascii, offs = synth.random_reads(seed, 300, 0, 60, p_invalid=0.08, p_lower=0.3)
    lens = np.diff(offs)
    assert (lens == 0).any(), "the case has empty reads"
    a = bytearray(ascii.tobytes())
    a[int(offs[5]):int(offs[6])] = b"N" * int(lens[5])   # a read of N only
    ascii = np.frombuffer(bytes(a), dtype=np.uint8)
    bases, fo, fr = oracle.fragments(ascii, offs)
    want_frags, want_read = [], []
    for r in range(len(offs) - 1):
        for f in brute.fragments([bytes(ascii[int(offs[r]):int(offs[r + 1])])]):
            want_frags.append(f)
            want_read.append(r)
    want_offs = np.concatenate([[0], np.cumsum([len(f) for f in want_frags])]).astype(np.uint64)
    assert bases == "".join(want_frags).encode()
    assert np.array_equal(fo, want_offs)
    assert np.array_equal(fr, np.array(want_read, dtype=np.uint32))


@pytest.mark.parametrize("k", [4, 40])
def test_find_windows_matches_brute_scan(k):
    """orc_find_windows against a scan of every read position: a hit is a
    position whose k+1 bases are all valid (any case) and spell a query."""
    ascii, offs = synth.random_reads(21 + k, 200, 0, 90, p_invalid=0.03, p_lower=0.2, alphabet=b"ACGT")
    nw = oracle.words_for(k)
    rng = np.random.default_rng(k)
    occ = []
    for r in range(len(offs) - 1):
        s = bytes(ascii[int(offs[r]):int(offs[r + 1])]).decode().upper()
        for p in range(len(s) - k):
            w = s[p:p + k + 1]
            if set(w) <= set("ACGT"):
                occ.append((w, r, p))
    picked = sorted({occ[i][0] for i in rng.choice(len(occ), size=40, replace=False)})
    absent = ["".join("ACGT"[c] for c in rng.integers(0, 4, size=k + 1)) for _ in range(10)]
    strs = picked + [a for a in absent if a not in {o[0] for o in occ}]
    qi = {s: i for i, s in enumerate(strs)}
    want = sorted((qi[w], r, p) for w, r, p in occ if w in qi)
    hq, hr, hp = oracle.find_windows(ascii, offs, k, oracle.strs_to_keys(strs, nw))
    got = sorted(zip(hq.tolist(), hr.tolist(), hp.tolist()))
    assert got == want and len(want) >= 40


@pytest.mark.parametrize("seed,k,d", [(3, 11, 2), (4, 21, 2), (5, 31, 1)])
def test_large_decoder_agrees_with_check_sdbg(seed, k, d):
    """The vectorised decoder that checks the full-size graph
    (tests/sdbg_scan.py) accepts what check.check_sdbg accepts and rejects
    every planted mistake that check.check_sdbg rejects (k = 31 with d = 1,
    so that error k-mers make targets with several in-edges)."""
    import sdbg_scan

    ascii, offs = synth.uniform_genome_reads(seed, 2000, 300, 60, 0.01)
    r = oracle.count(ascii, offs, k, d, mercy=True)
    edges = np.concatenate([r["solid_keys"], r["mercy_keys"]])
    sd = oracle.build_sdbg(k, r["solid_keys"], r["solid_cnt"], r["mercy_keys"], r["mercy_cnt"])
    assert np.any(sd["W"] > 4) and sd["t"] >= 2
    check.check_sdbg(sd, k, edges)
    got = sdbg_scan.check_sdbg_large(sd["W"], sd["last"], sd["dummy"], sd["F"], sd["aux"], k, edges)
    assert got["m"] == sd["m"] and got["t"] == sd["t"] and got["u"] == sd["u"] and got["n_nodes"] == sd["n_nodes"]
    shuffled = edges[np.random.default_rng(seed).permutation(len(edges))]
    sdbg_scan.check_sdbg_large(sd["W"], sd["last"], sd["dummy"], sd["F"], sd["aux"], k, shuffled)
    planted = 0
    for name, bad in _corruptions(sd):
        try:
            check.check_sdbg(bad, k, edges)
            continue  # the slip changed nothing here (e.g. two equal entries swapped)
        except AssertionError:
            planted += 1
        with pytest.raises(AssertionError):
            sdbg_scan.check_sdbg_large(bad["W"], bad["last"], bad["dummy"], bad["F"], bad["aux"], k, edges)
            raise RuntimeError("planted mistake not caught: " + name)
    assert planted >= 4
    # an edge missing from the graph
    with pytest.raises(AssertionError):
        sdbg_scan.check_sdbg_large(sd["W"], sd["last"], sd["dummy"], sd["F"], sd["aux"], k, edges[1:])


@pytest.mark.parametrize("k,threads", [(2, 3), (7, 8), (21, 5), (40, 4)])
def test_threaded_oracle_equals_single_thread(k, threads):
    """The threaded CPU baseline (counting split by 8-symbol prefix, mercy by
    fragment) gives exactly the single-thread oracle's tables."""
    ascii, offs = synth.random_reads(31 + k, 400, 0, 120, p_invalid=0.01, p_lower=0.1, alphabet=b"ACGT")
    g_ascii, g_offs = synth.uniform_genome_reads(k, 3000, 600, 80, 0.01)
    for a, o in ((ascii, offs), (g_ascii, g_offs)):
        one = oracle.count(a, o, k, 2, mercy=True)
        many = oracle.count(a, o, k, 2, mercy=True, threads=threads)
        for key in ("n_kmers", "n_distinct"):
            assert one[key] == many[key]
        for key in ("solid_keys", "solid_cnt", "mercy_keys", "mercy_cnt"):
            assert np.array_equal(one[key], many[key]), key
