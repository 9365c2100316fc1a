"""Parity at full size: the simulated metagenome (10 M read pairs, 3.0 Gbp,
k = 31, d = 2) through the C ABI, in the launch configuration bench.py
times (reads resident on the device).

The oracle cannot hold the whole multiset, so it computes sampled outputs one
by one (every count is a scan of all 3 Gbp of reads, on both strands):
  * the counts of randomly chosen solid and mercy (k+1)-mers;
  * the counts of randomly chosen read windows, which decide whether the
    window must (count >= d) or must not be in the solid table;
  * the mercy edges of randomly chosen reads, from the paper's rule with the
    solid graph's degrees taken from oracle counts of every neighbour;
  * the other way round, randomly chosen GPU mercy entries, each traced to
    the reads holding it (an oracle scan) and justified there by the rule;
and properties that hold at any size are checked on the whole output (sorted,
closed under reverse complement on a sample, totals, SdBG block structure),
and the whole SdBG is decoded (tests/sdbg_scan.py) and checked against its
definitions and the solid + mercy edge set.
All comparisons are exact (integers).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K, D = 31, 2
MASK = (1 << 64) - 1
LUT = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(b"ACGT"):
    LUT[_c] = _i


def _key(codes) -> int:
    v = 0
    for c in codes:
        v = (v << 2) | int(c)
    return v


def _rc(x: int) -> int:
    r = 0
    for i in range(K + 1):
        r = (r << 2) | (3 - ((x >> (2 * i)) & 3))
    return r


@pytest.fixture(scope="module")
def run():
    import torch

    import paper_1409_7208_gb300 as mh

    ascii, offs = synth.metagenome_reads()
    ctx = mh.Context(device=0)
    d_ascii = torch.from_numpy(ascii).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    reads = mh.mh_pack_reads(ctx, d_ascii, d_offs)
    solid = mh.mh_count_kmers(ctx, reads, K, D)
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    sdbg = mh.mh_build_sdbg(ctx, solid, mercy)
    out = {"ascii": ascii, "offs": offs, "solid": solid.numpy(), "mercy": mercy.numpy(), "sdbg": sdbg.numpy(),
           "n_frags": reads.view().n_frags}
    del sdbg, mercy, solid, reads
    return out


def _lookup(table_keys, table_counts, q):
    """Counts of the query keys in a sorted 1-word table (0 if absent)."""
    keys = table_keys[:, 0]
    pos = np.searchsorted(keys, q)
    pos = np.minimum(pos, len(keys) - 1)
    hit = keys[pos] == q
    return np.where(hit, table_counts[pos], 0).astype(np.uint64)


def test_totals(run):
    offs = run["offs"]
    lens = np.diff(offs).astype(np.int64)
    windows = int(np.maximum(lens - K, 0).sum())
    assert run["solid"]["n_kmers"] == 2 * windows
    assert run["n_frags"] == len(lens)          # no N in these reads


def test_solid_table_properties(run):
    s = run["solid"]
    keys, cnt = s["keys"][:, 0], s["counts"]
    assert np.all(keys[1:] > keys[:-1]), "solid keys strictly ascending"
    assert int(cnt.min()) >= D
    rng = np.random.default_rng(1)
    idx = rng.integers(0, len(keys), size=4000)
    rcs = np.array([_rc(int(x)) for x in keys[idx]], dtype=np.uint64)
    assert np.array_equal(_lookup(s["keys"], cnt, rcs), cnt[idx].astype(np.uint64)), "closed under rc"


def test_sampled_counts_against_oracle(run):
    s, m = run["solid"], run["mercy"]
    ascii, offs = run["ascii"], run["offs"]
    rng = np.random.default_rng(2)
    si = rng.integers(0, len(s["counts"]), size=300)
    mi = rng.integers(0, len(m["counts"]), size=300)
    # random read windows
    reads = rng.integers(0, len(offs) - 1, size=300)
    wins = []
    for r in reads:
        L = int(offs[r + 1] - offs[r])
        p = int(rng.integers(0, L - K))
        wins.append(_key(LUT[ascii[int(offs[r]) + p:int(offs[r]) + p + K + 1]]))
    wins = np.array(wins, dtype=np.uint64)
    queries = np.concatenate([s["keys"][si, 0], m["keys"][mi, 0], wins])
    want = oracle.count_queries(ascii, offs, K, queries.reshape(-1, 1))
    ns, nm = len(si), len(mi)
    assert np.array_equal(want[:ns], s["counts"][si].astype(np.uint64)), "solid counts"
    assert np.array_equal(want[ns:ns + nm], m["counts"][mi].astype(np.uint64)), "mercy counts"
    assert np.all((want[ns:ns + nm] >= 1) & (want[ns:ns + nm] < D))
    w = want[ns + nm:]
    got = _lookup(s["keys"], s["counts"], wins)
    assert np.array_equal(np.where(w >= D, w, 0), got), "window solid iff its count >= d, with that count"


def test_sampled_reads_mercy_against_oracle(run):
    """Mercy edges of 400 random reads, derived from oracle counts: solidity
    of each window and the degrees of each solid window (its 4 possible
    successors and 4 possible predecessors), then the paper's rule."""
    s, m = run["solid"], run["mercy"]
    ascii, offs = run["ascii"], run["offs"]
    rng = np.random.default_rng(3)
    reads = rng.integers(0, len(offs) - 1, size=400)
    per_read = []
    q = []
    for r in reads:
        seq = LUT[ascii[int(offs[r]):int(offs[r + 1])]]
        ws = [_key(seq[i:i + K + 1]) for i in range(len(seq) - K)]
        per_read.append(ws)
        for x in ws:
            q.append(x)
            q.extend(((x << 2) & MASK) | c for c in range(4))      # successors x[1..k] c
            q.extend((c << (2 * K)) | (x >> 2) for c in range(4))  # predecessors c x[0..k-1]
    qa = np.array(q, dtype=np.uint64)
    uq, inv = np.unique(qa, return_inverse=True)
    cnt = oracle.count_queries(ascii, offs, K, uq.reshape(-1, 1))[inv]
    mercy_keys = m["keys"][:, 0]
    expected = set()
    pos = 0
    for ws in per_read:
        info = []
        for x in ws:
            c9 = cnt[pos:pos + 9]
            pos += 9
            solid = c9[0] >= D
            out0 = not np.any(c9[1:5] >= D)
            in0 = not np.any(c9[5:9] >= D)
            info.append((solid, out0, in0))
        P = [i for i, t in enumerate(info) if t[0]]
        for a, b in zip(P, P[1:]):
            if b > a + 1 and info[a][1] and info[b][2]:
                expected.update(ws[a + 1:b])
    exp = np.array(sorted(expected), dtype=np.uint64)
    if len(exp):
        found = np.searchsorted(mercy_keys, exp)
        found = np.minimum(found, len(mercy_keys) - 1)
        assert np.all(mercy_keys[found] == exp), "a mercy edge of a sampled read is missing"
    # and the sampled reads must yield some mercy edges at this coverage
    assert len(exp) > 0


def test_sdbg_structure(run):
    g = run["sdbg"]
    s, m = run["solid"], run["mercy"]
    E = len(s["counts"]) + len(m["counts"])
    W, last, dummy = g["W"], g["last"].astype(bool), g["dummy"].astype(bool)
    assert g["m"] == E + g["t"] + g["u"] == len(W)
    assert int(dummy.sum()) == g["t"] and int((W == 0).sum()) == g["u"]
    assert int(last.sum()) == g["n_nodes"] and last[-1]
    assert np.all(g["valid"] == 1)
    assert W.max() <= 8 and not np.any((W > 4) & dummy)
    F = g["F"].astype(np.int64)
    assert F[0] == 0 and F[1] == 0 and F[5] == g["m"] and np.all(np.diff(F) >= 0)
    # every node lies inside one F block, and for each symbol the unflagged
    # entries equal the non-dummy nodes of its block (one in-edge per node)
    ends = np.nonzero(last)[0]
    starts = np.concatenate([[0], ends[:-1] + 1])
    blk = np.searchsorted(F, starts, side="right") - 1
    assert np.array_equal(blk, np.searchsorted(F, ends, side="right") - 1)
    node_dummy = dummy[starts]
    for c in range(1, 5):
        assert int((W == c).sum()) == int(((blk == c) & ~node_dummy).sum()), "symbol %d" % c
    # a $ entry is the only entry of its node
    dol = np.nonzero(W == 0)[0]
    assert np.all(last[dol]) and np.all((dol == 0) | last[np.maximum(dol - 1, 0)])
    # dummy nodes hold only dummy entries
    assert np.array_equal(np.add.reduceat(dummy.astype(np.int64), starts) > 0, node_dummy)
    assert np.all(np.add.reduceat(dummy.astype(np.int64), starts)[node_dummy] == (ends - starts + 1)[node_dummy])


def test_bucketed_count_matches_in_memory_count(run):
    """Under a 70 GB budget the same workload is counted in buckets of the
    mixed keys' top bits (reads resident, keys split); its solid and mercy
    tables must equal the in-memory ones exactly."""
    import torch

    import paper_1409_7208_gb300 as mh

    ctx = mh.Context(device=0, hbm_budget=70 << 30)
    d_ascii = torch.from_numpy(run["ascii"]).cuda()
    d_offs = torch.from_numpy(run["offs"].view(np.int64)).cuda()
    reads = mh.mh_pack_reads(ctx, d_ascii, d_offs)
    del d_ascii
    ctx.set_profile(True)
    solid = mh.mh_count_kmers(ctx, reads, K, D)
    ctx.set_profile(False)
    assert ctx.profile().get("extract_bucket", (0, 0, 0))[0] >= 2, "the budget should force buckets"
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    s, m = solid.numpy(), mercy.numpy()
    assert s["n_kmers"] == run["solid"]["n_kmers"] and s["n_distinct"] == run["solid"]["n_distinct"]
    assert np.array_equal(s["keys"], run["solid"]["keys"]) and np.array_equal(s["counts"], run["solid"]["counts"])
    assert np.array_equal(m["keys"], run["mercy"]["keys"]) and np.array_equal(m["counts"], run["mercy"]["counts"])
    del mercy, solid, reads
    ctx.close()


def test_sdbg_full_decode(run):
    """The whole 3.5e8-entry SdBG decoded and checked against its definitions
    (tests/sdbg_scan.py, vectorised on the GPU with torch; pinned against
    oracle/check.py on small graphs): colex order of every node, minus
    flags, the auxiliary store at zero-indegree vertices, '$' entries at
    zero-outdegree vertices, F, and decoded edges == solid + mercy exactly."""
    import torch

    import sdbg_scan

    g, s, m = run["sdbg"], run["solid"], run["mercy"]
    edges = np.concatenate([s["keys"][:, 0], m["keys"][:, 0]])
    got = sdbg_scan.check_sdbg_large(g["W"], g["last"], g["dummy"], g["F"], g["aux"], K, edges, device="cuda")
    assert got["m"] == g["m"] and got["t"] == g["t"] and got["u"] == g["u"] and got["n_nodes"] == g["n_nodes"]
    assert got["edges"] == len(edges)
    torch.cuda.empty_cache()


def test_sampled_gpu_mercy_edges_are_justified(run):
    """Every one of 300 randomly sampled GPU mercy entries is justified by a
    read, from oracle scans of all 3 Gbp (paper, Sec. 2, third paragraph):
    the entry or its reverse complement occurs as a window of some read,
    strictly between two consecutive solid windows of that read, the first
    without a solid successor and the second without a solid predecessor
    (degrees from oracle counts); and the occurrences add up to the entry's
    count.  Together with the subset check above, the mercy table is checked
    in both directions on samples."""
    s, m = run["solid"], run["mercy"]
    ascii, offs = run["ascii"], run["offs"]
    mk = m["keys"][:, 0]
    rng = np.random.default_rng(4)
    # sample among entries no larger than their reverse complement, so that no
    # two sampled queries are the same key
    idx = []
    while len(idx) < 300:
        i = int(rng.integers(0, len(mk)))
        if int(mk[i]) <= _rc(int(mk[i])) and i not in idx:
            idx.append(i)
    idx = np.array(idx)
    e = mk[idx]
    rce = np.array([_rc(int(x)) for x in e], dtype=np.uint64)
    pal = e == rce
    queries = np.concatenate([e, rce[~pal]])
    qpos = {int(x): i for i, x in enumerate(queries)}
    hq, hr, hp = oracle.find_windows(ascii, offs, K, queries.reshape(-1, 1), cap=1 << 16)
    occ = np.bincount(hq.astype(np.int64), minlength=len(queries))
    for i in range(len(e)):
        n_occ = occ[qpos[int(e[i])]] + (0 if pal[i] else occ[qpos[int(rce[i])]])
        want = 2 * n_occ if pal[i] else n_occ
        assert want == m["counts"][idx[i]], "mercy entry %d: count vs occurrences" % i
    # solidity and degrees of every window of the reads holding an occurrence
    reads = sorted(set(int(r) for r in hr))
    q = []
    windows = {}
    for r in reads:
        seq = LUT[ascii[int(offs[r]):int(offs[r + 1])]]
        ws = [_key(seq[i:i + K + 1]) for i in range(len(seq) - K)]
        windows[r] = ws
        for x in ws:
            q.append(x)
            q.extend(((x << 2) & MASK) | c for c in range(4))
            q.extend((c << (2 * K)) | (x >> 2) for c in range(4))
    qa = np.array(q, dtype=np.uint64)
    uq, inv = np.unique(qa, return_inverse=True)
    cnt = oracle.count_queries(ascii, offs, K, uq.reshape(-1, 1))[inv]
    info, pos = {}, 0
    for r in reads:
        rows = []
        for _ in windows[r]:
            c9 = cnt[pos:pos + 9]
            pos += 9
            rows.append((c9[0] >= D, not np.any(c9[1:5] >= D), not np.any(c9[5:9] >= D)))
        info[r] = rows
    justified = np.zeros(len(queries), dtype=bool)
    for qi, r, p in zip(hq.tolist(), hr.tolist(), hp.tolist()):
        rows = info[r]
        assert not rows[p][0], "a mercy entry occurs as a solid window"
        before = [a for a in range(p) if rows[a][0]]
        after = [b for b in range(p + 1, len(rows)) if rows[b][0]]
        if before and after and rows[before[-1]][1] and rows[after[0]][2]:
            justified[qi] = True
    for i in range(len(e)):
        ok = justified[qpos[int(e[i])]] or (not pal[i] and justified[qpos[int(rce[i])]])
        assert ok, "GPU mercy entry %d (key %d) is justified by no read" % (idx[i], int(e[i]))
