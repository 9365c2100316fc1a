"""Contig walks and the multiple-k iteration through the C ABI, bit-exact
against the oracle (oracle/walk.py): the walks on graphs of 1-, 2- and
4-word keys, and a three-step iteration (every table, SdBG array and contig
of every step)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import walk as ow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1409_7208_gb300 as mh
    return mh.Context(device=0)


@pytest.mark.parametrize("k,n_walks,max_len,seed", [(21, 300, 400, 1), (47, 200, 300, 2), (99, 100, 500, 3),
                                                    (11, 500, 2000, 4)])
def test_walks_match_oracle(ctx, k, n_walks, max_len, seed):
    import paper_1409_7208_gb300 as mh
    ascii, offs = synth.uniform_genome_reads(seed, 6000, 1500, 150, 0.01)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    solid = mh.mh_count_kmers(ctx, reads, k, 2)
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    got = mh.mh_walk_contigs(ctx, solid, mercy, n_walks, max_len, seed * 7).strings()
    s, m = solid.numpy(), mercy.numpy()
    want = ow.walk_contigs(ow.key_strings(s["keys"], k), ow.key_strings(m["keys"], k), k, n_walks, max_len,
                           seed * 7)
    assert got == want
    assert len(got) == n_walks and max(len(c) for c in got) <= max_len


def test_walks_without_mercy_and_on_empty_graph(ctx):
    import paper_1409_7208_gb300 as mh
    ascii, offs = synth.uniform_genome_reads(5, 3000, 800, 100, 0.01)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    solid = mh.mh_count_kmers(ctx, reads, 17, 2)
    got = mh.mh_walk_contigs(ctx, solid, None, 64, 250, 9).strings()
    assert got == ow.walk_contigs(ow.key_strings(solid.numpy()["keys"], 17), [], 17, 64, 250, 9)
    # d above every count: no edges, no contigs
    empty = mh.mh_count_kmers(ctx, reads, 17, 10_000)
    assert mh.mh_walk_contigs(ctx, empty, None, 10, 100, 1).strings() == []
    with pytest.raises(mh.MhError):
        mh.mh_walk_contigs(ctx, solid, None, 10, 17, 1)  # max_len < k + 1


def test_iteration_matches_oracle(ctx):
    import torch

    import paper_1409_7208_gb300 as mh
    from paper_1409_7208_gb300 import multik
    ascii, offs = synth.uniform_genome_reads(8, 8000, 1200, 120, 0.015)
    ks, d, n_walks, max_len, seed = (21, 33, 47), 2, 60, 600, 21
    d_ascii = torch.from_numpy(ascii).cuda()
    d_offs = torch.from_numpy(offs.view(np.int64)).cuda()
    steps = multik.iterate(ctx, d_ascii, d_offs, ks, d, n_walks, max_len, seed, keep=True)
    want = ow.iterate(ascii, offs, ks, d, n_walks, max_len, seed)
    for st, w in zip(steps, want):
        s, m, g = st["solid"].numpy(), st["mercy"].numpy(), st["sdbg"].numpy()
        wc = w["counts"]
        assert np.array_equal(s["keys"], wc["solid_keys"]) and np.array_equal(s["counts"], wc["solid_cnt"])
        assert np.array_equal(m["keys"], wc["mercy_keys"]) and np.array_equal(m["counts"], wc["mercy_cnt"])
        for key in ("W", "last", "dummy", "F", "aux"):
            assert np.array_equal(g[key], w["sdbg"][key]), (st["k"], key)
        assert st["contigs"].strings() == w["contigs"], st["k"]
