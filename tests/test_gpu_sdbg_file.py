"""The graph file (mh_sdbg_save / mh_sdbg_load): a graph written and read back
in a new context gives the same arrays, bit for bit, and the oracle's graph;
damaged, truncated and foreign files are rejected with MH_EINVAL and nothing
is returned."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graph(ctx, k, seed, with_mult=False):
    import paper_1409_7208_gb300 as mh
    ascii, offs = synth.uniform_genome_reads(seed, 20000, 3000, 120, 0.01)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    solid = mh.mh_count_kmers(ctx, reads, k, 2)
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    return mh.mh_build_sdbg(ctx, solid, mercy), (ascii, offs)


@pytest.mark.parametrize("k,mult", [(21, False), (47, True), (99, False)])
def test_saved_graph_loads_bit_identical(tmp_path, k, mult):
    import paper_1409_7208_gb300 as mh
    ctx = mh.Context(device=0, with_mult=mult)
    g, (ascii, offs) = _graph(ctx, k, 60 + k)
    path = str(tmp_path / "g.sdbg")
    mh.mh_sdbg_save(g, path)
    other = mh.Context(device=0)
    h = mh.mh_sdbg_load(other, path)
    a, b = g.numpy(), h.numpy()
    for key in ("k", "nw", "m", "t", "u", "n_nodes", "F", "W", "last", "valid", "dummy", "aux"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
    if mult:
        assert np.array_equal(g.tensors()["mult"].cpu().numpy(), h.tensors()["mult"].cpu().numpy())
    w = oracle.count(ascii, offs, k, 2, mercy=True)
    wg = oracle.build_sdbg(k, w["solid_keys"], w["solid_cnt"], w["mercy_keys"], w["mercy_cnt"])
    for key in ("W", "last", "dummy", "F", "aux"):
        assert np.array_equal(np.asarray(b[key]), np.asarray(wg[key])), key


def test_damaged_files_are_rejected(tmp_path):
    import paper_1409_7208_gb300 as mh
    ctx = mh.Context(device=0)
    g, _ = _graph(ctx, 31, 7)
    path = str(tmp_path / "g.sdbg")
    mh.mh_sdbg_save(g, path)
    raw = open(path, "rb").read()
    cases = {
        "flipped": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:],
        "truncated": raw[:-9],
        "longer": raw + b"\0",
        "foreign": b"NOTAGRAPH" + raw[9:],
        "empty": b"",
    }
    before = ctx.memory()[0]
    for name, data in cases.items():
        p = str(tmp_path / (name + ".sdbg"))
        open(p, "wb").write(data)
        with pytest.raises(mh.MhError) as e:
            mh.mh_sdbg_load(ctx, p)
        assert e.value.code == mh.MH_EINVAL, name
        assert ctx.memory()[0] == before, "nothing held after a rejected file (%s)" % name
    with pytest.raises(mh.MhError):
        mh.mh_sdbg_load(ctx, str(tmp_path / "missing.sdbg"))
    with pytest.raises(mh.MhError):
        mh.mh_sdbg_save(g, os.path.join(str(tmp_path), "no", "such", "dir", "g.sdbg"))
