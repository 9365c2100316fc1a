"""Batched runs (mh_run_batch): every set's outputs are bit-identical to the
plain calls on that set alone, whatever the worker count, the input memory
(device or host) or the memory plan; small sets match the oracle; the
autotuner picks one of the tile shapes and changes no output; a failing set
is reported and leaves no outputs."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1409_7208_gb300 as m
    return m


def _sets(n, seed=7):
    out = []
    for i in range(n):
        if i % 3 == 2:
            out.append(synth.random_reads(seed * 100 + i, 200 + 50 * i, 0, 180, p_invalid=0.01))
        else:
            out.append(synth.uniform_genome_reads(seed * 100 + i, 3000 + 400 * i, 300 + 150 * i, 120, 0.01))
    return out


def _plain(mh, ctx, a, o, k, d):
    reads = mh.mh_pack_reads(ctx, a, o)
    s = mh.mh_count_kmers(ctx, reads, k, d)
    m = mh.mh_mercy_kmers(ctx, reads, s)
    g = mh.mh_build_sdbg(ctx, s, m)
    return s.numpy(), m.numpy(), g.numpy()


def _same(r, want):
    gs, gm, gg = r["solid"].numpy(), r["mercy"].numpy(), r["sdbg"].numpy()
    ws, wm, wg = want
    for key in ("keys", "counts"):
        assert np.array_equal(gs[key], ws[key]) and np.array_equal(gm[key], wm[key]), key
    for key in ("m", "t", "u", "n_nodes"):
        assert gg[key] == wg[key], key
    for key in ("W", "last", "valid", "dummy", "F", "aux"):
        assert np.array_equal(gg[key], wg[key]), key


@pytest.mark.parametrize("k,workers", [(31, 1), (31, 3), (21, 8), (47, 2)])
def test_batch_matches_plain_calls(mh, k, workers):
    import torch
    sets = _sets(7)
    ctx = mh.Context(device=0)
    want = [_plain(mh, ctx, a, o, k, 2) for a, o in sets]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(o.view(np.int64)).cuda()) for a, o in sets]
    res = mh.mh_run_batch(ctx, dev, k, 2, workers=workers)
    assert [r["status"] for r in res] == [0] * len(sets)
    for r, w in zip(res, want):
        _same(r, w)
    ctx.close()


def test_batch_host_inputs_and_oracle(mh):
    sets = _sets(4, seed=8)
    ctx = mh.Context(device=0, torch_allocator=False)
    res = mh.mh_run_batch(ctx, sets, 31, 2, workers=2)
    for r, (a, o) in zip(res, sets):
        w = oracle.count(a, o, 31, 2, mercy=True)
        gs, gm = r["solid"].numpy(), r["mercy"].numpy()
        assert np.array_equal(gs["keys"], w["solid_keys"]) and np.array_equal(gs["counts"], w["solid_cnt"])
        assert np.array_equal(gm["keys"], w["mercy_keys"]) and np.array_equal(gm["counts"], w["mercy_cnt"])
        wg = oracle.build_sdbg(31, w["solid_keys"], w["solid_cnt"], w["mercy_keys"], w["mercy_cnt"])
        gg = r["sdbg"].numpy()
        for key in ("W", "last", "valid", "dummy", "F", "aux"):
            assert np.array_equal(gg[key], wg[key]), key
    ctx.close()


def test_batch_autotune_and_tight_budget(mh):
    sets = _sets(5, seed=9)
    ctx = mh.Context(device=0)
    want = [_plain(mh, ctx, a, o, 31, 2) for a, o in sets]
    assert mh.mh_sort_shape(ctx) == -1
    res = mh.mh_run_batch(ctx, sets, 31, 2, workers=3, autotune=True)
    assert mh.mh_sort_shape(ctx) in (0, 1, 2)
    for r, w in zip(res, want):
        _same(r, w)
    ctx.close()
    # a budget below every set's estimate: sets run one at a time, outputs unchanged
    tight = mh.Context(device=0, hbm_budget=1 << 20)
    res = mh.mh_run_batch(tight, sets, 31, 2, workers=4)
    for r, w in zip(res, want):
        _same(r, w)
    tight.close()


def test_batch_reports_a_failing_set(mh):
    sets = _sets(3, seed=10)
    a, o = sets[1]
    bad = o.copy()
    bad[-1] = bad[-1] + 5  # offsets run past the bases: rejected on the host
    ctx = mh.Context(device=0)
    with pytest.raises(mh.MhError) as e:
        mh.mh_run_batch(ctx, [sets[0], (a, bad), sets[2]], 31, 2, workers=2)
    assert e.value.code == mh.MH_EINVAL
    assert mh.mh_run_batch(ctx, [], 31, 2) == []
    ctx.close()


def _plans(nw):
    """The counting plans the batch autotuner tries (mh_batch.cu), plus
    forced out-of-core bucket counts."""
    p = []
    if nw == 1:
        p += [dict(path=0, sort_shape=s, unit_bits_delta=0, spread_bits_delta=0) for s in range(3)]
        p += [dict(path=0, sort_shape=0, unit_bits_delta=u, spread_bits_delta=0) for u in (-1, 1)]
    p += [dict(path=1, sort_shape=0, unit_bits_delta=0, spread_bits_delta=b) for b in (0, 8, -8)]
    return p + [dict(p[0], bucket_bits=1), dict(p[0], bucket_bits=3)]


@pytest.mark.parametrize("k", [31, 47])
def test_every_counting_plan_gives_the_same_outputs(mh, k):
    """Each plan the autotuner may pick (route, tile shape, unit or spread
    bits, bucket count) yields outputs bit-identical to the default plan's."""
    a, o = synth.uniform_genome_reads(61, 200_000, 40_000, 150, 0.01)
    ctx = mh.Context(device=0)
    want = _plain(mh, ctx, a, o, k, 2)
    for plan in _plans(1 if k <= 31 else 2):
        mh.mh_set_count_plan(ctx, **dict(dict(bucket_bits=-1), **plan))
        assert mh.mh_get_count_plan(ctx)["path"] == plan["path"]
        got = _plain(mh, ctx, a, o, k, 2)
        for i, part in enumerate(("keys", "counts")):
            assert np.array_equal(got[0][part], want[0][part]), (plan, part)
            assert np.array_equal(got[1][part], want[1][part]), (plan, part)
        for key in ("W", "last", "dummy", "F", "aux"):
            assert np.array_equal(got[2][key], want[2][key]), (plan, key)
    with pytest.raises(mh.MhError):
        mh.mh_set_count_plan(ctx, spread_bits_delta=4)


def test_autotuned_plan_is_no_slower_than_the_default(mh):
    """The plan the batch autotuner keeps counts the tuning set no slower
    than the default plan (best of five each, 15% allowed for noise)."""
    import time

    import torch
    sets = [synth.uniform_genome_reads(70 + i, 2_000_000, 400_000 - 50_000 * i, 150, 0.005) for i in range(4)]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(o.view(np.int64)).cuda()) for a, o in sets]
    ctx = mh.Context(device=0)
    res = mh.mh_run_batch(ctx, dev, 31, 2, workers=2, autotune=True)
    for r in res:
        for key in ("sdbg", "mercy", "solid"):
            r[key].free()
    tuned = mh.mh_get_count_plan(ctx)
    assert tuned["path"] in (0, 1)

    def best(plan):
        c = mh.Context(device=0)
        mh.mh_set_count_plan(c, **plan)
        reads = mh.mh_pack_reads(c, *dev[0])
        times = []
        for _ in range(6):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = mh.mh_count_kmers(c, reads, 31, 2)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            s.free()
        del reads
        c.close()
        return min(times[1:])

    default = dict(path=-1, sort_shape=-1, unit_bits_delta=0, spread_bits_delta=0, bucket_bits=-1)
    assert best(tuned) <= 1.15 * best(default), tuned
