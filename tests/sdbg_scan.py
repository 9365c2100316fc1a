"""A vectorised decode of the BOSS arrays for graphs far too large for
``oracle/check.py`` (hundreds of millions of entries), in torch on any device.

It checks the same definitions as ``check.check_sdbg`` (paper, Sec. 2: the
SdBG of Bowe et al. with validity bits and a 2kt-bit store of zero-indegree
vertices, edges in colex order of their k-prefixes), for 1-word keys
(k <= 31), holding every node as one 64-bit integer instead of a row of
symbols:

* every node lies in one F block, and dummy nodes hold only dummy entries;
* the r-th unflagged entry with label c is the in-edge of the r-th
  non-dummy node of block c, and that node is the edge's target;
* a node's string is read by walking k in-edges back (at a dummy in-edge the
  rest comes from the auxiliary record), and nodes are strictly increasing
  in colex order ('$' below A at position 0);
* the decoded real edges are exactly the given edge set;
* in each group of entries with the same target, the first (in entry order)
  is unflagged and the others carry the minus flag; dummy and '$' entries
  never do;
* the auxiliary records are exactly the zero-indegree vertices, one each, and
  agree with their dummy entries; the '$' entries are exactly the
  zero-outdegree vertices, each alone in its node;
* F counts the entries whose node ends below each symbol.

``tests/test_oracle_pins.py`` runs it beside ``check.check_sdbg`` on small
graphs (both must accept) and on planted mistakes (both must reject).
"""
from __future__ import annotations

import numpy as np


def _t(x, device, dtype=None):
    import torch

    if isinstance(x, torch.Tensor):
        t = x.to(device)
    else:
        t = torch.from_numpy(np.ascontiguousarray(x)).to(device)
    return t.to(dtype) if dtype is not None else t


def _rev_syms(key, n: int):
    """The n-symbol string held in `key` (first symbol most significant),
    reversed, as a key."""
    out = key & 0
    for i in range(n):
        out = (out << 2) | ((key >> (2 * i)) & 3)
    return out


def _mask(bits: int) -> int:
    return (1 << bits) - 1 if bits < 63 else -1


def check_sdbg_large(W, last, dummy, F, aux, k: int, edges, device="cpu") -> dict:
    """Decode and check the BOSS arrays (W codes $=0 A..T=1..4, +4 minus;
    last/dummy one 0/1 value per entry; F 6 counts; aux t 1-word keys) against
    ``edges``, the (k+1)-mer keys of the edge set (1 word each, any order).
    Raises AssertionError on the first violated definition; returns counts."""
    import torch

    assert 2 <= k <= 31, "1-word keys only"
    i64 = torch.int64
    W = _t(W, device, torch.int16)
    last = _t(last, device, torch.bool)
    dummy = _t(dummy, device, torch.bool)
    F = _t(np.asarray(F, dtype=np.int64), device, i64)
    aux = _t(np.asarray(aux, dtype=np.uint64).reshape(-1).view(np.int64), device, i64)
    E = _t(np.asarray(edges, dtype=np.uint64).reshape(-1).view(np.int64), device, i64)
    m = W.shape[0]
    assert last.shape[0] == m and dummy.shape[0] == m
    assert int(F[0]) == 0 and int(F[1]) == 0 and int(F[5]) == m, "F boundaries"
    assert bool((F[1:] >= F[:-1]).all()), "F not monotone"
    assert m == 0 or bool(last[-1]), "last entry must close a node"
    assert not bool((W > 8).any()) and not bool((W < 0).any())
    label = torch.where(W > 4, W - 4, W).to(i64)
    minus = W > 4
    assert not bool((minus & dummy).any()), "dummy edge with minus flag"
    # nodes
    ends = torch.nonzero(last).flatten()
    n_nodes = ends.shape[0]
    starts = torch.cat([torch.zeros(1, dtype=i64, device=device), ends[:-1] + 1])
    sizes = ends - starts + 1
    node_of_entry = torch.repeat_interleave(torch.arange(n_nodes, device=device), sizes)
    blk_s = torch.searchsorted(F, starts, right=True) - 1
    blk_e = torch.searchsorted(F, ends, right=True) - 1
    assert torch.equal(blk_s, blk_e), "a node straddles two F blocks"
    lastsym = blk_s
    assert n_nodes == 0 or (int(lastsym.min()) >= 1 and int(lastsym.max()) <= 4)
    dcount = torch.zeros(n_nodes, dtype=i64, device=device).index_add_(0, node_of_entry, dummy.to(i64))
    assert bool(((dcount == 0) | (dcount == sizes)).all()), "node mixes dummy and real edges"
    node_dummy = dcount > 0
    # aux rank of each dummy entry, and the aux records as keys
    t = int(dummy.sum())
    assert aux.shape[0] == t, "one auxiliary record per dummy entry"
    aux_rank = torch.cumsum(dummy.to(i64), 0) - 1
    # in-edge of each non-dummy node
    pred = torch.full((n_nodes,), -1, dtype=i64, device=device)
    for c in range(1, 5):
        e_c = torch.nonzero(W == c).flatten()
        n_c = torch.nonzero((lastsym == c) & ~node_dummy).flatten()
        assert e_c.shape[0] == n_c.shape[0], "symbol %d: %d in-edges for %d nodes" % (c, e_c.shape[0], n_c.shape[0])
        pred[n_c] = e_c
    # node strings by walking in-edges back (real nodes)
    real = torch.nonzero(~node_dummy).flatten()
    key = torch.zeros(real.shape[0], dtype=i64, device=device)
    cur = real.clone()
    done = torch.zeros(real.shape[0], dtype=torch.bool, device=device)
    for i in range(k):
        act = ~done
        key = torch.where(act, key | ((lastsym[cur] - 1) << (2 * i)), key)
        if i == k - 1:
            break
        pe = pred[cur]
        assert bool((pe[act] >= 0).all()), "a real node without an in-edge"
        via = act & dummy[pe.clamp(min=0)]
        if bool(via.any()):
            a = aux[aux_rank[pe[via]]]
            low = key[via] & _mask(2 * i)
            key[via] = ((a & _mask(2 * (k - i))) << (2 * i)) | low
            done = done | via
        cur = torch.where(done, cur, node_of_entry[pe.clamp(min=0)])
    node_key = torch.zeros(n_nodes, dtype=i64, device=device)
    node_key[real] = key
    # dummy nodes: '$' then the first k-1 symbols of their entries' record
    dn = torch.nonzero(node_dummy).flatten()
    dkey = aux[aux_rank[starts[dn]]] >> 2 if dn.numel() else torch.zeros(0, dtype=i64, device=device)
    if dn.numel():
        assert torch.equal(lastsym[dn] - 1, dkey & 3), "a dummy node outside the F block of its last symbol"
    de = torch.nonzero(dummy).flatten()
    if de.numel():
        a = aux[aux_rank[de]]
        assert torch.equal(a >> 2, (aux[aux_rank[starts[node_of_entry[de]]]] >> 2)), "dummy node vs aux"
        assert torch.equal(a & 3, label[de] - 1), "dummy label vs aux"
    # colex order: positions k-1 .. 1, then position 0 with '$' lowest
    ck = torch.zeros(n_nodes, dtype=i64, device=device)
    ck[real] = (_rev_syms(key & _mask(2 * (k - 1)), k - 1) << 3) | ((key >> (2 * (k - 1))) + 1)
    if dn.numel():
        ck[dn] = _rev_syms(dkey, k - 1) << 3
    assert bool((ck[1:] > ck[:-1]).all()), "nodes not strictly increasing in colex order"
    # labels strictly increasing inside a node
    if m > 1:
        inside = node_of_entry[1:] == node_of_entry[:-1]
        assert bool((label[1:][inside] > label[:-1][inside]).all()), "labels not increasing in a node"
    # real edges (non-dummy, label != $) decoded, as (k+1)-mer keys
    re_ = torch.nonzero((label > 0) & ~dummy).flatten()
    src = node_key[node_of_entry[re_]]
    ekey = (src << 2) | (label[re_] - 1)
    got = torch.sort(ekey).values
    want = torch.sort(E).values
    assert got.shape == want.shape and torch.equal(got, want), "decoded edges differ from the edge set"
    assert not bool((got[1:] == got[:-1]).any()), "an edge appears twice"
    # each unflagged in-edge leads to its node, and minus flags
    tgt = ekey & _mask(2 * k)
    for c in range(1, 5):
        e_c = torch.nonzero(W == c).flatten()
        n_c = torch.nonzero((lastsym == c) & ~node_dummy).flatten()
        real_tc = ((node_key[node_of_entry[e_c]] << 2) | (c - 1)) & _mask(2 * k)
        tc = torch.where(dummy[e_c], aux[aux_rank[e_c].clamp(min=0)], real_tc)
        assert torch.equal(node_key[n_c], tc), "an edge does not lead to its target node"
    order = torch.argsort(tgt, stable=True)
    ts = tgt[order]
    first = torch.ones_like(ts, dtype=torch.bool)
    if ts.numel() > 1:
        first[1:] = ts[1:] != ts[:-1]
    # within a target group the entries keep their order (stable sort), so
    # the group's first entry must be the unflagged one
    assert torch.equal(minus[re_][order], ~first), "minus flags"
    # padding
    srcs = torch.unique((E >> 2) & _mask(2 * k))
    tgts = torch.unique(E & _mask(2 * k))
    allv = torch.unique(torch.cat([srcs, tgts]))
    zero_in = allv[~torch.isin(allv, tgts)]
    zero_out = tgts[~torch.isin(tgts, srcs)]
    auxs = torch.sort(aux).values
    assert not bool((auxs[1:] == auxs[:-1]).any()) and torch.equal(auxs, zero_in), "dummy edges vs zero indegree"
    dol = torch.nonzero(label == 0).flatten()
    dn_keys = torch.sort(node_key[node_of_entry[dol]]).values
    assert torch.equal(dn_keys, zero_out) and not bool((dn_keys[1:] == dn_keys[:-1]).any()), \
        "$ edges vs zero outdegree"
    assert bool((starts[node_of_entry[dol]] == ends[node_of_entry[dol]]).all()), "$ edge shares its node"
    assert not bool(node_dummy[node_of_entry[dol]].any()), "$ edge in a dummy node"
    # F: entries whose node ends below c
    node_last = lastsym[node_of_entry]
    for c in range(5):
        assert int(F[c]) == int((node_last < c).sum()), "F[%d]" % c
    return {"m": m, "n_nodes": n_nodes, "t": t, "u": int(dol.numel()), "edges": int(got.numel())}
