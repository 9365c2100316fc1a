"""Properties that pin the outputs without reference to how they were built.

* ``check_kmers``  - a solid or mercy table: strictly ascending keys, closed
  under reverse complement with equal counts, counts in the allowed range.
* ``decode_sdbg``  - walks the BOSS arrays the way a user of the graph would
  (backward moves through F, W and last; the auxiliary store at dummy edges)
  and returns every node's string and every edge; ``check_sdbg`` then demands
  that the decoded graph is exactly the input edge set, that nodes are in
  strictly increasing colex order, that every in-edge after the first carries
  the minus flag, that each zero-indegree vertex has exactly one dummy edge and
  each zero-outdegree vertex one '$' edge, and that F counts the nodes' last
  symbols (paper, Sec. 2: SdBG of Bowe et al. with validity bits and a 2kt-bit
  store of zero-indegree vertices; colex order of the k-prefixes).

Everything works on numpy arrays and accepts either the oracle's output or
the CUDA library's (bit-vectors unpacked to one byte per entry first).
"""
from __future__ import annotations

import numpy as np

_ORDER = "$ACGT"


# ------------------------------------------------------------ packed keys

def _rows(keys) -> np.ndarray:
    keys = np.asarray(keys, dtype=np.uint64)
    if keys.ndim == 2:
        return keys
    return keys.reshape(keys.shape[0], -1) if keys.size else keys.reshape(keys.shape[0], 1)


def keys_to_syms(keys, n: int) -> np.ndarray:
    """(N, nw) packed keys -> (N, n) symbol codes 0..3, symbol 0 first."""
    keys = _rows(keys)
    out = np.empty((keys.shape[0], n), dtype=np.uint8)
    for i in range(n):
        bit = 2 * (n - 1 - i)
        out[:, i] = ((keys[:, bit // 64] >> np.uint64(bit % 64)) & np.uint64(3)).astype(np.uint8)
    return out


def syms_to_keys(syms, nw: int) -> np.ndarray:
    syms = np.asarray(syms, dtype=np.uint64)
    N, n = syms.shape
    out = np.zeros((N, nw), dtype=np.uint64)
    for i in range(n):
        bit = 2 * (n - 1 - i)
        out[:, bit // 64] |= syms[:, i] << np.uint64(bit % 64)
    return out


def lex_order_ok(keys) -> bool:
    """True iff the rows are strictly ascending as multiword integers."""
    keys = _rows(keys)
    if keys.shape[0] < 2:
        return True
    a, b = keys[:-1], keys[1:]
    less = np.zeros(a.shape[0], dtype=bool)
    eq = np.ones(a.shape[0], dtype=bool)
    for w in range(keys.shape[1] - 1, -1, -1):
        less |= eq & (a[:, w] < b[:, w])
        eq &= a[:, w] == b[:, w]
    return bool(less.all())


def sort_rows(keys) -> np.ndarray:
    keys = _rows(keys)
    if keys.shape[0] == 0:
        return keys
    return keys[np.lexsort([keys[:, w] for w in range(keys.shape[1])])]


def revcomp_keys(keys, k: int) -> np.ndarray:
    keys = _rows(keys)
    nw = keys.shape[1]
    s = keys_to_syms(keys, k + 1)
    return syms_to_keys(3 - s[:, ::-1], nw)


def check_kmers(keys, cnt, k: int, lo: int, hi: int | None = None) -> None:
    """Strictly ascending, closed under reverse complement with equal counts,
    and lo <= count <= hi."""
    keys = _rows(keys)
    cnt = np.asarray(cnt, dtype=np.uint64)
    assert keys.shape[0] == cnt.shape[0]
    assert lex_order_ok(keys), "keys not strictly ascending"
    if cnt.size:
        assert int(cnt.min()) >= lo, "count below %d" % lo
        if hi is not None:
            assert int(cnt.max()) <= hi, "count above %d" % hi
    r = revcomp_keys(keys, k)
    order = np.lexsort([r[:, w] for w in range(r.shape[1])])
    assert np.array_equal(r[order], keys.reshape(r.shape)), "not closed under reverse complement"
    assert np.array_equal(cnt[order], cnt), "a k-mer and its reverse complement differ in count"


# ------------------------------------------------------------ BOSS decode

def _colex_codes(node_syms: np.ndarray) -> list:
    """lexsort keys that order nodes colex: last symbol most significant."""
    # np.lexsort sorts by the LAST key first, so give symbol 0 first.
    return [node_syms[:, i] for i in range(node_syms.shape[1])]


def decode_sdbg(W, last, dummy, F, aux, k: int) -> dict:
    """Decode the BOSS arrays into node strings (codes $=0 A=1 C=2 G=3 T=4,
    one row per node) and per-entry data.

    Backward rule: the r-th entry with W == c (c in A..T, no minus flag) is the
    in-edge of the r-th non-dummy node whose entries lie in [F[c], F[c+1]).
    A node reached by a dummy edge is the auxiliary record of that edge;
    otherwise a node's symbols are read off k steps of in-edges (its own last
    symbol, its predecessor's, ...), stopping early at a dummy edge.
    """
    W = np.asarray(W, dtype=np.uint8)
    last = np.asarray(last, dtype=np.uint8)
    dummy = np.asarray(dummy, dtype=np.uint8)
    F = np.asarray(F, dtype=np.int64)
    m = W.shape[0]
    assert last.shape[0] == m and dummy.shape[0] == m
    assert F.shape[0] == 6 and F[5] == m and F[0] == 0 and F[1] == 0, "F boundaries"
    assert np.all(np.diff(F) >= 0), "F not monotone"
    assert m == 0 or last[m - 1] == 1, "last entry must close a node"
    ends = np.nonzero(last)[0]
    n_nodes = ends.shape[0]
    starts = np.concatenate([[0], ends[:-1] + 1]).astype(np.int64)
    node_of_entry = np.repeat(np.arange(n_nodes), ends - starts + 1)
    # block (last symbol) of each node; a node must not straddle blocks
    blk_start = np.searchsorted(F, starts, side="right") - 1
    blk_end = np.searchsorted(F, ends, side="right") - 1
    assert np.array_equal(blk_start, blk_end), "a node straddles two F blocks"
    lastsym = blk_start.astype(np.int64)        # 1..4
    assert n_nodes == 0 or (lastsym.min() >= 1 and lastsym.max() <= 4)
    # dummy nodes: all their entries dummy
    dcount = np.add.reduceat(dummy.astype(np.int64), starts) if m else np.zeros(0, np.int64)
    sizes = ends - starts + 1
    assert np.all((dcount == 0) | (dcount == sizes)), "node mixes dummy and real edges"
    node_dummy = dcount > 0
    label = np.where(W > 4, W - 4, W).astype(np.int64)
    minus = W > 4
    assert not np.any(minus & (dummy > 0)), "dummy edge with minus flag"
    assert not np.any(W > 8)
    # aux rank of each dummy entry
    aux = np.asarray(aux, dtype=np.uint64)
    aux_rank = np.cumsum(dummy) - 1
    t = int(dummy.sum())
    aux = aux.reshape(t, -1) if t else aux.reshape(0, 1)
    aux_syms = keys_to_syms(aux, k) + 1 if t else np.zeros((0, k), np.int64)
    # predecessor entry of each non-dummy node
    pred_entry = np.full(n_nodes, -1, dtype=np.int64)
    for c in range(1, 5):
        e_c = np.nonzero(W == c)[0]
        n_c = np.nonzero((lastsym == c) & ~node_dummy)[0]
        assert e_c.shape[0] == n_c.shape[0], \
            "symbol %s: %d in-edges for %d nodes" % (_ORDER[c], e_c.shape[0], n_c.shape[0])
        pred_entry[n_c] = e_c
    real = ~node_dummy
    # node symbols (codes 1..4; 0 = '$' at position 0 of dummy nodes)
    syms = np.zeros((n_nodes, k), dtype=np.int64)
    # dummy nodes: $ + aux[:k-1] of their first entry; every entry agrees
    dn = np.nonzero(node_dummy)[0]
    if dn.size:
        first_aux = aux_syms[aux_rank[starts[dn]]]
        syms[dn, 1:] = first_aux[:, :k - 1]
        syms[dn, 0] = 0
        de = np.nonzero(dummy)[0]
        a = aux_syms[aux_rank[de]]
        assert np.array_equal(a[:, :k - 1], syms[node_of_entry[de], 1:]), "dummy node vs aux"
        assert np.array_equal(a[:, k - 1], label[de]), "dummy label vs aux"
    # real nodes: walk in-edges back up to k-1 steps
    rn = np.nonzero(real)[0]
    cur = rn.copy()
    done = np.zeros(rn.shape[0], dtype=bool)
    for i in range(k):
        act = ~done
        syms[rn[act], k - 1 - i] = lastsym[cur[act]]
        if i == k - 1:
            break
        pe = pred_entry[cur]
        via_dummy = act & (dummy[pe] > 0)
        if via_dummy.any():
            a = aux_syms[aux_rank[pe[via_dummy]]]       # = string of node cur
            # node rn[j] = a[i..k-1] followed by the i symbols already read
            syms[rn[via_dummy], :k - i] = a[:, i:]
            done |= via_dummy
        cur = np.where(done, cur, node_of_entry[pe])
    return {"n_nodes": n_nodes, "starts": starts, "ends": ends, "node_syms": syms,
            "node_dummy": node_dummy, "node_of_entry": node_of_entry, "label": label,
            "minus": minus, "lastsym": lastsym, "pred_entry": pred_entry,
            "aux_syms": aux_syms, "aux_rank": aux_rank}


def check_sdbg(sd: dict, k: int, edge_keys, edge_mult=None) -> dict:
    """Decode ``sd`` (keys W, last, valid, dummy, F, aux; optional mult) and
    check it against the edge set ``edge_keys`` ((E, nw) packed (k+1)-mers).
    Returns the decode."""
    W = np.asarray(sd["W"], dtype=np.uint8)
    m = W.shape[0]
    if "valid" in sd:
        assert np.all(np.asarray(sd["valid"]) == 1), "validity bits at construction must be 1"
    dec = decode_sdbg(W, sd["last"], sd["dummy"], sd["F"], sd["aux"], k)
    syms = dec["node_syms"]
    n_nodes = dec["n_nodes"]
    noe = dec["node_of_entry"]
    label = dec["label"]
    dummy = np.asarray(sd["dummy"], dtype=np.uint8) > 0
    # nodes strictly increasing in colex order
    if n_nodes > 1:
        order = np.lexsort(_colex_codes(syms))
        assert np.array_equal(order, np.arange(n_nodes)), "nodes not in colex order"
        same = np.all(syms[1:] == syms[:-1], axis=1)
        assert not same.any(), "a node appears twice"
    # labels strictly increasing inside a node
    if m > 1:
        inside = noe[1:] == noe[:-1]
        assert np.all(label[1:][inside] > label[:-1][inside]), "labels not increasing in a node"
    # every in-edge maps to the node it points to: target = source[1:] + label
    nonminus_real = (label > 0) & ~dec["minus"]
    for c in range(1, 5):
        e_c = np.nonzero(W == c)[0]
        n_c = np.nonzero((dec["lastsym"] == c) & ~dec["node_dummy"])[0]
        src = syms[noe[e_c]]
        tgt = np.concatenate([src[:, 1:], np.full((e_c.shape[0], 1), c)], axis=1)
        assert np.array_equal(syms[n_c], tgt), "an edge does not lead to its target node"
    # minus edges: an earlier unflagged edge with the same target exists
    mi = np.nonzero(dec["minus"])[0]
    if mi.size:
        grp = {}
        for i in np.nonzero(nonminus_real)[0]:
            grp[(tuple(syms[noe[i], 1:]), int(label[i]))] = int(i)
        for i in mi:
            key = (tuple(syms[noe[i], 1:]), int(label[i]))
            assert key in grp and grp[key] < i, "minus flag without an earlier edge"
    # unflagged real edges have distinct targets (else one would need a minus)
    # (implied by the one-to-one mapping above)
    # the decoded edge set equals the input
    real_e = np.nonzero((label > 0) & ~dummy)[0]
    e_syms = np.concatenate([syms[noe[real_e]], label[real_e][:, None]], axis=1) - 1
    nw = np.asarray(edge_keys).reshape(len(edge_keys), -1).shape[1] if len(edge_keys) else 1
    got = syms_to_keys(e_syms, nw) if real_e.size else np.zeros((0, nw), np.uint64)
    want = sort_rows(np.asarray(edge_keys, dtype=np.uint64).reshape(-1, nw))
    got_sorted = sort_rows(got)
    assert got_sorted.shape == want.shape and np.array_equal(got_sorted, want), \
        "decoded edges differ from the edge set"
    if edge_mult is not None and "mult" in sd:
        gm = np.asarray(sd["mult"], dtype=np.uint32)[real_e]
        order = np.lexsort([got[:, w] for w in range(nw)])
        assert np.array_equal(gm[order], np.asarray(edge_mult, dtype=np.uint32)), "mult differs"
        assert np.all(np.asarray(sd["mult"])[np.nonzero(dummy | (label == 0))[0]] == 0)
    # padding: zero-indegree vertices <-> dummy edges, zero-outdegree <-> $ edges
    e_all = keys_to_syms(want, k + 1) + 1
    src_set = {tuple(r) for r in e_all[:, :k]}
    tgt_set = {tuple(r) for r in e_all[:, 1:]}
    zero_in = src_set - tgt_set
    zero_out = tgt_set - src_set
    aux_set = [tuple(r) for r in dec["aux_syms"]]
    assert len(aux_set) == len(set(aux_set)) and set(aux_set) == zero_in, "dummy edges vs zero indegree"
    dollar = np.nonzero(label == 0)[0]
    dollar_nodes = [tuple(syms[noe[i]]) for i in dollar]
    assert len(set(dollar_nodes)) == len(dollar_nodes) and set(dollar_nodes) == zero_out, \
        "$ edges vs zero outdegree"
    for i in dollar:
        n = noe[i]
        assert dec["starts"][n] == dec["ends"][n], "$ edge shares its node"
    # F counts the last symbols
    F = np.asarray(sd["F"], dtype=np.int64)
    node_last = syms[noe, k - 1] if m else np.zeros(0, np.int64)
    for c in range(5):
        assert F[c] == int(np.sum(node_last < c)), "F[%d]" % c
    return dec
