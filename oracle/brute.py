"""Brute force for tiny inputs: the paper's definitions taken literally, in
pure Python, with no sorting tricks and no packed keys.

Used only to pin the C++ oracle (``mh_oracle.cpp``) on small cases; each
function is written differently from the oracle's way of computing the same
thing (dictionaries instead of sort-and-scan, all pairs of solid positions
instead of consecutive ones, quadratic scans instead of sets).

Paper references: counting, solid and mercy k-mers - Sec. 2, third paragraph;
SdBG (BOSS) with validity bits and the zero-indegree store - Sec. 2, first
paragraph; colex ("reverse lexicographical") order - Sec. 2, second paragraph.
"""
from __future__ import annotations

_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def rc(s: str) -> str:
    return "".join(_COMP[c] for c in reversed(s))


def fragments(reads) -> list:
    """Maximal ACGT runs of each read, upper-cased ([reading]: other bytes split)."""
    out = []
    for r in reads:
        r = r.decode() if isinstance(r, (bytes, bytearray)) else r
        cur = ""
        for ch in r.upper():
            if ch in "ACGT":
                cur += ch
            else:
                if cur:
                    out.append(cur)
                cur = ""
        if cur:
            out.append(cur)
    return out


def count(reads, k: int) -> dict:
    """Every (k+1)-mer occurrence counted once as read and once reverse
    complemented (both strands)."""
    c: dict = {}
    for f in fragments(reads):
        for i in range(len(f) - k):
            e = f[i:i + k + 1]
            c[e] = c.get(e, 0) + 1
            c[rc(e)] = c.get(rc(e), 0) + 1
    return c


def solid(reads, k: int, d: int) -> dict:
    return {e: n for e, n in count(reads, k).items() if n >= d}


def mercy(reads, k: int, d: int) -> dict:
    """All pairs (x at p, y at q), p < q, in one fragment, with x solid and
    without a solid successor, y solid and without a solid predecessor, and
    every (k+1)-mer strictly between them not solid: the in-between
    (k+1)-mers are mercy edges.  Closed under reverse complement.  Returns
    edge -> count."""
    cnt = count(reads, k)
    sol = {e for e, n in cnt.items() if n >= d}

    def has_out(x):
        return any(z[:k] == x[1:] for z in sol)

    def has_in(y):
        return any(z[1:] == y[:k] for z in sol)

    found = set()
    for f in fragments(reads):
        edges = [f[i:i + k + 1] for i in range(len(f) - k)]
        for p in range(len(edges)):
            for q in range(p + 1, len(edges)):
                if edges[p] in sol and edges[q] in sol and not has_out(edges[p]) \
                        and not has_in(edges[q]) \
                        and all(edges[j] not in sol for j in range(p + 1, q)):
                    found.update(edges[p + 1:q])
    found |= {rc(e) for e in found}
    return {e: cnt[e] for e in found}


def boss(edges, k: int) -> dict:
    """String-level BOSS table of an edge set (iterable of (k+1)-mer strings).

    Returns a dict with ``rows`` (list of (node, label, minus, is_dummy,
    aux)), ``W``, ``last``, ``dummy``, ``F``, ``aux`` (list of strings).
    Colex: nodes compared from their last symbol back to their first, then the
    label, with '$' below every base.
    """
    edges = sorted(set(edges))
    nodes = {e[:k] for e in edges} | {e[1:] for e in edges}
    rows = []
    for e in edges:
        rows.append((e[:k], e[k], False, None))
    for v in sorted(nodes):
        if not any(e[1:] == v for e in edges):          # zero indegree
            rows.append(("$" + v[:k - 1], v[k - 1], True, v))
        if not any(e[:k] == v for e in edges):          # zero outdegree
            rows.append((v, "$", False, None))
    order = "$ACGT"
    rows.sort(key=lambda r: ([order.index(ch) for ch in reversed(r[0])], order.index(r[1])))
    m = len(rows)
    W, last, dummy, aux = [], [], [], []
    for i, (node, lab, is_dummy, v) in enumerate(rows):
        code = order.index(lab)
        minus = lab != "$" and any(rows[j][1] == lab and rows[j][0][1:] == node[1:] for j in range(i))
        W.append(code + 4 if minus else code)
        last.append(1 if i == m - 1 or rows[i + 1][0] != node else 0)
        dummy.append(1 if is_dummy else 0)
        if is_dummy:
            aux.append(v)
    F = [sum(1 for r in rows if order.index(r[0][k - 1]) < c) for c in range(5)] + [m]
    return {"rows": rows, "W": W, "last": last, "dummy": dummy, "F": F, "aux": aux, "m": m}
