"""Contig walks and the multiple-k iteration, written from their definitions.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import or run this module; the CUDA library
never calls it and shares no code with it.

The paper (Sec. 2, fourth paragraph; Sec. 3) builds the graph for a list of
increasing k and carries each k's contigs into the next graph.  Graph
cleaning and contig assembly are outside the hot path, so a contig is a
random walk of the graph E = solid + mercy, stated as follows:

* r(w, j) is SplitMix64 output number (w << 24) + j of the stream seeded
  with ``seed`` (:func:`splitmix64_at`).
* Walk w starts at edge number r(w, 0) mod |E| of the list solid (ascending)
  followed by mercy (ascending); the contig is that edge's k+1 symbols.
* Step j = 1, 2, ...: the node is the contig's last k symbols; its
  out-edges are the edges of E whose first k symbols are the node, in label
  order A < C < G < T.  With none the walk stops; otherwise it appends the
  label of out-edge r(w, j) mod (their number).  It stops at max_len symbols.

The multiple-k iteration (:func:`iterate`): for k_1 < k_2 < ..., the reads
of step i are the input reads plus ``d`` copies of every contig of step i-1
(so every (k_i+1)-mer of a contig reaches count d and is solid: the
contig-derived edges); walks of step i use seed + i.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_at(seed: int, c: int) -> int:
    """Output number c (counting from 0) of SplitMix64 seeded with seed."""
    z = (seed + (c + 1) * _GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def key_strings(keys: np.ndarray, k: int) -> list:
    """(n, nw) uint64 keys of (k+1)-mers -> strings over ACGT."""
    out = []
    keys = np.asarray(keys, dtype=np.uint64)
    if len(keys) == 0:
        return out
    for row in keys.reshape(len(keys), -1):
        v = 0
        for w in reversed(range(row.shape[0])):
            v = (v << 64) | int(row[w])
        out.append("".join("ACGT"[(v >> (2 * (k - i))) & 3] for i in range(k + 1)))
    return out


def walk_contigs(solid: list, mercy: list, k: int, n_walks: int, max_len: int, seed: int) -> list:
    """The contigs of n_walks walks (solid, mercy: sorted (k+1)-mer strings)."""
    edges = list(solid) + list(mercy)
    if not edges:
        return []
    out_labels = {}
    for e in edges:
        out_labels.setdefault(e[:k], []).append(e[k])
    for v in out_labels:
        out_labels[v].sort()
    contigs = []
    for w in range(n_walks):
        s = list(edges[splitmix64_at(seed, w << 24) % len(edges)])
        j = 1
        while len(s) < max_len:
            labels = out_labels.get("".join(s[len(s) - k:]))
            if not labels:
                break
            s.append(labels[splitmix64_at(seed, (w << 24) + j) % len(labels)])
            j += 1
        contigs.append("".join(s))
    return contigs


def with_contigs(ascii: np.ndarray, offs: np.ndarray, contigs: list, copies: int):
    """Reads followed by ``copies`` copies of every contig (contig i, copy c is
    read n_reads + i * copies + c)."""
    parts = [np.asarray(ascii, dtype=np.uint8)]
    lens = list(np.diff(np.asarray(offs, dtype=np.uint64)).astype(np.int64))
    for c in contigs:
        b = np.frombuffer(c.encode(), dtype=np.uint8)
        for _ in range(copies):
            parts.append(b)
            lens.append(len(b))
    a = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    o = np.zeros(len(lens) + 1, dtype=np.uint64)
    o[1:] = np.cumsum(np.array(lens, dtype=np.uint64))
    return a, o


def iterate(ascii, offs, ks, d: int, n_walks: int, max_len: int, seed: int, build=True):
    """The multiple-k iteration; per k: solid/mercy tables, SdBG, contigs."""
    from . import build_sdbg, count
    steps = []
    contigs = []
    for i, k in enumerate(ks):
        a, o = with_contigs(ascii, offs, contigs, d)
        w = count(a, o, k, d, mercy=True)
        g = build_sdbg(k, w["solid_keys"], w["solid_cnt"], w["mercy_keys"], w["mercy_cnt"]) if build else None
        contigs = walk_contigs(key_strings(w["solid_keys"], k), key_strings(w["mercy_keys"], k), k, n_walks,
                               max_len, seed + i)
        steps.append({"k": k, "counts": w, "sdbg": g, "contigs": contigs})
    return steps
