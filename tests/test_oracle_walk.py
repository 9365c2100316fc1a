"""Pins of the contig-walk oracle (oracle/walk.py) and the multiple-k
iteration, without the CUDA path.  CPU only.

* the generator against the reference outputs of SplitMix64 (golden file);
* closed form: on the graph of an error-free, high-coverage tiling of a
  random genome (two simple paths, one per strand) every walk is the genome
  (or its reverse complement) from the start edge to the path's end or to
  max_len;
* invariants on branching graphs: every (k+1)-window of a contig is an edge,
  a walk stops early only at a dead end, every out-edge of a branch is taken
  about equally often;
* the iteration: on error-free reads the contig-derived edges add nothing
  new, and with d = 1 the contigs' windows are all in the next graph.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import walk as ow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def _rc(s):
    return "".join(COMP[c] for c in reversed(s))


def test_splitmix64_reference_outputs():
    for line in open(os.path.join(ROOT, "tests", "golden", "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, idx, val = (int(x) for x in line.split())
        assert ow.splitmix64_at(seed, idx) == val


def _genome_graph(G, k, seed):
    ascii, offs, genome = synth.genome_tiling_reads(seed, G, 60, 3)
    w = oracle.count(ascii, offs, k, 2, mercy=True)
    return genome.decode(), w


def test_walks_on_two_simple_paths_follow_the_genome():
    k, G = 15, 3000
    genome, w = _genome_graph(G, k, 5)
    solid = ow.key_strings(w["solid_keys"], k)
    assert len(w["mercy_keys"]) == 0
    rc = _rc(genome)
    for max_len in (40, 500, 10_000):
        for s in ow.walk_contigs(solid, [], k, 30, max_len, 77):
            # the walk is the strand from its start edge, to the end or max_len
            src = genome if s[:k + 1] in genome else rc
            p = src.index(s[:k + 1])
            assert s == src[p:min(len(src), p + max_len)]


def test_walk_invariants_on_branching_graph():
    k = 11
    ascii, offs = synth.uniform_genome_reads(3, 3000, 1500, 100, 0.01)
    w = oracle.count(ascii, offs, k, 2, mercy=True)
    solid, mercy = ow.key_strings(w["solid_keys"], k), ow.key_strings(w["mercy_keys"], k)
    E = set(solid) | set(mercy)
    out = {}
    for e in E:
        out.setdefault(e[:k], set()).add(e[k])
    branch_seen = {}
    for s in ow.walk_contigs(solid, mercy, k, 400, 300, 9):
        assert len(s) >= k + 1
        for i in range(len(s) - k):
            assert s[i:i + k + 1] in E
            v = s[i + 1:i + k + 1]
            if i + k + 1 < len(s) and len(out.get(s[i:i + k], ())) == 2:
                key = s[i:i + k]
                branch_seen.setdefault(key, []).append(s[i + k])
        if len(s) < 300:
            assert s[-k:] not in out, "stopped before max_len at a node with out-edges"
    # every label of a 2-way branch is taken about half of the time
    taken = [lab for labs in branch_seen.values() for lab in labs]
    assert len(taken) > 200
    firsts = sum(1 for key, labs in branch_seen.items() for lab in labs if lab == min(out[key]))
    assert abs(firsts / len(taken) - 0.5) < 0.1


def test_walks_depend_on_seed_and_walk_index():
    k = 11
    ascii, offs = synth.uniform_genome_reads(3, 3000, 1500, 100, 0.01)
    w = oracle.count(ascii, offs, k, 2, mercy=True)
    solid, mercy = ow.key_strings(w["solid_keys"], k), ow.key_strings(w["mercy_keys"], k)
    a = ow.walk_contigs(solid, mercy, k, 50, 200, 1)
    b = ow.walk_contigs(solid, mercy, k, 50, 200, 2)
    assert a != b and len(set(a)) > 40
    assert ow.walk_contigs(solid, mercy, k, 50, 200, 1) == a


def test_iteration_on_error_free_reads_adds_no_edges():
    ascii, offs, genome = synth.genome_tiling_reads(6, 2500, 60, 3)
    genome = genome.decode()
    steps = ow.iterate(ascii, offs, (15, 21, 27), 2, 20, 400, 11, build=False)
    for st in steps:
        k = st["k"]
        plain = oracle.count(ascii, offs, k, 2, mercy=True)
        # contigs are genome substrings, so their windows are already solid
        assert np.array_equal(st["counts"]["solid_keys"], plain["solid_keys"])
        for c in st["contigs"]:
            assert c in genome or _rc(c) in genome


def test_iteration_contig_edges_enter_the_next_graph():
    ascii, offs = synth.uniform_genome_reads(4, 2000, 600, 100, 0.02)
    steps = ow.iterate(ascii, offs, (13, 19), 2, 40, 300, 5, build=False)
    nxt = steps[1]
    edges = set(ow.key_strings(nxt["counts"]["solid_keys"], 19))
    for c in steps[0]["contigs"]:
        for i in range(len(c) - 19):
            x = c[i:i + 20]
            assert x in edges and _rc(x) in edges
