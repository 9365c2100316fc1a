"""CPU oracle for the SdBG construction hot path (MEGAHIT, Li et al. 2015).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The CUDA library never calls it and shares no code, header or helper with it.

* ``mh_oracle.cpp`` - the oracle proper: plain C++ over ``std::string``
  k-mers, ``std::sort``, ``std::set``/``std::map`` (paper, Sec. 2).
* ``brute.py``      - pure-Python brute force used to pin the oracle on tiny
  inputs (all-pairs mercy, dictionary counting, string-level BOSS).
* ``check.py``      - invariants and the BOSS traversal that pin the SdBG
  arrays without reference to how they were built.

Output layout (shared with the CUDA library by definition, not by code): a
(k+1)-mer s is the integer sum s[i] * 4^(k-i) with A=0, C=1, G=2, T=3, held in
``nw`` little-endian 64-bit words, nw = 1, 2 or 4 for 2(k+1) <= 64, 128, 256.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mh_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``mh_oracle.cpp`` into ``liboracle.so`` next to it (host g++)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _KmerResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("k", ctypes.c_int), ("nw", ctypes.c_int),
                ("n_kmers", ctypes.c_uint64), ("n_distinct", ctypes.c_uint64),
                ("n_solid", ctypes.c_uint64), ("solid_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("solid_cnt", ctypes.POINTER(ctypes.c_uint32)),
                ("n_mercy", ctypes.c_uint64), ("mercy_keys", ctypes.POINTER(ctypes.c_uint64)),
                ("mercy_cnt", ctypes.POINTER(ctypes.c_uint32))]


class _SdbgResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("k", ctypes.c_int), ("nw", ctypes.c_int),
                ("m", ctypes.c_uint64), ("t", ctypes.c_uint64), ("u", ctypes.c_uint64),
                ("n_nodes", ctypes.c_uint64),
                ("W", ctypes.POINTER(ctypes.c_uint8)), ("last", ctypes.POINTER(ctypes.c_uint8)),
                ("valid", ctypes.POINTER(ctypes.c_uint8)), ("dummy", ctypes.POINTER(ctypes.c_uint8)),
                ("mult", ctypes.POINTER(ctypes.c_uint32)), ("F", ctypes.c_uint64 * 6),
                ("aux", ctypes.POINTER(ctypes.c_uint64))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p, u64p, u32p = (ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint32))
            lib.orc_count.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_count.restype = ctypes.POINTER(_KmerResult)
            lib.orc_count_threaded.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int]
            lib.orc_count_threaded.restype = ctypes.POINTER(_KmerResult)
            lib.orc_free_kmer_result.argtypes = [ctypes.POINTER(_KmerResult)]
            lib.orc_build_sdbg.argtypes = [ctypes.c_int, u64p, u32p, ctypes.c_uint64, u64p, u32p,
                                           ctypes.c_uint64]
            lib.orc_build_sdbg.restype = ctypes.POINTER(_SdbgResult)
            lib.orc_free_sdbg_result.argtypes = [ctypes.POINTER(_SdbgResult)]
            lib.orc_count_queries.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, u64p,
                                              ctypes.c_uint64, u64p, ctypes.c_int]
            lib.orc_count_queries.restype = ctypes.c_int
            lib.orc_fragments.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_char_p, u64p, u32p]
            lib.orc_fragments.restype = ctypes.c_uint64
            lib.orc_find_windows.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, u64p, ctypes.c_uint64,
                                             ctypes.c_uint64, u64p, u64p, u64p, ctypes.c_int]
            lib.orc_find_windows.restype = ctypes.c_int64
            _lib = lib
    return _lib


def words_for(k: int) -> int:
    """Number of 64-bit words of a (k+1)-mer key."""
    return 1 if 2 * (k + 1) <= 64 else (2 if 2 * (k + 1) <= 128 else 4)


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def fragments(ascii, offs):
    """(bases, frag_offs, frag_read): the fragments of every read (maximal
    ACGT runs, upper-cased) back to back as bytes, their offsets and reads."""
    lib = _load()
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    n_reads = len(offs) - 1
    buf = ctypes.create_string_buffer(max(1, len(ascii)))
    fo = np.zeros(len(ascii) + 2, dtype=np.uint64)
    fr = np.zeros(len(ascii) + 1, dtype=np.uint32)
    a = ascii if len(ascii) else np.zeros(1, dtype=np.uint8)
    nf = lib.orc_fragments(_p(a, ctypes.c_uint8), _p(offs, ctypes.c_uint64), n_reads, buf,
                           _p(fo, ctypes.c_uint64), _p(fr, ctypes.c_uint32))
    total = int(fo[nf])
    return buf.raw[:total], fo[:nf + 1].copy(), fr[:nf].copy()


def count(ascii, offs, k: int, d: int = 2, mercy: bool = True, threads: int = 1) -> dict:
    """Solid (k+1)-mers with counts and, if ``mercy``, mercy (k+1)-mers.
    ``threads`` > 1: the same computation split by 8-symbol prefix over that
    many threads (counting) and by fragment (mercy).

    Returns ``solid_keys`` (S x nw uint64, ascending), ``solid_cnt`` (uint32),
    ``mercy_keys``/``mercy_cnt`` likewise, ``n_kmers`` = |K| (both strands)
    and ``n_distinct``.
    """
    lib = _load()
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    n_reads = len(offs) - 1
    if len(ascii) == 0:
        ascii = np.zeros(1, dtype=np.uint8)
    if threads > 1:
        r = lib.orc_count_threaded(_p(ascii, ctypes.c_uint8), _p(offs, ctypes.c_uint64), n_reads, k, d,
                                   1 if mercy else 0, int(threads))
    else:
        r = lib.orc_count(_p(ascii, ctypes.c_uint8), _p(offs, ctypes.c_uint64), n_reads, k, d,
                          1 if mercy else 0)
    try:
        c = r.contents
        if c.status != 0:
            raise ValueError("oracle count failed with status %d" % c.status)
        nw = c.nw
        out = {
            "k": k, "d": d, "nw": nw, "n_kmers": c.n_kmers, "n_distinct": c.n_distinct,
            "solid_keys": _arr(c.solid_keys, c.n_solid * nw, np.uint64).reshape(-1, nw),
            "solid_cnt": _arr(c.solid_cnt, c.n_solid, np.uint32),
        }
        if mercy:
            out["mercy_keys"] = _arr(c.mercy_keys, c.n_mercy * nw, np.uint64).reshape(-1, nw)
            out["mercy_cnt"] = _arr(c.mercy_cnt, c.n_mercy, np.uint32)
        return out
    finally:
        lib.orc_free_kmer_result(r)


def build_sdbg(k: int, solid_keys, solid_cnt=None, mercy_keys=None, mercy_cnt=None) -> dict:
    """BOSS arrays of the edge set solid + mercy (paper, Sec. 2).

    Returns ``W`` (uint8 codes $=0 A=1 C=2 G=3 T=4, +4 for the minus flag),
    ``last``/``valid``/``dummy`` (uint8 0/1 per entry), ``mult`` (uint32),
    ``F`` (6 x uint64), ``aux`` (t x nw uint64, the zero-indegree vertices in
    the order of their dummy edges), ``m``, ``t``, ``u``, ``n_nodes``.
    """
    lib = _load()
    nw = words_for(k)
    sk = np.ascontiguousarray(np.asarray(solid_keys, dtype=np.uint64).reshape(-1, nw))
    n_s = sk.shape[0]
    sc = None if solid_cnt is None else np.ascontiguousarray(solid_cnt, dtype=np.uint32)
    if mercy_keys is None:
        mk = np.zeros((0, nw), dtype=np.uint64)
    else:
        mk = np.ascontiguousarray(np.asarray(mercy_keys, dtype=np.uint64).reshape(-1, nw))
    n_m = mk.shape[0]
    mc = None if mercy_cnt is None else np.ascontiguousarray(mercy_cnt, dtype=np.uint32)
    dummy64 = np.zeros(nw, dtype=np.uint64)
    r = lib.orc_build_sdbg(k, _p(sk if n_s else dummy64, ctypes.c_uint64),
                           None if sc is None else _p(sc, ctypes.c_uint32), n_s,
                           _p(mk if n_m else dummy64, ctypes.c_uint64),
                           None if mc is None else _p(mc, ctypes.c_uint32), n_m)
    try:
        c = r.contents
        if c.status != 0:
            raise ValueError("oracle build failed with status %d" % c.status)
        m = c.m
        return {
            "k": k, "nw": nw, "m": m, "t": c.t, "u": c.u, "n_nodes": c.n_nodes,
            "W": _arr(c.W, m, np.uint8), "last": _arr(c.last, m, np.uint8),
            "valid": _arr(c.valid, m, np.uint8), "dummy": _arr(c.dummy, m, np.uint8),
            "mult": _arr(c.mult, m, np.uint32), "F": np.array(list(c.F), dtype=np.uint64),
            "aux": _arr(c.aux, c.t * nw, np.uint64).reshape(-1, nw),
        }
    finally:
        lib.orc_free_sdbg_result(r)


def count_queries(ascii, offs, k: int, queries, n_threads: int | None = None) -> np.ndarray:
    """Multiplicity in K (both strands) of each query key, by scanning every
    read.  For sampled checks on read sets too large for ``count``."""
    lib = _load()
    nw = words_for(k)
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.uint64).reshape(-1, nw))
    out = np.zeros(q.shape[0], dtype=np.uint64)
    if q.shape[0] == 0:
        return out
    if n_threads is None:
        n_threads = max(1, min(64, os.cpu_count() or 1))
    rc = lib.orc_count_queries(_p(ascii, ctypes.c_uint8), _p(offs, ctypes.c_uint64), len(offs) - 1,
                               k, _p(q, ctypes.c_uint64), q.shape[0], _p(out, ctypes.c_uint64),
                               n_threads)
    if rc != 0:
        raise ValueError("oracle count_queries failed")
    return out


def find_windows(ascii, offs, k: int, queries, cap: int = 1 << 20, n_threads: int | None = None):
    """Every occurrence of the query keys as a forward window of a fragment:
    arrays (query index, read index, window position in the read), sorted,
    at most ``cap`` of them (ValueError beyond)."""
    lib = _load()
    nw = words_for(k)
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.uint64).reshape(-1, nw))
    hq = np.zeros(max(1, cap), dtype=np.uint64)
    hr = np.zeros(max(1, cap), dtype=np.uint64)
    hp = np.zeros(max(1, cap), dtype=np.uint64)
    if n_threads is None:
        n_threads = max(1, min(64, os.cpu_count() or 1))
    a = ascii if len(ascii) else np.zeros(1, dtype=np.uint8)
    qq = q if q.shape[0] else np.zeros((1, nw), dtype=np.uint64)
    n = lib.orc_find_windows(_p(a, ctypes.c_uint8), _p(offs, ctypes.c_uint64), len(offs) - 1, k,
                             _p(qq, ctypes.c_uint64), q.shape[0], cap, _p(hq, ctypes.c_uint64),
                             _p(hr, ctypes.c_uint64), _p(hp, ctypes.c_uint64), n_threads)
    if n < 0:
        raise ValueError("oracle find_windows failed")
    if n > cap:
        raise ValueError("%d hits, more than the cap of %d" % (n, cap))
    return hq[:n].copy(), hr[:n].copy(), hp[:n].copy()


# ------------------------------------------------------------ key helpers
# Conversions between packed keys and strings, for tests and checks.

_SYM = "ACGT"


def key_to_str(key_words, n: int) -> str:
    """Packed key (nw words) -> string of n symbols."""
    v = 0
    for w in reversed([int(x) for x in np.atleast_1d(key_words)]):
        v = (v << 64) | w
    return "".join(_SYM[(v >> (2 * (n - 1 - i))) & 3] for i in range(n))


def str_to_key(s: str, nw: int) -> np.ndarray:
    """String over ACGT -> packed key (nw words)."""
    v = 0
    for ch in s:
        v = v * 4 + _SYM.index(ch)
    return np.array([(v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(nw)], dtype=np.uint64)


def keys_to_strs(keys, n: int) -> list:
    keys = np.asarray(keys, dtype=np.uint64)
    keys = keys.reshape(keys.shape[0], -1) if keys.size else keys.reshape(0, 1)
    return [key_to_str(keys[i], n) for i in range(keys.shape[0])]


def strs_to_keys(strs, nw: int) -> np.ndarray:
    if not strs:
        return np.zeros((0, nw), dtype=np.uint64)
    return np.stack([str_to_key(s, nw) for s in strs])
