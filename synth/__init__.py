"""Seeded synthetic read sets (inputs only).

Every function returns ``(ascii, offs)``: ``ascii`` is a ``numpy.uint8`` array
holding all reads back to back, ``offs`` a ``numpy.uint64`` array of
``n_reads + 1`` offsets (read ``i`` is ``ascii[offs[i]:offs[i+1]]``).  Nothing
here computes any part of the SdBG method; the CUDA path and the CPU oracle
both read what these functions write.

The bulk generators (``uniform_genome_reads``, ``metagenome_reads``) run in C
(``synth.c``: xoshiro256** streams seeded through splitmix64, one stream per
read or pair), so a 3 Gbp read set takes seconds.  The small generators used
for edge cases are plain numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (host gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            f64p = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.synth_genome_lengths.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_uint64, u64p]
            lib.synth_abundances.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double, f64p]
            lib.synth_genome_codes.argtypes = [ctypes.c_uint64, ctypes.c_int, u64p, u8p]
            lib.synth_reads.argtypes = [ctypes.c_uint64, u8p, ctypes.c_int, u64p, f64p,
                                        ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, u8p, ctypes.c_int]
            lib.synth_reads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def genome_codes(seed: int, lens) -> np.ndarray:
    """Uniform random genome bases as codes 0..3 (A,C,G,T), one byte each."""
    lib = _load()
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    codes = np.empty(int(lens.sum()), dtype=np.uint8)
    lib.synth_genome_codes(seed, len(lens), _ptr(lens, ctypes.c_uint64), _ptr(codes, ctypes.c_uint8))
    return codes


def _sample(seed, codes, lens, weight, n_units, read_len, paired, insert_mean, insert_sd,
            err, err_ramp, out=None):
    lib = _load()
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    weight = np.ascontiguousarray(weight, dtype=np.float64)
    n_reads = n_units * (2 if paired else 1)
    if out is None:
        ascii = np.empty(n_reads * read_len, dtype=np.uint8)
    else:
        if out.dtype != np.uint8 or not out.flags.c_contiguous or len(out) < n_reads * read_len:
            raise ValueError("out must be a contiguous uint8 array of n_reads * read_len bytes")
        ascii = out[: n_reads * read_len]
    rc = lib.synth_reads(seed, _ptr(codes, ctypes.c_uint8), len(lens), _ptr(lens, ctypes.c_uint64),
                         _ptr(weight, ctypes.c_double), n_units, read_len, 1 if paired else 0,
                         insert_mean, insert_sd, err, 1 if err_ramp else 0,
                         _ptr(ascii, ctypes.c_uint8), _threads())
    if rc != 0:
        raise ValueError("a genome is shorter than one read")
    offs = np.arange(n_reads + 1, dtype=np.uint64) * np.uint64(read_len)
    return ascii, offs


def uniform_genome_reads(seed: int = 1, genome_len: int = 50_000, n_reads: int = 10_000,
                         read_len: int = 100, err: float = 0.01):
    """One uniform-ACGT genome; single-end reads from uniform positions on
    either strand (50/50); iid substitutions at rate ``err``.

    The defaults are the small plain job: 50 kbp genome, 10,000 x 100 bp
    reads (20x), 1% errors, seed 1.
    """
    lens = np.array([genome_len], dtype=np.uint64)
    codes = genome_codes(seed, lens)
    return _sample(seed, codes, lens, np.ones(1), n_reads, read_len, False, 0.0, 0.0, err, False)


def metagenome_genomes(seed: int = 2, n_genomes: int = 100, median_len: float = 2e6,
                       sigma_len: float = 0.5, sigma_ab: float = 1.5):
    """Genome lengths (lognormal), abundances (lognormal) and bases of a
    simulated community."""
    lib = _load()
    lens = np.empty(n_genomes, dtype=np.uint64)
    lib.synth_genome_lengths(seed, n_genomes, median_len, sigma_len, 1000, _ptr(lens, ctypes.c_uint64))
    ab = np.empty(n_genomes, dtype=np.float64)
    lib.synth_abundances(seed, n_genomes, sigma_ab, _ptr(ab, ctypes.c_double))
    return lens, ab, genome_codes(seed, lens)


def metagenome_reads(seed: int = 2, n_genomes: int = 100, median_len: float = 2e6,
                     sigma_len: float = 0.5, sigma_ab: float = 1.5, n_pairs: int = 10_000_000,
                     read_len: int = 150, insert_mean: float = 350.0, insert_sd: float = 35.0,
                     err_3p: float = 0.01, out=None):
    """Simulated metagenome: genomes picked with probability proportional to
    abundance x length; paired reads (mate 2 = reverse complement of the
    fragment's end; insert ~ N(350, 35)); substitution rate
    ``err_3p * (i + 0.5) / read_len`` at read position i (mean 0.5% for the
    default 1% at the 3' end).  ``out``: a uint8 buffer to write the reads
    into (pinned host memory, say); the returned ``ascii`` is a view of it.

    The defaults are the full simulated-metagenome workload: 100 genomes,
    median 2 Mbp, 10 M pairs of 2 x 150 bp (3.0 Gbp), seed 2.
    """
    lens, ab, codes = metagenome_genomes(seed, n_genomes, median_len, sigma_len, sigma_ab)
    weight = ab * lens.astype(np.float64)
    return _sample(seed, codes, lens, weight, n_pairs, read_len, True, insert_mean, insert_sd,
                   err_3p, True, out)


def batch_read_counts(seed: int = 5, n_sets: int = 64, lo: int = 50_000, hi: int = 5_000_000) -> np.ndarray:
    """Read counts of a batch: lognormal with ln-median halfway between ln lo
    and ln hi and sigma a quarter of that span, clipped to [lo, hi], rounded
    down to an even count (pairs)."""
    rng = np.random.default_rng(seed)
    mu = (np.log(lo) + np.log(hi)) / 2
    sigma = (np.log(hi) - np.log(lo)) / 4
    n = np.clip(np.exp(rng.normal(mu, sigma, size=n_sets)), lo, hi).astype(np.int64)
    return n // 2 * 2


def batch_sets(seed: int = 5, n_sets: int = 64, lo: int = 50_000, hi: int = 5_000_000,
               read_len: int = 150, err_3p: float = 0.01):
    """Independent read sets of a batch: set i is a 10-genome mini-metagenome
    (``metagenome_reads`` with 10 genomes, seed ``seed * 1000 + i``) of
    ``batch_read_counts`` reads in pairs of ``read_len`` bp, substitution rate
    rising to ``err_3p`` at the 3' end (mean 0.5%)."""
    counts = batch_read_counts(seed, n_sets, lo, hi)
    return [metagenome_reads(seed=seed * 1000 + i, n_genomes=10, n_pairs=int(c) // 2, read_len=read_len,
                             err_3p=err_3p) for i, c in enumerate(counts)]


def random_reads(seed: int, n_reads: int, min_len: int, max_len: int, p_invalid: float = 0.0,
                 p_lower: float = 0.0, alphabet: bytes = b"ACGT"):
    """Independent random reads with lengths uniform in [min_len, max_len].

    ``p_invalid``: chance that a base is replaced by ``N``; ``p_lower``: chance
    that a base is written in lower case.  Used for ragged and edge cases.
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(min_len, max_len + 1, size=n_reads).astype(np.uint64)
    offs = np.zeros(n_reads + 1, dtype=np.uint64)
    np.cumsum(lens, out=offs[1:])
    total = int(offs[-1])
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    ascii = alpha[rng.integers(0, len(alpha), size=total)]
    if p_invalid > 0:
        ascii[rng.random(total) < p_invalid] = ord("N")
    if p_lower > 0:
        low = rng.random(total) < p_lower
        ascii[low] = ascii[low] | 0x20
    return ascii.astype(np.uint8), offs


def reads_from_strings(reads) -> tuple:
    """Pack a list of str/bytes reads into (ascii, offs)."""
    bs = [r.encode() if isinstance(r, str) else bytes(r) for r in reads]
    offs = np.zeros(len(bs) + 1, dtype=np.uint64)
    np.cumsum([len(b) for b in bs], out=offs[1:]) if bs else None
    ascii = np.frombuffer(b"".join(bs), dtype=np.uint8).copy()
    return ascii, offs


def genome_tiling_reads(seed: int, genome_len: int, read_len: int, coverage: int):
    """Error-free reads tiling a uniform random genome: ``coverage`` copies of
    every read start 0, s, 2s, ... with s = read_len // 2, forward strand only,
    plus the last window.  Used for closed-form cases (solid set = all genome
    (k+1)-mers on both strands)."""
    codes = genome_codes(seed, np.array([genome_len], dtype=np.uint64))
    genome = np.frombuffer(b"ACGT", dtype=np.uint8)[codes]
    step = max(1, read_len // 2)
    starts = list(range(0, genome_len - read_len + 1, step))
    if starts[-1] != genome_len - read_len:
        starts.append(genome_len - read_len)
    reads = []
    for _ in range(coverage):
        for s in starts:
            reads.append(genome[s:s + read_len].tobytes())
    ascii, offs = reads_from_strings(reads)
    return ascii, offs, genome.tobytes()
