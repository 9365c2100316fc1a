"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

All outputs are integers, so every comparison is bit-exact (tolerance zero):
packed fragments, solid and mercy keys with counts, and every SdBG array.
Sizes span several radix tiles (4096 keys) with ragged tails; the edge cases
cover empty input, reads shorter than k+1, N and lower case, palindromes,
every key width (1, 2, 4 words) and the error codes.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1409_7208_gb300 as mh
    mh.load_library()
    return mh


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(device=0)


def _pack_expect(bases: bytes) -> np.ndarray:
    codes = np.frombuffer(bases, dtype=np.uint8)
    lut = np.zeros(256, dtype=np.uint32)
    for i, c in enumerate(b"ACGT"):
        lut[c] = i
    c = lut[codes]
    n_words = (len(c) + 15) // 16
    pad = np.zeros(n_words * 16, dtype=np.uint32)
    pad[: len(c)] = c
    pad = pad.reshape(n_words, 16)
    shifts = (30 - 2 * np.arange(16)).astype(np.uint32)
    return np.bitwise_or.reduce(pad << shifts, axis=1).astype(np.uint32) if n_words else np.zeros(0, np.uint32)


def _run(mh, ctx, ascii, offs, k, d):
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    solid = mh.mh_count_kmers(ctx, reads, k, d)
    mercy = mh.mh_mercy_kmers(ctx, reads, solid)
    sdbg = mh.mh_build_sdbg(ctx, solid, mercy)
    return reads, solid, mercy, sdbg


def _compare_all(mh, ctx, ascii, offs, k, d):
    reads, solid, mercy, sdbg = _run(mh, ctx, ascii, offs, k, d)
    want = oracle.count(ascii, offs, k, d, mercy=True)
    gs, gm = solid.numpy(), mercy.numpy()
    assert gs["n_kmers"] == want["n_kmers"]
    assert gs["n_distinct"] == want["n_distinct"]
    assert np.array_equal(gs["keys"], want["solid_keys"])
    assert np.array_equal(gs["counts"], want["solid_cnt"])
    assert np.array_equal(gm["keys"], want["mercy_keys"])
    assert np.array_equal(gm["counts"], want["mercy_cnt"])
    wg = oracle.build_sdbg(k, want["solid_keys"], want["solid_cnt"], want["mercy_keys"], want["mercy_cnt"])
    gg = sdbg.numpy()
    for key in ("m", "t", "u", "n_nodes"):
        assert gg[key] == wg[key], key
    for key in ("W", "last", "dummy", "valid", "F", "aux"):
        assert np.array_equal(gg[key], wg[key]), key
    return reads, gs, gm, gg


# ------------------------------------------------------------------- pack

@pytest.mark.parametrize("case", ["clean", "invalid", "empty_reads", "lower", "tiny"])
def test_pack_matches_oracle_fragments(mh, ctx, case):
    if case == "clean":
        ascii, offs = synth.random_reads(1, 500, 1, 300)
    elif case == "invalid":
        ascii, offs = synth.random_reads(2, 700, 0, 200, p_invalid=0.03)
    elif case == "empty_reads":
        ascii, offs = synth.reads_from_strings(["", "ACGT", "", "", "NNNN", "T"] * 50)
    elif case == "lower":
        ascii, offs = synth.random_reads(3, 300, 5, 90, p_lower=0.5, p_invalid=0.01)
    else:
        ascii, offs = synth.reads_from_strings(["A"])
    bases, fo, fr = oracle.fragments(ascii, offs)
    r = mh.mh_pack_reads(ctx, ascii, offs).tensors()
    assert r["n_frags"] == len(fr)
    assert r["n_packed"] == len(bases)
    got_words = r["packed"].cpu().numpy().view(np.uint32)
    assert np.array_equal(got_words, _pack_expect(bases))
    assert np.array_equal(r["frag_offs"].cpu().numpy().view(np.uint64), fo)
    assert np.array_equal(r["frag_read"].cpu().numpy().view(np.uint32), fr)


def test_pack_from_device_buffers(mh, ctx):
    import torch
    ascii, offs = synth.random_reads(4, 200, 10, 120, p_invalid=0.01)
    r_host = mh.mh_pack_reads(ctx, ascii, offs).tensors()
    r_dev = mh.mh_pack_reads(ctx, torch.from_numpy(ascii).cuda(), torch.from_numpy(offs.view(np.int64)).cuda()).tensors()
    for key in ("packed", "frag_offs", "frag_read"):
        assert torch.equal(r_host[key], r_dev[key])


# --------------------------------------------------- count, mercy, build

CASES = [
    # (name, k, d, generator)
    ("k21_d2_genome", 21, 2, lambda: synth.uniform_genome_reads(11, 3000, 900, 100, 0.01)),
    ("k31_d2_genome", 31, 2, lambda: synth.uniform_genome_reads(12, 4000, 800, 150, 0.01)),
    ("k31_d1", 31, 1, lambda: synth.uniform_genome_reads(13, 2000, 200, 120, 0.02)),
    ("k21_d3", 21, 3, lambda: synth.uniform_genome_reads(14, 2500, 1200, 80, 0.01)),
    ("k9_small_alphabet", 9, 2, lambda: synth.random_reads(15, 400, 0, 60, alphabet=b"AC")),
    ("k2", 2, 2, lambda: synth.random_reads(16, 200, 0, 12, p_invalid=0.05)),
    ("k3_palindromes", 3, 2, lambda: synth.reads_from_strings(["ACGT", "ACGTACGT", "AATT", "GGCC"] * 5 + ["ACGTT"])),
    ("k15_N_lower", 15, 2, lambda: synth.uniform_genome_reads(17, 1500, 600, 70, 0.0)),
    ("k32_two_words", 32, 2, lambda: synth.uniform_genome_reads(18, 3000, 600, 120, 0.01)),
    ("k47_two_words", 47, 2, lambda: synth.uniform_genome_reads(19, 3000, 700, 130, 0.01)),
    ("k63_two_words_full", 63, 2, lambda: synth.uniform_genome_reads(20, 3000, 700, 140, 0.01)),
    ("k64_four_words", 64, 2, lambda: synth.uniform_genome_reads(21, 3000, 700, 140, 0.01)),
    ("k99_four_words", 99, 2, lambda: synth.uniform_genome_reads(22, 3000, 900, 150, 0.005)),
    ("k127_four_words_full", 127, 2, lambda: synth.uniform_genome_reads(23, 2000, 900, 150, 0.003)),
]


@pytest.mark.parametrize("name,k,d,gen", CASES, ids=[c[0] for c in CASES])
def test_pipeline_parity(mh, ctx, name, k, d, gen):
    ascii, offs = gen()
    if name == "k15_N_lower":
        rng = np.random.default_rng(5)
        ascii = ascii.copy()
        ascii[rng.random(len(ascii)) < 0.01] = ord("N")
        low = rng.random(len(ascii)) < 0.2
        ascii[low] |= 0x20
    _compare_all(mh, ctx, ascii, offs, k, d)


def test_low_coverage_gaps_give_mercy(mh, ctx):
    """Flank / gap / flank reads (the shape mercy exists for) at k = 21."""
    rng = np.random.default_rng(7)
    reads = []
    for _ in range(40):
        g = "".join(rng.choice(list("ACGT"), size=260))
        reads += [g[0:100]] * 3 + [g[160:260]] * 3 + [g[50:210]]
    ascii, offs = synth.reads_from_strings(reads)
    _, gs, gm, _ = _compare_all(mh, ctx, ascii, offs, 21, 2)
    assert len(gm["counts"]) > 0


@pytest.mark.parametrize("n_windows", [1, 4095, 4096, 4097, 8191, 8193, 3 * 4096 + 17, 40961])
def test_tile_boundaries(mh, ctx, n_windows):
    """Reads of 64 windows plus one ragged read, so that the canonical sort
    sees exactly n_windows keys: on and around multiples of the 4096-key
    radix tile (and of the 2048-key run tile and the 4096-item scan tile)."""
    k = 20
    rng = np.random.default_rng(n_windows)
    q, r = divmod(n_windows, 64)
    lens = [k + 64] * q + ([k + r] if r else [])
    reads = ["".join(rng.choice(list("ACG"), size=L)) for L in lens]
    ascii, offs = synth.reads_from_strings(reads)
    _compare_all(mh, ctx, ascii, offs, k, 1)


@pytest.mark.parametrize("n_reads", [300, 1500, 3000])
def test_shared_prefix_groups(mh, ctx, n_reads):
    """Distinct keys sharing their top 40 bits (a 20-base common prefix): the
    sorts run their LSD passes over the top bits only and must put such groups
    in order afterwards (in shared memory, or by segment passes when a group is
    larger than a tile)."""
    rng = np.random.default_rng(n_reads)
    reads = ["A" * 20 + "".join(rng.choice(list("CGT"), size=12)) for _ in range(n_reads)]
    ascii, offs = synth.reads_from_strings(reads + reads)
    _compare_all(mh, ctx, ascii, offs, 31, 2)
    _compare_all(mh, ctx, ascii, offs, 25, 1)


def test_empty_and_short_inputs(mh, ctx):
    for reads in ([], [""], ["ACG"], ["NNNN", "AC"], ["ACGTACGTAC"]):
        ascii, offs = synth.reads_from_strings(reads)
        _compare_all(mh, ctx, ascii, offs, 5, 1)


def test_small_plain_job_end_to_end(mh, ctx):
    """The small plain workload at full size: 50 kbp genome, 10,000 x 100 bp
    reads, 1% errors, k = 21, d = 2, seed 1."""
    ascii, offs = synth.uniform_genome_reads()
    _, gs, gm, gg = _compare_all(mh, ctx, ascii, offs, 21, 2)
    edges = np.concatenate([gs["keys"], gm["keys"]])
    check.check_sdbg(gg, 21, edges)


def test_with_mult(mh):
    ctx = mh.Context(device=0, with_mult=True)
    ascii, offs = synth.uniform_genome_reads(31, 3000, 600, 100, 0.01)
    k = 21
    _, solid, mercy, sdbg = _run(mh, ctx, ascii, offs, k, 2)
    want = oracle.count(ascii, offs, k, 2, mercy=True)
    wg = oracle.build_sdbg(k, want["solid_keys"], want["solid_cnt"], want["mercy_keys"], want["mercy_cnt"])
    assert np.array_equal(sdbg.numpy()["mult"], wg["mult"])


def test_library_pool_allocator(mh):
    ctx = mh.Context(device=0, torch_allocator=False)
    ascii, offs = synth.uniform_genome_reads(32, 3000, 600, 100, 0.01)
    _compare_all(mh, ctx, ascii, offs, 21, 2)
    in_use, peak = ctx.memory()
    assert peak > 0


# ------------------------------------------------------------------ errors

def test_error_codes(mh, ctx):
    ascii, offs = synth.uniform_genome_reads(33, 2000, 100, 100, 0.01)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    for k, d in ((1, 2), (128, 2), (21, 0)):
        with pytest.raises(mh.MhError) as e:
            mh.mh_count_kmers(ctx, reads, k, d)
        assert e.value.code == mh.MH_EINVAL
    bad = offs.copy()
    bad[3], bad[4] = bad[4], bad[3]
    with pytest.raises(mh.MhError) as e:
        mh.mh_pack_reads(ctx, ascii, bad)
    assert e.value.code == mh.MH_EINVAL
    # the context stays usable after an error
    s = mh.mh_count_kmers(ctx, reads, 21, 2)
    assert s.n > 0


def test_budget_exceeded_is_enomem(mh):
    ctx = mh.Context(device=0, hbm_budget=1 << 16)
    ascii, offs = synth.uniform_genome_reads(34, 2000, 2000, 100, 0.01)
    with pytest.raises(mh.MhError) as e:
        reads = mh.mh_pack_reads(ctx, ascii, offs)
        mh.mh_count_kmers(ctx, reads, 21, 2)
    assert e.value.code == mh.MH_ENOMEM


def test_mismatched_k_is_einval(mh, ctx):
    ascii, offs = synth.uniform_genome_reads(35, 2000, 300, 100, 0.01)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    a = mh.mh_count_kmers(ctx, reads, 21, 2)
    b = mh.mh_count_kmers(ctx, reads, 23, 2)
    with pytest.raises(mh.MhError) as e:
        mh.mh_build_sdbg(ctx, a, b)
    assert e.value.code == mh.MH_EINVAL


def test_count_under_hbm_budget_matches_in_memory_count():
    """A budget too small for the whole key set makes counting go bucket by
    bucket; the tables must not change."""
    import paper_1409_7208_gb300 as mh
    ascii, offs = synth.uniform_genome_reads(1)
    free = mh.Context(device=0)
    want = mh.mh_count_kmers(free, mh.mh_pack_reads(free, ascii, offs), 21, 2)
    ctx = mh.Context(device=0, hbm_budget=40 << 20)
    reads = mh.mh_pack_reads(ctx, ascii, offs)
    got = mh.mh_count_kmers(ctx, reads, 21, 2)
    used, peak = ctx.memory()
    g, w = got.numpy(), want.numpy()
    assert np.array_equal(g["keys"], w["keys"]) and np.array_equal(g["counts"], w["counts"])
    assert g["n_distinct"] == w["n_distinct"] and peak <= 40 << 20
    # the bucketed spectrum serves the mercy step like the in-memory one
    m = mh.mh_mercy_kmers(free, reads, got).numpy()
    w_m = mh.mh_mercy_kmers(free, mh.mh_pack_reads(free, ascii, offs), want).numpy()
    assert np.array_equal(m["keys"], w_m["keys"]) and np.array_equal(m["counts"], w_m["counts"])
