"""mh_sort_keys_noalloc: the radix sort for callers that may not allocate
device memory (for example code running inside an engine that owns the whole
device memory budget and forbids others to call cudaMalloc or cudaFree).

Its output must equal the existing entry point's: the solid table that
mh_count_kmers returns is already sorted, so shuffling it and sorting it
again through the no-allocation entry point must give it back exactly (the
keys are integers: the tolerance is zero).  Several calls run in a row, with
different key widths, because every call reuses the same static scratch
array.  Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest


def _call(lib, src, dst, n, nw, key_bits, stream):
    return lib.mh_sort_keys_noalloc(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), n, nw,
                                    key_bits, ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.gpu
def test_noalloc_sort_matches_count_kmers_on_consecutive_calls():
    import torch

    import paper_1409_7208_gb300 as mh
    import synth

    lib = mh.load_library()
    ctx = mh.Context(device=0)
    stream = torch.cuda.current_stream()
    # one-, two-, four- and one-word keys again: every call reuses the array
    for call, (k, seed) in enumerate(((21, 41), (47, 42), (99, 44), (31, 43))):
        ascii, offs = synth.uniform_genome_reads(seed, 4000, 900, 130, 0.01)
        reads = mh.mh_pack_reads(ctx, ascii, offs)
        solid = mh.mh_count_kmers(ctx, reads, k, 2)
        want = solid.keys.clone()
        n, nw = want.shape
        assert n > 4096, "spans several radix tiles"
        perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).to(want.device)
        shuffled = want[perm].contiguous()
        out = torch.full_like(shuffled, -1)
        torch.cuda.synchronize()
        rc = _call(lib, shuffled, out, n, nw, 2 * (k + 1), stream)
        assert rc == mh.MH_OK, "call %d returned %d" % (call, rc)
        torch.cuda.synchronize()
        assert torch.equal(out, want), "call %d differs from mh_count_kmers" % call


@pytest.mark.gpu
def test_noalloc_sort_wide_keys_with_ragged_key_bits():
    """Four-word keys sorted by 200 bits (not a whole number of digits), twice
    in a row, against a lexicographic sort of the words on the host."""
    import torch

    import paper_1409_7208_gb300 as mh

    rng = np.random.default_rng(7)
    n = 9000
    for call in range(2):
        words = rng.integers(0, 1 << 63, size=(n, 4), dtype=np.int64).astype(np.uint64)
        words[:, 3] &= np.uint64((1 << 8) - 1)  # 200 bits: 3 full words + 8 bits
        words[: n // 3] = words[n // 3: 2 * (n // 3)]  # duplicates
        order = np.lexsort((words[:, 0], words[:, 1], words[:, 2], words[:, 3]))
        want = words[order]
        src = torch.from_numpy(words.view(np.int64)).cuda()
        dst = torch.full_like(src, -1)
        mh.mh_sort_keys_noalloc(src, dst, 4, 200)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy().view(np.uint64), want), "call %d" % call


def test_noalloc_sort_rejects_misaligned_buffers_before_touching_the_device():
    """The argument checks come before any CUDA call, so this runs without a
    GPU: the addresses are never dereferenced."""
    import paper_1409_7208_gb300 as mh

    lib = mh.load_library()
    a, b = 0x10000, 0x20000
    for nw in (2, 4):
        assert lib.mh_sort_keys_noalloc(ctypes.c_void_p(a + 8), ctypes.c_void_p(b), 10, nw, 64, None) == mh.MH_EINVAL
        assert lib.mh_sort_keys_noalloc(ctypes.c_void_p(a), ctypes.c_void_p(b + 8), 10, nw, 64, None) == mh.MH_EINVAL
    assert lib.mh_sort_keys_noalloc(ctypes.c_void_p(a + 4), ctypes.c_void_p(b), 10, 1, 64, None) == mh.MH_EINVAL
    assert lib.mh_sort_keys_noalloc(ctypes.c_void_p(a), ctypes.c_void_p(b), 0, 2, 64, None) == mh.MH_OK


@pytest.mark.gpu
def test_noalloc_sort_rejects_oversize_and_bad_arguments():
    import torch

    import paper_1409_7208_gb300 as mh

    lib = mh.load_library()
    stream = torch.cuda.current_stream()
    limit_words = 1 << 21
    big = torch.zeros(limit_words + 2, dtype=torch.int64, device="cuda")
    out = torch.full_like(big, 7)
    assert _call(lib, big, out, (limit_words + 2) // 2, 2, 100, stream) == mh.MH_EOVERFLOW
    assert _call(lib, big, out, limit_words + 1, 1, 64, stream) == mh.MH_EOVERFLOW
    torch.cuda.synchronize()
    assert bool((out == 7).all()), "a rejected call must not write"
    assert _call(lib, big, out, 10, 3, 64, stream) == mh.MH_EINVAL
    assert _call(lib, big, out, 10, 1, 65, stream) == mh.MH_EINVAL
    assert _call(lib, big, big, 10, 1, 64, stream) == mh.MH_EINVAL
    # at the limit it works, and agrees with a plain sort of the same values
    vals = torch.randint(0, 1 << 62, (limit_words,), dtype=torch.int64, device="cuda")
    dst = torch.empty_like(vals)
    assert _call(lib, vals, dst, limit_words, 1, 62, stream) == mh.MH_OK
    torch.cuda.synchronize()
    assert torch.equal(dst, torch.sort(vals).values)
