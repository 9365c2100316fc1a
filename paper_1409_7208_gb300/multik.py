"""Multiple-k iteration over the C ABI: for k_1 < k_2 < ..., the reads of
step i are the input reads plus ``d`` copies of every contig of step i-1
(mh_pack_reads_contigs), then counting, mercy, the SdBG and the contigs of
step i (mh_walk_contigs with seed + i).  Host logic only: every step runs in
libmh's kernels.  The paper (Sec. 2, fourth paragraph; Sec. 3) iterates k
the same way with assembled contigs; here a contig is a seeded walk."""
from __future__ import annotations

from . import (Context, mh_build_sdbg, mh_count_kmers, mh_mercy_kmers, mh_pack_reads_contigs,
               mh_walk_contigs)


def iterate(ctx: Context, ascii, offs, ks, d: int = 2, n_walks: int = 1000, max_len: int = 10_000,
            seed: int = 3, keep: bool = False) -> list:
    """Run the iteration on device reads (uint8 ``ascii``, int64 ``offs``
    CUDA tensors).  Returns one dict per k: the handles when ``keep``, else
    their sizes."""
    steps = []
    contigs = None
    for i, k in enumerate(ks):
        reads = mh_pack_reads_contigs(ctx, ascii, offs, contigs, d)
        solid = mh_count_kmers(ctx, reads, k, d)
        mercy = mh_mercy_kmers(ctx, reads, solid)
        sdbg = mh_build_sdbg(ctx, solid, mercy)
        nxt = mh_walk_contigs(ctx, solid, mercy, n_walks, max_len, seed + i)
        if keep:
            steps.append({"k": k, "reads": reads, "solid": solid, "mercy": mercy, "sdbg": sdbg,
                          "contigs": nxt})
        else:
            sv, mv, gv, cv = solid.view(), mercy.view(), sdbg.view(), nxt.view()
            steps.append({"k": k, "n_kmers": sv.n_kmers, "solid": sv.n, "mercy": mv.n, "m": gv.m,
                          "contigs": cv.n, "contig_bases": cv.n_bases})
            for h in (sdbg, mercy, solid, reads):
                h.free()
        if contigs is not None and not keep:
            contigs.free()
        contigs = nxt
    return steps
