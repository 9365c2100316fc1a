// Contigs for the next k of a multiple-k iteration (the paper, Sec. 2 fourth
// paragraph and Sec. 3, builds the graph for a list of increasing k and carries
// the previous k's contigs into the next graph).  Graph cleaning and contig
// assembly are not part of this library, so a contig here is a random walk of
// the graph E = solid + mercy:
//
//   walk w   counter-based random values r(w, j) = SplitMix64 output number
//            (w << 24) + j of the stream seeded with `seed` (Steele, Lea &
//            Flood 2014: state advanced by 0x9E3779B97F4A7C15, then two
//            xor-shift-multiply rounds);
//            start edge: index r(w, 0) mod |E| of solid followed by mercy
//            (each ascending), the contig is its k+1 symbols;
//            step j = 1, 2, ...: the node is the contig's last k symbols;
//            its out-edges are the edges of E with that k-prefix, taken in
//            label order; with none the walk stops (dead end), otherwise it
//            appends the label of out-edge r(w, j) mod (their number); it
//            also stops at max_len symbols.
//
// A thread runs one walk: each step is one lower-bound search per table
// (node.A) and a look at the next 4 entries, so the walk needs no index
// beyond the sorted tables.  Walks write into fixed slots of max_len bytes,
// compacted afterwards.
#include "mh_internal.cuh"

namespace mh {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Labels (bit c for label c) of the entries of a sorted table with k-prefix v.
template <int NW>
__device__ __forceinline__ uint32_t out_labels(const uint64_t* __restrict__ T, uint64_t n, const Key<NW>& v) {
    if (!n) return 0;
    const Key<NW> q = key_shl<NW>(v, 2);
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (key_less<NW>(load_key<NW>(T, mid), q)) lo = mid + 1; else hi = mid;
    }
    uint32_t mask = 0;
    for (uint64_t i = lo; i < lo + 4 && i < n; i++) {
        const Key<NW> e = load_key<NW>(T, i);
        if (!key_eq<NW>(key_shr<NW>(e, 2), v)) break;
        mask |= 1u << (uint32_t)(e.w[0] & 3u);
    }
    return mask;
}

template <int NW>
__global__ void walk_kernel(const uint64_t* __restrict__ S, uint64_t nS, const uint64_t* __restrict__ M, uint64_t nM,
                            int k, uint64_t n_walks, uint32_t max_len, uint64_t seed, uint8_t* __restrict__ slots,
                            uint64_t* __restrict__ lens) {
    const int K1 = k + 1;
    const uint64_t E = nS + nM;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < n_walks;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t* out = slots + w * max_len;
        const uint64_t s = splitmix64_at(seed, w << 24) % E;
        Key<NW> x = s < nS ? load_key<NW>(S, s) : load_key<NW>(M, s - nS);
        for (int i = 0; i < K1; i++) out[i] = "ACGT"[key_sym<NW>(x, K1, i)];
        uint32_t len = K1;
        for (uint32_t j = 1; len < max_len; j++) {
            const Key<NW> v = key_low<NW>(x, 2 * k);
            const uint32_t mask = out_labels<NW>(S, nS, v) | out_labels<NW>(M, nM, v);
            if (!mask) break;
            uint32_t r = (uint32_t)(splitmix64_at(seed, (w << 24) + j) % (uint64_t)__popc(mask));
            uint32_t m = mask;
            while (r--) m &= m - 1;
            const uint32_t c = __ffs(m) - 1;
            x = key_shl<NW>(v, 2);
            x.w[0] |= c;
            out[len++] = "ACGT"[c];
        }
        lens[w] = len;
    }
}

// contig w: lens[w] bytes from its slot to off[w]
__global__ void contig_compact_kernel(const uint8_t* __restrict__ slots, uint32_t max_len,
                                      const uint64_t* __restrict__ off, uint8_t* __restrict__ ascii) {
    const uint64_t w = blockIdx.x;
    const uint64_t o = off[w], len = off[w + 1] - o;
    for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) ascii[o + i] = slots[w * max_len + i];
}

template <int NW>
void walk_contigs(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, uint64_t n_walks, uint32_t max_len,
                  uint64_t seed, mh_contigs* out) {
    const int k = solid->k;
    const uint64_t nS = solid->n, nM = mercy ? mercy->n : 0;
    if (nS + nM == 0) n_walks = 0;
    Buf<uint8_t> slots(ctx, n_walks * max_len);
    Buf<uint64_t> lens(ctx, n_walks + 1), off(ctx, n_walks + 1);
    if (n_walks)
        MH_LAUNCH(ctx, "walk", grid_for(ctx, n_walks, 128), 128, 0, walk_kernel<NW>, solid->keys, nS,
                  mercy ? mercy->keys : nullptr, nM, k, n_walks, max_len, seed, slots.p, lens.p);
    exclusive_scan_u64(ctx, lens.p, off.p, n_walks);
    uint64_t total = 0;
    read_u64(ctx, off.p + n_walks, &total, 1);
    Buf<uint8_t> ascii(ctx, total + 16);
    if (n_walks)
        MH_LAUNCH(ctx, "contig_compact", (unsigned)n_walks, 256, 0, contig_compact_kernel, slots.p, max_len, off.p,
                  ascii.p);
    sync_and_check(ctx);
    out->k = k;
    out->n = n_walks;
    out->n_bases = total;
    out->ascii = ascii.release();
    out->offs = off.release();
}

template void walk_contigs<1>(mh_ctx*, const mh_kmers*, const mh_kmers*, uint64_t, uint32_t, uint64_t, mh_contigs*);
template void walk_contigs<2>(mh_ctx*, const mh_kmers*, const mh_kmers*, uint64_t, uint32_t, uint64_t, mh_contigs*);
template void walk_contigs<4>(mh_ctx*, const mh_kmers*, const mh_kmers*, uint64_t, uint32_t, uint64_t, mh_contigs*);

// ------------------------------------------------ reads plus contig copies
// out_ascii = reads, then `copies` copies of every contig (copy c of contig i
// is read n_reads + i * copies + c); out_offs the matching offsets.
__global__ void append_offs_kernel(const uint64_t* __restrict__ coffs, uint64_t n_contigs, uint32_t copies,
                                   uint64_t n_reads, uint64_t n_bases, uint64_t* __restrict__ out_offs) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= n_contigs * copies;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v;
        if (r == n_contigs * copies) {
            v = n_bases + coffs[n_contigs] * copies;
        } else {
            const uint64_t i = r / copies, c = r % copies;
            v = n_bases + coffs[i] * copies + c * (coffs[i + 1] - coffs[i]);
        }
        out_offs[n_reads + r] = v;
    }
}

__global__ void append_ascii_kernel(const uint8_t* __restrict__ cascii, const uint64_t* __restrict__ coffs,
                                    uint64_t n_contigs, uint32_t copies, uint64_t n_bases,
                                    uint8_t* __restrict__ out_ascii) {
    // block per contig
    for (uint64_t i = blockIdx.x; i < n_contigs; i += gridDim.x) {
        const uint64_t b = coffs[i], len = coffs[i + 1] - b;
        for (uint32_t c = 0; c < copies; c++) {
            uint8_t* dst = out_ascii + n_bases + b * copies + c * len;
            for (uint64_t j = threadIdx.x; j < len; j += blockDim.x) dst[j] = cascii[b + j];
        }
    }
}

void pack_reads(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs, uint64_t n_reads,
                mh_reads* out);

void pack_with_contigs(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs,
                       uint64_t n_reads, const mh_contigs* contigs, uint32_t copies, mh_reads* out) {
    const uint64_t nc = contigs ? contigs->n : 0;
    const uint64_t extra = contigs ? contigs->n_bases * copies : 0;
    const uint64_t N = n_bases + extra, R = n_reads + nc * copies;
    Buf<uint8_t> a(ctx, N + 16);
    Buf<uint64_t> o(ctx, R + 1);
    if (n_bases) MH_CUDA(cudaMemcpyAsync(a.p, d_ascii, n_bases, cudaMemcpyDeviceToDevice, ctx->stream));
    MH_CUDA(cudaMemcpyAsync(o.p, d_offs, sizeof(uint64_t) * (n_reads + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    if (nc && copies) {
        MH_LAUNCH(ctx, "append_offs", grid_for(ctx, nc * copies + 1, 256), 256, 0, append_offs_kernel, contigs->offs,
                  nc, copies, n_reads, n_bases, o.p);
        MH_LAUNCH(ctx, "append_ascii", (unsigned)std::min<uint64_t>(nc, (uint64_t)ctx->num_sms * 16), 256, 0,
                  append_ascii_kernel, contigs->ascii, contigs->offs, nc, copies, n_bases, a.p);
    }
    pack_reads(ctx, a.p, N, o.p, R, out);
}

}  // namespace mh
