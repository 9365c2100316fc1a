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
// A warp runs one walk: each step finds, in each table, the entries whose
// k-prefix is the node (node.A .. node.T) from a bucket index over the top
// bits of the keys (about 16 keys a bucket): the lanes read the bucket in one
// load and a ballot gives the first entry >= node.A, so a step costs a few
// dependent loads.  Walks write into fixed slots of max_len bytes, compacted
// afterwards.
#include <algorithm>

#include "mh_internal.cuh"

namespace mh {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Top `bits` bits of a (k+1)-mer key (bits <= 2(k+1), bits <= 32).
template <int NW>
__device__ __forceinline__ uint64_t top_bits(const Key<NW>& x, int K1, int bits) {
    return key_shr<NW>(x, 2 * K1 - bits).w[0];
}

// off[b] = first entry of the sorted table whose top bits are >= b, for
// b = 0 .. 2^bits (thread per entry; each boundary written by one thread).
template <int NW>
__global__ void table_index_kernel(const uint64_t* __restrict__ T, uint64_t n, int K1, int bits,
                                   uint64_t* __restrict__ off) {
    const uint64_t nb = 1ull << bits;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = top_bits<NW>(load_key<NW>(T, i), K1, bits);
        const uint64_t b0 = i == 0 ? 0 : top_bits<NW>(load_key<NW>(T, i - 1), K1, bits) + 1;
        for (uint64_t x = b0; x <= b; x++) off[x] = i;
        if (i == n - 1)
            for (uint64_t x = b + 1; x <= nb; x++) off[x] = n;
    }
}

// Labels (bit c for label c) of the out-edges of node v in both tables at
// once: half-warp 0 searches the solid table, half-warp 1 the mercy table,
// each within [lo, hi), the bucket of v.A in its own table.  A half reads
// the bucket 16 entries at a time and finds the first entry >= v.A by a
// ballot (the bucket's end if none); its lanes 0..3 then read the entries
// from there (into the next bucket when the index covers the label's bits,
// for tiny k).  Every lane gets the union of both masks.
template <int NW>
__device__ __forceinline__ uint32_t out_labels(const uint64_t* __restrict__ T, uint64_t n, uint64_t lo, uint64_t hi,
                                               const Key<NW>& v, int lane) {
    const int half = lane >> 4, hl = lane & 15;
    const Key<NW> q = key_shl<NW>(v, 2);
    uint64_t pos = hi, base = lo;
    bool done = base >= hi;
    while (__ballot_sync(0xFFFFFFFFu, !done)) {
        const uint64_t i = base + hl;
        const bool ge = !done && i < hi && !key_less<NW>(load_key<NW>(T, i), q);
        const uint32_t m = (__ballot_sync(0xFFFFFFFFu, ge) >> (16 * half)) & 0xFFFFu;
        if (!done) {
            if (m) {
                pos = base + __ffs(m) - 1;
                done = true;
            } else {
                base += 16;
                done = base >= hi;
            }
        }
    }
    bool hit = false;
    uint32_t label = 0;
    if (hl < 4 && pos + hl < n) {
        const Key<NW> e = load_key<NW>(T, pos + hl);
        hit = key_eq<NW>(key_shr<NW>(e, 2), v);
        label = (uint32_t)(e.w[0] & 3u);
    }
    // entries of prefix v are consecutive from pos: lane l counts if lanes 0..l of its half all match
    const uint32_t hm = (__ballot_sync(0xFFFFFFFFu, hit) >> (16 * half)) & 0xFu;
    const uint32_t run = __ffs(~hm) - 1;  // matching entries from pos (at most 4)
    uint32_t mask = (hl < (int)run) ? (1u << label) : 0u;
    for (int o = 16; o; o >>= 1) mask |= __shfl_xor_sync(0xFFFFFFFFu, mask, o);
    return mask;
}

// One warp per walk (the searches of a step are warp-wide).  The bucket of
// the next step's node does not depend on the label the step picks when the
// index's bits stop short of the last two symbols (2 K1 - bits >= 4): its
// bounds are then loaded one step ahead, while this step searches, so that
// a step waits for one memory access (the bucket) instead of two.
template <int NW>
__global__ void walk_kernel(const uint64_t* __restrict__ S, uint64_t nS, const uint64_t* __restrict__ offS,
                            const uint64_t* __restrict__ M, uint64_t nM, const uint64_t* __restrict__ offM,
                            int bits, int k, uint64_t n_walks, uint32_t max_len, uint64_t seed,
                            uint8_t* __restrict__ slots, uint64_t* __restrict__ lens,
                            unsigned long long* __restrict__ next_walk) {
    const int K1 = k + 1;
    const int lane = threadIdx.x & 31;
    const uint64_t E = nS + nM;
    // this lane's half-warp searches one table
    const bool mer = (lane >> 4) != 0;
    const uint64_t* T = mer ? M : S;
    const uint64_t n = mer ? nM : nS;
    const uint64_t* off = mer ? offM : offS;
    const bool ahead = 2 * K1 - bits >= 4;
    // bounds of the bucket of node v's query v.A
    auto bucket = [&](const Key<NW>& v, uint64_t& lo, uint64_t& hi) {
        lo = hi = 0;
        if (n) {
            const uint64_t b = top_bits<NW>(key_shl<NW>(v, 2), K1, bits);
            lo = off[b];
            hi = off[b + 1];
        }
    };
    // walks are taken one at a time from a counter: walks differ in length
    // (a dead end ends one early), and a warp that finishes takes the next
    for (;;) {
        uint64_t w = 0;
        if (lane == 0) w = atomicAdd(next_walk, 1ull);
        w = __shfl_sync(0xFFFFFFFFu, w, 0);
        if (w >= n_walks) break;
        uint8_t* out = slots + w * max_len;
        const uint64_t s = splitmix64_at(seed, w << 24) % E;
        Key<NW> x = s < nS ? load_key<NW>(S, s) : load_key<NW>(M, s - nS);
        for (int i = lane; i < K1; i += 32) out[i] = "ACGT"[key_sym<NW>(x, K1, i)];
        uint32_t len = K1;
        Key<NW> v = key_low<NW>(x, 2 * k);
        uint64_t lo, hi;
        bucket(v, lo, hi);
        for (uint32_t j = 1; len < max_len; j++) {
            // the next node's bucket, for any label (when `ahead`)
            uint64_t nlo = 0, nhi = 0;
            if (ahead) bucket(key_low<NW>(key_shl<NW>(v, 2), 2 * k), nlo, nhi);
            const uint32_t mask = out_labels<NW>(T, n, lo, hi, v, lane);
            if (!mask) break;
            uint32_t r = (uint32_t)(splitmix64_at(seed, (w << 24) + j) % (uint64_t)__popc(mask));
            uint32_t m = mask;
            while (r--) m &= m - 1;
            const uint32_t c = __ffs(m) - 1;
            x = key_shl<NW>(v, 2);
            x.w[0] |= c;
            if (lane == 0) out[len] = "ACGT"[c];
            len++;
            v = key_low<NW>(x, 2 * k);
            if (ahead) {
                lo = nlo;
                hi = nhi;
            } else {
                bucket(v, lo, hi);
            }
        }
        if (lane == 0) lens[w] = len;
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
    // bucket indexes over the top bits: about 16 entries a bucket
    int bits = 1;
    while (bits < 32 && bits < 2 * (k + 1) && (2ull << bits) * 16 <= std::max(nS, nM)) bits++;
    Buf<uint64_t> offS(ctx, (1ull << bits) + 1), offM(ctx, (1ull << bits) + 1);
    offS.zero();
    offM.zero();
    if (n_walks) {
        if (nS)
            MH_LAUNCH(ctx, "walk_index", grid_for(ctx, nS, 256), 256, 0, table_index_kernel<NW>, solid->keys, nS,
                      k + 1, bits, offS.p);
        if (nM)
            MH_LAUNCH(ctx, "walk_index", grid_for(ctx, nM, 256), 256, 0, table_index_kernel<NW>, mercy->keys, nM,
                      k + 1, bits, offM.p);
        Buf<uint64_t> next_walk(ctx, 1);
        next_walk.zero();
        MH_LAUNCH(ctx, "walk", grid_for(ctx, n_walks * 32, 256, 8), 256, 0, walk_kernel<NW>, solid->keys, nS, offS.p,
                  mercy ? mercy->keys : nullptr, nM, offM.p, bits, k, n_walks, max_len, seed, slots.p, lens.p,
                  (unsigned long long*)next_walk.p);
    }
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
