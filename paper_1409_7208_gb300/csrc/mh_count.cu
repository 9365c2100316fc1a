// mh_count_kmers: every (k+1)-mer on both strands, sorted and counted; the
// solid ones (count >= d) are kept (paper, Sec. 2, third paragraph).
//
// A window x and its reverse complement rc(x) always occur together in the
// both-strand multiset, so the library sorts one canonical key min(x, rc x)
// per window (half the keys of the literal multiset) and recovers the literal
// counts exactly: cnt(x) = cnt(rc x) = run length of canonical(x), doubled
// when x = rc(x) (a palindrome, counted twice per occurrence).
//
//   extract   fragments in groups of 32 a warp (a lane per short fragment,
//             its keys rolled on; a long one by the whole warp), window
//             keys from the packed words, canonical, stored as mix_key
//             images (their top bits evenly spread)
//   sort      8-bit LSD passes over the top bits only: 3 passes (24 bits)
//             leave every unit of keys sharing them contiguous.  From 2^22
//             keys on, the extraction makes the first pass itself: it
//             writes each tile's keys by digit into fixed-size segments,
//             and the next pass reads the segments (extract_scatter_kernel)
//   units     each unit sorted and run-length counted on chip by one warp,
//             the solid filter applied, both strands out (mh_group.cu)
//   sort      the solid table by the key-value spread sort, ascending
// The spread route (a plan's alternative): passes over the top ceil(log2 n)
// bits, a fix-up of keys sharing them, a run pass (runs_kernel: run heads
// in a shared-memory bitmask, run lengths from the next head, the solid
// filter, outputs placed by decoupled look-back), the expansion to both
// strands and the same key-value sort.  Read sets too large for device
// memory are counted in buckets of the mixed keys' top bits.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "mh_sort_kernels.cuh"

namespace mh {

// n windows of fragment f = max(0, L - k)
__global__ void frag_windows_kernel(const uint64_t* __restrict__ frag_offs, uint64_t n_frags, int k,
                                    uint64_t* __restrict__ nwin) {
    for (uint64_t f = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; f < n_frags;
         f += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t L = frag_offs[f + 1] - frag_offs[f];
        nwin[f] = L > (uint64_t)k ? L - k : 0;
    }
}

// Fragments of at most this many windows are extracted by one lane.
constexpr int kLaneWindows = 48;

// Canonical key of every window of every fragment, window i of fragment f
// written at woff[f] + i (MIXED: as its mix_key image).  With `hist` (1-word
// keys), the block also counts the digits the sort's passes will use
// (n_passes digits of rb bits from bit shift0; in dynamic shared memory,
// added to hist at the end), so the sort needs no histogram pass of its own.
template <int NW, bool MIXED>
__global__ void __launch_bounds__(256) extract_canonical_kernel(const uint32_t* __restrict__ packed,
                                                                const uint64_t* __restrict__ frag_offs,
                                                                const uint64_t* __restrict__ woff, uint64_t n_frags,
                                                                int k, uint64_t* __restrict__ out,
                                                                uint32_t* __restrict__ hist, int shift0,
                                                                int n_passes, int rb) {
    extern __shared__ uint32_t sh[];
    const int nbins = n_passes << rb;
    const uint32_t dmask = (1u << rb) - 1u;
    if (hist) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1;
    // the canonical key of window `at` (forward key x, reverse complement r)
    auto put = [&](uint64_t at, const Key<NW>& x, const Key<NW>& r) {
        Key<NW> c = key_less<NW>(r, x) ? r : x;
        if constexpr (MIXED) c = mix_key<NW>(c);
        store_key<NW>(out, at, c);
        if constexpr (NW == 1) {
            if (hist)
                for (int p = 0; p < n_passes; p++)
                    atomicAdd(&sh[(p << rb) + ((uint32_t)(c.w[0] >> (shift0 + rb * p)) & dmask)], 1u);
        }
    };
    // fragments in groups of 32 a warp: a fragment of at most kLaneWindows
    // windows is taken by one lane, which assembles its first key and its
    // reverse complement and rolls both on by one symbol a window (short
    // reads at a large k leave most lanes of a warp per fragment idle);
    // longer fragments are then taken by the whole warp, a window a lane
    for (uint64_t g = warp; g * 32 < n_frags; g += n_warps) {
        const uint64_t f = g * 32 + lane;
        uint64_t b = 0, w0 = 0, nw = 0;
        if (f < n_frags) {
            b = frag_offs[f];
            w0 = woff[f];
            nw = woff[f + 1] - w0;
        }
        const bool alone = nw <= (uint64_t)kLaneWindows;
        if (alone && nw) {
            Key<NW> x = load_window<NW>(packed, b, K1);
            Key<NW> r = key_rc<NW>(x, K1);
            for (uint64_t i = 0;;) {
                put(w0 + i, x, r);
                if (++i >= nw) break;
                roll_window<NW>(x, r, packed_sym(packed, b + i + K1 - 1), K1);
            }
        }
        uint32_t big = __ballot_sync(0xFFFFFFFFu, !alone);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint64_t fb = __shfl_sync(0xFFFFFFFFu, b, src);
            const uint64_t fw0 = __shfl_sync(0xFFFFFFFFu, w0, src);
            const uint64_t fnw = __shfl_sync(0xFFFFFFFFu, nw, src);
            for (uint64_t i = lane; i < fnw; i += 32) {
                const Key<NW> x = load_window<NW>(packed, fb + i, K1);
                put(fw0 + i, x, key_rc<NW>(x, K1));
            }
        }
    }
    if (hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

// Extraction fused with the first scatter pass of the unit counting (1-word
// keys, as mix_key images).  A CTA takes tiles of 256 * ITEMS consecutive
// windows in turn; a thread computes the keys of ITEMS consecutive windows
// (the first assembled from the packed words, the others rolled on by one
// symbol while they stay in one fragment), counts them by the pass's
// digit (bits [shift, shift + 8)) in its warp's histogram and by the next
// n_hist passes' digits in the CTA's histogram (added to hist at the end),
// ranks and stages them in digit order as the scatter pass does, and writes
// each digit's run to that digit's segment of `out`: segment d is the cap
// slots from d * cap, and the run's place in it comes from one atomic add
// on cursor[d] per tile and digit.  The keys of one segment land in no
// fixed order; they are keys alone, and the later stable passes and the
// unit sort bring equal keys together whatever that order is.  The digits
// of mix_key images are close to uniform, so cap is the mean count of a
// digit with a margin; a run that does not fit is not written and
// cursor[256] is set, and the caller then takes the unfused path.
constexpr int kXsTileMax = kSortThreads * 16;

// tfrag[t] = the fragment holding window t * tile (t < n_tiles) or the last
// window (t = n_tiles): the largest f < F with woff[f] <= that window.
__global__ void tile_frag_kernel(const uint64_t* __restrict__ woff, uint64_t F, uint64_t n, uint64_t tile,
                                 uint64_t n_tiles, uint64_t* __restrict__ tfrag) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= n_tiles;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w = t < n_tiles ? t * tile : n - 1;
        uint64_t lo = 0, hi = F - 1;
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo + 1) / 2;
            if (woff[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        tfrag[t] = lo;
    }
}

template <int ITEMS, int MINB>
__global__ void __launch_bounds__(kSortThreads, MINB)
    extract_scatter_kernel(const uint32_t* __restrict__ packed, const uint64_t* __restrict__ frag_offs,
                           const uint64_t* __restrict__ woff, const uint64_t* __restrict__ tfrag, uint64_t n, int k,
                           int shift, int n_hist, uint64_t cap, uint64_t* __restrict__ out,
                           unsigned long long* __restrict__ cursor, uint32_t* __restrict__ hist) {
    constexpr int TILE = kSortThreads * ITEMS;
    __shared__ uint32_t warp_hist[kSortWarps * 256];
    __shared__ uint32_t ghist[3 * 256];
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint64_t scatter_base[256];
    __shared__ uint64_t stage[TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K1 = k + 1;
    const uint32_t lt_mask = (1u << lane) - 1;
    for (int i = tid; i < 3 * 256; i += kSortThreads) ghist[i] = 0;
    const uint64_t n_tiles = ceil_div(n, TILE);
    uint32_t* wh = warp_hist + warp * 256;
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        // (the barrier also ends the previous tile's write-out)
        for (int i = tid; i < kSortWarps * 256; i += kSortThreads) warp_hist[i] = 0;
        __syncthreads();
        const uint64_t tb = t * TILE;
        const uint32_t tile_n = n - tb < (uint64_t)TILE ? (uint32_t)(n - tb) : (uint32_t)TILE;
        const uint32_t q0 = (uint32_t)tid * ITEMS;
        uint64_t key[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; i++) key[i] = 0;
        if (q0 < tile_n) {
            const uint64_t w = tb + q0;
            uint64_t lo = tfrag[t], hi = tfrag[t + 1];
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo + 1) / 2;
                if (woff[mid] <= w) lo = mid;
                else hi = mid - 1;
            }
            uint64_t f = lo, wend = woff[f + 1];
            uint64_t pos = frag_offs[f] + (w - woff[f]);
            Key<1> x = load_window<1>(packed, pos, K1);
            Key<1> r = key_rc<1>(x, K1);
#pragma unroll
            for (int i = 0; i < ITEMS; i++) {
                if (i > 0) {
                    if (q0 + i >= tile_n) break;
                    if (w + i == wend) {
                        // the next fragment with windows (empty ones skipped)
                        do {
                            f++;
                        } while (woff[f + 1] == wend);
                        wend = woff[f + 1];
                        pos = frag_offs[f];
                        x = load_window<1>(packed, pos, K1);
                        r = key_rc<1>(x, K1);
                    } else {
                        pos++;
                        roll_window<1>(x, r, packed_sym(packed, pos + K1 - 1), K1);
                    }
                }
                key[i] = mix_key<1>(key_less<1>(r, x) ? r : x).w[0];
            }
        }
        // counts: the pass's digit per warp, the later passes' per CTA
#pragma unroll
        for (int i = 0; i < ITEMS; i++)
            if (q0 + i < tile_n) {
                atomicAdd(&wh[(uint32_t)(key[i] >> shift) & 255u], 1u);
                for (int h = 0; h < n_hist; h++)
                    atomicAdd(&ghist[h * 256 + ((uint32_t)(key[i] >> (shift + 8 + 8 * h)) & 255u)], 1u);
            }
        __syncthreads();
        const int d = tid;  // kSortThreads == 256
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = warp_hist[w * 256 + d];
            warp_hist[w * 256 + d] = cnt;
            cnt += c;
        }
        // the digit's places in its segment (awaited only after the ranking)
        const unsigned long long at = cnt ? atomicAdd(&cursor[d], (unsigned long long)cnt) : 0ull;
        uint32_t start;
        {
            uint32_t x = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            uint32_t wpre = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; w++) wpre += w < warp ? wsum[w] : 0u;
            start = wpre + x - cnt;
        }
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) warp_hist[w * 256 + d] += start;
        __syncthreads();
        // rank and stage in tile digit order (as the scatter pass does)
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            const bool valid = q0 + i < tile_n;
            const uint32_t dg = (uint32_t)(key[i] >> shift) & 255u;
            const uint32_t peers = digit_peers(dg) & (__ballot_sync(0xFFFFFFFFu, valid) | (1u << lane));
            const int leader = __ffs(peers) - 1;
            uint32_t slot = 0;
            if (lane == leader && valid) slot = atomicAdd(&wh[dg], (uint32_t)__popc(peers));
            slot = __shfl_sync(0xFFFFFFFFu, slot, leader) + (uint32_t)__popc(peers & lt_mask);
            if (valid) stage[slot] = key[i];
        }
        const bool fits = at + cnt <= cap;
        scatter_base[d] = fits ? (uint64_t)d * cap + at - start : ~0ull;
        if (!fits) cursor[256] = 1ull;
        __syncthreads();
        // write out: consecutive staged keys of one digit to consecutive slots
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            const uint32_t j = tid + i * kSortThreads;
            if (j < tile_n) {
                const uint64_t kk = stage[j];
                const uint64_t b = scatter_base[(uint32_t)(kk >> shift) & 255u];
                if (b != ~0ull) out[b + j] = kk;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < n_hist * 256; i += kSortThreads)
        if (ghist[i]) atomicAdd(&hist[i], ghist[i]);
}

// Buckets of the mixed canonical keys: the top `bb` bits of the top word.
template <int NW>
__device__ __forceinline__ uint32_t key_bucket(const Key<NW>& m, int bb) {
    return bb ? (uint32_t)(m.w[NW - 1] >> (64 - bb)) : 0u;
}

// Bucketed extraction: fragments in tasks of kTaskFrags, a warp per task.
// A first pass computes every window's bucket (one byte a window, at its
// window index) and counts the windows of every (bucket, task).  After a
// scan of each bucket's row, a bucket's pass reads the bytes, queues the
// positions of its own windows in shared memory and computes keys for full
// warps of them only, writing them at exact offsets, in task order, without
// atomics.
constexpr int kTaskFrags = 64;

template <int NW>
__global__ void __launch_bounds__(256) task_hist_kernel(const uint32_t* __restrict__ packed,
                                                        const uint64_t* __restrict__ frag_offs,
                                                        const uint64_t* __restrict__ woff, uint64_t n_frags, int k,
                                                        int bb, uint64_t n_tasks, uint8_t* __restrict__ ids,
                                                        uint32_t* __restrict__ cnt) {
    __shared__ uint32_t h[8][64];  // per warp, up to 64 buckets
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1, nb = 1 << bb;
    for (uint64_t t = warp; t < n_tasks; t += n_warps) {
        for (int i = lane; i < nb; i += 32) h[wib][i] = 0;
        __syncwarp();
        const uint64_t f1 = (t + 1) * kTaskFrags < n_frags ? (t + 1) * kTaskFrags : n_frags;
        for (uint64_t f = t * kTaskFrags; f < f1; f++) {
            const uint64_t b = frag_offs[f], L = frag_offs[f + 1] - b, w0 = woff[f];
            const uint64_t nwin = L > (uint64_t)k ? L - k : 0;
            for (uint64_t i = lane; i < nwin; i += 32) {
                const Key<NW> x = load_window<NW>(packed, b + i, K1);
                const Key<NW> r = key_rc<NW>(x, K1);
                const uint32_t bk = key_bucket<NW>(mix_key<NW>(key_less<NW>(r, x) ? r : x), bb);
                ids[w0 + i] = (uint8_t)bk;
                atomicAdd(&h[wib][bk], 1u);
            }
        }
        __syncwarp();
        for (int i = lane; i < nb; i += 32) cnt[(uint64_t)i * n_tasks + t] = h[wib][i];
        __syncwarp();
    }
}

// The mixed canonical keys of bucket `bk`, task t's at off[t] onwards.  A
// warp reads its task's bucket bytes 16 a lane (the task's windows are
// contiguous), queues the window numbers of its bucket in shared memory and
// computes keys 32 at a time: each lane finds its window's fragment by a
// binary search over the task's fragment table, held in two registers a
// lane and read by shuffles.
constexpr int kQueue = 512 + 32;

template <int NW>
__global__ void __launch_bounds__(256) extract_bucket_kernel(const uint32_t* __restrict__ packed,
                                                             const uint64_t* __restrict__ frag_offs,
                                                             const uint64_t* __restrict__ woff,
                                                             const uint8_t* __restrict__ ids, uint64_t n_frags, int k,
                                                             uint32_t bk, uint64_t n_tasks,
                                                             const uint64_t* __restrict__ off,
                                                             uint64_t* __restrict__ out) {
    __shared__ uint64_t q[8][kQueue];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint64_t* qw = q[wib];
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1;
    const uint32_t bk4 = bk * 0x01010101u;
    for (uint64_t t = warp; t < n_tasks; t += n_warps) {
        const uint64_t f0 = t * kTaskFrags;
        const int nf = (int)((f0 + kTaskFrags < n_frags ? f0 + kTaskFrags : n_frags) - f0);
        // fragment j of the task: window offset and base, lane j % 32, register j / 32
        const uint64_t wA = lane < nf ? woff[f0 + lane] : ~0ull;
        const uint64_t wB = 32 + lane < nf ? woff[f0 + 32 + lane] : ~0ull;
        const uint64_t bA = lane < nf ? frag_offs[f0 + lane] : 0;
        const uint64_t bB = 32 + lane < nf ? frag_offs[f0 + 32 + lane] : 0;
        auto pick = [&](uint64_t ra, uint64_t rb, int j) {
            const uint64_t x = __shfl_sync(0xFFFFFFFFu, ra, j & 31);
            const uint64_t y = __shfl_sync(0xFFFFFFFFu, rb, j & 31);
            return j < 32 ? x : y;
        };
        const uint64_t W0 = woff[f0], W1 = woff[f0 + nf];
        // position in the packed stream of task window w (every lane at once)
        auto position = [&](uint64_t w) {
            int lo = 0;
            for (int step = 32; step; step >>= 1) {
                const int c = lo + step;
                const uint64_t wc = pick(wA, wB, c < nf ? c : nf - 1);
                if (c < nf && wc <= w) lo = c;
            }
            return pick(bA, bB, lo) + (w - pick(wA, wB, lo));
        };
        auto key_at = [&](uint64_t p) {
            const Key<NW> x = load_window<NW>(packed, p, K1);
            const Key<NW> r = key_rc<NW>(x, K1);
            return mix_key<NW>(key_less<NW>(r, x) ? r : x);
        };
        uint64_t at = off[t];
        int qn = 0;
        for (uint64_t g = W0 / 16; g * 16 < W1; g += 32) {
            const uint64_t gl = g + lane, w = gl * 16;
            uint32_t mask = 0;
            if (w < W1) {
                const uint4 v = *reinterpret_cast<const uint4*>(ids + w);
                const uint32_t e[4] = {v.x ^ bk4, v.y ^ bk4, v.z ^ bk4, v.w ^ bk4};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    // zero bytes of e[j]: windows of bucket bk
                    const uint32_t z = __vcmpeq4(e[j], 0u);
                    mask |= ((z & 1u) | ((z >> 7) & 2u) | ((z >> 14) & 4u) | ((z >> 21) & 8u)) << (4 * j);
                }
                const uint64_t lo = W0 > w ? W0 - w : 0, hi = W1 - w < 16 ? W1 - w : 16;
                mask &= (hi >= 16 ? 0xFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
            }
            const int c = __popc(mask);
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += y;
            }
            const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            int o = qn + incl - c;
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                qw[o++] = w + j;
            }
            qn += total;
            __syncwarp();
            int h = 0;
            for (; qn - h >= 32; h += 32) {
                const uint64_t p = position(qw[h + lane]);
                store_key<NW>(out, at + lane, key_at(p));
                at += 32;
            }
            if (h) {
                const int rem = qn - h;
                const uint64_t v = lane < rem ? qw[h + lane] : 0;
                __syncwarp();
                if (lane < rem) qw[lane] = v;
                qn = rem;
            }
            __syncwarp();
        }
        // the last, partial warp of positions
        const uint64_t p = position(lane < qn ? qw[lane] : W0);
        if (lane < qn) store_key<NW>(out, at + lane, key_at(p));
        __syncwarp();
    }
}

// ---------------------------------------------------------------- runs
// Run-length counting of a sorted key array in one read: a tile of keys is
// loaded to shared memory, run heads (key differs from its predecessor) are
// marked in a bitmask, each run's end is the next head (in the tile, or the
// first head of a later tile for the tile's last run), and the kept runs'
// outputs go to the tile's own slot of the output buffer (no dependence
// between tiles); a scan of the per-tile counts and a copy compact them.

constexpr int kRunThreads = 256;
constexpr int kRunItems = 8;
constexpr int kRunTile = kRunThreads * kRunItems;  // keys per tile
constexpr int kRunTilePad = kRunTile + kRunTile / 16;
__device__ __forceinline__ uint32_t rp(uint32_t i) { return i + (i >> 4); }
constexpr uint64_t kNoHead = ~0ull;

// first[t] = index of the first run head in tile t, or kNoHead (warp per tile).
template <int NW>
__global__ void run_first_head_kernel(const uint64_t* __restrict__ s, uint64_t n, uint64_t n_tiles,
                                      uint64_t* __restrict__ first) {
    const int lane = threadIdx.x & 31;
    for (uint64_t t = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; t < n_tiles;
         t += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        const uint64_t start = t * kRunTile, end = start + kRunTile < n ? start + kRunTile : n;
        uint64_t f = kNoHead;
        for (uint64_t base = start; base < end; base += 32) {
            const uint64_t i = base + lane;
            bool head = false;
            if (i < end) head = i == 0 || !key_eq<NW>(load_key<NW>(s, i), load_key<NW>(s, i - 1));
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, head);
            if (m) {
                f = base + __ffs(m) - 1;
                break;
            }
        }
        if (lane == 0) first[t] = f;
    }
}

// next[t] = first head after tile t (in tiles t+1, t+2, ...), or n.
__global__ void run_next_head_kernel(const uint64_t* __restrict__ first, uint64_t n_tiles, uint64_t n,
                                     uint64_t* __restrict__ next) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_tiles;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u = t + 1;
        while (u < n_tiles && first[u] == kNoHead) u++;
        next[t] = u < n_tiles ? first[u] : n;
    }
}

// Run length of x in the spectrum (distinct canonical keys, ascending, as
// mix_key images when spec_mixed, with the length of each key's run), or 0;
// the search starts from `hint`, left at the answer: a thread's queries
// ascend, so each search starts near the previous one.
template <int NW>
__device__ __forceinline__ uint64_t spectrum_count(const uint64_t* __restrict__ spec,
                                                   const uint32_t* __restrict__ spec_len, uint64_t n_spec, Key<NW> x,
                                                   bool spec_mixed, uint64_t& hint) {
    if (spec_mixed) x = mix_key<NW>(x);
    const uint64_t lb = gallop_lb<NW>(spec, n_spec, x, hint);
    hint = lb;
    if (lb >= n_spec || !key_eq<NW>(load_key<NW>(spec, lb), x)) return 0;
    return spec_len[lb];
}

// Counting mode (spec == nullptr): a run of length len is the canonical key
// of len windows; its literal count is len, doubled for a palindrome; it is
// kept if the count is >= d.  Lookup mode: every run is kept and its count
// is looked up in the spectrum.  A kept run outputs the key and, unless it is
// a palindrome, its reverse complement, both with the count.
//
// The tile's run heads are compacted into a list (head bitmask, word prefix
// counts), then each thread takes whole runs, so per-run work (unmixing,
// the palindrome test, output) is not repeated for every key of a run.
template <int NW, bool IN_MIXED>
__global__ void __launch_bounds__(kRunThreads) runs_kernel(const uint64_t* __restrict__ s, uint64_t n, int K1, int d,
                                                           const uint64_t* __restrict__ spec,
                                                           const uint32_t* __restrict__ spec_len, uint64_t n_spec,
                                                           bool spec_mixed,
                                                           const uint64_t* __restrict__ next_head,
                                                           uint64_t* __restrict__ out_keys,
                                                           uint32_t* __restrict__ out_cnt, uint32_t slot,
                                                           uint32_t* __restrict__ tile_count,
                                                           uint2* __restrict__ tile_stats,
                                                           uint64_t* __restrict__ run_keys,
                                                           uint32_t* __restrict__ run_len,
                                                           uint32_t* __restrict__ run_count,
                                                           uint32_t* __restrict__ err) {
    constexpr int kWords = kRunTile / 32;
    constexpr int kRunsPerThread = kRunTile / kRunThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    // tile keys, one pad key after every 16 (fewer bank conflicts for
    // threads reading keys far apart): key i at tk[rp(i) * NW]
    uint64_t* tk = reinterpret_cast<uint64_t*>(smem);                          // [(TILE + TILE/16) * NW]
    uint32_t* head_bits = reinterpret_cast<uint32_t*>(tk + kRunTilePad * NW);  // [TILE / 32]
    uint32_t* wpre = head_bits + kWords;                                       // [TILE / 32 + 1] (+7 pad)
    uint32_t* wsum = wpre + kWords + 8;                                        // [8]
    uint16_t* hp = reinterpret_cast<uint16_t*>(wsum + 8);                      // [TILE] head positions
    uint64_t* out_stage_k = reinterpret_cast<uint64_t*>(hp + kRunTile);        // [TILE] if NW == 1
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t tile = blockIdx.x;
    const uint64_t start = tile * kRunTile;
    const uint32_t tn = (uint32_t)(n - start < (uint64_t)kRunTile ? n - start : (uint64_t)kRunTile);
    if (tn == (uint32_t)kRunTile) {
        Key<NW> x[kRunsPerThread];
#pragma unroll
        for (int j = 0; j < kRunsPerThread; j++) x[j] = load_key<NW>(s, start + tid + j * kRunThreads);
#pragma unroll
        for (int j = 0; j < kRunsPerThread; j++)
#pragma unroll
            for (int w = 0; w < NW; w++) tk[rp(tid + j * kRunThreads) * NW + w] = x[j].w[w];
    } else {
        for (uint32_t i = tid; i < tn; i += kRunThreads) {
            Key<NW> x = load_key<NW>(s, start + i);
#pragma unroll
            for (int w = 0; w < NW; w++) tk[rp(i) * NW + w] = x.w[w];
        }
    }
    __syncthreads();
    // head bitmask, one warp per 32-key word
    for (uint32_t wd = warp; wd < kWords; wd += kRunThreads / 32) {
        const uint32_t i = wd * 32 + lane;
        bool head = false;
        if (i < tn) {
            Key<NW> x, y;
#pragma unroll
            for (int w = 0; w < NW; w++) x.w[w] = tk[rp(i) * NW + w];
            if (i > 0) {
#pragma unroll
                for (int w = 0; w < NW; w++) y.w[w] = tk[rp(i - 1) * NW + w];
            } else {
                y = start > 0 ? load_key<NW>(s, start - 1) : x;
            }
            head = (start + i == 0) || !key_eq<NW>(x, y);
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, head);
        if (lane == 0) head_bits[wd] = m;
    }
    __syncthreads();
    // heads before each word (warp 0: two words per lane)
    static_assert(kWords == 64, "two bitmask words per lane");
    if (warp == 0) {
        const uint32_t c0 = __popc(head_bits[2 * lane]), c1 = __popc(head_bits[2 * lane + 1]);
        uint32_t x = c0 + c1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        const uint32_t ex = x - c0 - c1;
        wpre[2 * lane] = ex;
        wpre[2 * lane + 1] = ex + c0;
        if (lane == 31) wpre[kWords] = x;
    }
    __syncthreads();
    for (uint32_t wd = warp; wd < kWords; wd += kRunThreads / 32) {
        const uint32_t m = head_bits[wd];
        if ((m >> lane) & 1u) hp[wpre[wd] + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(wd * 32 + lane);
    }
    __syncthreads();
    const uint32_t H = wpre[kWords];
    // thread per run: runs tid, tid + 256, ... (ascending, for the spectrum hint)
    uint32_t cnt[kRunsPerThread];
    uint8_t nout[kRunsPerThread];
    uint32_t outs = 0, palins = 0;
    uint64_t hint = n_spec / 2;
#pragma unroll
    for (int j = 0; j < kRunsPerThread; j++) {
        const uint32_t r = tid + j * kRunThreads;
        nout[j] = 0;
        cnt[j] = 0;
        if (r >= H) continue;
        const uint32_t i = hp[r];
        const uint64_t end = r + 1 < H ? start + hp[r + 1] : next_head[tile];
        Key<NW> x;
#pragma unroll
        for (int w = 0; w < NW; w++) x.w[w] = tk[rp(i) * NW + w];
        if constexpr (IN_MIXED) x = unmix_key<NW>(x);
        const bool palin = key_eq<NW>(key_rc<NW>(x, K1), x);
        const uint64_t len = spec ? spectrum_count<NW>(spec, spec_len, n_spec, x, spec_mixed, hint) : end - (start + i);
        if (run_keys) {
            // every run, in run order at the tile's own offset (mixed key, length)
#pragma unroll
            for (int w = 0; w < NW; w++) run_keys[(start + r) * NW + w] = tk[rp(i) * NW + w];
            run_len[start + r] = (uint32_t)(len < 0xFFFFFFFFull ? len : 0xFFFFFFFFull);
        }
        uint64_t c = palin ? 2 * len : len;
        if (c > 0xFFFFFFFFull) {
            atomicOr(err, ST_OVERFLOW);
            c = 0xFFFFFFFFull;
        }
        cnt[j] = (uint32_t)c;
        if (spec || c >= (uint64_t)d) nout[j] = palin ? 1 : 2;
        outs += nout[j];
        palins += palin;
    }
    // one block scan of (outputs | palindromic runs << 16): both fit 16 bits
    uint32_t total;
    const uint32_t excl_thread = block_excl_scan_256(outs | (palins << 16), wsum, &total) & 0xFFFFu;
    const uint32_t n_out = total & 0xFFFFu;
    if (tid == 0) {
        tile_stats[tile] = make_uint2(H, total >> 16);
        tile_count[tile] = n_out;
        if (run_count) run_count[tile] = H;
    }
    if (n_out > slot) {
        if (tid == 0) atomicOr(err, ST_TABLE_FULL);
        return;
    }
    const uint64_t toff = tile * (uint64_t)slot;
    // a tile's outputs fill [toff, toff + n_out): for 1-word keys that fit,
    // stage them in shared memory and write them out coalesced
    const bool staged = NW == 1 && n_out <= (uint32_t)kRunTile;
    uint32_t lpos = excl_thread;
    uint64_t pos = toff + excl_thread;
#pragma unroll
    for (int j = 0; j < kRunsPerThread; j++) {
        if (!nout[j]) continue;
        const uint32_t i = hp[tid + j * kRunThreads];
        Key<NW> xk;
#pragma unroll
        for (int w = 0; w < NW; w++) xk.w[w] = tk[rp(i) * NW + w];
        if constexpr (IN_MIXED) xk = unmix_key<NW>(xk);
        for (uint32_t o = 0; o < nout[j]; o++) {
            const Key<NW> y = o == 0 ? xk : key_rc<NW>(xk, K1);
            if (staged) {
                // keys staged for a coalesced write-out; counts go straight out
                out_stage_k[lpos] = y.w[0];
                out_cnt[toff + lpos] = cnt[j];
                lpos++;
            } else {
                store_key<NW>(out_keys, pos, y);
                out_cnt[pos] = cnt[j];
                pos++;
            }
        }
    }
    if (staged) {
        __syncthreads();
        for (uint32_t i = tid; i < n_out; i += kRunThreads) out_keys[toff + i] = out_stage_k[i];
    }
}

// totals[0] += sum of tile_stats[].x, totals[1] += sum of .y
__global__ void sum_tile_stats_kernel(const uint2* __restrict__ st, uint64_t n, unsigned long long* __restrict__ totals) {
    uint64_t a = 0, b = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        a += st[i].x;
        b += st[i].y;
    }
    for (int off = 16; off; off >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, off);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, off);
    }
    if ((threadIdx.x & 31) == 0 && (a || b)) {
        atomicAdd(&totals[0], (unsigned long long)a);
        atomicAdd(&totals[1], (unsigned long long)b);
    }
}

// Tile t's first cnt[t] outputs (at t * slot) move to off[t].
__global__ void runs_compact_kernel(const uint64_t* __restrict__ k, const uint32_t* __restrict__ c, uint32_t slot,
                                    const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                                    uint64_t* __restrict__ k2, uint32_t* __restrict__ c2, int nw) {
    const uint64_t t = blockIdx.x;
    const uint64_t src = t * (uint64_t)slot, dst = off[t];
    const uint32_t m = cnt[t];
    // 8 words per thread in flight
    for (uint32_t i0 = 0; i0 < m * nw; i0 += 8 * blockDim.x) {
        uint64_t v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t i = i0 + threadIdx.x + q * blockDim.x;
            if (i < m * nw) v[q] = k[src * nw + i];
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t i = i0 + threadIdx.x + q * blockDim.x;
            if (i < m * nw) k2[dst * nw + i] = v[q];
        }
    }
    for (uint32_t i0 = 0; i0 < m; i0 += 8 * blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t i = i0 + threadIdx.x + q * blockDim.x;
            if (i < m) v[q] = c[src + i];
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t i = i0 + threadIdx.x + q * blockDim.x;
            if (i < m) c2[dst + i] = v[q];
        }
    }
}

// Tile t's cnt[t] runs (keys of nw words and lengths, at t * kRunTile) move
// to off[t].
__global__ void run_list_compact_kernel(const uint64_t* __restrict__ kslot, const uint32_t* __restrict__ lslot,
                                        const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ off, int nw,
                                        uint64_t* __restrict__ keys, uint32_t* __restrict__ lens) {
    const uint64_t t = blockIdx.x;
    const uint64_t src = t * (uint64_t)kRunTile, dst = off[t];
    const uint32_t m = cnt[t];
    for (uint32_t i = threadIdx.x; i < m * nw; i += blockDim.x) keys[dst * nw + i] = kslot[src * nw + i];
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) lens[dst + i] = lslot[src + i];
}

// Sorted canonical keys -> both-strand keys of kept runs, sorted ascending.
// spectrum == nullptr: counting mode (keep count >= d).  Otherwise every run
// is kept with its count looked up in the spectrum.
template <int NW>
void expand_runs(mh_ctx* ctx, const uint64_t* sorted, uint64_t n, int k, int d, Buf<uint64_t>& out_keys,
                 Buf<uint32_t>& out_cnt, uint64_t* n_out, uint64_t* n_canon_runs, uint64_t* n_palin_runs,
                 const uint64_t* spectrum, const uint32_t* spectrum_len, uint64_t n_spectrum, bool in_mixed,
                 bool spec_mixed, RunList* list) {
    if (list && spectrum) fail(MH_EUNSUPPORTED, "run lists are made while counting");
    const int K1 = k + 1;
    const uint64_t tiles = ceil_div(n ? n : 1, kRunTile);
    // a tile's outputs: when every kept run has >= 2 keys or is a palindrome
    // (counting with d >= 2), the runs inside the tile give at most one
    // output per key and the run continuing past the tile at most two
    // (one more than its first key), so <= keys + 1; else <= twice its keys
    const uint32_t slot = (!spectrum && d >= 2) ? kRunTile + 2 : 2 * kRunTile;
    Buf<uint64_t> first(ctx, tiles), next(ctx, tiles), totals(ctx, 2), toff(ctx, tiles + 1);
    Buf<uint32_t> tcount(ctx, tiles);
    Buf<uint64_t> big_k(ctx, tiles * slot * NW);
    Buf<uint32_t> big_c(ctx, tiles * slot);
    totals.zero();
    uint64_t S = 0, tot[2] = {0, 0};
    if (n) {
        MH_LAUNCH(ctx, "runs_first_head", grid_for(ctx, tiles * 32, 256), 256, 0, run_first_head_kernel<NW>, sorted, n,
                  tiles, first.p);
        MH_LAUNCH(ctx, "runs_next_head", grid_for(ctx, tiles, 256), 256, 0, run_next_head_kernel, first.p, tiles, n,
                  next.p);
        const size_t smem = sizeof(uint64_t) * kRunTilePad * NW + sizeof(uint32_t) * (2 * (kRunTile / 32) + 16) +
                            sizeof(uint16_t) * kRunTile +
                            (NW == 1 ? sizeof(uint64_t) * kRunTile : 0);
        auto kern = in_mixed ? runs_kernel<NW, true> : runs_kernel<NW, false>;
        MH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        Buf<uint2> tstats(ctx, tiles);
        Buf<uint32_t> rcount(ctx, list ? tiles : 1);
        Buf<uint32_t> rlen(ctx, list ? tiles * (uint64_t)kRunTile : 1);
        MH_LAUNCH_B(ctx, "runs", n * 8 * NW, (unsigned)tiles, kRunThreads, smem, kern, sorted, n, K1, d, spectrum,
                    spectrum_len, n_spectrum, spec_mixed, next.p, big_k.p, big_c.p, slot, tcount.p, tstats.p,
                    list ? list->slot.p : nullptr, list ? rlen.p : nullptr, list ? rcount.p : nullptr,
                    ctx->d_status);
        if (list) {
            Buf<uint64_t> roff(ctx, tiles + 1);
            exclusive_scan_u32(ctx, rcount.p, roff.p, tiles);
            read_u64(ctx, roff.p + tiles, &list->n, 1);
            list->keys = Buf<uint64_t>(ctx, (list->n ? list->n : 1) * NW);
            list->lens = Buf<uint32_t>(ctx, list->n ? list->n : 1);
            if (list->n)
                MH_LAUNCH(ctx, "run_list_compact", (unsigned)tiles, 256, 0, run_list_compact_kernel, list->slot.p,
                          rlen.p, rcount.p, roff.p, NW, list->keys.p, list->lens.p);
            list->slot.reset();
        }
        MH_LAUNCH(ctx, "runs_totals", grid_for(ctx, tiles, 256, 2), 256, 0, sum_tile_stats_kernel, tstats.p, tiles,
                  (unsigned long long*)totals.p);
        exclusive_scan_u32(ctx, tcount.p, toff.p, tiles);
        read_u64(ctx, toff.p + tiles, &S, 1);
        read_u64(ctx, totals.p, tot, 2);
    }
    if (list && !list->keys.p) {  // no input: an empty spectrum
        list->keys = Buf<uint64_t>(ctx, NW);
        list->lens = Buf<uint32_t>(ctx, 1);
        list->slot.reset();
    }
    *n_out = S;
    *n_canon_runs = tot[0];
    *n_palin_runs = tot[1];
    first.reset();
    next.reset();
    Buf<uint64_t> keys(ctx, (S ? S : 1) * NW), alt(ctx, (S ? S : 1) * NW);
    Buf<uint32_t> cnt(ctx, S ? S : 1), calt(ctx, S ? S : 1);
    if (S)
        MH_LAUNCH(ctx, "runs_compact", (unsigned)tiles, 256, 0, runs_compact_kernel, big_k.p, big_c.p, slot, tcount.p,
                  toff.p, keys.p, cnt.p, NW);
    big_k.reset();
    big_c.reset();
    // the table's keys are distinct and, as (k+1)-mers of both strands, their
    // top bits spread: the spread order with counts attached
    const bool in_alt = radix_sort_spread_kv<NW>(ctx, keys.p, alt.p, cnt.p, calt.p, S, 64 * NW - 2 * K1);
    if (in_alt) {
        out_keys = std::move(alt);
        out_cnt = std::move(calt);
    } else {
        out_keys = std::move(keys);
        out_cnt = std::move(cnt);
    }
}

template void expand_runs<1>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, const uint32_t*, uint64_t, bool, bool,
                             RunList*);
template void expand_runs<2>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, const uint32_t*, uint64_t, bool, bool,
                             RunList*);
template void expand_runs<4>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, const uint32_t*, uint64_t, bool, bool,
                             RunList*);

// Buckets of the mixed canonical keys to count one at a time (0 = all at
// once).  Memory still free: the HBM budget, or without one 85% of the
// device's memory, less what the context holds.  All at once if the count's
// working set (keys, sort buffer, run slots: about 24 nw + 12 bytes a
// window) fits in 90% of it; otherwise enough buckets (up to 64) that one
// bucket's working set and the byte a window of bucket numbers take at most
// 60% of it.  MH_COUNT_BUCKET_BITS (0..6) forces the number (tests).
int count_bucket_bits(mh_ctx* ctx, uint64_t n, int nw) {
    static const int forced = [] {
        const char* e = std::getenv("MH_COUNT_BUCKET_BITS");
        const int v = e ? std::atoi(e) : -1;
        return v >= 0 && v <= 6 ? v : -1;
    }();
    if (forced >= 0) return forced;
    if (ctx->bucket_bits >= 0) return ctx->bucket_bits;
    if (!n) return 0;
    const double per = 24.0 * nw + 12.0;
    const uint64_t budget = ctx->budget ? ctx->budget : ctx->device_bytes / 20 * 17;
    const double avail = budget > ctx->in_use ? (double)(budget - ctx->in_use) : 0.0;
    // in memory if the whole count fits in 90% of what is free; bucketed, the
    // buckets' outputs accumulate beside the next bucket's working set, and
    // one byte a window (its bucket) stays for the whole count
    if ((double)n * 1.05 * per <= 0.9 * avail) return 0;
    auto need = [&](int bb) { return (double)n + (double)n / (double)(1ull << bb) * 1.05 * per; };
    int bb = 1;
    while (bb < 6 && need(bb) > 0.6 * avail) bb++;
    return bb;
}

// The unit counting (8-bit passes over the top bits, units sorted and
// counted by a warp each), unless the context's plan or MH_COUNT_PATH=spread
// selects the spread sort with the fix-up and the run pass.
static bool use_unit_count(const mh_ctx* ctx) {
    static const bool v = [] {
        const char* e = std::getenv("MH_COUNT_PATH");
        return !(e && std::string(e) == "spread");
    }();
    return ctx->count_path >= 0 ? ctx->count_path == 0 : v;
}

// The extraction fused with the first pass (extract_scatter_kernel), for
// 1-word keys sorted by two passes or more, from 2^22 keys on;
// MH_EXTRACT_SCATTER=0 turns it off, =1 on at any size (tests).
static bool use_extract_scatter(uint64_t n) {
    static const int v = [] {
        const char* e = std::getenv("MH_EXTRACT_SCATTER");
        return e ? std::atoi(e) : -1;
    }();
    return v == 0 ? false : (v == 1 || n >= (1ull << 22));
}

// Shape of the fused pass (MH_XS_VARIANT): 0 = 14 items a thread and 4
// CTAs an SM (measured fastest), 1 = (16, 4), 2 = (16, 3), 3 = (12, 5).
static int xs_variant() {
    static const int v = [] {
        const char* e = std::getenv("MH_XS_VARIANT");
        return e ? std::atoi(e) : 0;
    }();
    return v;
}

// Slots of a segment of the fused pass: the mean count of a digit, plus
// 1/32 of it and eight standard deviations of a binomial count (the digits
// of mix_key images are nearly uniform; a k-mer seen m times adds m to one
// digit, which the 1/32 covers at the coverages met), at least one scatter
// tile.  MH_SCATTER_CAP sets it (at least a tile): tests make segments
// overflow with it.
static uint64_t scatter_cap(uint64_t n) {
    static const uint64_t forced = [] {
        const char* e = std::getenv("MH_SCATTER_CAP");
        return e ? std::strtoull(e, nullptr, 10) : 0ull;
    }();
    const uint64_t tile = (uint64_t)std::max(kXsTileMax, sort_tile<1>());
    if (forced) return std::max(forced, tile);
    const uint64_t mean = ceil_div(n, 256);
    return std::max(tile, mean + mean / 32 + 8 * (uint64_t)std::sqrt((double)mean) + 64);
}

template <int NW>
void count_kmers(mh_ctx* ctx, const mh_reads* reads, int k, int d, mh_kmers* out) {
    const uint64_t F = reads->n_frags;
    Buf<uint64_t> nwin(ctx, F + 1), woff(ctx, F + 1);
    if (F)
        MH_LAUNCH(ctx, "frag_windows", grid_for(ctx, F, 256), 256, 0, frag_windows_kernel, reads->frag_offs, F, k,
                  nwin.p);
    exclusive_scan_u64(ctx, nwin.p, woff.p, F);
    uint64_t n;
    read_u64(ctx, woff.p + F, &n, 1);
    nwin.reset();
    // keys are sorted as mix_key images: their evenly spread top bits let
    // the sort run its passes over the top ceil(log2 n) bits only
    constexpr bool kMixed = true;
    out->k = k;
    out->nw = NW;
    out->d = d;
    out->n_kmers = 2 * n;
    out->spectrum_mixed = kMixed;
    const int bb = count_bucket_bits(ctx, n, NW);
    const GroupPlan gp = group_plan(ctx, n, 0, NW);
    if (bb == 0 && use_unit_count(ctx) && gp.passes >= 0) {
        // 8-bit passes over the top bits, then the units sorted and counted
        // by a warp each (mh_group.cu); the extraction counts the passes'
        // digits for 1-word keys, or (two passes or more) makes the first
        // pass itself
        const int G = 8 * gp.passes;
        Buf<uint64_t> keys, alt;
        bool in_alt = false, fused = false;
        if (NW == 1 && n && gp.passes >= 2 && use_extract_scatter(n)) {
            const uint64_t cap = scatter_cap(n);
            keys = Buf<uint64_t>(ctx, 256 * cap);
            alt = Buf<uint64_t>(ctx, n);
            Buf<unsigned long long> cursor(ctx, 257);
            Buf<uint32_t> hist(ctx, (size_t)(gp.passes - 1) * 256);
            cursor.zero();
            hist.zero();
            // (items a thread, resident CTAs an SM)
            static const int shapes[4][2] = {{14, 4}, {16, 4}, {16, 3}, {12, 5}};
            const int* shape = shapes[xs_variant() & 3];
            const uint64_t tile = (uint64_t)kSortThreads * shape[0];
            const uint64_t n_tiles = ceil_div(n, tile);
            Buf<uint64_t> tfrag(ctx, n_tiles + 1);
            MH_LAUNCH(ctx, "tile_frag", grid_for(ctx, n_tiles + 1, 256), 256, 0, tile_frag_kernel, woff.p, F, n, tile,
                      n_tiles, tfrag.p);
            const unsigned xgrid = (unsigned)std::min<uint64_t>(n_tiles, (uint64_t)ctx->num_sms * shape[1]);
#define MH_XS_LAUNCH(I, B)                                                                                   \
    MH_LAUNCH_B(ctx, "extract_scatter", reads->n_packed / 4 + n * 8, xgrid, kSortThreads, 0,                 \
                (extract_scatter_kernel<I, B>), reads->packed, reads->frag_offs, woff.p, tfrag.p, n, k, 64 - G, \
                gp.passes - 1, cap, keys.p, cursor.p, hist.p)
            switch (xs_variant() & 3) {
                case 1: MH_XS_LAUNCH(16, 4); break;
                case 2: MH_XS_LAUNCH(16, 3); break;
                case 3: MH_XS_LAUNCH(12, 5); break;
                default: MH_XS_LAUNCH(14, 4);
            }
#undef MH_XS_LAUNCH
            uint64_t over = 0;
            read_u64(ctx, reinterpret_cast<const uint64_t*>(cursor.p) + 256, &over, 1);
            if (!over) {
                in_alt = radix_sort_segmented(ctx, keys.p, alt.p, n, cursor.p, cap, 64 - G + 8, 64, hist.p);
                fused = true;
            }
        }
        if (!fused) {
            keys.reset();
            alt.reset();
            keys = Buf<uint64_t>(ctx, (n ? n : 1) * NW);
            alt = Buf<uint64_t>(ctx, (n ? n : 1) * NW);
            const bool fuse = NW == 1 && gp.passes > 0;
            Buf<uint32_t> hist(ctx, fuse ? (size_t)gp.passes * 256 : 1);
            if (fuse) hist.zero();
            if (n)
                MH_LAUNCH_B(ctx, "extract_canonical", reads->n_packed / 4 + n * 8 * NW,
                            grid_for(ctx, F * 32, 256, 8), 256, fuse ? sizeof(uint32_t) * gp.passes * 256 : 0,
                            (extract_canonical_kernel<NW, kMixed>), reads->packed, reads->frag_offs, woff.p, F, k,
                            keys.p, fuse ? hist.p : nullptr, 64 - G, gp.passes, 8);
            in_alt = G ? radix_sort<NW>(ctx, keys.p, alt.p, nullptr, nullptr, n, 64 * NW - G, 64 * NW,
                                        fuse ? hist.p : nullptr)
                       : false;
        }
        woff.reset();
        Buf<uint64_t>& sorted = in_alt ? alt : keys;
        Buf<uint64_t>& other = in_alt ? keys : alt;
        Buf<uint64_t> sk;
        Buf<uint32_t> sc;
        uint64_t S = 0, runs = 0, palins = 0;
        RunList list;
        group_count<NW>(ctx, sorted, other, n, k, d, 0, gp, sk, sc, &S, &runs, &palins, &list);
        sync_and_check(ctx);
        out->n = S;
        out->n_distinct = 2 * runs - palins;
        out->keys = sk.release();
        out->counts = sc.release();
        out->n_spectrum = list.n;
        out->spectrum = list.keys.release();
        out->spectrum_len = list.lens.release();
        return;
    }
    if (bb == 0) {
        Buf<uint64_t> keys(ctx, (n ? n : 1) * NW), alt(ctx, (n ? n : 1) * NW);
        // the extraction counts the digits of the spread sort's passes (1-word
        // keys: for wider keys it measured no faster than the histogram pass)
        const int P = spread_pass_bits(ctx, n);
        const bool fuse = NW == 1 && n > 1 && P < 64;
        const int n_passes = (P + 7) / 8;
        Buf<uint32_t> hist(ctx, fuse ? (size_t)n_passes * 256 : 1);
        if (fuse) hist.zero();
        if (n)
            MH_LAUNCH_B(ctx, "extract_canonical", reads->n_packed / 4 + n * 8 * NW, grid_for(ctx, F * 32, 256, 8),
                        256, fuse ? sizeof(uint32_t) * n_passes * 256 : 0, (extract_canonical_kernel<NW, kMixed>),
                        reads->packed, reads->frag_offs, woff.p, F, k, keys.p, fuse ? hist.p : nullptr,
                        64 * NW - P, n_passes, 8);
        woff.reset();
        bool in_alt = radix_sort_spread<NW>(ctx, keys.p, alt.p, n, 0, fuse ? hist.p : nullptr);
        hist.reset();
        Buf<uint64_t>& sorted = in_alt ? alt : keys;
        Buf<uint64_t>& other = in_alt ? keys : alt;
        Buf<uint64_t> sk;
        Buf<uint32_t> sc;
        uint64_t S = 0, runs = 0, palins = 0;
        // every run (mixed key, length) is listed too, in the free sort buffer:
        // the spectrum the mercy step looks counts up in
        RunList list;
        list.slot = std::move(other);
        other.reset();
        expand_runs<NW>(ctx, sorted.p, n, k, d, sk, sc, &S, &runs, &palins, nullptr, nullptr, 0, kMixed, false,
                        &list);
        sorted.reset();
        sync_and_check(ctx);
        out->n = S;
        out->n_distinct = 2 * runs - palins;
        out->keys = sk.release();
        out->counts = sc.release();
        out->n_spectrum = list.n;
        out->spectrum = list.keys.release();
        out->spectrum_len = list.lens.release();
        return;
    }
    // Out of core: one bucket of the mixed canonical keys at a time (the
    // paper partitions its sort by k-mer prefix blocks the same way, Sec. 2
    // second paragraph).  Every window is extracted once per bucket and kept
    // if its key falls in it; each bucket is sorted (skipping its constant
    // top bits) and counted alone.  The spectrum is the buckets' spectra in
    // bucket order; the solid tables (both strands, real key order) of the
    // buckets are merged.
    const uint32_t nb = 1u << bb;
    const uint64_t n_tasks = ceil_div(F ? F : 1, (uint64_t)kTaskFrags);
    Buf<uint32_t> tcnt(ctx, nb * n_tasks);
    Buf<uint8_t> ids(ctx, n + 16);  // read 16 at a time
    if (F)
        MH_LAUNCH_B(ctx, "bucket_hist", reads->n_packed / 4 + n, grid_for(ctx, n_tasks * 32, 256, 8), 256, 0,
                    task_hist_kernel<NW>, reads->packed, reads->frag_offs, woff.p, F, k, bb, n_tasks, ids.p,
                    tcnt.p);
    else
        tcnt.zero();
    std::vector<uint64_t> hist(nb, 0);
    std::vector<Buf<uint64_t>> toff;
    for (uint32_t b = 0; b < nb; b++) {
        toff.emplace_back(ctx, n_tasks + 1);
        exclusive_scan_u32(ctx, tcnt.p + (uint64_t)b * n_tasks, toff[b].p, n_tasks);
    }
    for (uint32_t b = 0; b < nb; b++) read_u64(ctx, toff[b].p + n_tasks, &hist[b], 1);
    tcnt.reset();
    std::vector<Buf<uint64_t>> part_k, part_sk;
    std::vector<Buf<uint32_t>> part_l, part_sc;
    std::vector<uint64_t> part_n, part_S;
    uint64_t runs_tot = 0, palins_tot = 0;
    for (uint32_t b = 0; b < nb; b++) {
        const uint64_t m = hist[b];
        Buf<uint64_t> keys(ctx, (m ? m : 1) * NW), alt(ctx, (m ? m : 1) * NW);
        if (m)
            MH_LAUNCH_B(ctx, "extract_bucket", n + m * 8 * NW, grid_for(ctx, n_tasks * 32, 256, 8), 256, 0,
                        extract_bucket_kernel<NW>, reads->packed, reads->frag_offs, woff.p, ids.p, F, k, b, n_tasks,
                        toff[b].p, keys.p);
        toff[b].reset();
        Buf<uint64_t> sk;
        Buf<uint32_t> sc;
        uint64_t S = 0, runs = 0, palins = 0;
        RunList list;
        const GroupPlan bp = group_plan(ctx, m, bb, NW);
        if (use_unit_count(ctx) && bp.passes >= 0) {
            const bool in_alt = bp.passes ? radix_sort<NW>(ctx, keys.p, alt.p, nullptr, nullptr, m,
                                                           64 * NW - bb - 8 * bp.passes, 64 * NW - bb)
                                          : false;
            Buf<uint64_t>& sorted = in_alt ? alt : keys;
            Buf<uint64_t>& other = in_alt ? keys : alt;
            group_count<NW>(ctx, sorted, other, m, k, d, bb, bp, sk, sc, &S, &runs, &palins, &list);
        } else {
            const bool in_alt = radix_sort_spread<NW>(ctx, keys.p, alt.p, m, bb);
            Buf<uint64_t>& sorted = in_alt ? alt : keys;
            Buf<uint64_t>& other = in_alt ? keys : alt;
            list.slot = std::move(other);
            other.reset();
            expand_runs<NW>(ctx, sorted.p, m, k, d, sk, sc, &S, &runs, &palins, nullptr, nullptr, 0, kMixed, false,
                            &list);
            sorted.reset();
        }
        keys.reset();
        alt.reset();
        runs_tot += runs;
        palins_tot += palins;
        part_k.push_back(std::move(list.keys));
        part_l.push_back(std::move(list.lens));
        part_n.push_back(list.n);
        part_sk.push_back(std::move(sk));
        part_sc.push_back(std::move(sc));
        part_S.push_back(S);
    }
    ids.reset();
    woff.reset();
    // spectrum: the buckets' spectra back to back
    uint64_t n_spec = 0, S_tot = 0;
    for (uint32_t b = 0; b < nb; b++) {
        n_spec += part_n[b];
        S_tot += part_S[b];
    }
    Buf<uint64_t> spec(ctx, (n_spec ? n_spec : 1) * NW);
    Buf<uint32_t> spec_len(ctx, n_spec ? n_spec : 1);
    for (uint64_t b = 0, o = 0; b < nb; o += part_n[b], b++) {
        if (part_n[b]) {
            MH_CUDA(cudaMemcpyAsync(spec.p + o * NW, part_k[b].p, part_n[b] * NW * 8, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
            MH_CUDA(cudaMemcpyAsync(spec_len.p + o, part_l[b].p, part_n[b] * 4, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
        }
        part_k[b].reset();
        part_l[b].reset();
    }
    // solid: the buckets' tables back to back, then merged
    Buf<uint64_t> sk(ctx, (S_tot ? S_tot : 1) * NW), sk2(ctx, (S_tot ? S_tot : 1) * NW);
    Buf<uint32_t> sc(ctx, S_tot ? S_tot : 1), sc2(ctx, S_tot ? S_tot : 1);
    std::vector<uint64_t> bounds(1, 0);
    for (uint64_t b = 0, o = 0; b < nb; o += part_S[b], b++) {
        if (part_S[b]) {
            MH_CUDA(cudaMemcpyAsync(sk.p + o * NW, part_sk[b].p, part_S[b] * NW * 8, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
            MH_CUDA(cudaMemcpyAsync(sc.p + o, part_sc[b].p, part_S[b] * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        part_sk[b].reset();
        part_sc[b].reset();
        bounds.push_back(o + part_S[b]);
    }
    if (merge_runs<NW>(ctx, sk.p, sk2.p, sc.p, sc2.p, bounds)) {
        std::swap(sk, sk2);
        std::swap(sc, sc2);
    }
    sk2.reset();
    sc2.reset();
    sync_and_check(ctx);
    out->n = S_tot;
    out->n_distinct = 2 * runs_tot - palins_tot;
    out->keys = sk.release();
    out->counts = sc.release();
    out->n_spectrum = n_spec;
    out->spectrum = spec.release();
    out->spectrum_len = spec_len.release();
}

template void count_kmers<1>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);
template void count_kmers<2>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);
template void count_kmers<4>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);

}  // namespace mh
