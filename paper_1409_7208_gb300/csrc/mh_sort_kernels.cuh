// Radix sort kernels shared by the allocating sort (mh_sort.cu) and the
// static-scratch sort (mh_noalloc.cu).  See mh_sort.cu for the method.
#pragma once

#include "mh_internal.cuh"

namespace mh {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint64_t kMaxTilesPerChunk = (1ull << 18) - 1;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 23;  // default bound of a look-back wait (polls)

template <int NW>
struct SortItems;
template <>
struct SortItems<1> {
    static constexpr int v = 16;
};
template <>
struct SortItems<2> {
    static constexpr int v = 12;
};
template <>
struct SortItems<4> {
    static constexpr int v = 8;
};

template <int NW, int ITEMS = SortItems<NW>::v>
__host__ __device__ constexpr int sort_tile() {
    return kSortThreads * ITEMS;
}

template <int NW, bool HV, int ITEMS = SortItems<NW>::v>
constexpr size_t onesweep_smem() {
    return sizeof(uint32_t) * (kSortWarps * 256 + 256 + 256 + 8) + sizeof(uint64_t) * 256 +
           sizeof(uint64_t) * NW * sort_tile<NW, ITEMS>() + (HV ? sizeof(uint32_t) * sort_tile<NW, ITEMS>() : 0);
}

// ------------------------------------------------------------ histogram
// hist[p * 256 + digit] over all n keys, digit of pass p = bits
// [shift0 + 8p, +8).
template <int NW>
__global__ void __launch_bounds__(256) radix_hist_kernel(const uint64_t* __restrict__ keys, uint64_t n, int shift0,
                                                         int n_passes, uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t sh[];
    const int nb = n_passes * 256;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    // four independent loads in flight per thread before the counting
    constexpr int U = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < n; i += U * stride) {
        Key<NW> k[U];
#pragma unroll
        for (int u = 0; u < U; u++) k[u] = load_key<NW>(keys, i + u * stride);
#pragma unroll
        for (int u = 0; u < U; u++)
            for (int p = 0; p < n_passes; p++) atomicAdd(&sh[p * 256 + key_digit<NW>(k[u], shift0 + 8 * p)], 1u);
    }
    for (; i < n; i += stride) {
        Key<NW> k = load_key<NW>(keys, i);
        for (int p = 0; p < n_passes; p++) atomicAdd(&sh[p * 256 + key_digit<NW>(k, shift0 + 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// base[p * 256 + d] = sum over d' < d of hist[p][d'] (where chunk 0 of pass
// p starts writing digit d).  One block of 256 threads per pass.
static __global__ void radix_base_kernel(const uint32_t* __restrict__ hist, uint64_t* __restrict__ base,
                                  uint64_t base_stride) {
    __shared__ uint64_t s[256];
    int p = blockIdx.x, d = threadIdx.x;
    uint64_t tot = hist[p * 256 + d];
    s[d] = tot;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        uint64_t v = d >= off ? s[d - off] : 0;
        __syncthreads();
        s[d] += v;
        __syncthreads();
    }
    base[p * base_stride + d] = s[d] - tot;
}

// The lanes of the warp whose digit (8 bits) equals this lane's.  A warp
// match instruction finds such sets, but it runs on the SM's divergence
// unit, one per SM, for about one cycle per distinct value among the lanes:
// on a whole random digit (some 30 values) that unit bound the scatter
// pass.  So the match takes the top kMatchBits bits only (at most 8
// values), and one ballot per remaining bit keeps the lanes that agree
// with this lane on that bit (ordinary instructions).
constexpr int kMatchBits = 3;
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg) {
    uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg >> (8 - kMatchBits));
#pragma unroll
    for (int b = 0; b < 8 - kMatchBits; b++) {
        const uint32_t bit = (dg >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// --------------------------------------------------------------- onesweep
// A segmented input (SEG): the slots [r * cap, r * cap + cnt[r]) hold
// segment r's keys and the rest of the slots are unused.  Slot 0 of the
// launch is slot slot0 of the whole input; cap is at least one tile, so a
// tile meets at most two segments.
struct SegIn {
    const unsigned long long* cnt = nullptr;
    uint64_t cap = 0;
    uint64_t slot0 = 0;
};

template <int NW, bool HV, int ITEMS = SortItems<NW>::v, int MINB = 2, bool SEG = false>
__global__ void __launch_bounds__(kSortThreads, MINB)
    onesweep_kernel(const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ vout, uint64_t n, int shift, const uint64_t* __restrict__ digit_base,
                    uint64_t* __restrict__ next_base, uint32_t* __restrict__ status,
                    uint32_t* __restrict__ tile_counter, uint32_t* __restrict__ err, int spin_limit,
                    int withhold_first, SegIn seg) {
    constexpr int TILE = sort_tile<NW, ITEMS>();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* warp_hist = reinterpret_cast<uint32_t*>(smem);          // [warps][256]
    uint32_t* misc = warp_hist + kSortWarps * 256 + 512;               // [8]
    uint64_t* scatter_base = reinterpret_cast<uint64_t*>(misc + 8);    // [256]
    uint64_t* stage = scatter_base + 256;                              // [NW][TILE]
    uint32_t* vstage = reinterpret_cast<uint32_t*>(stage + NW * TILE); // [TILE]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) misc[0] = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) warp_hist[i] = 0;
    __syncthreads();
    const uint32_t tile = misc[0];
    const uint64_t tile_base = (uint64_t)tile * TILE;
    const uint64_t rem = n - tile_base;
    const uint32_t tile_n = rem < (uint64_t)TILE ? (uint32_t)rem : (uint32_t)TILE;
    // the tile's keys: positions [0, va) and [vb, vc) (one run unless the
    // input is segmented and the tile crosses into the next segment)
    uint32_t va = tile_n, vb = TILE, vc = TILE;
    if constexpr (SEG) {
        const uint64_t s = seg.slot0 + tile_base;
        const uint64_t r0 = s / seg.cap;
        const uint64_t e0 = r0 * seg.cap + seg.cnt[r0];
        va = e0 > s ? (uint32_t)(e0 - s < (uint64_t)tile_n ? e0 - s : tile_n) : 0u;
        const uint64_t nb = (r0 + 1) * seg.cap - s;
        if (nb < tile_n) {
            vb = (uint32_t)nb;
            const uint64_t e1 = nb + seg.cnt[r0 + 1];
            vc = (uint32_t)(e1 < (uint64_t)tile_n ? e1 : tile_n);
        }
    }
    const bool full = SEG ? va == (uint32_t)TILE : tile_n == (uint32_t)TILE;
    const uint32_t n_valid = SEG ? va + (vc - vb) : tile_n;
#define MH_PRESENT(q) (SEG ? ((q) < va || (q) - vb < vc - vb) : ((q) < tile_n))
    const uint64_t* kt = kin + tile_base * NW;
    const uint32_t* vt = HV ? vin + tile_base : nullptr;

    // load: warp-striped, item i of lane l is tile key warp*32*ITEMS + 32*i + l
    Key<NW> k[ITEMS];
    uint32_t v[HV ? ITEMS : 1];
    const uint32_t w0 = (uint32_t)warp * 32 * ITEMS + lane;
    if (full) {
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            k[i] = load_key<NW>(kt, w0 + 32 * i);
            if constexpr (HV) v[i] = vt[w0 + 32 * i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            if (MH_PRESENT(w0 + 32 * i)) {
                k[i] = load_key<NW>(kt, w0 + 32 * i);
                if constexpr (HV) v[i] = vt[w0 + 32 * i];
            } else {
#pragma unroll
                for (int w = 0; w < NW; w++) k[i].w[w] = 0;
                if constexpr (HV) v[i] = 0;
            }
        }
    }
    // counts first: each warp counts its keys' digits in its own histogram
    uint32_t* wh = warp_hist + warp * 256;
    const uint32_t lt_mask = (1u << lane) - 1;
#pragma unroll
    for (int i = 0; i < ITEMS; i++)
        if (full || MH_PRESENT(w0 + 32 * i)) atomicAdd(&wh[key_digit<NW>(k[i], shift)], 1u);
    __syncthreads();
    // per digit: exclusive prefix over warps, tile total
    const int d = tid;  // kSortThreads == 256
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
        uint32_t c = warp_hist[w * 256 + d];
        warp_hist[w * 256 + d] = cnt;
        cnt += c;
    }
    // publish this tile's count before ranking, so later tiles can proceed (a
    // test hook, withhold_first, keeps tile 0 from publishing: the next
    // tiles' bounded waits then run out and report it)
    uint32_t* st = status + (uint64_t)tile * 256 + d;
    if (!(withhold_first && tile == 0)) st_relaxed_u32(st, (tile == 0 ? kFlagInc : kFlagAgg) | cnt);
    // block exclusive scan of the tile counts -> start of digit d in the tile
    uint32_t start;
    {
        uint32_t x = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) misc[warp] = x;  // misc[0..7]; misc[0] (tile) already read
        __syncthreads();
        uint32_t wpre = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) wpre += w < warp ? misc[w] : 0u;
        start = wpre + x - cnt;
    }
    // each warp's first staging slot for digit d
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) warp_hist[w * 256 + d] += start;
    __syncthreads();
    // rank and stage in tile digit order, stable by item then lane: the
    // lanes holding one digit in one item find each other (digit_peers), the
    // lowest of them takes their slots from the warp's counter in one
    // atomic add and hands the first slot on; each lane adds the number of
    // its lower peers.  Staging needs no global prefix, and by the time it
    // is done the earlier tiles have published more of theirs.
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const bool valid = full || MH_PRESENT(w0 + 32 * i);
        const uint32_t dg = key_digit<NW>(k[i], shift);
        // (a lane past the tile's end counts itself only among the valid)
        const uint32_t peers =
            digit_peers(dg) & (full ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid) | (1u << lane));
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (lane == leader && valid) slot = atomicAdd(&wh[dg], (uint32_t)__popc(peers));
        slot = __shfl_sync(0xFFFFFFFFu, slot, leader) + (uint32_t)__popc(peers & lt_mask);
        if (valid) {
#pragma unroll
            for (int w = 0; w < NW; w++) stage[w * TILE + slot] = k[i].w[w];
            if constexpr (HV) vstage[slot] = v[i];
        }
    }
    // look back over earlier tiles for this digit
    uint64_t excl = 0;
    if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        bool ok = true;
        while (j >= 0) {
            const uint32_t* sp = status + (uint64_t)j * 256 + d;
            uint32_t s = ld_relaxed_u32(sp);
            int spins = 0;
            while ((s & ~kCountMask) == 0) {
                if (++spins > spin_limit) {
                    ok = false;
                    break;
                }
                if (spins > 64) __nanosleep(128);
                s = ld_relaxed_u32(sp);
            }
            if (!ok) break;
            excl += s & kCountMask;
            if ((s & ~kCountMask) == kFlagInc) break;
            j--;
        }
        if (!ok) atomicOr(err, ST_SPIN_TIMEOUT);
        st_relaxed_u32(st, kFlagInc | (uint32_t)((excl + cnt) & kCountMask));
    }
    scatter_base[d] = digit_base[d] + excl - start;
    // the chunk's last tile: where the next chunk starts writing digit d
    if (next_base && (uint64_t)(tile + 1) * TILE >= n) next_base[d] = digit_base[d] + excl + cnt;
    __syncthreads();
    // write out: consecutive staged keys of one digit go to consecutive addresses
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const uint32_t j = tid + i * kSortThreads;
        if (full || j < n_valid) {
            Key<NW> kk;
#pragma unroll
            for (int w = 0; w < NW; w++) kk.w[w] = stage[w * TILE + j];
            const uint64_t dst = scatter_base[key_digit<NW>(kk, shift)] + j;
            store_key<NW>(kout, dst, kk);
            if constexpr (HV) vout[dst] = vstage[j];
        }
    }
}
#undef MH_PRESENT

}  // namespace mh
