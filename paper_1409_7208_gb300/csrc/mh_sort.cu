// LSD radix sort of multiword keys (optionally with a 32-bit payload) and
// device-wide exclusive scans.
//
// Sort: one histogram kernel counts every 8-bit digit of every pass in a
// single read of the keys; then each pass is one "onesweep" kernel: a CTA
// takes the next tile (dynamic tile id, so every earlier tile already runs),
// ranks its keys by digit with warp match/ballot and shared-memory warp
// histograms (stable: rank follows input order), publishes its per-digit
// counts, looks back over earlier tiles' published counts (decoupled
// look-back, every wait bounded), stages the tile in shared memory in digit
// order and writes it out in coalesced runs.  Look-back counts are 30-bit,
// so a pass runs in chunks of at most (2^18 - 1) tiles, one launch per chunk,
// each with its own look-back chain.  Chunk 0 starts from the global digit
// offsets of the histogram (the same for every pass); the last tile of chunk
// c writes the digit offsets where chunk c+1 starts.
#include <cstdlib>

#include "mh_internal.cuh"

namespace mh {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint64_t kMaxTilesPerChunk = (1ull << 18) - 1;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 23;

template <int NW>
struct SortItems;
template <>
struct SortItems<1> {
    static constexpr int v = 16;
};
template <>
struct SortItems<2> {
    static constexpr int v = 10;
};
template <>
struct SortItems<4> {
    static constexpr int v = 6;
};

template <int NW>
__host__ __device__ constexpr int sort_tile() {
    return kSortThreads * SortItems<NW>::v;
}

template <int NW, bool HV>
constexpr size_t onesweep_smem() {
    return sizeof(uint32_t) * (kSortWarps * 256 + 256 + 256 + 8) + sizeof(uint64_t) * 256 +
           sizeof(uint64_t) * NW * sort_tile<NW>() + (HV ? sizeof(uint32_t) * sort_tile<NW>() : 0);
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
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> k = load_key<NW>(keys, i);
        for (int p = 0; p < n_passes; p++) atomicAdd(&sh[p * 256 + key_digit<NW>(k, shift0 + 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// base[p * 256 + d] = sum over d' < d of hist[p][d'] (where chunk 0 of pass
// p starts writing digit d).  One block of 256 threads per pass.
__global__ void radix_base_kernel(const uint32_t* __restrict__ hist, uint64_t* __restrict__ base,
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

// --------------------------------------------------------------- onesweep
template <int NW, bool HV>
__global__ void __launch_bounds__(kSortThreads, 2)
    onesweep_kernel(const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ vout, uint64_t n, int shift, const uint64_t* __restrict__ digit_base,
                    uint64_t* __restrict__ next_base, uint32_t* __restrict__ status,
                    uint32_t* __restrict__ tile_counter, uint32_t* __restrict__ err) {
    constexpr int ITEMS = SortItems<NW>::v;
    constexpr int TILE = sort_tile<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* warp_hist = reinterpret_cast<uint32_t*>(smem);          // [warps][256]
    uint32_t* tile_cnt = warp_hist + kSortWarps * 256;                 // [256]
    uint32_t* tile_start = tile_cnt + 256;                             // [256]
    uint32_t* misc = tile_start + 256;                                 // [8]
    uint64_t* scatter_base = reinterpret_cast<uint64_t*>(misc + 8);    // [256]
    uint64_t* stage = scatter_base + 256;                              // [NW][TILE]
    uint32_t* vstage = reinterpret_cast<uint32_t*>(stage + NW * TILE); // [TILE]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) misc[0] = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) warp_hist[i] = 0;
    __syncthreads();
    const uint32_t tile = misc[0];
    const uint64_t tile_base = (uint64_t)tile * TILE;

    // load: warp-striped, item i of lane l is key tile_base + warp*32*ITEMS + 32*i + l
    Key<NW> k[ITEMS];
    uint32_t v[HV ? ITEMS : 1];
    uint32_t rank[ITEMS];
    const uint64_t wbase = tile_base + (uint64_t)warp * 32 * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        uint64_t idx = wbase + 32 * i + lane;
        if (idx < n) {
            k[i] = load_key<NW>(kin, idx);
            if constexpr (HV) v[i] = vin[idx];
        } else {
#pragma unroll
            for (int w = 0; w < NW; w++) k[i].w[w] = 0;
            if constexpr (HV) v[i] = 0;
        }
    }
    // rank within the warp, stable by item then lane
    uint32_t* wh = warp_hist + warp * 256;
    const uint32_t lt_mask = (1u << lane) - 1;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        uint64_t idx = wbase + 32 * i + lane;
        uint32_t dg = idx < n ? key_digit<NW>(k[i], shift) : 256u;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && dg < 256u) {
            old = wh[dg];
            wh[dg] = old + __popc(peers);
        }
        old = __shfl_sync(0xFFFFFFFFu, old, leader);
        rank[i] = old + __popc(peers & lt_mask);
        __syncwarp();
    }
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
    tile_cnt[d] = cnt;
    // publish this tile's count early so later tiles can proceed
    uint32_t* st = status + (uint64_t)tile * 256 + d;
    st_relaxed_u32(st, (tile == 0 ? kFlagInc : kFlagAgg) | cnt);
    // block exclusive scan of tile_cnt -> tile_start
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
        for (int w = 0; w < warp; w++) wpre += misc[w];
        tile_start[d] = wpre + x - cnt;
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
                if (++spins > kSpinLimit) {
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
    scatter_base[d] = digit_base[d] + excl - tile_start[d];
    // the chunk's last tile: where the next chunk starts writing digit d
    if (next_base && (uint64_t)(tile + 1) * TILE >= n) next_base[d] = digit_base[d] + excl + cnt;
    __syncthreads();
    // stage in tile digit order
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        uint64_t idx = wbase + 32 * i + lane;
        if (idx < n) {
            uint32_t dg = key_digit<NW>(k[i], shift);
            uint32_t pos = tile_start[dg] + warp_hist[warp * 256 + dg] + rank[i];
#pragma unroll
            for (int w = 0; w < NW; w++) stage[w * TILE + pos] = k[i].w[w];
            if constexpr (HV) vstage[pos] = v[i];
        }
    }
    __syncthreads();
    const uint64_t rem = n - tile_base;
    const int n_valid = rem < (uint64_t)TILE ? (int)rem : TILE;
    for (int j = tid; j < n_valid; j += kSortThreads) {
        Key<NW> kk;
#pragma unroll
        for (int w = 0; w < NW; w++) kk.w[w] = stage[w * TILE + j];
        uint32_t dg = key_digit<NW>(kk, shift);
        uint64_t dst = scatter_base[dg] + j;
        store_key<NW>(kout, dst, kk);
        if constexpr (HV) vout[dst] = vstage[j];
    }
}

// Tiles per look-back chunk: (2^18 - 1), or MH_SORT_CHUNK_TILES (>= 1) when
// set, which tests use to run the multi-chunk path on small inputs.
static uint64_t chunk_tiles() {
    static uint64_t v = [] {
        const char* e = std::getenv("MH_SORT_CHUNK_TILES");
        uint64_t t = e ? std::strtoull(e, nullptr, 10) : 0;
        return (t >= 1 && t <= kMaxTilesPerChunk) ? t : kMaxTilesPerChunk;
    }();
    return v;
}

template <int NW, bool HV>
static bool radix_sort_impl(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                            int bit_lo, int bit_hi) {
    if (n <= 1 || bit_hi <= bit_lo) return false;
    constexpr int TILE = sort_tile<NW>();
    const int n_passes = (bit_hi - bit_lo + 7) / 8;
    const uint64_t chunk_len = chunk_tiles() * TILE;
    const int n_chunks = (int)ceil_div(n, chunk_len);
    Buf<uint32_t> hist(ctx, (size_t)n_passes * 256);
    // base[(p * n_chunks + c) * 256 + d]: where chunk c of pass p starts writing digit d
    Buf<uint64_t> base(ctx, (size_t)n_passes * n_chunks * 256);
    hist.zero();
    MH_LAUNCH_B(ctx, "radix_hist", n * 8 * NW, grid_for(ctx, n, 256, 4), 256, sizeof(uint32_t) * n_passes * 256,
                radix_hist_kernel<NW>, keys, n, bit_lo, n_passes, hist.p);
    MH_LAUNCH(ctx, "radix_base", n_passes, 256, 0, radix_base_kernel, hist.p, base.p, (uint64_t)n_chunks * 256);
    const uint64_t max_tiles = std::min<uint64_t>(chunk_tiles(), ceil_div(n, TILE));
    Buf<uint32_t> status(ctx, max_tiles * 256);
    Buf<uint32_t> counter(ctx, 64);
    constexpr size_t smem = onesweep_smem<NW, HV>();
    MH_CUDA(cudaFuncSetAttribute(onesweep_kernel<NW, HV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    uint64_t *kin = keys, *kout = alt;
    uint32_t *vin = vals, *vout = valt;
    for (int p = 0; p < n_passes; p++) {
        for (int c = 0; c < n_chunks; c++) {
            uint64_t c0 = (uint64_t)c * chunk_len;
            uint64_t len = std::min(chunk_len, n - c0);
            uint64_t tiles = ceil_div(len, TILE);
            MH_CUDA(cudaMemsetAsync(status.p, 0, tiles * 256 * sizeof(uint32_t), ctx->stream));
            MH_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(uint32_t), ctx->stream));
            MH_LAUNCH_B(ctx, "radix_onesweep", len * (16 * NW + (HV ? 8 : 0)), (unsigned)tiles, kSortThreads, smem,
                        (onesweep_kernel<NW, HV>), kin + c0 * NW, kout, HV ? vin + c0 : nullptr, vout, len,
                        bit_lo + 8 * p, base.p + ((uint64_t)p * n_chunks + c) * 256,
                        c + 1 < n_chunks ? base.p + ((uint64_t)p * n_chunks + c + 1) * 256 : nullptr, status.p,
                        counter.p, ctx->d_status);
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return (n_passes & 1) != 0;
}

template <int NW>
bool radix_sort(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n, int bit_lo,
                int bit_hi) {
    if (vals) return radix_sort_impl<NW, true>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
    return radix_sort_impl<NW, false>(ctx, keys, alt, nullptr, nullptr, n, bit_lo, bit_hi);
}

template bool radix_sort<1>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int);
template bool radix_sort<2>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int);
template bool radix_sort<4>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int);

// ------------------------------------------------------------------ scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, uint64_t n, uint64_t* __restrict__ sums) {
    uint64_t b0 = (uint64_t)blockIdx.x * kScanTile;
    uint64_t acc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        uint64_t idx = b0 + i;
        if (idx < n) acc += (uint64_t)in[idx];
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    __shared__ uint64_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kScanThreads / 32; w++) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// In-place exclusive scan of at most kScanTile values by one block; writes the total to a[n].
__global__ void scan_small_kernel(uint64_t* a, uint64_t n) {
    __shared__ uint64_t s[kScanTile];
    __shared__ uint64_t ws[kScanThreads / 32];
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) s[i] = (uint64_t)i < n ? a[i] : 0;
    __syncthreads();
    uint64_t loc[kScanItems];
    uint64_t t = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        loc[j] = t;
        t += s[threadIdx.x * kScanItems + j];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = t;
    for (int off = 1; off < 32; off <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += ws[w];
    uint64_t pre = wpre + x - t;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; j++) s[threadIdx.x * kScanItems + j] = pre + loc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
        if ((uint64_t)i < n) a[i] = s[i];
    if (threadIdx.x == kScanThreads - 1) a[n] = pre + t;
}

template <class T>
__global__ void scan_down_kernel(const T* __restrict__ in, uint64_t n, const uint64_t* __restrict__ offs,
                                 uint64_t* __restrict__ out) {
    __shared__ uint64_t s[kScanTile];
    __shared__ uint64_t ws[kScanThreads / 32];
    uint64_t b0 = (uint64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        uint64_t idx = b0 + i;
        s[i] = idx < n ? (uint64_t)in[idx] : 0;
    }
    __syncthreads();
    uint64_t loc[kScanItems];
    uint64_t t = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        loc[j] = t;
        t += s[threadIdx.x * kScanItems + j];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = t;
    for (int off = 1; off < 32; off <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += ws[w];
    uint64_t pre = offs[blockIdx.x] + wpre + x - t;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; j++) s[threadIdx.x * kScanItems + j] = pre + loc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        uint64_t idx = b0 + i;
        if (idx < n) out[idx] = s[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = offs[gridDim.x];
}

template <class T>
static void exclusive_scan_impl(mh_ctx* ctx, const T* in, uint64_t* out, uint64_t n) {
    if (n == 0) {
        MH_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), ctx->stream));
        return;
    }
    uint64_t nb = ceil_div(n, kScanTile);
    Buf<uint64_t> sums(ctx, nb + 1);
    MH_LAUNCH(ctx, "scan_reduce", (unsigned)nb, kScanThreads, 0, scan_reduce_kernel<T>, in, n, sums.p);
    if (nb <= (uint64_t)kScanTile) {
        MH_LAUNCH(ctx, "scan_small", 1, kScanThreads, 0, scan_small_kernel, sums.p, nb);
    } else {
        Buf<uint64_t> sums2(ctx, nb + 1);
        exclusive_scan_impl<uint64_t>(ctx, sums.p, sums2.p, nb);
        MH_CUDA(cudaMemcpyAsync(sums.p, sums2.p, sizeof(uint64_t) * (nb + 1), cudaMemcpyDeviceToDevice,
                                ctx->stream));
    }
    MH_LAUNCH(ctx, "scan_down", (unsigned)nb, kScanThreads, 0, scan_down_kernel<T>, in, n, sums.p, out);
}

void exclusive_scan_u64(mh_ctx* ctx, const uint64_t* in, uint64_t* out, uint64_t n) {
    exclusive_scan_impl<uint64_t>(ctx, in, out, n);
}
void exclusive_scan_u32(mh_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n) {
    exclusive_scan_impl<uint32_t>(ctx, in, out, n);
}

}  // namespace mh
