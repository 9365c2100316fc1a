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

#include "mh_sort_kernels.cuh"

namespace mh {

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

template <int NW, bool HV, int ITEMS, int MINB>
static bool radix_sort_impl(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                            int bit_lo, int bit_hi) {
    if (n <= 1 || bit_hi <= bit_lo) return false;
    constexpr int TILE = sort_tile<NW, ITEMS>();
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
    constexpr size_t smem = onesweep_smem<NW, HV, ITEMS>();
    MH_CUDA(cudaFuncSetAttribute(onesweep_kernel<NW, HV, ITEMS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
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
                        (onesweep_kernel<NW, HV, ITEMS, MINB>), kin + c0 * NW, kout, HV ? vin + c0 : nullptr, vout, len,
                        bit_lo + 8 * p, base.p + ((uint64_t)p * n_chunks + c) * 256,
                        c + 1 < n_chunks ? base.p + ((uint64_t)p * n_chunks + c + 1) * 256 : nullptr, status.p,
                        counter.p, ctx->d_status);
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return (n_passes & 1) != 0;
}

// Tile shape of the scatter pass for 1-word keys: (items per thread,
// resident CTAs per SM).  The default (12, 3) measured fastest on GB300;
// MH_SORT_VARIANT selects another shape for tuning runs.
static int sort_variant() {
    static int v = [] {
        const char* e = std::getenv("MH_SORT_VARIANT");
        return e ? std::atoi(e) : 0;
    }();
    return v;
}

template <int NW, bool HV>
static bool radix_sort_dispatch(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt,
                                uint64_t n, int bit_lo, int bit_hi) {
    if constexpr (NW == 1) {
        switch (sort_variant()) {
            case 1: return radix_sort_impl<NW, HV, 16, 2>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
            case 2: return radix_sort_impl<NW, HV, 8, 4>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
            default: return radix_sort_impl<NW, HV, 12, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
        }
    }
    return radix_sort_impl<NW, HV, SortItems<NW>::v, 2>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
}

template <int NW>
bool radix_sort(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n, int bit_lo,
                int bit_hi) {
    if (vals) return radix_sort_dispatch<NW, true>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
    return radix_sort_dispatch<NW, false>(ctx, keys, alt, nullptr, nullptr, n, bit_lo, bit_hi);
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
