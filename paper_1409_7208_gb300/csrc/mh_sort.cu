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
#include <vector>

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
    MH_LAUNCH_B(ctx, "radix_hist", n * 8 * NW, grid_for(ctx, n, 256, 8), 256, sizeof(uint32_t) * n_passes * 256,
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
// resident CTAs per SM).  The defaults, (12, 4) for keys alone and (12, 3)
// with a payload (which needs more than 64 registers), measured fastest on
// GB300; MH_SORT_VARIANT selects another key-only shape for tuning runs.
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
        if constexpr (HV) {
            return radix_sort_impl<NW, HV, 12, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
        } else {
            switch (sort_variant()) {
                case 1: return radix_sort_impl<NW, HV, 14, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
                case 2: return radix_sort_impl<NW, HV, 12, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
                default: return radix_sort_impl<NW, HV, 12, 4>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi);
            }
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

// ------------------------------------------------------------ spread sort
// After LSD passes over bits [lo, 64), keys are ordered by their top bits;
// every position whose key is below its predecessor's within a group of
// equal top bits marks the group (once, through a bitmap of group starts),
// and each marked group is sorted in shared memory.  Groups larger than
// kSpreadFix keys (rare) are sorted by passes over the low bits, one
// segment at a time.

constexpr int kSpreadFix = 2048;

__global__ void spread_mark_kernel(const uint64_t* __restrict__ keys, uint64_t n, int lo,
                                   uint32_t* __restrict__ marked, uint64_t* __restrict__ list, uint64_t cap,
                                   unsigned long long* __restrict__ count) {
    for (uint64_t i = 1 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = keys[i], y = keys[i - 1];
        const uint64_t px = x >> lo;
        if (!(x < y && px == (y >> lo))) continue;
        // first index of the group (gallop back, then bisect)
        uint64_t hi = i - 1, step = 1, lb;
        while (true) {
            if (hi < step) {
                lb = 0;
                break;
            }
            if ((keys[hi - step] >> lo) != px) {
                lb = hi - step + 1;
                break;
            }
            hi -= step;
            step <<= 1;
        }
        while (lb < hi) {
            const uint64_t mid = (lb + hi) / 2;
            if ((keys[mid] >> lo) == px) hi = mid; else lb = mid + 1;
        }
        const uint64_t gs = lb;
        const uint32_t bit = 1u << (gs & 31);
        if (atomicOr(&marked[gs >> 5], bit) & bit) continue;
        const uint64_t slot = atomicAdd(count, 1ull);
        if (slot < cap) list[slot] = gs;
    }
}

__global__ void __launch_bounds__(256) spread_group_kernel(uint64_t* __restrict__ keys, uint64_t n, int lo,
                                                           const uint64_t* __restrict__ list, uint64_t n_groups,
                                                           ulonglong2* __restrict__ big,
                                                           unsigned long long* __restrict__ n_big) {
    __shared__ uint64_t sk[kSpreadFix];
    __shared__ uint64_t s_end;
    for (uint64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const uint64_t gs = list[g];
        if (threadIdx.x == 0) {
            const uint64_t px = keys[gs] >> lo;
            uint64_t l = gs + 1, step = 1, h;
            while (true) {  // first index with other top bits
                const uint64_t probe = l + step - 1;
                if (probe >= n) {
                    h = n;
                    break;
                }
                if ((keys[probe] >> lo) != px) {
                    h = probe;
                    break;
                }
                l = probe + 1;
                step <<= 1;
            }
            while (l < h) {
                const uint64_t mid = (l + h) / 2;
                if ((keys[mid] >> lo) == px) l = mid + 1; else h = mid;
            }
            s_end = l;
        }
        __syncthreads();
        const uint64_t size = s_end - gs;
        if (size > (uint64_t)kSpreadFix) {
            if (threadIdx.x == 0) big[atomicAdd(n_big, 1ull)] = make_ulonglong2(gs, s_end);
            __syncthreads();
            continue;
        }
        int p2 = 2;
        while ((uint64_t)p2 < size) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += blockDim.x) sk[i] = (uint64_t)i < size ? keys[gs + i] : ~0ull;
        __syncthreads();
        for (int kk = 2; kk <= p2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l <= i) continue;
                    const uint64_t a = sk[i], b = sk[l];
                    if ((a > b) == ((i & kk) == 0)) {
                        sk[i] = b;
                        sk[l] = a;
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; (uint64_t)i < size; i += blockDim.x) keys[gs + i] = sk[i];
        __syncthreads();
    }
}

static int ceil_log2(uint64_t n) {
    int b = 0;
    while (b < 64 && (1ull << b) < n) b++;
    return b;
}

// MH_SPREAD_BITS (a multiple of 8 in [8, 64]) fixes the number of top bits
// sorted by passes; tests use small values to run the fix-up on small inputs.
static int spread_bits(uint64_t n) {
    static int forced = [] {
        const char* e = std::getenv("MH_SPREAD_BITS");
        int v = e ? std::atoi(e) : 0;
        return (v >= 8 && v <= 64 && v % 8 == 0) ? v : 0;
    }();
    return forced ? forced : ((ceil_log2(n) + 8 + 7) / 8) * 8;
}

bool radix_sort_spread(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint64_t n) {
    const int P = spread_bits(n);
    if (n <= 1 || P >= 64) return radix_sort<1>(ctx, keys, alt, nullptr, nullptr, n, 0, 64);
    const int lo = 64 - P;
    const bool in_alt = radix_sort<1>(ctx, keys, alt, nullptr, nullptr, n, lo, 64);
    uint64_t* k = in_alt ? alt : keys;
    uint64_t* other = in_alt ? keys : alt;
    const uint64_t cap = std::max<uint64_t>(1 << 16, n / 256);
    Buf<uint32_t> marked(ctx, ceil_div(n, 32));
    Buf<uint64_t> list(ctx, cap), cnt(ctx, 2);
    marked.zero();
    cnt.zero();
    MH_LAUNCH(ctx, "spread_fixup_mark", grid_for(ctx, n, 256), 256, 0, spread_mark_kernel, k, n, lo, marked.p, list.p,
              cap, (unsigned long long*)cnt.p);
    uint64_t n_groups = 0;
    read_u64(ctx, cnt.p, &n_groups, 1);
    if (n_groups > cap) {
        // far more shared prefixes than uniform keys would have: sort fully
        return in_alt != radix_sort<1>(ctx, k, other, nullptr, nullptr, n, 0, 64);
    }
    if (n_groups) {
        Buf<ulonglong2> big(ctx, n_groups);
        MH_LAUNCH(ctx, "spread_fixup_groups", (unsigned)std::min<uint64_t>(n_groups, (uint64_t)ctx->num_sms * 16), 256,
                  0, spread_group_kernel, k, n, lo, list.p, n_groups, big.p, (unsigned long long*)(cnt.p + 1));
        uint64_t n_big = 0;
        read_u64(ctx, cnt.p + 1, &n_big, 1);
        if (n_big) {
            std::vector<ulonglong2> h(n_big);
            MH_CUDA(cudaMemcpyAsync(h.data(), big.p, sizeof(ulonglong2) * n_big, cudaMemcpyDeviceToHost, ctx->stream));
            sync_and_check(ctx);
            for (const ulonglong2& seg : h) {
                const uint64_t len = seg.y - seg.x;
                Buf<uint64_t> tmp(ctx, len);
                if (radix_sort<1>(ctx, k + seg.x, tmp.p, nullptr, nullptr, len, 0, lo))
                    MH_CUDA(cudaMemcpyAsync(k + seg.x, tmp.p, len * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            }
        }
    }
    return in_alt;
}

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
