// LSD radix sort of multiword keys (optionally with a 32-bit payload) and
// device-wide exclusive scans.
//
// Sort: one histogram kernel counts every 8-bit digit of every pass in a
// single read of the keys; then each pass is one "onesweep" kernel: a CTA
// takes the next tile (dynamic tile id, so every earlier tile already runs),
// counts its keys' digits in per-warp shared-memory histograms, publishes
// the tile's per-digit counts, ranks the keys by digit (a warp match on the
// digit's top bits, ballots on the rest) with one shared atomic per group of
// equal digits (stable: rank follows input order) while staging them in
// shared memory in digit order, looks back over earlier tiles' published
// counts (decoupled look-back, every wait bounded) and writes the tile out
// in coalesced runs.  Look-back counts are 30-bit, so a pass runs in chunks of at most (2^18 - 1) tiles, one launch per chunk,
// each with its own look-back chain.  Chunk 0 starts from the global digit
// offsets of the histogram (the same for every pass); the last tile of chunk
// c writes the digit offsets where chunk c+1 starts.  The first pass may
// read a segmented input (radix_sort_segmented: the keys of each value of
// the previous digit in a segment of fixed size, as the fused extraction
// of mh_count.cu writes them); its tiles then skip the unused slots.
#include <atomic>
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

// Polls a look-back wait may make before it gives up (MH_SPIN_LIMIT, >= 1;
// default kSpinLimit, about a second with the back-off).
static int spin_limit() {
    static const int v = [] {
        const char* e = std::getenv("MH_SPIN_LIMIT");
        const long x = e ? std::strtol(e, nullptr, 10) : 0;
        return x >= 1 && x <= kSpinLimit ? (int)x : kSpinLimit;
    }();
    return v;
}

// Test hook: MH_TEST_WITHHOLD_TILE0=N makes the first N scatter launches of
// the process keep their tile 0 from publishing its counts, so that the
// bounded waits of the tiles after it run out (MH_ETIMEOUT); later launches
// are normal.
static int take_withhold() {
    static std::atomic<int> left{[] {
        const char* e = std::getenv("MH_TEST_WITHHOLD_TILE0");
        return e ? std::atoi(e) : 0;
    }()};
    int v = left.load();
    while (v > 0 && !left.compare_exchange_weak(v, v - 1)) {
    }
    return v > 0 ? 1 : 0;
}

// seg.cnt set: the first pass reads a segmented input of 256 * seg.cap
// slots holding the n keys (SegIn); every pass writes n contiguous keys.
template <int NW, bool HV, int ITEMS, int MINB>
static bool radix_sort_impl(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                            int bit_lo, int bit_hi, const uint32_t* hist_in, SegIn seg = SegIn{}) {
    if (n <= 1 || bit_hi <= bit_lo) return false;
    constexpr int TILE = sort_tile<NW, ITEMS>();
    const int n_passes = (bit_hi - bit_lo + 7) / 8;
    const uint64_t chunk_len = chunk_tiles() * TILE;
    // positions pass p reads: the segment slots in the first pass
    auto span = [&](int p) { return p == 0 && seg.cnt ? 256 * seg.cap : n; };
    const int max_chunks = (int)ceil_div(span(0), chunk_len);
    Buf<uint32_t> hist(ctx, hist_in ? 1 : (size_t)n_passes * 256);
    // base[(p * max_chunks + c) * 256 + d]: where chunk c of pass p starts writing digit d
    Buf<uint64_t> base(ctx, (size_t)n_passes * max_chunks * 256);
    if (!hist_in) {
        hist.zero();
        MH_LAUNCH_B(ctx, "radix_hist", n * 8 * NW, grid_for(ctx, n, 256, 8), 256, sizeof(uint32_t) * n_passes * 256,
                    radix_hist_kernel<NW>, keys, n, bit_lo, n_passes, hist.p);
    }
    MH_LAUNCH(ctx, "radix_base", n_passes, 256, 0, radix_base_kernel, hist_in ? hist_in : hist.p, base.p,
              (uint64_t)max_chunks * 256);
    const uint64_t max_tiles = std::min<uint64_t>(chunk_tiles(), ceil_div(span(0), TILE));
    Buf<uint32_t> status(ctx, max_tiles * 256);
    Buf<uint32_t> counter(ctx, 64);
    constexpr size_t smem = onesweep_smem<NW, HV, ITEMS>();
    MH_CUDA(cudaFuncSetAttribute(onesweep_kernel<NW, HV, ITEMS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    uint64_t *kin = keys, *kout = alt;
    uint32_t *vin = vals, *vout = valt;
    for (int p = 0; p < n_passes; p++) {
        const uint64_t np = span(p);
        const int n_chunks = (int)ceil_div(np, chunk_len);
        for (int c = 0; c < n_chunks; c++) {
            uint64_t c0 = (uint64_t)c * chunk_len;
            uint64_t len = std::min(chunk_len, np - c0);
            uint64_t tiles = ceil_div(len, TILE);
            MH_CUDA(cudaMemsetAsync(status.p, 0, tiles * 256 * sizeof(uint32_t), ctx->stream));
            MH_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(uint32_t), ctx->stream));
            uint64_t* nb = c + 1 < n_chunks ? base.p + ((uint64_t)p * max_chunks + c + 1) * 256 : nullptr;
            if constexpr (NW == 1 && !HV) {
                if (p == 0 && seg.cnt) {
                    SegIn sp = seg;
                    sp.slot0 = c0;
                    MH_CUDA(cudaFuncSetAttribute(onesweep_kernel<NW, HV, ITEMS, MINB, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                    MH_LAUNCH_B(ctx, "radix_onesweep", len * 16, (unsigned)tiles, kSortThreads, smem,
                                (onesweep_kernel<NW, HV, ITEMS, MINB, true>), kin + c0, kout, nullptr, nullptr, len,
                                bit_lo, base.p + (uint64_t)c * 256, nb, status.p, counter.p, ctx->d_status,
                                spin_limit(), take_withhold(), sp);
                    continue;
                }
            }
            MH_LAUNCH_B(ctx, "radix_onesweep", len * (16 * NW + (HV ? 8 : 0)), (unsigned)tiles, kSortThreads, smem,
                        (onesweep_kernel<NW, HV, ITEMS, MINB>), kin + c0 * NW, kout, HV ? vin + c0 : nullptr, vout, len,
                        bit_lo + 8 * p, base.p + ((uint64_t)p * max_chunks + c) * 256, nb, status.p, counter.p,
                        ctx->d_status, spin_limit(), take_withhold(), SegIn{});
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return (n_passes & 1) != 0;
}

// Tile shape of the scatter pass for 1-word keys: (items per thread,
// resident CTAs per SM).  The defaults, (16, 3) for keys alone and (14, 3)
// with a payload, measured fastest on GB300; a context's tuned shape
// (mh_run_batch's autotuner) or MH_SORT_VARIANT selects another key-only
// shape: 1 = (12, 4), 2 = (14, 3).
static int sort_variant() {
    static int v = [] {
        const char* e = std::getenv("MH_SORT_VARIANT");
        return e ? std::atoi(e) : 0;
    }();
    return v;
}

template <int NW, bool HV>
static bool radix_sort_dispatch(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt,
                                uint64_t n, int bit_lo, int bit_hi, const uint32_t* h, SegIn seg = SegIn{}) {
    if constexpr (NW == 1) {
        if constexpr (HV) {
            return radix_sort_impl<NW, HV, 14, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, h, seg);
        } else {
            switch (ctx->sort_shape >= 0 ? ctx->sort_shape : sort_variant()) {
                case 1: return radix_sort_impl<NW, HV, 12, 4>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, h, seg);
                case 2: return radix_sort_impl<NW, HV, 14, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, h, seg);
                default: return radix_sort_impl<NW, HV, 16, 3>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, h, seg);
            }
        }
    }
    return radix_sort_impl<NW, HV, SortItems<NW>::v, 2>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, h, seg);
}

bool radix_sort_segmented(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint64_t n,
                          const unsigned long long* seg_cnt, uint64_t seg_cap, int bit_lo, int bit_hi,
                          const uint32_t* hist) {
    if (seg_cap < (uint64_t)sort_tile<1>() || !hist) throw Error{MH_EINVAL, "segmented sort: bad segments"};
    SegIn seg;
    seg.cnt = seg_cnt;
    seg.cap = seg_cap;
    return radix_sort_dispatch<1, false>(ctx, keys, alt, nullptr, nullptr, n, bit_lo, bit_hi, hist, seg);
}

template <int NW>
bool radix_sort(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n, int bit_lo,
                int bit_hi, const uint32_t* hist) {
    if (vals) return radix_sort_dispatch<NW, true>(ctx, keys, alt, vals, valt, n, bit_lo, bit_hi, hist);
    return radix_sort_dispatch<NW, false>(ctx, keys, alt, nullptr, nullptr, n, bit_lo, bit_hi, hist);
}

template bool radix_sort<1>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int, const uint32_t*);
template bool radix_sort<2>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int, const uint32_t*);
template bool radix_sort<4>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int, int, const uint32_t*);

// ------------------------------------------------------------ spread sort
// The keys are mix_key images, so the top bits of their top word are evenly
// spread: LSD passes over the top P bits only (P = ceil(log2 n) rounded up
// to a digit) leave every group of equal top bits in input order, and a
// group holds more than one distinct key only where two keys collide on
// those P bits (about D^2 / 2^(P+1) groups for D distinct keys).  The fix-up
// sorts such groups.  A tile kernel reads a window of keys (2048 / nw plus
// 256 / nw past the tile, for the group that crosses its end), finds the
// groups that start in the tile and contain a descent, and sorts them: up to
// 16 keys by one thread (insertion sort), larger ones by one warp
// (successive minima: each round finds the smallest key above the previous
// one and its count, then writes that run).  Groups that do not end inside
// the window, or have more than 64 distinct keys, go to a list for a CTA
// each (successive minima over the group in global memory, written through
// the free buffer); more than 256 distinct keys there (pathological) fall
// back to a radix sort of the segment.

template <int NW>
struct Fix {
    static constexpr int kTile = 2048 / NW;
    static constexpr int kExt = 256 / NW;
    static constexpr int kWin = kTile + kExt;
    static constexpr int kWords = kWin / 32;
    static constexpr int kThreadSort = 16;
    static constexpr int kQueue = kWin / (kThreadSort + 1) + 1;  // groups of > 16 keys in a window
};
constexpr int kFixWarpRounds = 64;
constexpr int kFixBlockRounds = 256;

template <int NW>
__device__ __forceinline__ Key<NW> shfl_key(const Key<NW>& a, int src_lane_xor) {
    Key<NW> r;
#pragma unroll
    for (int w = 0; w < NW; w++) r.w[w] = __shfl_xor_sync(0xFFFFFFFFu, a.w[w], src_lane_xor);
    return r;
}

template <int NW>
__device__ __forceinline__ Key<NW> key_ones() {
    Key<NW> r;
#pragma unroll
    for (int w = 0; w < NW; w++) r.w[w] = ~0ull;
    return r;
}

template <int NW>
__global__ void __launch_bounds__(256) spread_fix_kernel(uint64_t* __restrict__ keys, uint64_t n, int lo,
                                                         uint64_t* __restrict__ big, uint64_t big_cap,
                                                         unsigned long long* __restrict__ n_big) {
    using F = Fix<NW>;
    __shared__ uint64_t K[F::kWin * NW];
    __shared__ uint32_t head[F::kWords], desc[F::kWords];
    __shared__ uint32_t queue[2 * F::kQueue];  // (start, end) of the groups for warps
    __shared__ uint32_t n_queue;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t s = blockIdx.x * (uint64_t)F::kTile;
    const uint32_t W = (uint32_t)(n - s < (uint64_t)F::kWin ? n - s : (uint64_t)F::kWin);
    const uint32_t len = W < (uint32_t)F::kTile ? W : (uint32_t)F::kTile;
    const bool window_ends_array = s + W == n;
    auto kget = [&](uint32_t i) {
        Key<NW> r;
#pragma unroll
        for (int w = 0; w < NW; w++) r.w[w] = K[i * NW + w];
        return r;
    };
    auto kset = [&](uint32_t i, const Key<NW>& x) {
#pragma unroll
        for (int w = 0; w < NW; w++) K[i * NW + w] = x.w[w];
    };
    if (W == (uint32_t)F::kWin) {
        // all loads in flight at once
        uint64_t v[F::kWin * NW / 256];
#pragma unroll
        for (int q = 0; q < F::kWin * NW / 256; q++) v[q] = keys[s * NW + tid + q * 256];
#pragma unroll
        for (int q = 0; q < F::kWin * NW / 256; q++) K[tid + q * 256] = v[q];
    } else {
        for (uint32_t i = tid; i < W * NW; i += 256) K[i] = keys[s * NW + i];
    }
    if (tid == 0) n_queue = 0;
    __syncthreads();
    // a and b share their top bits iff (a ^ b) < 2^lo in the top word
    const uint64_t same_top = 1ull << lo;
    for (uint32_t wd = warp; wd < (uint32_t)F::kWords; wd += 8) {
        const uint32_t i = wd * 32 + lane;
        bool h = false, d = false;
        if (i < W) {
            const Key<NW> x = kget(i);
            const Key<NW> y = i > 0 ? kget(i - 1) : (s > 0 ? load_key<NW>(keys, s - 1) : key_ones<NW>());
            h = i == 0 && s == 0 ? true : (x.w[NW - 1] ^ y.w[NW - 1]) >= same_top;
            d = i > 0 && !h && key_less<NW>(x, y);
        }
        const uint32_t hb = __ballot_sync(0xFFFFFFFFu, h), db = __ballot_sync(0xFFFFFFFFu, d);
        if (lane == 0) {
            head[wd] = hb;
            desc[wd] = db;
        }
    }
    __syncthreads();
    // groups starting in this tile that hold a descent, each found from its
    // first descent (a word of descent bits a thread; descents are few: a
    // group holds two distinct keys only where keys collide on the top bits)
    auto to_big = [&](uint32_t h) {
        const unsigned long long q = atomicAdd(n_big, 1ull);
        if (q < big_cap) big[q] = s + h;
    };
    if (tid == 0 && !window_ends_array) {
        // the tile's last group, if it may run past the window with no descent
        // inside it: checked by a CTA of its own
        const uint32_t h = prev_bit(head, len - 1);
        if (h != ~0u && next_bit(head, h + 1, W) == W && !any_bit(desc, h + 1, W)) to_big(h);
    }
    for (uint32_t wd = tid; wd < (uint32_t)F::kWords; wd += 256) {
        uint32_t dm = desc[wd];
        while (dm) {
            const uint32_t jd = wd * 32 + __ffs(dm) - 1;
            dm &= dm - 1;
            const uint32_t h = prev_bit(head, jd);
            if (h == ~0u || h >= len) continue;  // the group starts in another tile
            if (any_bit(desc, h + 1, jd)) continue;  // not its first descent
            const uint32_t g1 = next_bit(head, jd + 1, W);
            if (g1 == W && !window_ends_array) {
                to_big(h);  // may run past the window
                continue;
            }
            if (g1 - h <= (uint32_t)F::kThreadSort) {
                for (uint32_t j = h + 1; j < g1; j++) {
                    const Key<NW> x = kget(j);
                    uint32_t i = j;
                    while (i > h && key_less<NW>(x, kget(i - 1))) {
                        kset(i, kget(i - 1));
                        i--;
                    }
                    kset(i, x);
                }
                for (uint32_t j = h; j < g1; j++) store_key<NW>(keys, s + j, kget(j));
            } else {
                const uint32_t q = atomicAdd(&n_queue, 1u);
                queue[2 * q] = h;
                queue[2 * q + 1] = g1;
            }
        }
    }
    __syncthreads();
    // larger groups: a warp each, by successive minima, from K to keys
    const uint32_t nq = n_queue;
    for (uint32_t q = warp; q < nq; q += 8) {
        const uint32_t g0 = queue[2 * q], g1 = queue[2 * q + 1];
        uint32_t pos = g0;
        Key<NW> prev = key_zero<NW>();
        bool first = true;
        int rounds = 0;
        while (pos < g1 && rounds < kFixWarpRounds) {
            // smallest key above prev, and its count
            Key<NW> mn = key_ones<NW>();
            bool have = false;
            for (uint32_t i = g0 + lane; i < g1; i += 32) {
                const Key<NW> x = kget(i);
                if ((first || key_less<NW>(prev, x)) && (!have || key_less<NW>(x, mn))) {
                    mn = x;
                    have = true;
                }
            }
            for (int off = 16; off; off >>= 1) {
                const Key<NW> o = shfl_key<NW>(mn, off);
                const bool oh = __shfl_xor_sync(0xFFFFFFFFu, have, off);
                if (oh && (!have || key_less<NW>(o, mn))) {
                    mn = o;
                    have = true;
                }
            }
            uint32_t c = 0;
            for (uint32_t i = g0 + lane; i < g1; i += 32) c += key_eq<NW>(kget(i), mn);
            for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
            for (uint32_t i = lane; i < c; i += 32) store_key<NW>(keys, s + pos + i, mn);
            pos += c;
            prev = mn;
            first = false;
            rounds++;
        }
        if (pos < g1 && lane == 0) {
            // too many distinct keys: rewrite the group as it was and defer it
            for (uint32_t i = g0; i < g1; i++) store_key<NW>(keys, s + i, kget(i));
            const unsigned long long b = atomicAdd(n_big, 1ull);
            if (b < big_cap) big[b] = s + g0;
        }
    }
}

// A CTA per listed group start: find the group's end, skip it if sorted,
// else sort it by successive minima through tmp (the free buffer).
template <int NW>
__global__ void __launch_bounds__(256) spread_big_kernel(uint64_t* __restrict__ keys, uint64_t* __restrict__ tmp,
                                                         uint64_t n, int lo, const uint64_t* __restrict__ list,
                                                         uint64_t n_list, ulonglong2* __restrict__ rest,
                                                         unsigned long long* __restrict__ n_rest) {
    __shared__ uint64_t s_end;
    __shared__ uint64_t redk[8 * NW];
    __shared__ uint32_t redh[8];
    __shared__ uint32_t red32[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto top = [&](uint64_t i) { return keys[i * NW + NW - 1] >> lo; };
    for (uint64_t g = blockIdx.x; g < n_list; g += gridDim.x) {
        const uint64_t gs = list[g];
        if (tid == 0) {
            const uint64_t px = top(gs);
            uint64_t l = gs + 1, step = 1, h;
            while (true) {  // first index with other top bits
                const uint64_t probe = l + step - 1;
                if (probe >= n) {
                    h = n;
                    break;
                }
                if (top(probe) != px) {
                    h = probe;
                    break;
                }
                l = probe + 1;
                step <<= 1;
            }
            while (l < h) {
                const uint64_t mid = (l + h) / 2;
                if (top(mid) == px) l = mid + 1; else h = mid;
            }
            s_end = l;
        }
        __syncthreads();
        const uint64_t ge = s_end;
        // sorted already?
        uint32_t d = 0;
        for (uint64_t i = gs + 1 + tid; i < ge; i += 256)
            d |= key_less<NW>(load_key<NW>(keys, i), load_key<NW>(keys, i - 1));
        d = __syncthreads_or(d);
        if (!d) continue;
        uint64_t pos = gs;
        Key<NW> prev = key_zero<NW>();
        bool first = true;
        int rounds = 0;
        while (pos < ge && rounds < kFixBlockRounds) {
            Key<NW> mn = key_ones<NW>();
            bool have = false;
            for (uint64_t i = gs + tid; i < ge; i += 256) {
                const Key<NW> x = load_key<NW>(keys, i);
                if ((first || key_less<NW>(prev, x)) && (!have || key_less<NW>(x, mn))) {
                    mn = x;
                    have = true;
                }
            }
            for (int off = 16; off; off >>= 1) {
                const Key<NW> o = shfl_key<NW>(mn, off);
                const bool oh = __shfl_xor_sync(0xFFFFFFFFu, have, off);
                if (oh && (!have || key_less<NW>(o, mn))) {
                    mn = o;
                    have = true;
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int w = 0; w < NW; w++) redk[warp * NW + w] = mn.w[w];
                redh[warp] = have;
            }
            __syncthreads();
            have = false;
            for (int wv = 0; wv < 8; wv++) {
                Key<NW> o;
#pragma unroll
                for (int w = 0; w < NW; w++) o.w[w] = redk[wv * NW + w];
                if (redh[wv] && (!have || key_less<NW>(o, mn))) {
                    mn = o;
                    have = true;
                }
            }
            uint32_t c = 0;
            for (uint64_t i = gs + tid; i < ge; i += 256) c += key_eq<NW>(load_key<NW>(keys, i), mn);
            for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
            __syncthreads();
            if (lane == 0) red32[warp] = c;
            __syncthreads();
            c = 0;
            for (int w = 0; w < 8; w++) c += red32[w];
            for (uint64_t i = tid; i < c; i += 256) store_key<NW>(tmp, pos + i, mn);
            pos += c;
            prev = mn;
            first = false;
            rounds++;
            __syncthreads();
        }
        if (pos < ge) {
            if (tid == 0) rest[atomicAdd(n_rest, 1ull)] = make_ulonglong2(gs, ge);
        } else {
            for (uint64_t i = gs * NW + tid; i < ge * NW; i += 256) keys[i] = tmp[i];
        }
        __syncthreads();
    }
}

// a and b agree on every bit at or above bit lo of the whole key (bit 0 the
// lowest bit of word 0).
template <int NW>
__device__ __forceinline__ bool same_above(const Key<NW>& a, const Key<NW>& b, int lo) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const int b0 = 64 * w;
        if (lo >= b0 + 64) continue;
        const uint64_t x = a.w[w] ^ b.w[w];
        eq &= (lo <= b0) ? x == 0 : (x >> (lo - b0)) == 0;
    }
    return eq;
}

// Key-value fix-up (keys with a 32-bit payload): groups of up to 16 keys
// are sorted by one thread each, pairs moving together; larger groups inside
// the window by one warp (successive minima: each round writes every copy
// of the smallest key above the previous one with its payloads); groups that
// run past the window or hold more than 64 distinct keys go to a list, each
// listed group then to a segment sort of its own (few, for spread keys).
template <int NW>
__global__ void __launch_bounds__(256) spread_fix_kv_kernel(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                            uint64_t n, int lo, uint64_t* __restrict__ big,
                                                            uint64_t big_cap, unsigned long long* __restrict__ n_big) {
    using F = Fix<NW>;
    __shared__ uint64_t K[F::kWin * NW];
    __shared__ uint32_t V[F::kWin];
    __shared__ uint32_t head[F::kWords], desc[F::kWords];
    __shared__ uint32_t queue[2 * F::kQueue];  // (start, end) of the groups for warps
    __shared__ uint32_t n_queue;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t s = blockIdx.x * (uint64_t)F::kTile;
    const uint32_t W = (uint32_t)(n - s < (uint64_t)F::kWin ? n - s : (uint64_t)F::kWin);
    const uint32_t len = W < (uint32_t)F::kTile ? W : (uint32_t)F::kTile;
    const bool window_ends_array = s + W == n;
    auto kget = [&](uint32_t i) {
        Key<NW> r;
#pragma unroll
        for (int w = 0; w < NW; w++) r.w[w] = K[i * NW + w];
        return r;
    };
    auto kset = [&](uint32_t i, const Key<NW>& x) {
#pragma unroll
        for (int w = 0; w < NW; w++) K[i * NW + w] = x.w[w];
    };
    for (uint32_t i = tid; i < W * NW; i += 256) K[i] = keys[s * NW + i];
    for (uint32_t i = tid; i < W; i += 256) V[i] = vals[s + i];
    if (tid == 0) n_queue = 0;
    __syncthreads();
    for (uint32_t wd = warp; wd < (uint32_t)F::kWords; wd += 8) {
        const uint32_t i = wd * 32 + lane;
        bool h = false, d = false;
        if (i < W) {
            const Key<NW> x = kget(i);
            const Key<NW> y = i > 0 ? kget(i - 1) : (s > 0 ? load_key<NW>(keys, s - 1) : key_ones<NW>());
            h = i == 0 && s == 0 ? true : !same_above<NW>(x, y, lo);
            d = i > 0 && !h && key_less<NW>(x, y);
        }
        const uint32_t hb = __ballot_sync(0xFFFFFFFFu, h), db = __ballot_sync(0xFFFFFFFFu, d);
        if (lane == 0) {
            head[wd] = hb;
            desc[wd] = db;
        }
    }
    __syncthreads();
    // groups found from their first descent, as in spread_fix_kernel
    auto to_big = [&](uint32_t h) {
        const unsigned long long q = atomicAdd(n_big, 1ull);
        if (q < big_cap) big[q] = s + h;
    };
    if (tid == 0 && !window_ends_array) {
        const uint32_t h = prev_bit(head, len - 1);
        if (h != ~0u && next_bit(head, h + 1, W) == W && !any_bit(desc, h + 1, W)) to_big(h);
    }
    for (uint32_t wd = tid; wd < (uint32_t)F::kWords; wd += 256) {
        uint32_t dm = desc[wd];
        while (dm) {
            const uint32_t jd = wd * 32 + __ffs(dm) - 1;
            dm &= dm - 1;
            const uint32_t h = prev_bit(head, jd);
            if (h == ~0u || h >= len) continue;
            if (any_bit(desc, h + 1, jd)) continue;
            const uint32_t g1 = next_bit(head, jd + 1, W);
            if (g1 == W && !window_ends_array) {
                to_big(h);
                continue;
            }
            if (g1 - h > (uint32_t)F::kThreadSort) {
                const uint32_t q = atomicAdd(&n_queue, 1u);
                queue[2 * q] = h;
                queue[2 * q + 1] = g1;
                continue;
            }
            for (uint32_t j = h + 1; j < g1; j++) {
                const Key<NW> x = kget(j);
                const uint32_t v = V[j];
                uint32_t i = j;
                while (i > h && key_less<NW>(x, kget(i - 1))) {
                    kset(i, kget(i - 1));
                    V[i] = V[i - 1];
                    i--;
                }
                kset(i, x);
                V[i] = v;
            }
            for (uint32_t j = h; j < g1; j++) {
                store_key<NW>(keys, s + j, kget(j));
                vals[s + j] = V[j];
            }
        }
    }
    __syncthreads();
    // larger groups: a warp each, from K and V to keys and vals
    const uint32_t nq = n_queue;
    for (uint32_t q = warp; q < nq; q += 8) {
        const uint32_t g0 = queue[2 * q], g1 = queue[2 * q + 1];
        uint32_t pos = g0;
        Key<NW> prev = key_zero<NW>();
        bool first = true;
        int rounds = 0;
        while (pos < g1 && rounds < kFixWarpRounds) {
            Key<NW> mn = key_ones<NW>();
            bool have = false;
            for (uint32_t i = g0 + lane; i < g1; i += 32) {
                const Key<NW> x = kget(i);
                if ((first || key_less<NW>(prev, x)) && (!have || key_less<NW>(x, mn))) {
                    mn = x;
                    have = true;
                }
            }
            for (int off = 16; off; off >>= 1) {
                const Key<NW> o = shfl_key<NW>(mn, off);
                const bool oh = __shfl_xor_sync(0xFFFFFFFFu, have, off);
                if (oh && (!have || key_less<NW>(o, mn))) {
                    mn = o;
                    have = true;
                }
            }
            // every copy of mn, with its payload, in group order
            for (uint32_t b0 = g0; b0 < g1; b0 += 32) {
                const uint32_t i = b0 + lane;
                const bool eq = i < g1 && key_eq<NW>(kget(i), mn);
                const uint32_t m = __ballot_sync(0xFFFFFFFFu, eq);
                if (eq) {
                    const uint32_t o = pos + __popc(m & ((1u << lane) - 1u));
                    store_key<NW>(keys, s + o, mn);
                    vals[s + o] = V[i];
                }
                pos += __popc(m);
            }
            prev = mn;
            first = false;
            rounds++;
        }
        __syncwarp();
        if (pos < g1) {
            // too many distinct keys: rewrite the group as it was and defer it
            for (uint32_t i = g0 + lane; i < g1; i += 32) {
                store_key<NW>(keys, s + i, kget(i));
                vals[s + i] = V[i];
            }
            if (lane == 0) to_big(g0);
        }
    }
}

// A CTA per listed group start: the group's end (the first key differing at
// or above bit lo), and (start, end) out if the group holds a descent.
template <int NW>
__global__ void __launch_bounds__(256) spread_bounds_kernel(const uint64_t* __restrict__ keys, uint64_t n, int lo,
                                                            const uint64_t* __restrict__ list, uint64_t n_list,
                                                            ulonglong2* __restrict__ rest,
                                                            unsigned long long* __restrict__ n_rest) {
    __shared__ uint64_t s_end;
    const int tid = threadIdx.x;
    for (uint64_t g = blockIdx.x; g < n_list; g += gridDim.x) {
        const uint64_t gs = list[g];
        if (tid == 0) {
            const Key<NW> px = load_key<NW>(keys, gs);
            uint64_t l = gs + 1, step = 1, h;
            while (true) {
                const uint64_t probe = l + step - 1;
                if (probe >= n) {
                    h = n;
                    break;
                }
                if (!same_above<NW>(load_key<NW>(keys, probe), px, lo)) {
                    h = probe;
                    break;
                }
                l = probe + 1;
                step <<= 1;
            }
            while (l < h) {
                const uint64_t mid = (l + h) / 2;
                if (same_above<NW>(load_key<NW>(keys, mid), px, lo)) l = mid + 1; else h = mid;
            }
            s_end = l;
        }
        __syncthreads();
        const uint64_t ge = s_end;
        uint32_t d = 0;
        for (uint64_t i = gs + 1 + tid; i < ge; i += 256)
            d |= key_less<NW>(load_key<NW>(keys, i), load_key<NW>(keys, i - 1));
        d = __syncthreads_or(d);
        if (d && tid == 0) rest[atomicAdd(n_rest, 1ull)] = make_ulonglong2(gs, ge);
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
    return forced ? forced : std::max(8, ((ceil_log2(n) + 7) / 8) * 8);
}

// The count sort's spread bits: the default moved by the context's plan
// (a multiple of 8, kept in [8, 64]).
int spread_pass_bits(mh_ctx* ctx, uint64_t n) {
    const int P = spread_bits(n) + (ctx ? ctx->spread_bits_delta : 0);
    return std::min(64, std::max(8, P / 8 * 8));
}

template <int NW>
bool radix_sort_spread(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint64_t n, int skip, const uint32_t* hist) {
    using F = Fix<NW>;
    const int P = spread_pass_bits(ctx, n);
    const int bits = 64 * NW;
    if (n <= 1 || P + skip >= 64) return radix_sort<NW>(ctx, keys, alt, nullptr, nullptr, n, 0, bits - skip);
    // the top `skip` bits are equal in every key: passes over the P bits below
    const int lo = 64 - skip - P;  // within the top word
    const bool in_alt = radix_sort<NW>(ctx, keys, alt, nullptr, nullptr, n, bits - skip - P, bits - skip, hist);
    uint64_t* k = in_alt ? alt : keys;
    uint64_t* other = in_alt ? keys : alt;
    const uint64_t cap = std::max<uint64_t>(1 << 16, n / 64);
    Buf<uint64_t> list(ctx, cap), cnt(ctx, 2);
    cnt.zero();
    MH_LAUNCH_B(ctx, "spread_fixup", n * 8 * NW, (unsigned)ceil_div(n, F::kTile), 256, 0, spread_fix_kernel<NW>, k,
                n, lo, list.p, cap, (unsigned long long*)cnt.p);
    uint64_t n_big = 0;
    read_u64(ctx, cnt.p, &n_big, 1);
    if (n_big > cap) {
        // far more long or crowded groups than evenly spread keys give: sort fully
        return in_alt != radix_sort<NW>(ctx, k, other, nullptr, nullptr, n, 0, bits - skip);
    }
    if (n_big) {
        Buf<ulonglong2> rest(ctx, n_big);
        MH_LAUNCH(ctx, "spread_fixup_big", (unsigned)std::min<uint64_t>(n_big, (uint64_t)ctx->num_sms * 8), 256, 0,
                  spread_big_kernel<NW>, k, other, n, lo, list.p, n_big, rest.p, (unsigned long long*)(cnt.p + 1));
        uint64_t n_rest = 0;
        read_u64(ctx, cnt.p + 1, &n_rest, 1);
        if (n_rest) {
            std::vector<ulonglong2> h(n_rest);
            MH_CUDA(cudaMemcpyAsync(h.data(), rest.p, sizeof(ulonglong2) * n_rest, cudaMemcpyDeviceToHost,
                                    ctx->stream));
            sync_and_check(ctx);
            for (const ulonglong2& seg : h) {
                const uint64_t len = seg.y - seg.x;
                if (radix_sort<NW>(ctx, k + seg.x * NW, other + seg.x * NW, nullptr, nullptr, len, 0,
                                   bits - skip - P))
                    MH_CUDA(cudaMemcpyAsync(k + seg.x * NW, other + seg.x * NW, len * 8 * NW, cudaMemcpyDeviceToDevice,
                                            ctx->stream));
            }
        }
    }
    return in_alt;
}

// Distinct keys with a 32-bit payload (a solid table and its counts): the
// same spread order (passes over the top P bits of the top word below
// `skip` constant bits, then the key-value fix-up).  Keys whose top bits are
// crowded (more than 256 groups past the thread sorts) are sorted fully.
// Returns true when the result is in alt / valt.
template <int NW>
bool radix_sort_spread_kv(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                          int skip) {
    using F = Fix<NW>;
    const int P = spread_bits(n);
    const int bits = 64 * NW;
    // small tables (below 2^20 keys, or MH_SPREAD_KV_MIN for tests): the full
    // sort, which needs no read-back of the fix-up's list
    static const uint64_t kv_min = [] {
        const char* e = std::getenv("MH_SPREAD_KV_MIN");
        return e ? (uint64_t)std::strtoull(e, nullptr, 10) : (uint64_t)1 << 20;
    }();
    if (n < std::max<uint64_t>(kv_min, 2) || P + skip >= bits)
        return radix_sort<NW>(ctx, keys, alt, vals, valt, n, 0, bits - skip);
    const int lo = bits - skip - P;  // groups: keys equal at and above bit lo of the whole key
    const bool in_alt = radix_sort<NW>(ctx, keys, alt, vals, valt, n, bits - skip - P, bits - skip);
    uint64_t* k = in_alt ? alt : keys;
    uint64_t* ko = in_alt ? keys : alt;
    uint32_t* v = in_alt ? valt : vals;
    uint32_t* vo = in_alt ? vals : valt;
    constexpr uint64_t kMaxSegments = 256;
    Buf<uint64_t> list(ctx, kMaxSegments), cnt(ctx, 2);
    cnt.zero();
    MH_LAUNCH_B(ctx, "spread_fixup_kv", n * (8 * NW + 4), (unsigned)ceil_div(n, F::kTile), 256, 0,
                spread_fix_kv_kernel<NW>, k, v, n, lo, list.p, kMaxSegments, (unsigned long long*)cnt.p);
    uint64_t n_big = 0;
    read_u64(ctx, cnt.p, &n_big, 1);
    if (n_big > kMaxSegments) return in_alt != radix_sort<NW>(ctx, k, ko, v, vo, n, 0, bits - skip);
    if (!n_big) return in_alt;
    Buf<ulonglong2> rest(ctx, n_big);
    MH_LAUNCH(ctx, "spread_bounds", (unsigned)n_big, 256, 0, spread_bounds_kernel<NW>, k, n, lo, list.p, n_big,
              rest.p, (unsigned long long*)(cnt.p + 1));
    uint64_t n_rest = 0;
    read_u64(ctx, cnt.p + 1, &n_rest, 1);
    if (!n_rest) return in_alt;
    std::vector<ulonglong2> h(n_rest);
    MH_CUDA(cudaMemcpyAsync(h.data(), rest.p, sizeof(ulonglong2) * n_rest, cudaMemcpyDeviceToHost, ctx->stream));
    sync_and_check(ctx);
    for (const ulonglong2& seg : h) {
        const uint64_t len = seg.y - seg.x;
        if (radix_sort<NW>(ctx, k + seg.x * NW, ko + seg.x * NW, v + seg.x, vo + seg.x, len, 0, bits - skip - P)) {
            MH_CUDA(cudaMemcpyAsync(k + seg.x * NW, ko + seg.x * NW, len * 8 * NW, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
            MH_CUDA(cudaMemcpyAsync(v + seg.x, vo + seg.x, len * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    return in_alt;
}

template bool radix_sort_spread_kv<1>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int);
template bool radix_sort_spread_kv<2>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int);
template bool radix_sort_spread_kv<4>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, uint64_t, int);

template bool radix_sort_spread<1>(mh_ctx*, uint64_t*, uint64_t*, uint64_t, int, const uint32_t*);
template bool radix_sort_spread<2>(mh_ctx*, uint64_t*, uint64_t*, uint64_t, int, const uint32_t*);
template bool radix_sort_spread<4>(mh_ctx*, uint64_t*, uint64_t*, uint64_t, int, const uint32_t*);

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

// Each thread scans its own run of kScanItems consecutive inputs in
// registers (read and written straight from and to global memory: a warp's
// runs are one contiguous span), then the block adds the runs' prefixes.
template <class T>
__global__ void scan_down_kernel(const T* __restrict__ in, uint64_t n, const uint64_t* __restrict__ offs,
                                 uint64_t* __restrict__ out) {
    __shared__ uint64_t ws[kScanThreads / 32];
    const uint64_t b = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t loc[kScanItems];
    uint64_t t = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        loc[j] = t;
        t += b + j < n ? (uint64_t)in[b + j] : 0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = t;
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += ws[w];
    const uint64_t pre = offs[blockIdx.x] + wpre + x - t;
#pragma unroll
    for (int j = 0; j < kScanItems; j++)
        if (b + j < n) out[b + j] = pre + loc[j];
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
