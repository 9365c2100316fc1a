// Unit counting: the sort-and-count of mh_count_kmers (paper, Sec. 2, third
// paragraph: every (k+1)-mer on both strands sorted and counted, those seen
// at least d times solid), for keys of 1, 2 or 4 words.  A key of NW words
// is stored as NW consecutive words, the top word last; its mix_key image
// spreads every word into the top word's top bits, which the passes and
// the units use.
//
// The canonical keys are mix_key images, so their top bits are evenly
// spread.  LSD passes of 8-bit digits sort them by their top 8 * passes bits
// only; that leaves every "unit" (the keys sharing their top unit_bits <=
// 8 * passes bits, about 100-200 keys) contiguous.  One warp then finishes a
// unit, with no block-wide barrier:
//
//   find      the warp streams over a tile of the sorted keys through a
//             window of 512 / NW keys in its shared memory (filled by
//             asynchronous copies, one round trip for several units) and
//             finds the units
//             that start in the tile (a unit id is the key's top bits; the
//             tile's last unit may run past its end)
//   bucket    a counting sort from the window into the warp's sort buffer by
//             the next 8 bits (256 sub-buckets; equal keys share a
//             sub-bucket, so stability is not needed)
//   fix       sub-buckets holding a descent (two or more distinct keys) are
//             flagged and sorted by the warp: up to 32 keys by counting, for
//             each key, the keys that go before it; larger ones by listing
//             their distinct keys and multiplicities (successive minima), then
//             writing them out
//   runs      run heads listed in order, a lane per run: the literal count
//             (run length, doubled for a palindrome), the solid filter
//   output    the spectrum (every run's mixed key and length) and the kept
//             runs' key and reverse complement with the count go to the
//             unit's own slots (a unit has no more runs, and with d >= 2 no
//             more kept outputs, than keys), compacted afterwards in unit
//             order; the solid table is then sorted.
//
// A unit of more than 512 / NW keys (keys of very high multiplicity, or
// many error k-mers in one unit) is counted
// straight from global memory by successive minima: each round the smallest
// key above the previous one and its multiplicity, one run.  A unit with
// more than 64 distinct keys as well, or a sub-bucket of more than 32 keys
// with more than 32 distinct ones (neither is met with mixed keys, but both
// are possible for skewed input), is set aside: it is sorted afterwards by
// the general radix sort and its runs counted from the sorted keys.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "mh_internal.cuh"

namespace mh {

namespace {

constexpr int kSubBits = 8;
constexpr int kSubBuckets = 1 << kSubBits;
constexpr uint32_t kTileKeys = 4096;          // keys a warp's tile holds
constexpr uint64_t kMaxRounds = 64;           // runs of a large unit counted from global memory

// Per key width: the keys a warp sorts on chip (its window and its sort
// buffer each hold that many: 4 KB a buffer; wider keys' units, richer in
// error k-mers, overflow it more often and are then set aside and sorted
// together), the warps a CTA, the keys an average unit aims at, and the
// most an average unit may hold when that saves a pass.
template <int NW>
struct UnitCfg {
    static constexpr int kCap = 512 / NW;
    static constexpr int kWarps = 8;
    static constexpr int kThreads = 32 * kWarps;
    static constexpr uint64_t kTarget = NW == 1 ? 160 : NW == 2 ? 96 : 56;
    static constexpr uint64_t kMax = NW == 1 ? 256 : NW == 2 ? 160 : 96;
    // per-warp shared memory (bytes): window, sort buffer, sub-bucket
    // counts (then run heads), flags of the sub-buckets to sort
    static constexpr size_t kWWin = 0;
    static constexpr size_t kWK = kWWin + sizeof(uint64_t) * NW * kCap;
    static constexpr size_t kWCnt = kWK + sizeof(uint64_t) * NW * kCap;
    static constexpr size_t kWDb = kWCnt + sizeof(uint32_t) * kSubBuckets;
    static constexpr size_t kWarpSmem = kWDb + sizeof(uint32_t) * (kSubBuckets / 32);
    static constexpr size_t kSmem = kWarpSmem * kWarps;
    static_assert(sizeof(uint32_t) * kSubBuckets >= sizeof(uint16_t) * kCap, "run heads fit over the counts");
    static_assert(kWarpSmem % 16 == 0, "16-byte aligned warp areas");
};
constexpr int kWarpCapMax = 512;

template <int NW>
__device__ __forceinline__ Key<NW> shfl_key(const Key<NW>& a, int src) {
    Key<NW> r;
#pragma unroll
    for (int w = 0; w < NW; w++) r.w[w] = __shfl_sync(0xFFFFFFFFu, a.w[w], src);
    return r;
}

template <int NW>
__device__ __forceinline__ Key<NW> shfl_xor_key(const Key<NW>& a, int m) {
    Key<NW> r;
#pragma unroll
    for (int w = 0; w < NW; w++) r.w[w] = __shfl_xor_sync(0xFFFFFFFFu, a.w[w], m);
    return r;
}

template <int NW>
__device__ __forceinline__ Key<NW> key_max() {
    Key<NW> r;
#pragma unroll
    for (int w = 0; w < NW; w++) r.w[w] = ~0ull;
    return r;
}

// The sub-bucket bits and the unit bits lie in the top word.
template <int NW>
__device__ __forceinline__ uint64_t top_word(const Key<NW>& x) {
    return x.w[NW - 1];
}

// Sorts K[g0, g1) (g1 - g0 >= 2) by one warp.  Up to 32 keys: each lane
// holds one and counts the keys that go before it (smaller, or equal and
// earlier).  Larger: the distinct keys are listed with their multiplicities
// by successive minima (reads only), then written out in order.  Returns
// false, with K unchanged, for more than 32 distinct keys in more than 32.
template <int NW>
__device__ __forceinline__ bool warp_sort(uint64_t* K, uint32_t g0, uint32_t g1) {
    const int lane = threadIdx.x & 31;
    const uint32_t size = g1 - g0;
    if (size <= 32) {
        const bool have = (uint32_t)lane < size;
        const Key<NW> x = have ? load_key<NW>(K, g0 + lane) : Key<NW>{};
        uint32_t r = 0;
        for (uint32_t j = 0; j < size; j++) {
            const Key<NW> y = shfl_key<NW>(x, (int)j);
            r += key_less<NW>(y, x) || (key_eq<NW>(y, x) && j < (uint32_t)lane);
        }
        __syncwarp();
        if (have) store_key<NW>(K, g0 + r, x);
        __syncwarp();
        return true;
    }
    Key<NW> val{}, prev{};
    uint32_t vcnt = 0, got = 0;
    int rounds = 0;
    while (got < size && rounds < 32) {
        Key<NW> mn = key_max<NW>();
        for (uint32_t j = g0 + lane; j < g1; j += 32) {
            const Key<NW> x = load_key<NW>(K, j);
            if ((rounds == 0 || key_less<NW>(prev, x)) && key_less<NW>(x, mn)) mn = x;
        }
        for (int off = 16; off; off >>= 1) {
            const Key<NW> o = shfl_xor_key<NW>(mn, off);
            mn = key_less<NW>(o, mn) ? o : mn;
        }
        uint32_t c = 0;
        for (uint32_t j = g0 + lane; j < g1; j += 32) c += key_eq<NW>(load_key<NW>(K, j), mn);
        for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
        if (lane == rounds) {
            val = mn;
            vcnt = c;
        }
        got += c;
        prev = mn;
        rounds++;
    }
    __syncwarp();
    if (got < size) return false;
    uint32_t at = g0;
    for (int r = 0; r < rounds; r++) {
        const Key<NW> v = shfl_key<NW>(val, r);
        const uint32_t c = __shfl_sync(0xFFFFFFFFu, vcnt, r);
        for (uint32_t i = lane; i < c; i += 32) store_key<NW>(K, at + i, v);
        at += c;
    }
    __syncwarp();
    return true;
}

// Window fill: keys[from, from + min(cap, n - from)) into the warp's
// window by asynchronous copies of 8 or 16 bytes (no registers held), then
// waited for.
template <int NW>
__device__ __forceinline__ uint32_t fill_window(uint64_t* win, const uint64_t* keys, uint64_t n, uint64_t from) {
    constexpr int kWin = UnitCfg<NW>::kCap;
    const int lane = threadIdx.x & 31;
    const uint32_t len = (uint32_t)(n - from < (uint64_t)kWin ? n - from : (uint64_t)kWin);
    if constexpr (NW == 1) {
        for (uint32_t i = lane; i < len; i += 32) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(win + i);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(keys + from + i) : "memory");
        }
    } else {
        // 16-byte pieces: NW / 2 a key
        const uint32_t pieces = len * (NW / 2);
        const uint64_t* src = keys + from * NW;
        for (uint32_t i = lane; i < pieces; i += 32) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(win + 2 * i);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + 2 * i) : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    return len;
}

// Unit id of a key: bits [lo, lo + unit_bits) of its top word (0 for a
// single unit).
template <int NW>
__device__ __forceinline__ uint32_t unit_of(const Key<NW>& x, int lo, uint32_t umask) {
    return umask ? (uint32_t)(top_word<NW>(x) >> lo) & umask : 0u;
}

template <int NW>
__device__ __forceinline__ uint32_t sub_of(const Key<NW>& x, int sb_shift) {
    return (uint32_t)(top_word<NW>(x) >> sb_shift) & (kSubBuckets - 1);
}

// What a run (mixed key x, length len) gives: its real key, literal count
// (length, doubled for a palindrome) and number of solid outputs.
template <int NW>
struct RunOut {
    Key<NW> c;
    uint32_t count;
    uint32_t nout;
    bool palin;
};

template <int NW>
__device__ __forceinline__ RunOut<NW> run_out(const Key<NW>& x, uint64_t len, int K1, int d, uint32_t* err) {
    RunOut<NW> o;
    o.c = unmix_key<NW>(x);
    o.palin = key_eq<NW>(key_rc<NW>(o.c, K1), o.c);
    uint64_t count = o.palin ? 2 * len : len;
    if (count > 0xFFFFFFFFull) {
        atomicOr(err, ST_OVERFLOW);
        count = 0xFFFFFFFFull;
    }
    o.count = (uint32_t)count;
    o.nout = count >= (uint64_t)d ? (o.palin ? 1u : 2u) : 0u;
    return o;
}

// The solid outputs of one run at index `at`: its key and, unless it is a
// palindrome, its reverse complement, each with the count.
template <int NW>
__device__ __forceinline__ void put_solid(uint64_t* solid_k, uint32_t* solid_c, uint64_t at, const RunOut<NW>& o,
                                          int K1) {
    store_key<NW>(solid_k, at, o.c);
    solid_c[at] = o.count;
    if (o.nout == 2) {
        store_key<NW>(solid_k, at + 1, key_rc<NW>(o.c, K1));
        solid_c[at + 1] = o.count;
    }
}

}  // namespace

// Warps over tiles of kTileKeys sorted keys; every unit that starts in a
// warp's tile is counted by that warp.  Unit [us, ue): spectrum entries at
// spec_k / spec_len [us + r], solid outputs at solid_k / solid_c [so0 + i]
// with so0 = us (d >= 2) or 2 us (d = 1); its start, run and output counts
// at ustart / ucount / scount [its unit id].  totals[0] += palindromic runs.
template <int NW>
__global__ void __launch_bounds__(UnitCfg<NW>::kThreads, 3)
    unit_count_kernel(const uint64_t* __restrict__ keys, uint64_t n, int lo, uint32_t umask, int sb_shift, int K1,
                      int d, uint32_t cap, uint64_t* __restrict__ spec_k, uint32_t* __restrict__ spec_len,
                      uint64_t* __restrict__ solid_k, uint32_t* __restrict__ solid_c,
                      uint64_t* __restrict__ ustart, uint32_t* __restrict__ ucount,
                      uint32_t* __restrict__ scount, ulonglong2* __restrict__ deferred,
                      unsigned long long* __restrict__ totals, uint32_t* __restrict__ err) {
    using C = UnitCfg<NW>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* ws = smem + C::kWarpSmem * wib;
    uint64_t* Wb = reinterpret_cast<uint64_t*>(ws + C::kWWin);
    uint64_t* K = reinterpret_cast<uint64_t*>(ws + C::kWK);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(ws + C::kWCnt);
    uint32_t* db = reinterpret_cast<uint32_t*>(ws + C::kWDb);
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t n_tiles = ceil_div(n, kTileKeys);
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t palins = 0;

    for (uint64_t t = gwarp; t < n_tiles; t += n_warps) {
        const uint64_t t0 = t * kTileKeys, t1 = t0 + kTileKeys < n ? t0 + kTileKeys : n;
        // the window holds keys [wbase, wbase + wlen)
        uint64_t wbase = t0 > 0 ? t0 - 1 : 0;
        uint32_t wlen = fill_window<NW>(Wb, keys, n, wbase);
        // first unit start at or after t0
        uint64_t pos = t0;
        if (t0 > 0) {
            const uint32_t before = unit_of<NW>(load_key<NW>(Wb, 0), lo, umask);
            pos = t1;
            while (true) {
                uint32_t found = wlen;
                for (uint32_t c = 0; c < wlen; c += 32) {
                    const uint32_t i = c + lane;
                    const bool h =
                        i < wlen && wbase + i >= t0 && unit_of<NW>(load_key<NW>(Wb, i), lo, umask) != before;
                    const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
                    if (b) {
                        found = c + __ffs(b) - 1;
                        break;
                    }
                }
                if (found < wlen) {
                    pos = wbase + found;
                    break;
                }
                if (wbase + wlen >= t1) break;  // no unit starts in the tile
                wbase += wlen;
                wlen = fill_window<NW>(Wb, keys, n, wbase);
            }
        }
        while (pos < t1) {
            if (pos >= wbase + wlen) {
                wbase = pos;
                wlen = fill_window<NW>(Wb, keys, n, wbase);
            }
            const uint64_t us = pos;
            uint32_t i0 = (uint32_t)(us - wbase);
            const uint32_t uid = unit_of<NW>(load_key<NW>(Wb, i0), lo, umask);
            // the unit's end inside the window, else refill from its start
            uint64_t ue = 0;
            while (true) {
                uint32_t found = wlen;
                for (uint32_t c = i0 + 1; c < wlen; c += 32) {
                    const uint32_t i = c + lane;
                    const bool h = i < wlen && unit_of<NW>(load_key<NW>(Wb, i), lo, umask) != uid;
                    const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
                    if (b) {
                        found = c + __ffs(b) - 1;
                        break;
                    }
                }
                if (found < wlen) {
                    ue = wbase + found;
                    break;
                }
                if (wbase + wlen >= n) {
                    ue = n;
                    break;
                }
                if (i0 == 0) break;  // longer than the window
                wbase = us;
                wlen = fill_window<NW>(Wb, keys, n, wbase);
                i0 = 0;
            }
            if (ue == 0) {
                // longer than the window: its end from global memory
                ue = wbase + wlen;
                while (ue < n) {
                    const uint64_t j = ue + lane;
                    const bool h = j >= n || unit_of<NW>(load_key<NW>(keys, j), lo, umask) != uid;
                    const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
                    if (b) {
                        ue += __ffs(b) - 1;
                        break;
                    }
                    ue += 32;
                }
                if (ue > n) ue = n;
            }
            pos = ue;
            const uint64_t m64 = ue - us;
            const uint64_t so0 = d >= 2 ? us : 2 * us;
            if (m64 > cap) {
                // ---- from global memory, one run a round (at most kMaxRounds)
                Key<NW> prev{};
                uint64_t got = 0, r = 0, so = 0, pal = 0;
                while (got < m64 && r < kMaxRounds) {
                    Key<NW> mn = key_max<NW>();
                    for (uint64_t j = us + lane; j < ue; j += 32) {
                        const Key<NW> x = load_key<NW>(keys, j);
                        if ((r == 0 || key_less<NW>(prev, x)) && key_less<NW>(x, mn)) mn = x;
                    }
                    for (int off = 16; off; off >>= 1) {
                        const Key<NW> o = shfl_xor_key<NW>(mn, off);
                        mn = key_less<NW>(o, mn) ? o : mn;
                    }
                    uint64_t c = 0;
                    for (uint64_t j = us + lane; j < ue; j += 32) c += key_eq<NW>(load_key<NW>(keys, j), mn);
                    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
                    const RunOut<NW> o = run_out<NW>(mn, c, K1, d, err);
                    if (lane == 0) {
                        store_key<NW>(spec_k, us + r, mn);
                        spec_len[us + r] = (uint32_t)(c < 0xFFFFFFFFull ? c : 0xFFFFFFFFull);
                        if (o.nout) put_solid<NW>(solid_k, solid_c, so0 + so, o, K1);
                        pal += o.palin;
                    }
                    so += o.nout;
                    got += c;
                    prev = mn;
                    r++;
                }
                if (lane == 0) {
                    if (got < m64) {
                        // too many distinct keys: sorted and counted afterwards
                        // (its slots are rewritten then)
                        deferred[atomicAdd(&totals[1], 1ull)] = make_ulonglong2(us, ue);
                    } else {
                        ustart[uid] = us;
                        ucount[uid] = (uint32_t)r;
                        scount[uid] = (uint32_t)so;
                        palins += pal;
                    }
                }
                continue;
            }
            // ---- on chip: counting sort by the next 8 bits
            const uint32_t m = (uint32_t)m64;
#pragma unroll
            for (int i = 0; i < kSubBuckets / 32; i++) cnt[lane + 32 * i] = 0;
            __syncwarp();
            const uint64_t* U = Wb + (size_t)i0 * NW;  // the unit, in the window
            for (uint32_t j = lane; j < m; j += 32) atomicAdd(&cnt[sub_of<NW>(load_key<NW>(U, j), sb_shift)], 1u);
            __syncwarp();
            {
                // exclusive scan of the 256 counts, 8 a lane
                constexpr int per = kSubBuckets / 32;
                uint32_t v[per], s = 0;
#pragma unroll
                for (int q = 0; q < per; q++) {
                    v[q] = cnt[per * lane + q];
                    s += v[q];
                }
                uint32_t x = s;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
                    if (lane >= off) x += y;
                }
                uint32_t e = x - s;
#pragma unroll
                for (int q = 0; q < per; q++) {
                    cnt[per * lane + q] = e;
                    e += v[q];
                }
            }
            __syncwarp();
            for (uint32_t j = lane; j < m; j += 32) {
                const Key<NW> x = load_key<NW>(U, j);
                store_key<NW>(K, atomicAdd(&cnt[sub_of<NW>(x, sb_shift)], 1u), x);
            }
            __syncwarp();
            // sub-buckets holding a descent, flagged by id (256 bits in db),
            // then each sorted by the warp over its range from the counting
            // sort's offsets (cnt[b] is now the end of sub-bucket b)
            const uint32_t nwords = (m + 31) / 32;
            if (lane < kSubBuckets / 32) db[lane] = 0;
            __syncwarp();
            for (uint32_t j = lane + 1; j < m; j += 32) {
                const Key<NW> x = load_key<NW>(K, j), y = load_key<NW>(K, j - 1);
                const uint32_t b = sub_of<NW>(x, sb_shift);
                if (key_less<NW>(x, y) && sub_of<NW>(y, sb_shift) == b) atomicOr(&db[b >> 5], 1u << (b & 31));
            }
            __syncwarp();
            bool sorted_ok = true;
            {
                uint32_t fw = __ballot_sync(0xFFFFFFFFu, lane < kSubBuckets / 32 && db[lane] != 0);
                while (fw && sorted_ok) {
                    const int w = __ffs(fw) - 1;
                    fw &= fw - 1;
                    uint32_t f = db[w];
                    while (f && sorted_ok) {
                        const uint32_t b = 32 * w + __ffs(f) - 1;
                        f &= f - 1;
                        sorted_ok = warp_sort<NW>(K, b ? cnt[b - 1] : 0u, cnt[b]);
                    }
                }
            }
            if (!sorted_ok) {
                // a sub-bucket with more than 32 distinct keys: the unit is
                // sorted and counted afterwards
                if (lane == 0) deferred[atomicAdd(&totals[1], 1ull)] = make_ulonglong2(us, ue);
                __syncwarp();
                continue;
            }
            // runs: their heads listed in order (hp, over the free counts),
            // then a lane per run
            uint16_t* hp = reinterpret_cast<uint16_t*>(cnt);
            uint32_t H = 0;
            for (uint32_t wd = 0; wd < nwords; wd++) {
                const uint32_t j = wd * 32 + lane;
                const bool h = j < m && (j == 0 || !key_eq<NW>(load_key<NW>(K, j), load_key<NW>(K, j - 1)));
                const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
                if (h) hp[H + __popc(b & lt)] = (uint16_t)j;
                H += __popc(b);
            }
            __syncwarp();
            uint32_t r0 = H, so = 0;
            for (uint32_t rb = 0; rb < H; rb += 32) {
                const uint32_t r = rb + lane;
                RunOut<NW> o{};
                if (r < H) {
                    const uint32_t j = hp[r];
                    const uint32_t end = r + 1 < H ? (uint32_t)hp[r + 1] : m;
                    const Key<NW> x = load_key<NW>(K, j);
                    o = run_out<NW>(x, end - j, K1, d, err);
                    store_key<NW>(spec_k, us + r, x);
                    spec_len[us + r] = end - j;
                    palins += o.palin;
                }
                // solid outputs in run order
                uint32_t incl = o.nout;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                    if (lane >= off) incl += y;
                }
                const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                if (o.nout) put_solid<NW>(solid_k, solid_c, so0 + so + incl - o.nout, o, K1);
                so += tot;
            }
            if (lane == 0) {
                ustart[uid] = us;
                ucount[uid] = r0;
                scount[uid] = so;
            }
            __syncwarp();
        }
    }
    for (int off = 16; off; off >>= 1) palins += __shfl_xor_sync(0xFFFFFFFFu, palins, off);
    if (lane == 0 && palins) atomicAdd(&totals[0], (unsigned long long)palins);
}

// x + 1 over all NW words (x below the largest key).
template <int NW>
__device__ __forceinline__ Key<NW> key_next(const Key<NW>& x) {
    Key<NW> r = x;
    bool carry = true;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        r.w[w] = x.w[w] + (carry ? 1ull : 0ull);
        carry = carry && x.w[w] == ~0ull;
    }
    return r;
}

// The set-aside units, each already sorted: a warp per unit streams its keys
// 32 at a time, a lane per run head; the run's end is found by galloping to
// the first larger key.  Slots and counts as in unit_count_kernel.
template <int NW>
__global__ void __launch_bounds__(256)
    sorted_units_kernel(const uint64_t* __restrict__ keys, const ulonglong2* __restrict__ list, uint64_t n_list,
                        int lo, uint32_t umask, int K1, int d, uint64_t* __restrict__ spec_k,
                        uint32_t* __restrict__ spec_len, uint64_t* __restrict__ solid_k,
                        uint32_t* __restrict__ solid_c, uint64_t* __restrict__ ustart,
                        uint32_t* __restrict__ ucount, uint32_t* __restrict__ scount,
                        unsigned long long* __restrict__ totals, uint32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t palins = 0;
    for (uint64_t q = gwarp; q < n_list; q += n_warps) {
        const uint64_t us = list[q].x, ue = list[q].y;
        const uint64_t so0 = d >= 2 ? us : 2 * us;
        uint64_t r0 = 0, so = 0;
        for (uint64_t c0 = us; c0 < ue; c0 += 32) {
            const uint64_t j = c0 + lane;
            bool h = false;
            Key<NW> x{};
            if (j < ue) {
                x = load_key<NW>(keys, j);
                h = j == us || !key_eq<NW>(x, load_key<NW>(keys, j - 1));
            }
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
            RunOut<NW> o{};
            if (h) {
                const bool top = key_eq<NW>(x, key_max<NW>());
                const uint64_t end =
                    top ? ue : j + 1 + gallop_lb<NW>(keys + (j + 1) * NW, ue - j - 1, key_next<NW>(x), 0);
                const uint64_t len = end - j;
                o = run_out<NW>(x, len, K1, d, err);
                const uint64_t r = r0 + __popc(b & lt);
                store_key<NW>(spec_k, us + r, x);
                spec_len[us + r] = (uint32_t)(len < 0xFFFFFFFFull ? len : 0xFFFFFFFFull);
                palins += o.palin;
            }
            uint32_t incl = o.nout;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                if (lane >= off) incl += y;
            }
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (o.nout) put_solid<NW>(solid_k, solid_c, so0 + so + incl - o.nout, o, K1);
            so += tot;
            r0 += __popc(b);
        }
        if (lane == 0) {
            const uint32_t uid = unit_of<NW>(load_key<NW>(keys, us), lo, umask);
            ustart[uid] = us;
            ucount[uid] = (uint32_t)r0;
            scount[uid] = (uint32_t)so;
        }
    }
    for (int off = 16; off; off >>= 1) palins += __shfl_xor_sync(0xFFFFFFFFu, palins, off);
    if (lane == 0 && palins) atomicAdd(&totals[0], (unsigned long long)palins);
}

// The units' slot entries compacted in unit order: unit u (starting at key
// ustart[u]; ucount[u] = scount[u] = 0 for an empty unit) moves ucount[u]
// spectrum entries from its slot to uoff[u] and scount[u] solid entries to
// soff[u].  A warp per unit.
template <int NW>
__global__ void __launch_bounds__(256) unit_compact_kernel(const uint64_t* __restrict__ spec_k,
                                                           const uint32_t* __restrict__ spec_len,
                                                           const uint64_t* __restrict__ solid_k,
                                                           const uint32_t* __restrict__ solid_c,
                                                           const uint64_t* __restrict__ ustart,
                                                           const uint32_t* __restrict__ ucount,
                                                           const uint32_t* __restrict__ scount,
                                                           const uint64_t* __restrict__ uoff,
                                                           const uint64_t* __restrict__ soff, uint64_t n_units, int d,
                                                           uint64_t* __restrict__ out_sk,
                                                           uint32_t* __restrict__ out_sl,
                                                           uint64_t* __restrict__ out_k,
                                                           uint32_t* __restrict__ out_c) {
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = gwarp; u < n_units; u += n_warps) {
        const uint32_t nu = ucount[u], ns = scount[u];
        if (!(nu | ns)) continue;
        const uint64_t us = ustart[u], a = uoff[u], so = soff[u], so0 = d >= 2 ? us : 2 * us;
        for (uint32_t q = lane; q < nu; q += 32) {
            store_key<NW>(out_sk, a + q, load_key<NW>(spec_k, us + q));
            out_sl[a + q] = spec_len[us + q];
        }
        for (uint32_t q = lane; q < ns; q += 32) {
            store_key<NW>(out_k, so + q, load_key<NW>(solid_k, so0 + q));
            out_c[so + q] = solid_c[so0 + q];
        }
    }
}

// The set-aside units between their places in the sorted keys and one
// contiguous buffer: unit q, keys [list[q].x, list[q].y), is at [off[q],
// off[q] + its length) of buf.  A warp per unit.
template <int NW>
__global__ void __launch_bounds__(256) move_units_kernel(uint64_t* __restrict__ keys,
                                                         const ulonglong2* __restrict__ list,
                                                         const uint64_t* __restrict__ off, uint64_t n_list,
                                                         uint64_t* __restrict__ buf, int to_buf) {
    const int lane = threadIdx.x & 31;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = gwarp; q < n_list; q += n_warps) {
        uint64_t* k = keys + list[q].x * NW;
        uint64_t* b = buf + off[q] * NW;
        const uint64_t words = (list[q].y - list[q].x) * NW;
        for (uint64_t t = lane; t < words; t += 32) {
            if (to_buf) b[t] = k[t];
            else k[t] = b[t];
        }
    }
}

// ------------------------------------------------------------------ host

static int env_int(const char* name, int dflt) {
    const char* e = std::getenv(name);
    return e ? std::atoi(e) : dflt;
}

// MH_GROUP_UNIT_BITS (0..30) forces the unit bits; tests use it for one
// unit or many small ones.  Otherwise the fewest bits that leave about
// the key width's target keys a unit, moved by the context's plan.
GroupPlan group_plan(mh_ctx* ctx, uint64_t n, int skip, int nw) {
    static const int forced = env_int("MH_GROUP_UNIT_BITS", -1);
    const uint64_t target = nw == 1 ? UnitCfg<1>::kTarget : nw == 2 ? UnitCfg<2>::kTarget : UnitCfg<4>::kTarget;
    const uint64_t most = nw == 1 ? UnitCfg<1>::kMax : nw == 2 ? UnitCfg<2>::kMax : UnitCfg<4>::kMax;
    GroupPlan p;
    int ub = 0;
    if (forced >= 0 && forced <= 30) {
        ub = forced;
    } else {
        while (ub < 30 && ceil_div(n, 1ull << ub) > target) ub++;
        // one bit past a whole number of passes costs a whole pass: units of
        // up to `most` keys on average are cheaper than that pass
        if (ub % 8 == 1 && ceil_div(n, 1ull << (ub - 1)) <= most) ub--;
        if (ub > 0 && ctx) ub = std::max(1, std::min(30, ub + ctx->unit_bits_delta));
    }
    p.unit_bits = ub;
    p.passes = (ub + 7) / 8;
    if (skip + 8 * p.passes + kSubBits > 64) p.passes = -1;
    return p;
}

// MH_GROUP_CAP (1..512) lowers the most keys a unit is sorted with on chip
// (never above the key width's own most); tests use it to send units
// through the global-memory path.
template <int NW>
static uint32_t group_cap() {
    static const int v = env_int("MH_GROUP_CAP", kWarpCapMax);
    constexpr int most = UnitCfg<NW>::kCap;
    return (uint32_t)(v >= 1 && v <= most ? v : most);
}

template <int NW>
void group_count(mh_ctx* ctx, Buf<uint64_t>& sorted, Buf<uint64_t>& other, uint64_t n, int k, int d, int skip,
                 const GroupPlan& plan, Buf<uint64_t>& out_keys, Buf<uint32_t>& out_cnt, uint64_t* n_out,
                 uint64_t* n_runs, uint64_t* n_palin_runs, RunList* list) {
    using C = UnitCfg<NW>;
    const int K1 = k + 1;
    const int ub = plan.unit_bits;
    const int lo = 64 - skip - ub;  // unit bits [lo, lo + ub) of the top word
    const int sb_shift = lo - kSubBits;
    if (sb_shift < 0) fail(MH_EINVAL, "unit counting: keys too narrow");
    const uint32_t umask = ub ? (uint32_t)((1ull << ub) - 1) : 0u;
    const uint32_t cap = group_cap<NW>();
    // slots: spectrum keys in `other`, lengths, solid outputs; per unit id its
    // start and counts
    const uint64_t n_units = 1ull << ub;
    const uint64_t out_cap = (d >= 2 ? n : 2 * n);
    Buf<uint32_t> spec_len(ctx, n ? n : 1);
    Buf<uint64_t> sk(ctx, (out_cap ? out_cap : 1) * NW);
    Buf<uint32_t> sc(ctx, out_cap ? out_cap : 1);
    Buf<uint64_t> ustart(ctx, n_units);
    Buf<uint32_t> ucount(ctx, n_units), scount(ctx, n_units);
    Buf<uint64_t> totals(ctx, 4);  // palindromic runs, units set aside
    Buf<ulonglong2> deferred(ctx, n / ((uint64_t)cap + 1) + 1);
    ucount.zero();
    scount.zero();
    totals.zero();
    if (n) {
        MH_CUDA(cudaFuncSetAttribute(unit_count_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)C::kSmem));
        int per_sm = 0;
        MH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unit_count_kernel<NW>, C::kThreads,
                                                              C::kSmem));
        const uint64_t tiles = ceil_div(n, kTileKeys);
        const unsigned grid = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>(ceil_div(tiles, C::kWarps), (uint64_t)ctx->num_sms * std::max(1, per_sm)));
        MH_LAUNCH_B(ctx, "unit_count", n * 8 * NW, grid, C::kThreads, C::kSmem, unit_count_kernel<NW>, sorted.p, n,
                    lo, umask, sb_shift, K1, d, cap, other.p, spec_len.p, sk.p, sc.p, ustart.p, ucount.p, scount.p,
                    deferred.p, (unsigned long long*)totals.p, ctx->d_status);
        // units set aside: sorted in place (their slot range of `other` as the
        // second buffer), then counted from the sorted keys
        uint64_t n_def = 0;
        read_u64(ctx, totals.p + 1, &n_def, 1);
        if (n_def) {
            std::vector<ulonglong2> h(n_def);
            MH_CUDA(cudaMemcpyAsync(h.data(), deferred.p, sizeof(ulonglong2) * n_def, cudaMemcpyDeviceToHost,
                                    ctx->stream));
            sync_and_check(ctx);
            // in key order, so that their concatenation is in unit order
            std::sort(h.begin(), h.end(), [](const ulonglong2& a, const ulonglong2& b) { return a.x < b.x; });
            std::vector<uint64_t> off(n_def + 1, 0);
            for (uint64_t q = 0; q < n_def; q++) off[q + 1] = off[q] + (h[q].y - h[q].x);
            const uint64_t total = off[n_def];
            if (n_def > 1 && total <= n / 2) {
                // many units: gathered into one buffer and sorted there at once
                // (their top bits order them by unit, so each comes back to its
                // own range), then moved back
                MH_CUDA(cudaMemcpyAsync(deferred.p, h.data(), sizeof(ulonglong2) * n_def, cudaMemcpyHostToDevice,
                                        ctx->stream));
                Buf<uint64_t> doff(ctx, n_def + 1), g(ctx, total * NW), g2(ctx, total * NW);
                MH_CUDA(cudaMemcpyAsync(doff.p, off.data(), sizeof(uint64_t) * (n_def + 1), cudaMemcpyHostToDevice,
                                        ctx->stream));
                const unsigned mgrid = grid_for(ctx, n_def * 32, 256);
                MH_LAUNCH(ctx, "move_units", mgrid, 256, 0, move_units_kernel<NW>, sorted.p, deferred.p, doff.p,
                          n_def, g.p, 1);
                const bool alt = radix_sort_spread<NW>(ctx, g.p, g2.p, total, skip);
                MH_LAUNCH(ctx, "move_units", mgrid, 256, 0, move_units_kernel<NW>, sorted.p, deferred.p, doff.p,
                          n_def, alt ? g2.p : g.p, 0);
                // the host copies must not be freed before the stream has read them
                sync_and_check(ctx);
            } else {
                for (const ulonglong2& seg : h) {
                    const uint64_t len = seg.y - seg.x;
                    if (radix_sort_spread<NW>(ctx, sorted.p + seg.x * NW, other.p + seg.x * NW, len, skip + ub))
                        MH_CUDA(cudaMemcpyAsync(sorted.p + seg.x * NW, other.p + seg.x * NW, len * 8 * NW,
                                                cudaMemcpyDeviceToDevice, ctx->stream));
                }
            }
            MH_LAUNCH(ctx, "sorted_units", grid_for(ctx, n_def * 32, 256), 256, 0, sorted_units_kernel<NW>, sorted.p,
                      deferred.p, n_def, lo, umask, K1, d, other.p, spec_len.p, sk.p, sc.p, ustart.p, ucount.p,
                      scount.p, (unsigned long long*)totals.p, ctx->d_status);
        }
    }
    // offsets of the units' entries, then the compaction
    Buf<uint64_t> uoff(ctx, n_units + 1), soff(ctx, n_units + 1);
    exclusive_scan_u32(ctx, ucount.p, uoff.p, n_units);
    exclusive_scan_u32(ctx, scount.p, soff.p, n_units);
    uint64_t R = 0, S = 0, pal = 0;
    read_u64(ctx, uoff.p + n_units, &R, 1);
    read_u64(ctx, soff.p + n_units, &S, 1);
    read_u64(ctx, totals.p, &pal, 1);
    sync_and_check(ctx);
    *n_out = S;
    *n_runs = R;
    *n_palin_runs = pal;
    list->n = R;
    list->keys = Buf<uint64_t>(ctx, (R ? R : 1) * NW);
    list->lens = Buf<uint32_t>(ctx, R ? R : 1);
    Buf<uint64_t> keys(ctx, (S ? S : 1) * NW), alt(ctx, (S ? S : 1) * NW);
    Buf<uint32_t> cnt(ctx, S ? S : 1), calt(ctx, S ? S : 1);
    if (n)
        MH_LAUNCH_B(ctx, "unit_compact", (R + S) * (16 * NW + 8), grid_for(ctx, n_units * 32, 256, 8), 256, 0,
                    unit_compact_kernel<NW>, other.p, spec_len.p, sk.p, sc.p, ustart.p, ucount.p, scount.p, uoff.p,
                    soff.p, n_units, d, list->keys.p, list->lens.p, keys.p, cnt.p);
    ustart.reset();
    uoff.reset();
    soff.reset();
    ucount.reset();
    scount.reset();
    spec_len.reset();
    sk.reset();
    sc.reset();
    sorted.reset();
    other.reset();
    // the solid table: S distinct keys with their counts, sorted
    const bool in_alt = radix_sort_spread_kv<NW>(ctx, keys.p, alt.p, cnt.p, calt.p, S, 64 * NW - 2 * K1);
    if (in_alt) {
        out_keys = std::move(alt);
        out_cnt = std::move(calt);
    } else {
        out_keys = std::move(keys);
        out_cnt = std::move(cnt);
    }
}

#define MH_GROUP_COUNT(NW)                                                                                          \
    template void group_count<NW>(mh_ctx*, Buf<uint64_t>&, Buf<uint64_t>&, uint64_t, int, int, int,               \
                                  const GroupPlan&, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*, uint64_t*, uint64_t*, \
                                  RunList*);
MH_GROUP_COUNT(1)
MH_GROUP_COUNT(2)
MH_GROUP_COUNT(4)
#undef MH_GROUP_COUNT

}  // namespace mh
