// Internal declarations of the SdBG construction library (sm_103a).
//
// Keys are multiword integers (Key<NW>, NW = 1, 2, 4 little-endian 64-bit
// words) holding 2-bit symbols, first symbol most significant; see mh.h for
// the layout.  Every kernel runs on the context's stream; every device-side
// wait is bounded and reports through the context's status word.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mh.h"

namespace mh {

// ------------------------------------------------------------ status bits
// Set by kernels with atomicOr on ctx->d_status, checked by the host after
// the call's synchronising copy.
constexpr uint32_t ST_SPIN_TIMEOUT = 1u;  // a bounded look-back wait gave up
constexpr uint32_t ST_OVERFLOW = 2u;      // a count did not fit 32 bits
constexpr uint32_t ST_TABLE_FULL = 4u;    // a hash probe sequence ran out
constexpr uint32_t ST_BAD_INPUT = 8u;     // read offsets not monotone or out of range
constexpr uint32_t ST_BAD_TABLE = 16u;    // a solid table with more than 4 entries per node

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define MH_CUDA(call) ::mh::cuda_check((call), #call)

}  // namespace mh

struct KernelStat {
    uint64_t launches = 0;
    double total_ms = 0.0;
    uint64_t bytes = 0;  // algorithmic bytes (reads + writes the kernel must do)
};

struct mh_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // host uploads overlapped with packing (created on first use)
    cudaEvent_t pack_ev[5] = {};         // the staged upload's events (created on first use)
    std::vector<mh_ctx*> workers;        // worker contexts of mh_run_batch (created on first use)
    int sort_shape = -1;                 // scatter tile shape for 1-word keys (-1: default)
    // the counting plan (mh_set_count_plan, or the batch autotuner); defaults: -1 / 0
    int count_path = -1;                 // 0: unit counting, 1: spread sort, fix-up, run pass
    int unit_bits_delta = 0;             // added to the unit bits of the unit counting
    int spread_bits_delta = 0;           // added to the bits the count's spread passes cover (x 8)
    int bucket_bits = -1;                // out-of-core buckets (0..6); -1: the memory plan's choice
    std::map<std::tuple<int, int, int>, std::vector<int>> tuned;  // (nw, k, size class) -> plan
    uint64_t device_bytes = 0;           // the device's memory, for plans when no budget is set
    mh_alloc_fn alloc = nullptr;
    mh_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0, in_use = 0, peak = 0;
    std::unordered_map<void*, size_t> sizes;
    std::mutex alloc_mu;  // the handles' frees may come from other threads
    int with_mult = 0;
    int num_sms = 0;
    uint32_t* d_status = nullptr;  // device status word (ST_* bits)
    uint64_t* h_pinned = nullptr;  // small pinned buffer for read-backs (64 words)
    // profiling
    int profile = 0;
    std::vector<cudaEvent_t> ev_free;
    struct Pending {
        int name;
        cudaEvent_t a, b;
        uint64_t bytes;
    };
    std::vector<Pending> pending;
    std::vector<std::string> names;
    std::unordered_map<std::string, int> name_id;
    std::vector<KernelStat> stats;
    std::string last_error;
};

struct mh_reads {
    uint64_t n_reads = 0, n_bases = 0, n_frags = 0, n_packed = 0;
    uint32_t* packed = nullptr;     // ceil(n_packed/16) + kPackPad words
    uint64_t* frag_offs = nullptr;  // n_frags + 1
    uint32_t* frag_read = nullptr;  // n_frags
    mh_ctx* ctx = nullptr;
};

struct mh_kmers {
    int k = 0, nw = 1, d = 0;
    uint64_t n = 0;
    uint64_t* keys = nullptr;   // n * nw
    uint32_t* counts = nullptr; // n
    // counting handles: the spectrum, every distinct canonical (k+1)-mer
    // (min(x, rc x)) as a mix_key image, ascending, with the number of
    // windows it has (before doubling for a palindrome); the mercy step
    // looks counts up in it
    uint64_t* spectrum = nullptr;      // n_spectrum * nw
    uint32_t* spectrum_len = nullptr;  // n_spectrum
    uint64_t n_spectrum = 0;
    bool spectrum_mixed = false;
    uint64_t n_kmers = 0, n_distinct = 0;
    mh_ctx* ctx = nullptr;
};

struct mh_contigs {
    int k = 0;
    uint64_t n = 0, n_bases = 0;
    uint8_t* ascii = nullptr;   // n_bases (+16) bytes, ACGT
    uint64_t* offs = nullptr;   // n + 1
    mh_ctx* ctx = nullptr;
};

struct mh_sdbg {
    int k = 0, nw = 1;
    uint64_t m = 0, t = 0, u = 0, n_nodes = 0;
    uint64_t F[6] = {0, 0, 0, 0, 0, 0};
    uint8_t* W = nullptr;
    uint32_t* last = nullptr;
    uint32_t* valid = nullptr;
    uint32_t* dummy = nullptr;
    uint64_t* aux = nullptr;
    uint32_t* mult = nullptr;
    mh_ctx* ctx = nullptr;
};

namespace mh {

constexpr int kPackPad = 12;  // zero words after the packed stream (window loads read ahead)

// ----------------------------------------------------------- allocation
void* ctx_alloc(mh_ctx* ctx, size_t bytes);
void ctx_free(mh_ctx* ctx, void* p);

// Owning device buffer; frees through the context unless released.
template <class T>
struct Buf {
    mh_ctx* ctx = nullptr;
    T* p = nullptr;
    size_t n = 0;
    Buf() = default;
    Buf(mh_ctx* c, size_t count) : ctx(c), n(count) {
        p = static_cast<T*>(ctx_alloc(c, (count ? count : 1) * sizeof(T)));
    }
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; }
    Buf& operator=(Buf&& o) noexcept {
        reset();
        ctx = o.ctx; p = o.p; n = o.n; o.p = nullptr;
        return *this;
    }
    ~Buf() { reset(); }
    void reset() {
        if (p) ctx_free(ctx, p);
        p = nullptr;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
    void zero() { MH_CUDA(cudaMemsetAsync(p, 0, (n ? n : 1) * sizeof(T), ctx->stream)); }
};

// ------------------------------------------------------ launch profiling
// An NVTX range (named in a profiler's timeline) for the scope: every public
// call and every kernel launch opens one.  Without a tool attached the calls
// return at once.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Prof {
    NvtxRange range;
    mh_ctx* ctx;
    int id = -1;
    uint64_t bytes = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    Prof(mh_ctx* c, const char* name, uint64_t algo_bytes = 0);
    ~Prof();
};

// Launch a kernel on the context stream, timed when profiling is on.
#define MH_LAUNCH(ctx, name, grid, block, smem, kernel, ...)                          \
    do {                                                                               \
        ::mh::Prof _mh_prof((ctx), (name));                                            \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);               \
        ::mh::cuda_check(cudaGetLastError(), (name));                                  \
    } while (0)

// Same, also recording the launch's algorithmic bytes for the roofline.
#define MH_LAUNCH_B(ctx, name, algo_bytes, grid, block, smem, kernel, ...)            \
    do {                                                                               \
        ::mh::Prof _mh_prof((ctx), (name), (algo_bytes));                              \
        kernel<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);               \
        ::mh::cuda_check(cudaGetLastError(), (name));                                  \
    } while (0)

// Wait for the stream, then raise the first status bit the kernels set.
void sync_and_check(mh_ctx* ctx);
// Copy `count` uint64 from device to host through the pinned buffer (waits).
void read_u64(mh_ctx* ctx, const uint64_t* d, uint64_t* h, int count);

__host__ __device__ inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline int words_for(int k) { return 2 * (k + 1) <= 64 ? 1 : (2 * (k + 1) <= 128 ? 2 : 4); }
int grid_for(mh_ctx* ctx, uint64_t work_items, int per_block, int blocks_per_sm = 8);

// ------------------------------------------------------------ key helpers
template <int NW>
struct Key {
    uint64_t w[NW];
};

template <int NW>
__host__ __device__ __forceinline__ bool key_less(const Key<NW>& a, const Key<NW>& b) {
#pragma unroll
    for (int i = NW - 1; i >= 0; i--)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
    return false;
}

template <int NW>
__host__ __device__ __forceinline__ bool key_eq(const Key<NW>& a, const Key<NW>& b) {
    bool e = true;
#pragma unroll
    for (int i = 0; i < NW; i++) e &= a.w[i] == b.w[i];
    return e;
}

template <int NW>
__device__ __forceinline__ Key<NW> key_zero() {
    Key<NW> r;
#pragma unroll
    for (int i = 0; i < NW; i++) r.w[i] = 0;
    return r;
}

// Word j of a key (0 past the top), without a run-time array index (which
// would move the key to local memory).
template <int NW>
__device__ __forceinline__ uint64_t key_word(const Key<NW>& a, int j) {
    uint64_t v = 0;
#pragma unroll
    for (int m = 0; m < NW; m++) v = (j == m) ? a.w[m] : v;
    return v;
}

// Bits [shift, shift+8) of the key, 0 <= shift < 64*NW (bits past the top read 0).
template <int NW>
__device__ __forceinline__ uint32_t key_digit(const Key<NW>& a, int shift) {
    if constexpr (NW == 1) {
        return (uint32_t)(a.w[0] >> shift) & 0xFFu;
    } else {
        int wi = shift >> 6, sb = shift & 63;
        uint64_t v = key_word<NW>(a, wi) >> sb;
        if (sb > 56) v |= key_word<NW>(a, wi + 1) << (64 - sb);
        return (uint32_t)(v & 0xFF);
    }
}

// a >> s for 0 <= s < 64*NW
template <int NW>
__device__ __forceinline__ Key<NW> key_shr(const Key<NW>& a, int s) {
    Key<NW> r;
    if constexpr (NW == 1) {
        r.w[0] = a.w[0] >> s;
    } else {
        int ws = s >> 6, bs = s & 63;
#pragma unroll
        for (int i = 0; i < NW; i++) {
            uint64_t lo = key_word<NW>(a, i + ws), hi = key_word<NW>(a, i + ws + 1);
            r.w[i] = bs ? ((lo >> bs) | (hi << (64 - bs))) : lo;
        }
    }
    return r;
}

// a << s for 0 <= s < 64*NW (bits shifted past the top are dropped)
template <int NW>
__device__ __forceinline__ Key<NW> key_shl(const Key<NW>& a, int s) {
    Key<NW> r;
    if constexpr (NW == 1) {
        r.w[0] = a.w[0] << s;
    } else {
        int ws = s >> 6, bs = s & 63;
#pragma unroll
        for (int i = 0; i < NW; i++) {
            uint64_t hi = key_word<NW>(a, i - ws), lo = key_word<NW>(a, i - ws - 1);
            r.w[i] = bs ? ((hi << bs) | (lo >> (64 - bs))) : hi;
        }
    }
    return r;
}

// Keep the low `bits` bits (0 <= bits <= 64*NW).
template <int NW>
__device__ __forceinline__ Key<NW> key_low(const Key<NW>& a, int bits) {
    Key<NW> r;
#pragma unroll
    for (int i = 0; i < NW; i++) {
        int lo = 64 * i;
        r.w[i] = bits <= lo ? 0 : (bits >= lo + 64 ? a.w[i] : (a.w[i] & ((1ull << (bits - lo)) - 1)));
    }
    return r;
}

template <int NW>
__device__ __forceinline__ Key<NW> key_or_low(Key<NW> a, uint64_t v) {
    a.w[0] |= v;
    return a;
}

// The next window of a read from the current one: x (the window, K1
// symbols, first symbol most significant) shifted up by one symbol with the
// new symbol s appended and its first symbol dropped; r, its reverse
// complement, shifted down by one symbol with the complement of s put in
// front (symbol position K1 - 1).
template <int NW>
__device__ __forceinline__ void roll_window(Key<NW>& x, Key<NW>& r, uint32_t s, int K1) {
#pragma unroll
    for (int i = NW - 1; i > 0; i--) x.w[i] = (x.w[i] << 2) | (x.w[i - 1] >> 62);
    x.w[0] = (x.w[0] << 2) | s;
    x = key_low<NW>(x, 2 * K1);
#pragma unroll
    for (int i = 0; i + 1 < NW; i++) r.w[i] = (r.w[i] >> 2) | (r.w[i + 1] << 62);
    r.w[NW - 1] >>= 2;
    const int top = 2 * (K1 - 1);
#pragma unroll
    for (int i = 0; i < NW; i++)
        if ((top >> 6) == i) r.w[i] |= (uint64_t)(3u - s) << (top & 63);
}

// The forward half of roll_window: the next window from the current one.
template <int NW>
__device__ __forceinline__ void roll_forward(Key<NW>& x, uint32_t s, int K1) {
#pragma unroll
    for (int i = NW - 1; i > 0; i--) x.w[i] = (x.w[i] << 2) | (x.w[i - 1] >> 62);
    x.w[0] = (x.w[0] << 2) | s;
    x = key_low<NW>(x, 2 * K1);
}

// Symbol j of the packed stream (base j at bits 31-2(j%16) of word j/16).
__device__ __forceinline__ uint32_t packed_sym(const uint32_t* __restrict__ packed, uint64_t j) {
    return (packed[j >> 4] >> (30 - 2 * (uint32_t)(j & 15))) & 3u;
}

// Reverse the order of the 2-bit symbols of a 64-bit word.
__device__ __forceinline__ uint64_t rev2_u64(uint64_t x) {
    uint64_t y = __brevll(x);
    return ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
}

// Reverse the order of the low n symbols (n >= 1) of a key.
template <int NW>
__device__ __forceinline__ Key<NW> key_rev(const Key<NW>& a, int n) {
    Key<NW> r;
#pragma unroll
    for (int i = 0; i < NW; i++) r.w[i] = rev2_u64(a.w[NW - 1 - i]);
    return key_shr<NW>(r, 64 * NW - 2 * n);
}

// Reverse complement of a string of n symbols (n >= 1).
template <int NW>
__device__ __forceinline__ Key<NW> key_rc(const Key<NW>& a, int n) {
    Key<NW> c;
#pragma unroll
    for (int i = 0; i < NW; i++) c.w[i] = ~a.w[i];
    return key_rev<NW>(key_low<NW>(c, 2 * n), n);
}

// Symbol i (0 = first) of a string of n symbols.
template <int NW>
__device__ __forceinline__ uint32_t key_sym(const Key<NW>& a, int n, int i) {
    int bit = 2 * (n - 1 - i);
    return (uint32_t)(key_word<NW>(a, bit >> 6) >> (bit & 63)) & 3u;
}

template <int NW>
__device__ __forceinline__ Key<NW> load_key(const uint64_t* p, uint64_t i) {
    Key<NW> r;
    if constexpr (NW == 1) {
        r.w[0] = p[i];
    } else if constexpr (NW == 2) {
        ulonglong2 v = reinterpret_cast<const ulonglong2*>(p)[i];
        r.w[0] = v.x; r.w[1] = v.y;
    } else {
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p) + 2 * i;
        ulonglong2 v0 = q[0], v1 = q[1];
        r.w[0] = v0.x; r.w[1] = v0.y; r.w[2] = v1.x; r.w[3] = v1.y;
    }
    return r;
}

template <int NW>
__device__ __forceinline__ void store_key(uint64_t* p, uint64_t i, const Key<NW>& k) {
    if constexpr (NW == 1) {
        p[i] = k.w[0];
    } else if constexpr (NW == 2) {
        reinterpret_cast<ulonglong2*>(p)[i] = make_ulonglong2(k.w[0], k.w[1]);
    } else {
        ulonglong2* q = reinterpret_cast<ulonglong2*>(p) + 2 * i;
        q[0] = make_ulonglong2(k.w[0], k.w[1]);
        q[1] = make_ulonglong2(k.w[2], k.w[3]);
    }
}

// The n symbols starting at base p of the packed stream (base j at bits
// 31-2(j%16) of word j/16), as a key.  Reads up to 2*NW+1 words from p/16.
template <int NW>
__device__ __forceinline__ Key<NW> load_window(const uint32_t* __restrict__ packed, uint64_t p, int n) {
    const uint32_t* w = packed + (p >> 4);
    int o = 2 * (int)(p & 15);
    uint32_t s32[2 * NW];
    uint32_t cur = w[0];
#pragma unroll
    for (int t = 0; t < 2 * NW; t++) {
        uint32_t nxt = w[t + 1];
        s32[t] = o ? ((cur << o) | (nxt >> (32 - o))) : cur;
        cur = nxt;
    }
    Key<NW> r;
#pragma unroll
    for (int j = 0; j < NW; j++) r.w[NW - 1 - j] = ((uint64_t)s32[2 * j] << 32) | s32[2 * j + 1];
    return key_shr<NW>(r, 64 * NW - 2 * n);
}

// ------------------------------------------------------ bounded waits
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------ searching
// First index in [0, n) with a[i] >= q, searched outward from `hint` (any
// value in [0, n]): exponential steps towards the answer, then bisection.
template <int NW>
__device__ __forceinline__ uint64_t gallop_lb(const uint64_t* __restrict__ a, uint64_t n, const Key<NW>& q,
                                              uint64_t hint) {
    uint64_t lo, hi;  // answer in [lo, hi]
    if (hint < n && key_less<NW>(load_key<NW>(a, hint), q)) {
        // a[hint] < q: answer > hint
        lo = hint + 1;
        uint64_t step = 1;
        while (true) {
            uint64_t probe = lo + step - 1;
            if (probe >= n) {
                hi = n;
                break;
            }
            if (!key_less<NW>(load_key<NW>(a, probe), q)) {
                hi = probe;
                break;
            }
            lo = probe + 1;
            step <<= 1;
        }
    } else {
        // a[hint] >= q (or hint == n): answer <= hint
        hi = hint;
        uint64_t step = 1;
        while (true) {
            if (hi < step) {
                lo = 0;
                break;
            }
            uint64_t probe = hi - step;
            if (key_less<NW>(load_key<NW>(a, probe), q)) {
                lo = probe + 1;
                break;
            }
            hi = probe;
            step <<= 1;
        }
    }
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (key_less<NW>(load_key<NW>(a, mid), q)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------ bitmask scans
// First set bit at or after i in b (bits [0, n)), or n.
__device__ __forceinline__ uint32_t next_bit(const uint32_t* b, uint32_t i, uint32_t n) {
    if (i >= n) return n;
    uint32_t w = i >> 5;
    uint32_t m = b[w] & ~((1u << (i & 31)) - 1u);
    while (true) {
        if (m) {
            const uint32_t r = w * 32 + __ffs(m) - 1;
            return r < n ? r : n;
        }
        if (++w * 32 >= n) return n;
        m = b[w];
    }
}

// Last set bit at or before i in b, or ~0u.
__device__ __forceinline__ uint32_t prev_bit(const uint32_t* b, uint32_t i) {
    int w = (int)(i >> 5);
    uint32_t m = b[w] & (0xFFFFFFFFu >> (31 - (i & 31)));
    while (true) {
        if (m) return (uint32_t)w * 32 + 31 - __clz(m);
        if (--w < 0) return ~0u;
        m = b[w];
    }
}

// Any set bit in [i, j)?
__device__ __forceinline__ bool any_bit(const uint32_t* b, uint32_t i, uint32_t j) {
    return next_bit(b, i, j) < j;
}

// ------------------------------------------------ tile compaction helpers
// 64-bit per-tile status words for decoupled look-back: flag in the top two
// bits (aggregate / inclusive), count in the low 62.
constexpr uint64_t kLbAgg = 1ull << 62;
constexpr uint64_t kLbInc = 2ull << 62;
constexpr uint64_t kLbCountMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Called by one whole warp of the tile: publishes the tile's total, looks
// back over earlier tiles (lane l reads tile j - l, the window is used up to
// the nearest inclusive entry; every wait is bounded) and returns the sum of
// all earlier tiles' totals.  Tiles must be numbered in launch-claim order
// (a dynamic tile id) so that every earlier tile is running or done.
__device__ __forceinline__ uint64_t warp_lookback_u64(uint64_t* status, uint64_t tile, uint64_t total,
                                                      uint32_t* err) {
    const int lane = threadIdx.x & 31;
    uint64_t* st = status + tile;
    if (lane == 0) st_relaxed_u64(st, (tile == 0 ? kLbInc : kLbAgg) | total);
    uint64_t excl = 0;
    bool ok = true;
    for (int64_t j = (int64_t)tile - 1; j >= 0 && ok; j -= 32) {
        const int64_t idx = j - lane;
        uint64_t v = idx >= 0 ? ld_relaxed_u64(status + idx) : kLbInc;
        int spins = 0;
        uint32_t inc;
        while (true) {
            inc = __ballot_sync(0xFFFFFFFFu, (v & ~kLbCountMask) == kLbInc);
            const uint32_t need = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xFFFFFFFFu;
            const uint32_t waiting = __ballot_sync(0xFFFFFFFFu, (v & ~kLbCountMask) == 0) & need;
            if (!waiting) break;
            if (++spins > (1 << 23)) {
                ok = false;
                break;
            }
            if (spins > 64) __nanosleep(128);
            if (idx >= 0 && (v & ~kLbCountMask) == 0) v = ld_relaxed_u64(status + idx);
        }
        const uint32_t need = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xFFFFFFFFu;
        uint64_t c = ((need >> lane) & 1u) ? (v & kLbCountMask) : 0;
        for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
        excl += c;
        if (inc) break;
    }
    if (lane == 0) {
        if (!ok) atomicOr(err, 1u);  // ST_SPIN_TIMEOUT
        if (tile > 0) st_relaxed_u64(st, kLbInc | (excl + total));
    }
    return excl;
}

// Exclusive prefix of a per-thread count over a block of 256 threads (8
// warps); `scratch` holds 8 words of shared memory.  Also returns the total.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* scratch, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const uint32_t sw = scratch[w];
        pre += w < warp ? sw : 0u;
        tot += sw;
    }
    __syncthreads();
    *total = tot;
    return pre + x - v;
}

// ----------------------------------------------------------- hashing
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Invertible 64-bit mixer: multiplication by an odd constant is a bijection
// of 64-bit words, so mix_bij permutes the keys (equal keys stay equal,
// distinct keys stay distinct), and every bit of the key reaches the top
// bits of the product, which is all the sorts use (Fibonacci hashing: keys
// that differ in a few symbols differ in their top bits).
constexpr uint64_t kMixC1 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMixC1Inv = 0xF1DE83E19937733Dull;  // its inverse mod 2^64
__host__ __device__ __forceinline__ uint64_t mix_bij(uint64_t x) { return x * kMixC1; }
__host__ __device__ __forceinline__ uint64_t unmix_bij(uint64_t h) { return h * kMixC1Inv; }

// Multiword keys: word i is mixed together with the mixed word below it, so
// the top word depends on every word (its top bits spread evenly) and each
// step can be undone given the word below (a bijection of keys).  One word:
// mix_bij.
template <int NW>
__host__ __device__ __forceinline__ Key<NW> mix_key(Key<NW> a) {
    a.w[0] = mix_bij(a.w[0]);
#pragma unroll
    for (int i = 1; i < NW; i++) a.w[i] = mix_bij(a.w[i] ^ a.w[i - 1]);
    return a;
}
template <int NW>
__host__ __device__ __forceinline__ Key<NW> unmix_key(const Key<NW>& m) {
    Key<NW> a;
#pragma unroll
    for (int i = NW - 1; i >= 1; i--) a.w[i] = unmix_bij(m.w[i]) ^ m.w[i - 1];
    a.w[0] = unmix_bij(m.w[0]);
    return a;
}

template <int NW>
__device__ __forceinline__ uint64_t key_hash(const Key<NW>& a) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int i = 0; i < NW; i++) h = mix64(h ^ a.w[i]);
    return h;
}

// ------------------------------------------------------------- sorting
// LSD radix sort (one digit histogram pass, then one onesweep pass per
// 8-bit digit of bits [bit_lo, bit_hi)).  keys/alt (and vals/valt when
// vals != nullptr) are n-element buffers; returns true if the sorted data
// ended in alt/valt, false if in keys/vals.  `hist`, when given, holds the
// digit counts of the passes (pass p's 256 counts at p * 256), counted by
// the caller while it wrote the keys; the histogram pass is then skipped.
template <int NW>
bool radix_sort(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                int bit_lo, int bit_hi, const uint32_t* hist = nullptr);
// The same for n 1-word keys held in 256 segments of seg_cap slots each
// (segment r's seg_cnt[r] keys at r * seg_cap; seg_cap at least one scatter
// tile): the first pass reads the segments, and every pass writes n
// contiguous keys.  `hist` is required.
bool radix_sort_segmented(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint64_t n,
                          const unsigned long long* seg_cnt, uint64_t seg_cap, int bit_lo, int bit_hi,
                          const uint32_t* hist);

// Sort of mix_key images (evenly spread top bits): LSD passes over the top
// P = spread_pass_bits(n) bits below the top `skip` bits (equal in every
// key), then a fix-up of the keys that share them.  `hist`: the counts of
// those passes' digits (as for radix_sort), or nullptr.  Returns true if the
// result is in alt.
int spread_pass_bits(mh_ctx* ctx, uint64_t n);
template <int NW>
bool radix_sort_spread(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint64_t n, int skip = 0,
                       const uint32_t* hist = nullptr);
template <int NW>
bool radix_sort_spread_kv(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt, uint64_t n,
                          int skip);

// ---------------------------------------------------------------- scans
// out[i] = sum of in[0..i-1] for i in [0, n]; out has n+1 entries.
void exclusive_scan_u64(mh_ctx* ctx, const uint64_t* in, uint64_t* out, uint64_t n);
void exclusive_scan_u32(mh_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n);

// ------------------------------------------------- counting stages
// Merge of sorted runs [bounds[i], bounds[i+1]) of keys (and payload, when
// vals) into one sorted sequence; returns true when the result is in alt/valt.
template <int NW>
bool merge_runs(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt,
                const std::vector<uint64_t>& bounds);

// X \ Y and Y \ X of two sorted arrays without repeats, each in order.
template <int NW>
void set_differences(mh_ctx* ctx, const uint64_t* X, uint64_t nx, const uint64_t* Y, uint64_t ny, uint64_t* outX,
                     uint64_t* n_outX, uint64_t* outY, uint64_t* n_outY);

// One read set through pack, count and (by flags) mercy and build on
// context w (mh_batch.cu); a failed set keeps no outputs.
int run_set_job(mh_ctx* w, const mh_read_set& s, int k, int d, int flags, mh_set_result& r);
void free_set_result(mh_set_result& r);

template <int NW>
void walk_contigs(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, uint64_t n_walks, uint32_t max_len,
                  uint64_t seed, mh_contigs* out);
void pack_reads(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs, uint64_t n_reads,
                mh_reads* out);
void pack_reads_host(mh_ctx* ctx, const uint8_t* h_ascii, uint64_t n_bases, const uint64_t* h_offs, uint64_t n_reads,
                     mh_reads* out);
void pack_with_contigs(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs,
                       uint64_t n_reads, const mh_contigs* contigs, uint32_t copies, mh_reads* out);

// Optional output of expand_runs in counting mode: every run's input key
// and length, in input order.  `slot` is scratch of >= n keys, freed once
// the list is compacted.
struct RunList {
    Buf<uint64_t> slot;
    Buf<uint64_t> keys;
    Buf<uint32_t> lens;
    uint64_t n = 0;
};

// Out-of-core buckets of the count of n canonical windows of nw-word keys:
// 0 (all in memory) or bits of 2^bits buckets (mh_count.cu).
int count_bucket_bits(mh_ctx* ctx, uint64_t n, int nw);

// How the unit counting splits n keys of nw words whose top `skip` bits
// are equal: units of the next unit_bits bits of the top word (about
// 160 / 96 / 56 keys each for 1 / 2 / 4 words), sorted into place by
// `passes` 8-bit LSD passes over the next 8 * passes bits.  passes < 0: the
// keys are too narrow for it (the spread path is used).
struct GroupPlan {
    int unit_bits = 0;
    int passes = 0;
};
GroupPlan group_plan(mh_ctx* ctx, uint64_t n, int skip, int nw);

// Unit counting of mixed canonical keys of NW words (defined in
// mh_group.cu): `sorted` holds n keys sorted by the top skip + 8 *
// plan.passes bits of their top word, `other` n free keys.  Each unit is
// sorted on chip and run-length counted: out_keys / out_cnt get the kept
// (k+1)-mers of both strands (count >= d, ascending), list the spectrum
// (every run's mixed key and length, ascending).  Both input buffers are
// consumed (freed).
template <int NW>
void group_count(mh_ctx* ctx, Buf<uint64_t>& sorted, Buf<uint64_t>& other, uint64_t n, int k, int d, int skip,
                 const GroupPlan& plan, Buf<uint64_t>& out_keys, Buf<uint32_t>& out_cnt, uint64_t* n_out,
                 uint64_t* n_runs, uint64_t* n_palin_runs, RunList* list);


// Sorted canonical keys -> solid (k+1)-mers, both strands, sorted.  Defined
// in mh_count.cu, used by mercy too (d = 1, counts looked up in the
// spectrum).  in_mixed: `sorted` holds mix_key images of the canonical keys;
// spec_mixed: likewise for the spectrum.
template <int NW>
void expand_runs(mh_ctx* ctx, const uint64_t* sorted, uint64_t n, int k, int d, Buf<uint64_t>& out_keys,
                 Buf<uint32_t>& out_cnt, uint64_t* n_out, uint64_t* n_canon_runs, uint64_t* n_palin_runs,
                 const uint64_t* spectrum, const uint32_t* spectrum_len, uint64_t n_spectrum, bool in_mixed = false,
                 bool spec_mixed = false, RunList* list = nullptr);

}  // namespace mh
