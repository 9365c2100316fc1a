// mh_count_kmers: every (k+1)-mer on both strands, sorted and counted; the
// solid ones (count >= d) are kept (paper, Sec. 2, third paragraph).
//
// A window x and its reverse complement rc(x) always occur together in the
// both-strand multiset, so the library sorts one canonical key min(x, rc x)
// per window (half the keys of the literal multiset) and recovers the literal
// counts exactly: cnt(x) = cnt(rc x) = run length of canonical(x), doubled
// when x = rc(x) (a palindrome, counted twice per occurrence).
//
//   extract   warp per fragment, window keys from the packed words, canonical
//   sort      LSD radix over the 2(k+1) key bits
//   runs      run heads, run lengths by galloping search, solid filter
//   expand    each solid canonical key -> itself and its reverse complement
//   sort      key-value LSD radix -> solid table in ascending key order
#include "mh_internal.cuh"

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

// Warp per fragment: canonical key of every window, written at woff[f] + i.
template <int NW>
__global__ void __launch_bounds__(256) extract_canonical_kernel(const uint32_t* __restrict__ packed,
                                                                const uint64_t* __restrict__ frag_offs,
                                                                const uint64_t* __restrict__ woff, uint64_t n_frags,
                                                                int k, uint64_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1;
    for (uint64_t f = warp; f < n_frags; f += n_warps) {
        uint64_t b = frag_offs[f];
        uint64_t w0 = woff[f], nw = woff[f + 1] - w0;
        for (uint64_t i = lane; i < nw; i += 32) {
            Key<NW> x = load_window<NW>(packed, b + i, K1);
            Key<NW> r = key_rc<NW>(x, K1);
            store_key<NW>(out, w0 + i, key_less<NW>(r, x) ? r : x);
        }
    }
}

constexpr int kRunThreads = 256;
constexpr int kRunItems = 8;
constexpr int kRunTile = kRunThreads * kRunItems;

// First index j > i with s[j] != s[i] (or n), by galloping then bisection.
template <int NW>
__device__ __forceinline__ uint64_t run_end(const uint64_t* __restrict__ s, uint64_t n, uint64_t i,
                                            const Key<NW>& x) {
    uint64_t step = 1, lo = i;  // s[lo] == x
    while (true) {
        uint64_t j = i + step;
        if (j >= n) {
            j = n;
            // bisection on (lo, n]
            uint64_t hi = n;
            while (hi - lo > 1) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (key_eq<NW>(load_key<NW>(s, mid), x)) lo = mid; else hi = mid;
            }
            return hi;
        }
        if (!key_eq<NW>(load_key<NW>(s, j), x)) {
            uint64_t hi = j;
            while (hi - lo > 1) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (key_eq<NW>(load_key<NW>(s, mid), x)) lo = mid; else hi = mid;
            }
            return hi;
        }
        lo = j;
        step <<= 1;
    }
}

// What a run contributes.  mode 0 (counting): literal count = len (x2 for a
// palindrome); kept if >= d; outputs 1 (palindrome) or 2 keys.  mode 1
// (dedup with counts from a spectrum): every run kept, count looked up.
struct RunOut {
    uint32_t n_out;
    uint32_t count;
    bool palin;
};

template <int NW>
__device__ __forceinline__ uint64_t spectrum_count(const uint64_t* __restrict__ spec, uint64_t n_spec,
                                                   const Key<NW>& x) {
    // lower bound
    uint64_t lo = 0, hi = n_spec;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (key_less<NW>(load_key<NW>(spec, mid), x)) lo = mid + 1; else hi = mid;
    }
    if (lo >= n_spec || !key_eq<NW>(load_key<NW>(spec, lo), x)) return 0;
    return run_end<NW>(spec, n_spec, lo, x) - lo;
}

template <int NW>
__device__ __forceinline__ RunOut run_info(const uint64_t* __restrict__ s, uint64_t n, uint64_t i, const Key<NW>& x,
                                           int K1, int d, const uint64_t* __restrict__ spec, uint64_t n_spec,
                                           uint32_t* __restrict__ err) {
    Key<NW> r = key_rc<NW>(x, K1);
    bool palin = key_eq<NW>(r, x);
    uint64_t len = spec ? spectrum_count<NW>(spec, n_spec, x) : run_end<NW>(s, n, i, x) - i;
    uint64_t c = palin ? 2 * len : len;
    if (c > 0xFFFFFFFFull) {
        atomicOr(err, ST_OVERFLOW);
        c = 0xFFFFFFFFull;
    }
    RunOut o;
    o.palin = palin;
    o.count = (uint32_t)c;
    o.n_out = (spec || c >= (uint64_t)d) ? (palin ? 1u : 2u) : 0u;
    return o;
}

// Pass 1: per tile, the number of output keys; also distinct-run totals.
template <int NW>
__global__ void __launch_bounds__(kRunThreads) runs_count_kernel(const uint64_t* __restrict__ s, uint64_t n, int K1,
                                                                 int d, const uint64_t* __restrict__ spec,
                                                                 uint64_t n_spec, uint64_t* __restrict__ tile_out,
                                                                 unsigned long long* __restrict__ totals,
                                                                 uint32_t* __restrict__ err) {
    uint64_t t0 = (uint64_t)blockIdx.x * kRunTile;
    uint32_t outs = 0, heads = 0, palins = 0;
#pragma unroll
    for (int it = 0; it < kRunItems; it++) {
        uint64_t i = t0 + it * kRunThreads + threadIdx.x;
        if (i >= n) break;
        Key<NW> x = load_key<NW>(s, i);
        if (i > 0 && key_eq<NW>(load_key<NW>(s, i - 1), x)) continue;
        RunOut o = run_info<NW>(s, n, i, x, K1, d, spec, n_spec, err);
        outs += o.n_out;
        heads++;
        palins += o.palin;
    }
    __shared__ uint32_t red[3][kRunThreads / 32];
    for (int off = 16; off; off >>= 1) {
        outs += __shfl_xor_sync(0xFFFFFFFFu, outs, off);
        heads += __shfl_xor_sync(0xFFFFFFFFu, heads, off);
        palins += __shfl_xor_sync(0xFFFFFFFFu, palins, off);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = outs;
        red[1][warp] = heads;
        red[2][warp] = palins;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t a = 0, b = 0, c = 0;
        for (int w = 0; w < kRunThreads / 32; w++) {
            a += red[0][w];
            b += red[1][w];
            c += red[2][w];
        }
        tile_out[blockIdx.x] = a;
        atomicAdd(&totals[0], (unsigned long long)b);
        atomicAdd(&totals[1], (unsigned long long)c);
    }
}

// Pass 2: write the kept runs' keys (and reverse complements) with counts.
template <int NW>
__global__ void __launch_bounds__(kRunThreads) runs_write_kernel(const uint64_t* __restrict__ s, uint64_t n, int K1,
                                                                 int d, const uint64_t* __restrict__ spec,
                                                                 uint64_t n_spec, const uint64_t* __restrict__ tile_off,
                                                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ cnt,
                                                                 uint32_t* __restrict__ err) {
    uint64_t t0 = (uint64_t)blockIdx.x * kRunTile;
    uint32_t mine = 0;
    RunOut o[kRunItems];
    Key<NW> xs[kRunItems];
#pragma unroll
    for (int it = 0; it < kRunItems; it++) {
        o[it].n_out = 0;
        uint64_t i = t0 + it * kRunThreads + threadIdx.x;
        if (i >= n) continue;
        xs[it] = load_key<NW>(s, i);
        if (i > 0 && key_eq<NW>(load_key<NW>(s, i - 1), xs[it])) continue;
        o[it] = run_info<NW>(s, n, i, xs[it], K1, d, spec, n_spec, err);
        mine += o[it].n_out;
    }
    // block exclusive scan of per-thread output counts (thread order)
    __shared__ uint32_t ws[kRunThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = mine;
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; w++) pre += ws[w];
    uint64_t pos = tile_off[blockIdx.x] + pre + x - mine;
#pragma unroll
    for (int it = 0; it < kRunItems; it++) {
        if (!o[it].n_out) continue;
        store_key<NW>(keys, pos, xs[it]);
        cnt[pos] = o[it].count;
        pos++;
        if (o[it].n_out == 2) {
            store_key<NW>(keys, pos, key_rc<NW>(xs[it], K1));
            cnt[pos] = o[it].count;
            pos++;
        }
    }
}

// Sorted canonical keys -> both-strand keys of kept runs, sorted ascending.
// spectrum == nullptr: counting mode (keep count >= d).  Otherwise every run
// is kept with its count looked up in the spectrum.
template <int NW>
void expand_runs(mh_ctx* ctx, const uint64_t* sorted, uint64_t n, int k, int d, Buf<uint64_t>& out_keys,
                 Buf<uint32_t>& out_cnt, uint64_t* n_out, uint64_t* n_canon_runs, uint64_t* n_palin_runs,
                 const uint64_t* spectrum, uint64_t n_spectrum) {
    const int K1 = k + 1;
    const uint64_t tiles = ceil_div(n ? n : 1, kRunTile);
    Buf<uint64_t> tile_out(ctx, tiles + 1), tile_off(ctx, tiles + 1);
    Buf<uint64_t> totals(ctx, 2);
    totals.zero();
    tile_out.zero();
    if (n)
        MH_LAUNCH_B(ctx, "runs_count", n * 8 * NW, (unsigned)tiles, kRunThreads, 0, runs_count_kernel<NW>, sorted, n, K1,
                    d, spectrum, n_spectrum, tile_out.p, (unsigned long long*)totals.p, ctx->d_status);
    exclusive_scan_u64(ctx, tile_out.p, tile_off.p, tiles);
    uint64_t tot[3];
    read_u64(ctx, tile_off.p + tiles, &tot[0], 1);
    read_u64(ctx, totals.p, &tot[1], 2);
    const uint64_t S = tot[0];
    *n_out = S;
    *n_canon_runs = tot[1];
    *n_palin_runs = tot[2];
    Buf<uint64_t> keys(ctx, (S ? S : 1) * NW), alt(ctx, (S ? S : 1) * NW);
    Buf<uint32_t> cnt(ctx, S ? S : 1), calt(ctx, S ? S : 1);
    if (n && S)
        MH_LAUNCH(ctx, "runs_write", (unsigned)tiles, kRunThreads, 0, runs_write_kernel<NW>, sorted, n, K1, d, spectrum,
                  n_spectrum, tile_off.p, keys.p, cnt.p, ctx->d_status);
    bool in_alt = radix_sort<NW>(ctx, keys.p, alt.p, cnt.p, calt.p, S, 0, 2 * K1);
    if (in_alt) {
        out_keys = std::move(alt);
        out_cnt = std::move(calt);
    } else {
        out_keys = std::move(keys);
        out_cnt = std::move(cnt);
    }
}

template void expand_runs<1>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, uint64_t);
template void expand_runs<2>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, uint64_t);
template void expand_runs<4>(mh_ctx*, const uint64_t*, uint64_t, int, int, Buf<uint64_t>&, Buf<uint32_t>&, uint64_t*,
                             uint64_t*, uint64_t*, const uint64_t*, uint64_t);

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
    Buf<uint64_t> keys(ctx, (n ? n : 1) * NW), alt(ctx, (n ? n : 1) * NW);
    if (n)
        MH_LAUNCH_B(ctx, "extract_canonical", reads->n_packed / 4 + n * 8 * NW, grid_for(ctx, F * 32, 256, 8), 256, 0,
                    extract_canonical_kernel<NW>, reads->packed, reads->frag_offs, woff.p, F, k, keys.p);
    woff.reset();
    bool in_alt = radix_sort<NW>(ctx, keys.p, alt.p, nullptr, nullptr, n, 0, 2 * (k + 1));
    Buf<uint64_t>& spec = in_alt ? alt : keys;
    (in_alt ? keys : alt).reset();
    Buf<uint64_t> sk;
    Buf<uint32_t> sc;
    uint64_t S = 0, runs = 0, palins = 0;
    expand_runs<NW>(ctx, spec.p, n, k, d, sk, sc, &S, &runs, &palins, nullptr, 0);
    sync_and_check(ctx);
    out->k = k;
    out->nw = NW;
    out->d = d;
    out->n = S;
    out->n_kmers = 2 * n;
    out->n_distinct = 2 * runs - palins;
    out->keys = sk.release();
    out->counts = sc.release();
    out->n_spectrum = n;
    out->spectrum = spec.release();
}

template void count_kmers<1>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);
template void count_kmers<2>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);
template void count_kmers<4>(mh_ctx*, const mh_reads*, int, int, mh_kmers*);

}  // namespace mh
