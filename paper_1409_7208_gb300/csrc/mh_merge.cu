// Merge of sorted runs (keys of NW words, optional 32-bit payload): a tree of
// two-way merges, each a merge-path merge.  A partition kernel finds, for
// every CTA's first output position d, how many of the first d outputs come
// from the first run (a binary search along the diagonal); each CTA then
// loads its two input slices into shared memory, each thread finds its own
// diagonal split there and merges its items, and the CTA writes its output
// slice in one coalesced sweep.  Equal keys take the first run's key first,
// so the merge is stable.
#include <vector>

#include "mh_internal.cuh"

namespace mh {

constexpr int kMergeThreads = 256;

template <int NW>
__host__ __device__ constexpr int merge_items() {
    return 4 / NW;  // 1024, 512 or 256 keys a CTA: 8 KB of keys
}
template <int NW>
__host__ __device__ constexpr int merge_tile() {
    return kMergeThreads * merge_items<NW>();
}
// The set differences stage both inputs' slices and walk twice the merge's
// items a thread (the tile sizes measured fastest for each).
template <int NW>
__host__ __device__ constexpr int diff_items() {
    return 8 / NW;
}
template <int NW>
__host__ __device__ constexpr int diff_tile() {
    return kMergeThreads * diff_items<NW>();
}

// Runs [a, a + na) and [a + na, a + na + nb) merge into [a, a + na + nb) of
// the other buffer; CTAs cta0 .. cta0 + ceil((na + nb) / tile) - 1 do it.
struct MergePair {
    uint64_t a, na, nb, cta0;
};

template <int NW>
__device__ __forceinline__ bool key_le(const Key<NW>& a, const Key<NW>& b) {
    return !key_less<NW>(b, a);
}

// Number of the first d outputs that come from x (length nx), the rest from y.
template <int NW>
__device__ __forceinline__ uint64_t merge_path(const uint64_t* __restrict__ x, uint64_t nx,
                                               const uint64_t* __restrict__ y, uint64_t ny, uint64_t d) {
    uint64_t lo = d > ny ? d - ny : 0, hi = d < nx ? d : nx;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (key_le<NW>(load_key<NW>(x, mid), load_key<NW>(y, d - 1 - mid))) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int pair_of(const MergePair* __restrict__ pairs, int n_pairs, uint64_t c) {
    int p = 0;
    while (p + 1 < n_pairs && pairs[p + 1].cta0 <= c) p++;
    return p;
}

// part[c] = the first-run count at CTA c's first output.
template <int NW>
__global__ void merge_partition_kernel(const uint64_t* __restrict__ keys, const MergePair* __restrict__ pairs,
                                       int n_pairs, uint64_t n_ctas, uint64_t* __restrict__ part) {
    constexpr int T = merge_tile<NW>();
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_ctas;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const MergePair P = pairs[pair_of(pairs, n_pairs, c)];
        const uint64_t d = (c - P.cta0) * T;
        const uint64_t* x = keys + P.a * NW;
        part[c] = merge_path<NW>(x, P.na, x + P.na * NW, P.nb, d);
    }
}

template <int NW, bool HV>
__global__ void __launch_bounds__(kMergeThreads) merge_kernel(const uint64_t* __restrict__ keys,
                                                              const uint32_t* __restrict__ vals,
                                                              uint64_t* __restrict__ out, uint32_t* __restrict__ vout,
                                                              const MergePair* __restrict__ pairs, int n_pairs,
                                                              const uint64_t* __restrict__ part) {
    constexpr int ITEMS = merge_items<NW>();
    constexpr int T = merge_tile<NW>();
    __shared__ uint64_t sk[T * NW];
    __shared__ uint32_t sv[HV ? T : 1];
    const uint64_t c = blockIdx.x;
    const int p = pair_of(pairs, n_pairs, c);
    const MergePair P = pairs[p];
    const uint64_t cl = c - P.cta0, total = P.na + P.nb;
    const uint64_t d0 = cl * T, d1 = d0 + T < total ? d0 + T : total;
    const uint64_t i0 = part[c];
    const bool last = (p + 1 < n_pairs) ? (c + 1 == pairs[p + 1].cta0) : (d1 == total);
    const uint64_t i1 = last ? P.na : part[c + 1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    const uint32_t la = (uint32_t)(i1 - i0), lb = (uint32_t)(j1 - j0), n = la + lb;
    const uint64_t* xa = keys + (P.a + i0) * NW;
    const uint64_t* xb = keys + (P.a + P.na + j0) * NW;
    // n <= T keys: every thread has ITEMS loads in flight
#pragma unroll
    for (int q = 0; q < ITEMS; q++) {
        const uint32_t t = threadIdx.x + q * kMergeThreads;
        if (t < n) {
            const Key<NW> v = t < la ? load_key<NW>(xa, t) : load_key<NW>(xb, t - la);
#pragma unroll
            for (int w = 0; w < NW; w++) sk[t * NW + w] = v.w[w];
            if constexpr (HV) sv[t] = t < la ? vals[P.a + i0 + t] : vals[P.a + P.na + j0 + t - la];
        }
    }
    __syncthreads();
    auto skey = [&](uint32_t i) {
        Key<NW> r;
#pragma unroll
        for (int w = 0; w < NW; w++) r.w[w] = sk[i * NW + w];
        return r;
    };
    // this thread's outputs dt .. dt + ITEMS - 1
    const uint32_t dt = threadIdx.x * ITEMS;
    Key<NW> ok[ITEMS];
    uint32_t ov[HV ? ITEMS : 1];
    if (dt < n) {
        uint32_t lo = dt > lb ? dt - lb : 0, hi = dt < la ? dt : la;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (key_le<NW>(skey(mid), skey(la + dt - 1 - mid))) lo = mid + 1; else hi = mid;
        }
        uint32_t ia = lo, ib = dt - lo;
#pragma unroll
        for (int q = 0; q < ITEMS; q++) {
            if (dt + q < n) {
                const bool take_a = ib >= lb || (ia < la && key_le<NW>(skey(ia), skey(la + ib)));
                const uint32_t src = take_a ? ia : la + ib;
                ok[q] = skey(src);
                if constexpr (HV) ov[q] = sv[src];
                if (take_a) ia++; else ib++;
            }
        }
    }
    __syncthreads();
    if (dt < n) {
#pragma unroll
        for (int q = 0; q < ITEMS; q++) {
            if (dt + q < n) {
#pragma unroll
                for (int w = 0; w < NW; w++) sk[(dt + q) * NW + w] = ok[q].w[w];
                if constexpr (HV) sv[dt + q] = ov[q];
            }
        }
    }
    __syncthreads();
    uint64_t* o = out + (P.a + d0) * NW;
    for (uint32_t t = threadIdx.x; t < n * NW; t += kMergeThreads) o[t] = sk[t];
    if constexpr (HV)
        for (uint32_t t = threadIdx.x; t < n; t += kMergeThreads) vout[P.a + d0 + t] = sv[t];
}

template <int NW>
bool merge_runs(mh_ctx* ctx, uint64_t* keys, uint64_t* alt, uint32_t* vals, uint32_t* valt,
                const std::vector<uint64_t>& bounds) {
    constexpr int T = merge_tile<NW>();
    // runs [bounds[i], bounds[i+1]), empty ones dropped
    std::vector<std::pair<uint64_t, uint64_t>> runs;
    for (size_t i = 0; i + 1 < bounds.size(); i++)
        if (bounds[i + 1] > bounds[i]) runs.push_back({bounds[i], bounds[i + 1] - bounds[i]});
    bool in_alt = false;
    while (runs.size() > 1) {
        const uint64_t* src = in_alt ? alt : keys;
        uint64_t* dst = in_alt ? keys : alt;
        const uint32_t* vsrc = in_alt ? valt : vals;
        uint32_t* vdst = in_alt ? vals : valt;
        std::vector<MergePair> pairs;
        std::vector<std::pair<uint64_t, uint64_t>> next;
        uint64_t ctas = 0;
        for (size_t r = 0; r + 1 < runs.size(); r += 2) {
            const uint64_t na = runs[r].second, nb = runs[r + 1].second;
            pairs.push_back({runs[r].first, na, nb, ctas});
            ctas += ceil_div(na + nb, (uint64_t)T);
            next.push_back({runs[r].first, na + nb});
        }
        if (runs.size() % 2) {
            const auto& r = runs.back();
            MH_CUDA(cudaMemcpyAsync(dst + r.first * NW, src + r.first * NW, r.second * NW * sizeof(uint64_t),
                                    cudaMemcpyDeviceToDevice, ctx->stream));
            if (vals)
                MH_CUDA(cudaMemcpyAsync(vdst + r.first, vsrc + r.first, r.second * sizeof(uint32_t),
                                        cudaMemcpyDeviceToDevice, ctx->stream));
            next.push_back(r);
        }
        Buf<MergePair> dpairs(ctx, pairs.size());
        Buf<uint64_t> part(ctx, ctas);
        MH_CUDA(cudaMemcpyAsync(dpairs.p, pairs.data(), pairs.size() * sizeof(MergePair), cudaMemcpyHostToDevice,
                                ctx->stream));
        MH_LAUNCH(ctx, "merge_partition", grid_for(ctx, ctas, 256), 256, 0, merge_partition_kernel<NW>, src, dpairs.p,
                  (int)pairs.size(), ctas, part.p);
        uint64_t bytes = 0;
        for (const auto& q : pairs) bytes += 2 * (q.na + q.nb) * (8 * NW + (vals ? 4 : 0));
        if (vals)
            MH_LAUNCH_B(ctx, "merge", bytes, (unsigned)ctas, kMergeThreads, 0, (merge_kernel<NW, true>), src, vsrc, dst,
                        vdst, dpairs.p, (int)pairs.size(), part.p);
        else
            MH_LAUNCH_B(ctx, "merge", bytes, (unsigned)ctas, kMergeThreads, 0, (merge_kernel<NW, false>), src, nullptr,
                        dst, nullptr, dpairs.p, (int)pairs.size(), part.p);
        runs.swap(next);
        in_alt = !in_alt;
    }
    return in_alt;
}

// --------------------------------------------------------- set differences
// X and Y sorted, each without repeats.  In their merge (ties: X first) an
// element of both sets has its Y copy right after its X copy, so x in X is
// in Y iff the next merged element equals x, and y in Y is in X iff the
// previous one equals y; across a CTA's slice boundary that neighbour is
// Y[j1] (next) or X[i0 - 1] (previous).

template <int NW>
__global__ void diff_partition_kernel(const uint64_t* __restrict__ X, uint64_t nx, const uint64_t* __restrict__ Y,
                                      uint64_t ny, uint64_t n_ctas, uint64_t* __restrict__ part) {
    constexpr int T = diff_tile<NW>();
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c <= n_ctas;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = c * T < nx + ny ? c * T : nx + ny;
        part[c] = merge_path<NW>(X, nx, Y, ny, d);
    }
}

// The elements of X \ Y and Y \ X of each CTA's slice, compacted in order
// into outX / outY (one decoupled look-back per output over dynamic tile ids).
template <int NW>
__global__ void __launch_bounds__(kMergeThreads) diff_kernel(const uint64_t* __restrict__ X, uint64_t nx,
                                                             const uint64_t* __restrict__ Y, uint64_t ny,
                                                             const uint64_t* __restrict__ part,
                                                             uint64_t* __restrict__ status_x,
                                                             uint64_t* __restrict__ status_y,
                                                             uint32_t* __restrict__ tile_counter,
                                                             uint64_t* __restrict__ outX, uint64_t* __restrict__ outY,
                                                             uint32_t* __restrict__ err) {
    constexpr int ITEMS = diff_items<NW>();
    constexpr int T = diff_tile<NW>();
    __shared__ uint64_t sx[T * NW], sy[T * NW];
    __shared__ uint32_t scratch[8];
    __shared__ uint64_t offs[2];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint64_t c = s_tile;
    const uint64_t d0 = c * T, d1 = d0 + T < nx + ny ? d0 + T : nx + ny;
    const uint64_t i0 = part[c], i1 = part[c + 1];
    const uint64_t j0 = d0 - i0, j1 = d1 - i1;
    const uint32_t la = (uint32_t)(i1 - i0), lb = (uint32_t)(j1 - j0);
    for (uint32_t t = threadIdx.x; t < la * NW; t += kMergeThreads) sx[t] = X[i0 * NW + t];
    for (uint32_t t = threadIdx.x; t < lb * NW; t += kMergeThreads) sy[t] = Y[j0 * NW + t];
    __syncthreads();
    auto get = [&](const uint64_t* a, uint32_t i) {
        Key<NW> r;
#pragma unroll
        for (int w = 0; w < NW; w++) r.w[w] = a[i * NW + w];
        return r;
    };
    // the neighbours outside the slice: the Y element after it, the X element before it
    const bool has_next = j1 < ny, has_prev = i0 > 0;
    Key<NW> next_y, prev_x;
    if (has_next) next_y = load_key<NW>(Y, j1);
    if (has_prev) prev_x = load_key<NW>(X, i0 - 1);
    // this thread's merged positions dt .. dt + ITEMS - 1: split, then walk
    const uint32_t n = la + lb, dt = threadIdx.x * ITEMS;
    uint32_t mx = 0, my = 0;
    Key<NW> val[ITEMS];
    if (dt < n) {
        uint32_t lo = dt > lb ? dt - lb : 0, hi = dt < la ? dt : la;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (key_le<NW>(get(sx, mid), get(sy, dt - 1 - mid))) lo = mid + 1; else hi = mid;
        }
        uint32_t ia = lo, ib = dt - lo;
#pragma unroll
        for (int q = 0; q < ITEMS; q++) {
            if (dt + q >= n) continue;
            const bool take_x = ib >= lb || (ia < la && key_le<NW>(get(sx, ia), get(sy, ib)));
            if (take_x) {
                const Key<NW> x = get(sx, ia);
                val[q] = x;
                const bool in_y = ib < lb ? key_eq<NW>(get(sy, ib), x) : (has_next && key_eq<NW>(next_y, x));
                if (!in_y) mx |= 1u << q;
                ia++;
            } else {
                const Key<NW> y = get(sy, ib);
                val[q] = y;
                const bool in_x = ia > 0 ? key_eq<NW>(get(sx, ia - 1), y) : (has_prev && key_eq<NW>(prev_x, y));
                if (!in_x) my |= 1u << q;
                ib++;
            }
        }
    }
    uint32_t tx, ty;
    const uint32_t ex = block_excl_scan_256(__popc(mx), scratch, &tx);
    const uint32_t ey = block_excl_scan_256(__popc(my), scratch, &ty);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        const uint64_t o = warp_lookback_u64(status_x, c, tx, err);
        if ((threadIdx.x & 31) == 0) offs[0] = o;
    } else if (warp == 1) {
        const uint64_t o = warp_lookback_u64(status_y, c, ty, err);
        if ((threadIdx.x & 31) == 0) offs[1] = o;
    }
    __syncthreads();
    uint64_t px = offs[0] + ex, py = offs[1] + ey;
#pragma unroll
    for (int q = 0; q < ITEMS; q++) {
        if ((mx >> q) & 1u) store_key<NW>(outX, px++, val[q]);
        if ((my >> q) & 1u) store_key<NW>(outY, py++, val[q]);
    }
}

template <int NW>
void set_differences(mh_ctx* ctx, const uint64_t* X, uint64_t nx, const uint64_t* Y, uint64_t ny, uint64_t* outX,
                     uint64_t* n_outX, uint64_t* outY, uint64_t* n_outY) {
    constexpr int T = diff_tile<NW>();
    *n_outX = *n_outY = 0;
    if (nx + ny == 0) return;
    const uint64_t ctas = ceil_div(nx + ny, (uint64_t)T);
    Buf<uint64_t> part(ctx, ctas + 1), st(ctx, 2 * ctas);
    Buf<uint32_t> counter(ctx, 1);
    st.zero();
    counter.zero();
    MH_LAUNCH(ctx, "diff_partition", grid_for(ctx, ctas + 1, 256), 256, 0, diff_partition_kernel<NW>, X, nx, Y, ny,
              ctas, part.p);
    MH_LAUNCH_B(ctx, "set_differences", (nx + ny) * 8 * NW, (unsigned)ctas, kMergeThreads, 0, diff_kernel<NW>, X, nx,
                Y, ny, part.p, st.p, st.p + ctas, counter.p, outX, outY, ctx->d_status);
    uint64_t last[2];
    read_u64(ctx, st.p + ctas - 1, &last[0], 1);
    read_u64(ctx, st.p + 2 * ctas - 1, &last[1], 1);
    *n_outX = last[0] & kLbCountMask;
    *n_outY = last[1] & kLbCountMask;
}

template void set_differences<1>(mh_ctx*, const uint64_t*, uint64_t, const uint64_t*, uint64_t, uint64_t*, uint64_t*,
                                 uint64_t*, uint64_t*);
template void set_differences<2>(mh_ctx*, const uint64_t*, uint64_t, const uint64_t*, uint64_t, uint64_t*, uint64_t*,
                                 uint64_t*, uint64_t*);
template void set_differences<4>(mh_ctx*, const uint64_t*, uint64_t, const uint64_t*, uint64_t, uint64_t*, uint64_t*,
                                 uint64_t*, uint64_t*);

template bool merge_runs<1>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, const std::vector<uint64_t>&);
template bool merge_runs<2>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, const std::vector<uint64_t>&);
template bool merge_runs<4>(mh_ctx*, uint64_t*, uint64_t*, uint32_t*, uint32_t*, const std::vector<uint64_t>&);

}  // namespace mh
