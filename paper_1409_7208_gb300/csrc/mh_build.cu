// mh_build_sdbg: the BOSS arrays of E = solid + mercy (paper, Sec. 2, first
// and second paragraphs).
//
//   colex     ck(e) = (e[k-1], ..., e[0], e[k]) packed, so integer order of ck
//             is colex order of the k-prefix, then the label
//   order     no sort: solid and mercy are lex-sorted and closed under
//             reverse complement, and for f = rc(e), ck(e) is ~f rotated by
//             one symbol ((f[1..k] complemented, then comp f[0])).  Walking a
//             table backwards from its end, each block of equal first symbol
//             f[0] gives ck ascending; so the ck of solid and mercy edges are
//             8 sorted runs, merged by a tree of merge-path merges
//   analyse   per entry: minus flag (an earlier entry of the same group
//             e[1..k-1] has the same label; groups are contiguous and hold at
//             most 16 entries), node head/last flags
//   nodes     B = reversed source nodes (ck >> 2 at heads), ascending
//   targets   A = reversed targets (label, e[k-1], ..., e[1]) of unflagged
//             entries; already ascending within each label, so one stable
//             radix pass on their top 8 bits sorts them
//   joins     zero indegree = B \ A, zero outdegree = A \ B, both from one
//             merge-path merge of A and B (an element of both has its copies
//             adjacent in the merge); B and A are tile compactions with a
//             decoupled look-back
//   padding   dummy entries (node $ v[0..k-2], label v[k-1]) sorted by
//             (v[k-2..0], v[k-1]); $ entries in the order of A \ B
//   merge     final position of every entry: its rank in its own list plus
//             the number of entries of the other lists below it, by binary
//             search and a scan of insertion counts over E
//   emit      W with minus flag, last, dummy, valid bit-vectors, aux, F, mult
#include "mh_internal.cuh"

namespace mh {

// ck -> group G = ck >> 4 (node symbols k-1..1), tail = pos0' * 5 + label',
// with pos0' = node symbol 0 + 1 and label' = label + 1 ($ = 0 for both).
template <int NW>
__device__ __forceinline__ bool ext_less(const Key<NW>& ga, uint32_t ta, const Key<NW>& gb, uint32_t tb) {
    if (!key_eq<NW>(ga, gb)) return key_less<NW>(ga, gb);
    return ta < tb;
}

template <int NW>
__device__ __forceinline__ void ext_of_ck(const Key<NW>& ck, Key<NW>& g, uint32_t& tail) {
    g = key_shr<NW>(ck, 4);
    uint32_t lo = (uint32_t)(ck.w[0] & 15u);
    tail = ((lo >> 2) + 1) * 5 + (lo & 3) + 1;
}

// dummy key dk = (v[k-2], ..., v[0], v[k-1]) (k symbols): G = dk >> 2, tail = label'
template <int NW>
__device__ __forceinline__ void ext_of_dummy(const Key<NW>& dk, Key<NW>& g, uint32_t& tail) {
    g = key_shr<NW>(dk, 2);
    tail = (uint32_t)(dk.w[0] & 3u) + 1;
}

// $ entry of reversed node u_rev = (u[k-1], ..., u[0]): G = u_rev >> 2, tail = (u[0]+1)*5
template <int NW>
__device__ __forceinline__ void ext_of_dollar(const Key<NW>& ur, Key<NW>& g, uint32_t& tail) {
    g = key_shr<NW>(ur, 2);
    tail = ((uint32_t)(ur.w[0] & 3u) + 1) * 5;
}

// Lower bound of (g, t) in a sorted list whose i-th element's ext key is given by ExtOf.
template <int NW, int KIND>
__device__ __forceinline__ uint64_t lb_ext(const uint64_t* __restrict__ a, uint64_t n, const Key<NW>& g, uint32_t t) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        Key<NW> x = load_key<NW>(a, mid), gx;
        uint32_t tx;
        if (KIND == 0) ext_of_ck<NW>(x, gx, tx);
        else if (KIND == 1) ext_of_dummy<NW>(x, gx, tx);
        else ext_of_dollar<NW>(x, gx, tx);
        if (ext_less<NW>(gx, tx, g, t)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Colex keys of the reverse complements of the tables, read backwards:
// out[i] = ck(rc(s[ns-1-i])) for i < ns, then the same for m; counts move
// along as payload.  ck(rc(f)) = (~f[1..k] << 2) | comp f[0].
template <int NW>
__global__ void colex_kernel(const uint64_t* __restrict__ s, const uint32_t* __restrict__ sc, uint64_t ns,
                             const uint64_t* __restrict__ m, const uint32_t* __restrict__ mc, uint64_t nm, int k,
                             uint64_t* __restrict__ ck, uint32_t* __restrict__ cv) {
    const uint64_t n = ns + nm;
    const int K1 = k + 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t src = i < ns ? ns - 1 - i : nm - 1 - (i - ns);
        Key<NW> f = i < ns ? load_key<NW>(s, src) : load_key<NW>(m, src);
#pragma unroll
        for (int w = 0; w < NW; w++) f.w[w] = ~f.w[w];
        f = key_low<NW>(f, 2 * K1);
        const uint32_t top = (uint32_t)(key_shr<NW>(f, 2 * k).w[0] & 3u);
        const Key<NW> c = key_or_low<NW>(key_low<NW>(key_shl<NW>(f, 2), 2 * K1), top);
        store_key<NW>(ck, i, c);
        if (cv) cv[i] = i < ns ? sc[src] : mc[src];
    }
}

// bounds[3 t + c - 1] = first index of table t (0 solid, 1 mercy) whose
// first symbol is >= c, for c = 1, 2, 3.
template <int NW>
__global__ void first_symbol_bounds_kernel(const uint64_t* __restrict__ s, uint64_t ns,
                                           const uint64_t* __restrict__ m, uint64_t nm, int k,
                                           uint64_t* __restrict__ bounds) {
    const int t = threadIdx.x / 3, c = threadIdx.x % 3 + 1;
    if (t >= 2) return;
    const uint64_t* a = t == 0 ? s : m;
    const uint64_t n = t == 0 ? ns : nm;
    Key<NW> q = key_zero<NW>();
    q.w[0] = (uint64_t)c;
    q = key_shl<NW>(q, 2 * k);
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (key_less<NW>(load_key<NW>(a, mid), q)) lo = mid + 1; else hi = mid;
    }
    bounds[threadIdx.x] = lo;
}

// Per sorted entry: flags (bit0 minus, bit1 node head, bit2 node last in E).
template <int NW>
__global__ void analyse_kernel(const uint64_t* __restrict__ ck, uint64_t E, uint8_t* __restrict__ fl) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(ck, i);
        Key<NW> g = key_shr<NW>(x, 4), node = key_shr<NW>(x, 2);
        uint32_t lab = (uint32_t)(x.w[0] & 3u);
        bool minus = false;
        for (uint64_t j = i; j > 0; j--) {
            Key<NW> y = load_key<NW>(ck, j - 1);
            if (!key_eq<NW>(key_shr<NW>(y, 4), g)) break;
            if ((uint32_t)(y.w[0] & 3u) == lab) {
                minus = true;
                break;
            }
        }
        bool head = i == 0 || !key_eq<NW>(key_shr<NW>(load_key<NW>(ck, i - 1), 2), node);
        bool last = i + 1 == E || !key_eq<NW>(key_shr<NW>(load_key<NW>(ck, i + 1), 2), node);
        fl[i] = (minus ? 1 : 0) | (head ? 2 : 0) | (last ? 4 : 0);
    }
}

// Tile compaction: 256 threads x 8 consecutive entries per tile, a block
// scan of the per-thread counts and a decoupled look-back for the tile's
// output offset (one read of the input, no flag or position arrays).
constexpr int kCmpItems = 8;
constexpr int kCmpTile = 256 * kCmpItems;

// Heads (new nodes) -> B = reversed source nodes; unflagged entries -> A =
// reversed targets (label, e[k-1], ..., e[1]).  Two output streams.
template <int NW>
__global__ void __launch_bounds__(256) nodes_targets_kernel(const uint64_t* __restrict__ ck,
                                                            const uint8_t* __restrict__ fl, uint64_t E, int k,
                                                            uint64_t* __restrict__ B, uint64_t* __restrict__ A,
                                                            uint64_t* __restrict__ status_b,
                                                            uint64_t* __restrict__ status_a,
                                                            uint32_t* __restrict__ tile_counter,
                                                            uint32_t* __restrict__ err) {
    __shared__ uint32_t scratch[8];
    __shared__ uint64_t offs[2];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t i0 = tile * kCmpTile + (uint64_t)threadIdx.x * kCmpItems;
    uint32_t hm = 0, pm = 0;
    // the 8 flags in one load, and the keys loaded before the look-back waits
    static_assert(kCmpItems == 8, "one 8-byte flag load per thread");
    uint8_t f8[kCmpItems];
    if (i0 + kCmpItems <= E) {
        const uint2 v = *reinterpret_cast<const uint2*>(fl + i0);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            f8[j] = (uint8_t)(v.x >> (8 * j));
            f8[4 + j] = (uint8_t)(v.y >> (8 * j));
        }
    } else {
#pragma unroll
        for (int j = 0; j < kCmpItems; j++) f8[j] = i0 + j < E ? fl[i0 + j] : 0;
    }
    Key<NW> xs[kCmpItems];
#pragma unroll
    for (int j = 0; j < kCmpItems; j++) {
        if (i0 + j < E) {
            hm |= ((f8[j] >> 1) & 1u) << j;
            pm |= ((f8[j] & 1u) ^ 1u) << j;
            if ((f8[j] & 3u) != 1u) xs[j] = load_key<NW>(ck, i0 + j);
        }
    }
    uint32_t tot_b, tot_a;
    const uint32_t eb = block_excl_scan_256(__popc(hm), scratch, &tot_b);
    const uint32_t ea = block_excl_scan_256(__popc(pm), scratch, &tot_a);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        const uint64_t o = warp_lookback_u64(status_b, tile, tot_b, err);
        if ((threadIdx.x & 31) == 0) offs[0] = o;
    } else if (warp == 1) {
        const uint64_t o = warp_lookback_u64(status_a, tile, tot_a, err);
        if ((threadIdx.x & 31) == 0) offs[1] = o;
    }
    __syncthreads();
    uint64_t pb = offs[0] + eb, pa = offs[1] + ea;
#pragma unroll
    for (int j = 0; j < kCmpItems; j++) {
        if (!(((hm | pm) >> j) & 1u)) continue;
        const Key<NW> x = xs[j];
        if ((hm >> j) & 1u) store_key<NW>(B, pb++, key_shr<NW>(x, 2));
        if ((pm >> j) & 1u) {
            Key<NW> t = key_shr<NW>(x, 4);
            Key<NW> lab = key_zero<NW>();
            lab.w[0] = x.w[0] & 3u;
            lab = key_shl<NW>(lab, 2 * (k - 1));
#pragma unroll
            for (int w = 0; w < NW; w++) t.w[w] |= lab.w[w];
            store_key<NW>(A, pa++, t);
        }
    }
}

// zero-indegree reversed node v_rev -> dummy key (v[k-2], ..., v[0], v[k-1])
template <int NW>
__global__ void dummy_keys_kernel(const uint64_t* __restrict__ zin, uint64_t t, int k, uint64_t* __restrict__ dk) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> v = load_key<NW>(zin, i);
        Key<NW> low = key_low<NW>(v, 2 * (k - 1));
        Key<NW> top = key_shr<NW>(v, 2 * (k - 1));
        store_key<NW>(dk, i, key_or_low<NW>(key_shl<NW>(low, 2), top.w[0] & 3u));
    }
}

// Final positions of dummy (KIND 1) or $ (KIND 2) entries; insertion counts over E.
template <int NW, int KIND>
__global__ void place_pad_kernel(const uint64_t* __restrict__ own, uint64_t n_own, const uint64_t* __restrict__ ck,
                                 uint64_t E, const uint64_t* __restrict__ other, uint64_t n_other,
                                 uint64_t* __restrict__ final_pos, uint32_t* __restrict__ ins) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_own;
         i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(own, i), g;
        uint32_t t;
        if (KIND == 1) ext_of_dummy<NW>(x, g, t); else ext_of_dollar<NW>(x, g, t);
        uint64_t le = lb_ext<NW, 0>(ck, E, g, t);
        uint64_t lo = KIND == 1 ? lb_ext<NW, 2>(other, n_other, g, t) : lb_ext<NW, 1>(other, n_other, g, t);
        final_pos[i] = le + i + lo;
        atomicAdd(&ins[le], 1u);
    }
}

// Add a thread's 4 symbol counts to the global histogram (warp-reduced first).
__device__ __forceinline__ void flush_hist4(const uint32_t h[4], unsigned long long* __restrict__ hist) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint32_t v = h[c];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&hist[c], (unsigned long long)v);
    }
}

// W byte: low 4 bits W code, bit 4 last, bit 5 dummy.
template <int NW>
__global__ void emit_edges_kernel(const uint64_t* __restrict__ ck, const uint32_t* __restrict__ cv, uint64_t E, int K1,
                                  const uint8_t* __restrict__ fl, const uint64_t* __restrict__ shift,
                                  uint8_t* __restrict__ wf, uint32_t* __restrict__ mult,
                                  unsigned long long* __restrict__ hist) {
    uint32_t h[4] = {0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(ck, i);
        uint8_t f = fl[i];
        uint32_t lab = (uint32_t)(x.w[0] & 3u) + 1;
        uint64_t p = i + shift[i + 1];
        wf[p] = (uint8_t)((lab + ((f & 1) ? 4 : 0)) | ((f & 4) ? 16 : 0));
        if (mult) mult[p] = cv ? cv[i] : 0;
        h[key_sym<NW>(x, K1, 0)]++;
    }
    flush_hist4(h, hist);
}

template <int NW>
__global__ void emit_dummy_kernel(const uint64_t* __restrict__ dk, uint64_t t, int k, const uint64_t* __restrict__ pos,
                                  uint8_t* __restrict__ wf, uint32_t* __restrict__ mult, uint64_t* __restrict__ aux,
                                  unsigned long long* __restrict__ hist) {
    uint32_t h[4] = {0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < t; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(dk, i);
        Key<NW> g = key_shr<NW>(x, 2);
        bool last = i + 1 == t || !key_eq<NW>(key_shr<NW>(load_key<NW>(dk, i + 1), 2), g);
        uint32_t lab = (uint32_t)(x.w[0] & 3u);
        uint64_t p = pos[i];
        wf[p] = (uint8_t)((lab + 1) | (last ? 16 : 0) | 32);
        if (mult) mult[p] = 0;
        // v = reverse of v_rev, v_rev = (v[k-1], v[k-2], ..., v[0]) = lab * 4^(k-1) + g
        Key<NW> top = key_zero<NW>();
        top.w[0] = lab;
        top = key_shl<NW>(top, 2 * (k - 1));
        Key<NW> vr = g;
#pragma unroll
        for (int w = 0; w < NW; w++) vr.w[w] |= top.w[w];
        store_key<NW>(aux, i, key_rev<NW>(vr, k));
        h[key_sym<NW>(x, k, 0)]++;  // node symbol k-1 = v[k-2], the top symbol of x
    }
    flush_hist4(h, hist);
}

template <int NW>
__global__ void emit_dollar_kernel(const uint64_t* __restrict__ ur, uint64_t u, int k, const uint64_t* __restrict__ pos,
                                   uint8_t* __restrict__ wf, uint32_t* __restrict__ mult,
                                   unsigned long long* __restrict__ hist) {
    uint32_t h[4] = {0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < u; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(ur, i);
        uint64_t p = pos[i];
        wf[p] = (uint8_t)(0 | 16);
        if (mult) mult[p] = 0;
        h[key_sym<NW>(x, k, 0)]++;  // u[k-1], the top symbol of u_rev
    }
    flush_hist4(h, hist);
}

// W bytes -> W codes and the last / dummy / valid bit-vectors (warp per 32 entries).
__global__ void pack_bits_kernel(const uint8_t* __restrict__ wf, uint64_t m, uint8_t* __restrict__ W,
                                 uint32_t* __restrict__ last, uint32_t* __restrict__ dummy,
                                 uint32_t* __restrict__ valid, unsigned long long* __restrict__ n_last) {
    const int lane = threadIdx.x & 31;
    const uint64_t n_words = ceil_div(m, 32);
    uint32_t cnt = 0;
    for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < n_words;
         w += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        uint64_t i = w * 32 + lane;
        uint8_t b = i < m ? wf[i] : 0;
        if (i < m) W[i] = b & 15;
        uint32_t lb = __ballot_sync(0xFFFFFFFFu, (b & 16) != 0);
        uint32_t db = __ballot_sync(0xFFFFFFFFu, (b & 32) != 0);
        uint32_t vb = __ballot_sync(0xFFFFFFFFu, i < m);
        if (lane == 0) {
            last[w] = lb;
            dummy[w] = db;
            valid[w] = vb;
            cnt += __popc(lb);
        }
    }
    if (lane == 0 && cnt) atomicAdd(n_last, (unsigned long long)cnt);
}

template <int NW>
void build_sdbg(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, mh_sdbg* out) {
    const int k = solid->k, K1 = k + 1;
    const uint64_t nS = solid->n, nM = mercy ? mercy->n : 0, E = nS + nM;
    const bool want_mult = ctx->with_mult != 0;
    out->k = k;
    out->nw = NW;
    // colex keys, sorted
    Buf<uint64_t> ck(ctx, (E ? E : 1) * NW), ck2(ctx, (E ? E : 1) * NW);
    Buf<uint32_t> cv, cv2;
    if (want_mult) {
        cv = Buf<uint32_t>(ctx, E ? E : 1);
        cv2 = Buf<uint32_t>(ctx, E ? E : 1);
    }
    if (E) {
        Buf<uint64_t> fb(ctx, 6);
        MH_LAUNCH(ctx, "first_symbol_bounds", 1, 32, 0, first_symbol_bounds_kernel<NW>, solid->keys, nS,
                  mercy ? mercy->keys : nullptr, nM, k, fb.p);
        MH_LAUNCH(ctx, "colex_keys", grid_for(ctx, E, 256), 256, 0, colex_kernel<NW>, solid->keys, solid->counts, nS,
                  mercy ? mercy->keys : nullptr, mercy ? mercy->counts : nullptr, nM, k, ck.p,
                  want_mult ? cv.p : nullptr);
        uint64_t b[6];
        read_u64(ctx, fb.p, b, 6);
        // runs (label A, C, G, T) of each table: its first-symbol blocks T, G, C, A
        const std::vector<uint64_t> runs = {0, nS - b[2], nS - b[1], nS - b[0], nS,
                                            nS + nM - b[5], nS + nM - b[4], nS + nM - b[3], E};
        if (merge_runs<NW>(ctx, ck.p, ck2.p, want_mult ? cv.p : nullptr, want_mult ? cv2.p : nullptr, runs)) {
            std::swap(ck, ck2);
            std::swap(cv, cv2);
        }
    }
    ck2.reset();
    cv2.reset();
    // per-entry flags, node list B, target list A
    Buf<uint8_t> fl(ctx, E ? E : 1);
    if (E) MH_LAUNCH(ctx, "analyse", grid_for(ctx, E, 256), 256, 0, analyse_kernel<NW>, ck.p, E, fl.p);
    Buf<uint64_t> B(ctx, (E ? E : 1) * NW), A(ctx, (E ? E : 1) * NW);
    uint64_t nB = 0, nA = 0;
    if (E) {
        const uint64_t tiles = ceil_div(E, kCmpTile);
        Buf<uint64_t> st(ctx, 2 * tiles);
        Buf<uint32_t> counter(ctx, 1);
        st.zero();
        counter.zero();
        MH_LAUNCH(ctx, "nodes_targets", (unsigned)tiles, 256, 0, nodes_targets_kernel<NW>, ck.p, fl.p, E, k, B.p, A.p,
                  st.p, st.p + tiles, counter.p, ctx->d_status);
        uint64_t last[2];
        read_u64(ctx, st.p + tiles - 1, &last[0], 1);
        read_u64(ctx, st.p + 2 * tiles - 1, &last[1], 1);
        nB = last[0] & kLbCountMask;
        nA = last[1] & kLbCountMask;
    }
    Buf<uint64_t> A2(ctx, (nA ? nA : 1) * NW);
    if (radix_sort<NW>(ctx, A.p, A2.p, nullptr, nullptr, nA, std::max(0, 2 * k - 8), 2 * k)) std::swap(A, A2);
    A2.reset();
    // zero indegree: B \ A; zero outdegree: A \ B
    Buf<uint64_t> zin(ctx, (nB ? nB : 1) * NW), zout(ctx, (nA ? nA : 1) * NW);
    uint64_t t = 0, u = 0;
    set_differences<NW>(ctx, B.p, nB, A.p, nA, zin.p, &t, zout.p, &u);
    B.reset();
    A.reset();
    // dummy entries in colex order
    Buf<uint64_t> dk(ctx, (t ? t : 1) * NW), dk2(ctx, (t ? t : 1) * NW);
    if (t) MH_LAUNCH(ctx, "dummy_keys", grid_for(ctx, t, 256), 256, 0, dummy_keys_kernel<NW>, zin.p, t, k, dk.p);
    if (radix_sort<NW>(ctx, dk.p, dk2.p, nullptr, nullptr, t, 0, 2 * k)) std::swap(dk, dk2);
    dk2.reset();
    zin.reset();
    // merge positions
    const uint64_t m = E + t + u;
    Buf<uint32_t> ins(ctx, E + 1);
    ins.zero();
    Buf<uint64_t> pos_d(ctx, t ? t : 1), pos_u(ctx, u ? u : 1), shift(ctx, E + 2);
    if (t)
        MH_LAUNCH(ctx, "place_dummy", grid_for(ctx, t, 256), 256, 0, (place_pad_kernel<NW, 1>), dk.p, t, ck.p, E,
                  zout.p, u, pos_d.p, ins.p);
    if (u)
        MH_LAUNCH(ctx, "place_dollar", grid_for(ctx, u, 256), 256, 0, (place_pad_kernel<NW, 2>), zout.p, u, ck.p, E,
                  dk.p, t, pos_u.p, ins.p);
    exclusive_scan_u32(ctx, ins.p, shift.p, E + 1);
    ins.reset();
    // emit
    Buf<uint8_t> wf(ctx, m ? m : 1);
    Buf<unsigned long long> hist(ctx, 8);
    hist.zero();
    Buf<uint32_t> mult;
    if (want_mult) mult = Buf<uint32_t>(ctx, m ? m : 1);
    if (E)
        MH_LAUNCH(ctx, "emit_edges", grid_for(ctx, E, 256), 256, 0, emit_edges_kernel<NW>, ck.p,
                  want_mult ? cv.p : nullptr, E, K1, fl.p, shift.p, wf.p, want_mult ? mult.p : nullptr, hist.p);
    const uint64_t nwk = (uint64_t)NW;
    Buf<uint64_t> aux(ctx, (t ? t : 1) * nwk);
    if (t)
        MH_LAUNCH(ctx, "emit_dummy", grid_for(ctx, t, 256), 256, 0, emit_dummy_kernel<NW>, dk.p, t, k, pos_d.p, wf.p,
                  want_mult ? mult.p : nullptr, aux.p, hist.p);
    if (u)
        MH_LAUNCH(ctx, "emit_dollar", grid_for(ctx, u, 256), 256, 0, emit_dollar_kernel<NW>, zout.p, u, k, pos_u.p, wf.p,
                  want_mult ? mult.p : nullptr, hist.p);
    ck.reset();
    cv.reset();
    fl.reset();
    shift.reset();
    const uint64_t n_words = ceil_div(m, 32);
    Buf<uint8_t> W(ctx, m ? m : 1);
    Buf<uint32_t> last(ctx, n_words ? n_words : 1), dummy(ctx, n_words ? n_words : 1), valid(ctx, n_words ? n_words : 1);
    if (m)
        MH_LAUNCH(ctx, "pack_bits", grid_for(ctx, n_words * 32, 256), 256, 0, pack_bits_kernel, wf.p, m, W.p, last.p,
                  dummy.p, valid.p, hist.p + 4);
    uint64_t h[5];
    read_u64(ctx, reinterpret_cast<const uint64_t*>(hist.p), h, 5);
    out->m = m;
    out->t = t;
    out->u = u;
    out->n_nodes = h[4];
    out->F[0] = 0;
    out->F[1] = 0;
    out->F[2] = h[0];
    out->F[3] = h[0] + h[1];
    out->F[4] = h[0] + h[1] + h[2];
    out->F[5] = m;
    out->W = W.release();
    out->last = last.release();
    out->dummy = dummy.release();
    out->valid = valid.release();
    out->aux = aux.release();
    out->mult = want_mult ? mult.release() : nullptr;
}

template void build_sdbg<1>(mh_ctx*, const mh_kmers*, const mh_kmers*, mh_sdbg*);
template void build_sdbg<2>(mh_ctx*, const mh_kmers*, const mh_kmers*, mh_sdbg*);
template void build_sdbg<4>(mh_ctx*, const mh_kmers*, const mh_kmers*, mh_sdbg*);

}  // namespace mh
