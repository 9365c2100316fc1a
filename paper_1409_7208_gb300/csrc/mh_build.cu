// mh_build_sdbg: the BOSS arrays of E = solid + mercy (paper, Sec. 2, first
// and second paragraphs).
//
//   colex     ck(e) = (e[k-1], ..., e[0], e[k]) packed, so integer order of ck
//             is colex order of the k-prefix, then the label
//   sort      LSD radix over ck
//   analyse   per entry: minus flag (an earlier entry of the same group
//             e[1..k-1] has the same label; groups are contiguous and hold at
//             most 16 entries), node head/last flags
//   nodes     B = reversed source nodes (ck >> 2 at heads), ascending
//   targets   A = reversed targets (label, e[k-1], ..., e[1]) of unflagged
//             entries; already ascending within each label, so one stable
//             radix pass on their top 8 bits sorts them
//   joins     zero indegree = B \ A, zero outdegree = A \ B (sorted queries
//             in sorted arrays: each thread gallops through 16 consecutive
//             queries)
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

// Edge keys (solid then mercy) -> colex keys, with counts as payload.
template <int NW>
__global__ void colex_kernel(const uint64_t* __restrict__ s, const uint32_t* __restrict__ sc, uint64_t ns,
                             const uint64_t* __restrict__ m, const uint32_t* __restrict__ mc, uint64_t nm, int k,
                             uint64_t* __restrict__ ck, uint32_t* __restrict__ cv) {
    uint64_t n = ns + nm;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> e = i < ns ? load_key<NW>(s, i) : load_key<NW>(m, i - ns);
        Key<NW> node = key_shr<NW>(e, 2);
        Key<NW> c = key_or_low<NW>(key_shl<NW>(key_rev<NW>(node, k), 2), e.w[0] & 3u);
        store_key<NW>(ck, i, c);
        if (cv) cv[i] = i < ns ? sc[i] : mc[i - ns];
    }
}

// Per sorted entry: flags (bit0 minus, bit1 node head, bit2 node last in E),
// and selection flags for B (heads) and A (unflagged entries).
template <int NW>
__global__ void analyse_kernel(const uint64_t* __restrict__ ck, uint64_t E, uint8_t* __restrict__ fl,
                               uint32_t* __restrict__ is_head, uint32_t* __restrict__ is_plain) {
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
        is_head[i] = head;
        is_plain[i] = !minus;
    }
}

template <int NW>
__global__ void select_nodes_targets_kernel(const uint64_t* __restrict__ ck, uint64_t E, int k,
                                            const uint32_t* __restrict__ is_head, const uint64_t* __restrict__ pos_b,
                                            const uint32_t* __restrict__ is_plain, const uint64_t* __restrict__ pos_a,
                                            uint64_t* __restrict__ B, uint64_t* __restrict__ A) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(ck, i);
        if (is_head[i]) store_key<NW>(B, pos_b[i], key_shr<NW>(x, 2));
        if (is_plain[i]) {
            // reversed target (label, e[k-1], ..., e[1]) = label * 4^(k-1) + G
            Key<NW> t = key_shr<NW>(x, 4);
            Key<NW> lab = key_zero<NW>();
            lab.w[0] = x.w[0] & 3u;
            lab = key_shl<NW>(lab, 2 * (k - 1));
#pragma unroll
            for (int w = 0; w < NW; w++) t.w[w] |= lab.w[w];
            store_key<NW>(A, pos_a[i], t);
        }
    }
}

// flag[i] = 1 iff q[i] is absent from the sorted array a.  The queries are
// sorted too: each thread takes 16 consecutive ones and gallops from the
// previous answer.
constexpr int kAbsentRun = 16;
template <int NW>
__global__ void absent_kernel(const uint64_t* __restrict__ q, uint64_t nq, const uint64_t* __restrict__ a, uint64_t na,
                              uint32_t* __restrict__ flag) {
    for (uint64_t i0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * kAbsentRun; i0 < nq;
         i0 += (uint64_t)gridDim.x * blockDim.x * kAbsentRun) {
        uint64_t hint = na / 2;
        const uint64_t i1 = i0 + kAbsentRun < nq ? i0 + kAbsentRun : nq;
        for (uint64_t i = i0; i < i1; i++) {
            Key<NW> x = load_key<NW>(q, i);
            uint64_t lb = gallop_lb<NW>(a, na, x, hint);
            hint = lb;
            flag[i] = !(lb < na && key_eq<NW>(load_key<NW>(a, lb), x));
        }
    }
}

template <int NW>
__global__ void select_kernel(const uint64_t* __restrict__ in, const uint32_t* __restrict__ flag,
                              const uint64_t* __restrict__ pos, uint64_t n, uint64_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (flag[i]) store_key<NW>(out, pos[i], load_key<NW>(in, i));
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
    for (int c = 0; c < 4; c++)
        if (h[c]) atomicAdd(&hist[c], (unsigned long long)h[c]);
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
    for (int c = 0; c < 4; c++)
        if (h[c]) atomicAdd(&hist[c], (unsigned long long)h[c]);
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
    for (int c = 0; c < 4; c++)
        if (h[c]) atomicAdd(&hist[c], (unsigned long long)h[c]);
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

// Exclusive positions of set flags: pos has n+1 entries, pos[n] = count.
static uint64_t flag_positions(mh_ctx* ctx, const uint32_t* flag, uint64_t n, Buf<uint64_t>& pos) {
    pos = Buf<uint64_t>(ctx, n + 1);
    exclusive_scan_u32(ctx, flag, pos.p, n);
    uint64_t c;
    read_u64(ctx, pos.p + n, &c, 1);
    return c;
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
    if (E)
        MH_LAUNCH(ctx, "colex_keys", grid_for(ctx, E, 256), 256, 0, colex_kernel<NW>, solid->keys, solid->counts, nS,
                  mercy ? mercy->keys : nullptr, mercy ? mercy->counts : nullptr, nM, k, ck.p,
                  want_mult ? cv.p : nullptr);
    if (radix_sort<NW>(ctx, ck.p, ck2.p, want_mult ? cv.p : nullptr, want_mult ? cv2.p : nullptr, E, 0, 2 * K1)) {
        std::swap(ck, ck2);
        std::swap(cv, cv2);
    }
    ck2.reset();
    cv2.reset();
    // per-entry flags, node list B, target list A
    Buf<uint8_t> fl(ctx, E ? E : 1);
    Buf<uint32_t> is_head(ctx, E ? E : 1), is_plain(ctx, E ? E : 1);
    if (E)
        MH_LAUNCH(ctx, "analyse", grid_for(ctx, E, 256), 256, 0, analyse_kernel<NW>, ck.p, E, fl.p, is_head.p,
                  is_plain.p);
    Buf<uint64_t> pos_b, pos_a;
    const uint64_t nB = flag_positions(ctx, is_head.p, E, pos_b);
    const uint64_t nA = flag_positions(ctx, is_plain.p, E, pos_a);
    Buf<uint64_t> B(ctx, (nB ? nB : 1) * NW), A(ctx, (nA ? nA : 1) * NW), A2(ctx, (nA ? nA : 1) * NW);
    if (E)
        MH_LAUNCH(ctx, "select_nodes_targets", grid_for(ctx, E, 256), 256, 0, select_nodes_targets_kernel<NW>, ck.p, E,
                  k, is_head.p, pos_b.p, is_plain.p, pos_a.p, B.p, A.p);
    is_head.reset();
    is_plain.reset();
    pos_a.reset();
    pos_b.reset();
    if (radix_sort<NW>(ctx, A.p, A2.p, nullptr, nullptr, nA, std::max(0, 2 * k - 8), 2 * k)) std::swap(A, A2);
    A2.reset();
    // zero indegree: B \ A; zero outdegree: A \ B
    Buf<uint32_t> zf_b(ctx, nB ? nB : 1), zf_a(ctx, nA ? nA : 1);
    if (nB)
        MH_LAUNCH(ctx, "absent_nodes", grid_for(ctx, ceil_div(nB, kAbsentRun), 256), 256, 0, absent_kernel<NW>, B.p, nB,
                  A.p, nA, zf_b.p);
    if (nA)
        MH_LAUNCH(ctx, "absent_targets", grid_for(ctx, ceil_div(nA, kAbsentRun), 256), 256, 0, absent_kernel<NW>, A.p,
                  nA, B.p, nB, zf_a.p);
    Buf<uint64_t> pz_b, pz_a;
    const uint64_t t = flag_positions(ctx, zf_b.p, nB, pz_b);
    const uint64_t u = flag_positions(ctx, zf_a.p, nA, pz_a);
    Buf<uint64_t> zin(ctx, (t ? t : 1) * NW), zout(ctx, (u ? u : 1) * NW);
    if (nB) MH_LAUNCH(ctx, "select_zin", grid_for(ctx, nB, 256), 256, 0, select_kernel<NW>, B.p, zf_b.p, pz_b.p, nB, zin.p);
    if (nA)
        MH_LAUNCH(ctx, "select_zout", grid_for(ctx, nA, 256), 256, 0, select_kernel<NW>, A.p, zf_a.p, pz_a.p, nA, zout.p);
    B.reset();
    A.reset();
    zf_a.reset();
    zf_b.reset();
    pz_a.reset();
    pz_b.reset();
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
