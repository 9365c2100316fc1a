// mh_mercy_kmers: mercy (k+1)-mers (paper, Sec. 2, third paragraph).
//
//   degrees  for each canonical solid edge c: out0(c) = no solid edge starts
//            with c[1..k]; in0(c) = no solid edge ends with c[0..k-1], i.e. no
//            solid edge starts with rc(c)[1..k] (the solid set is closed under
//            reverse complement).  Both are one lower-bound search in the
//            sorted solid table.
//   table    open-addressing hash set of the canonical solid edges with the
//            two flags (linear probing, 32-bit tags, load <= 1/2).
//   scan     warp per fragment, 32 windows at a time: lookup of each window,
//            ballot of the solid ones, previous solid position by bit scan
//            (carried across rounds); a solid window q whose previous solid
//            window p has no outdegree, with q > p+1 and no indegree at q,
//            emits the canonical keys of windows p+1..q-1.
//   finish   sort + dedup of the canonical candidates, counts looked up in the
//            counting spectrum, both strands, sorted.
#include "mh_internal.cuh"

namespace mh {

template <int NW>
struct Slot {
    uint64_t k[NW];
    uint32_t tag;
    uint32_t flags;
};

// First index in the sorted table with key >= q.
template <int NW>
__device__ __forceinline__ uint64_t lower_bound_keys(const uint64_t* __restrict__ a, uint64_t n, const Key<NW>& q) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (key_less<NW>(load_key<NW>(a, mid), q)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Is there a solid (k+1)-mer whose k-prefix is P (a k-symbol key)?
template <int NW>
__device__ __forceinline__ bool has_prefix(const uint64_t* __restrict__ solid, uint64_t S, const Key<NW>& P) {
    Key<NW> q = key_shl<NW>(P, 2);  // P followed by A: the smallest edge with that prefix
    uint64_t lb = lower_bound_keys<NW>(solid, S, q);
    if (lb >= S) return false;
    return key_eq<NW>(key_shr<NW>(load_key<NW>(solid, lb), 2), P);
}

__device__ __forceinline__ uint32_t slot_tag(uint64_t h) { return (uint32_t)(h >> 32) | 1u; }

// For each canonical solid edge: degree flags, then insertion.
template <int NW>
__global__ void __launch_bounds__(256) degree_insert_kernel(const uint64_t* __restrict__ solid, uint64_t S, int k,
                                                            Slot<NW>* __restrict__ table, uint64_t cap_mask,
                                                            unsigned long long* __restrict__ n_out0,
                                                            uint32_t* __restrict__ err) {
    const int K1 = k + 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(solid, i);
        Key<NW> r = key_rc<NW>(x, K1);
        if (key_less<NW>(r, x)) continue;  // only the canonical orientation
        bool out0 = !has_prefix<NW>(solid, S, key_low<NW>(x, 2 * k));
        bool in0 = !has_prefix<NW>(solid, S, key_low<NW>(r, 2 * k));
        uint64_t h = key_hash<NW>(x);
        uint32_t tag = slot_tag(h);
        uint64_t s = h & cap_mask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= cap_mask; probe++) {
            if (atomicCAS(&table[s].tag, 0u, tag) == 0u) {
#pragma unroll
                for (int w = 0; w < NW; w++) table[s].k[w] = x.w[w];
                table[s].flags = (out0 ? 1u : 0u) | (in0 ? 2u : 0u);
                placed = true;
                break;
            }
            s = (s + 1) & cap_mask;
        }
        if (!placed) atomicOr(err, ST_TABLE_FULL);
        if (out0) atomicAdd(n_out0, 1ull);
    }
}

// Flags of canonical key c (bit0 out0, bit1 in0), or -1 if c is not solid.
template <int NW>
__device__ __forceinline__ int table_find(const Slot<NW>* __restrict__ table, uint64_t cap_mask, const Key<NW>& c) {
    uint64_t h = key_hash<NW>(c);
    uint32_t tag = slot_tag(h);
    uint64_t s = h & cap_mask;
    for (uint64_t probe = 0; probe <= cap_mask; probe++) {
        uint32_t t = table[s].tag;
        if (t == 0u) return -1;
        if (t == tag) {
            bool eq = true;
#pragma unroll
            for (int w = 0; w < NW; w++) eq &= table[s].k[w] == c.w[w];
            if (eq) return (int)table[s].flags;
        }
        s = (s + 1) & cap_mask;
    }
    return -1;
}

template <int NW>
__global__ void __launch_bounds__(256) mercy_scan_kernel(const uint32_t* __restrict__ packed,
                                                         const uint64_t* __restrict__ frag_offs, uint64_t n_frags,
                                                         int k, const Slot<NW>* __restrict__ table, uint64_t cap_mask,
                                                         uint64_t* __restrict__ out, uint64_t out_cap,
                                                         unsigned long long* __restrict__ counter) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1;
    for (uint64_t f = warp; f < n_frags; f += n_warps) {
        const uint64_t b = frag_offs[f];
        const uint64_t L = frag_offs[f + 1] - b;
        const uint64_t nwin = L > (uint64_t)k ? L - k : 0;
        int64_t carry_pos = -1;
        bool carry_out0 = false;
        for (uint64_t base = 0; base < nwin; base += 32) {
            const uint64_t i = base + lane;
            bool solid = false, o0 = false, i0 = false;
            if (i < nwin) {
                Key<NW> x = load_window<NW>(packed, b + i, K1);
                Key<NW> r = key_rc<NW>(x, K1);
                bool fwd_canon = !key_less<NW>(r, x);
                int fl = table_find<NW>(table, cap_mask, fwd_canon ? x : r);
                if (fl >= 0) {
                    solid = true;
                    // flags are stored for the canonical orientation; the
                    // reverse orientation swaps outdegree and indegree
                    o0 = fwd_canon ? (fl & 1) : ((fl >> 1) & 1);
                    i0 = fwd_canon ? ((fl >> 1) & 1) : (fl & 1);
                }
            }
            const uint32_t mask = __ballot_sync(0xFFFFFFFFu, solid);
            const uint32_t below = mask & lt_mask;
            const int p_lane = below ? 31 - __clz(below) : 0;
            const bool p_o0_lane = __shfl_sync(0xFFFFFFFFu, o0, p_lane);
            int64_t p = below ? (int64_t)(base + p_lane) : carry_pos;
            bool p_o0 = below ? p_o0_lane : carry_out0;
            if (solid && p >= 0 && (int64_t)i > p + 1 && p_o0 && i0) {
                uint64_t cnt = i - (uint64_t)p - 1;
                uint64_t idx = atomicAdd(counter, (unsigned long long)cnt);
                for (uint64_t j = (uint64_t)p + 1; j < i; j++, idx++) {
                    if (idx >= out_cap) continue;
                    Key<NW> y = load_window<NW>(packed, b + j, K1);
                    Key<NW> ry = key_rc<NW>(y, K1);
                    store_key<NW>(out, idx, key_less<NW>(ry, y) ? ry : y);
                }
            }
            if (mask) {
                const int hl = 31 - __clz(mask);
                const bool hl_o0 = __shfl_sync(0xFFFFFFFFu, o0, hl);
                carry_pos = (int64_t)(base + hl);
                carry_out0 = hl_o0;
            }
        }
    }
}

static uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <int NW>
void mercy_kmers(mh_ctx* ctx, const mh_reads* reads, const mh_kmers* solid, mh_kmers* out) {
    const int k = solid->k;
    const uint64_t S = solid->n;
    const uint64_t cap = next_pow2(std::max<uint64_t>(2 * S, 64));
    Buf<Slot<NW>> table(ctx, cap);
    table.zero();
    Buf<uint64_t> stats(ctx, 2);
    stats.zero();
    if (S)
        MH_LAUNCH(ctx, "degree_insert", grid_for(ctx, S, 256), 256, 0, degree_insert_kernel<NW>, solid->keys, S, k,
                  table.p, cap - 1, (unsigned long long*)stats.p, ctx->d_status);
    uint64_t out_cap = std::max<uint64_t>(1u << 20, reads->n_packed / 32);
    Buf<uint64_t> cand;
    uint64_t n_cand = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        cand = Buf<uint64_t>(ctx, out_cap * NW);
        MH_CUDA(cudaMemsetAsync(stats.p + 1, 0, sizeof(uint64_t), ctx->stream));
        if (reads->n_frags && S)
            MH_LAUNCH(ctx, "mercy_scan", grid_for(ctx, reads->n_frags * 32, 256, 8), 256, 0, mercy_scan_kernel<NW>,
                      reads->packed, reads->frag_offs, reads->n_frags, k, table.p, cap - 1, cand.p, out_cap,
                      (unsigned long long*)(stats.p + 1));
        read_u64(ctx, stats.p + 1, &n_cand, 1);
        if (n_cand <= out_cap) break;
        out_cap = n_cand;
    }
    table.reset();
    Buf<uint64_t> alt(ctx, (n_cand ? n_cand : 1) * NW);
    bool in_alt = radix_sort<NW>(ctx, cand.p, alt.p, nullptr, nullptr, n_cand, 0, 2 * (k + 1));
    Buf<uint64_t>& sorted = in_alt ? alt : cand;
    Buf<uint64_t> mk;
    Buf<uint32_t> mc;
    uint64_t M = 0, runs = 0, palins = 0;
    expand_runs<NW>(ctx, sorted.p, n_cand, k, 1, mk, mc, &M, &runs, &palins, solid->spectrum, solid->n_spectrum);
    sync_and_check(ctx);
    out->k = k;
    out->nw = NW;
    out->d = solid->d;
    out->n = M;
    out->n_kmers = n_cand;
    out->n_distinct = M;
    out->keys = mk.release();
    out->counts = mc.release();
}

template void mercy_kmers<1>(mh_ctx*, const mh_reads*, const mh_kmers*, mh_kmers*);
template void mercy_kmers<2>(mh_ctx*, const mh_reads*, const mh_kmers*, mh_kmers*);
template void mercy_kmers<4>(mh_ctx*, const mh_reads*, const mh_kmers*, mh_kmers*);

}  // namespace mh
