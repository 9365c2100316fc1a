// mh_mercy_kmers: mercy (k+1)-mers (paper, Sec. 2, third paragraph).
//
//   degrees  for every solid edge x (both orientations are in the sorted
//            solid table S): out0(x) = no solid edge starts with x[1..k];
//            in0(x) = no solid edge ends with x[0..k-1].  With P = the
//            k-prefixes of S (sorted, as S is) both are a join of the
//            suffixes x[1..k] against P: out0(x) iff x's suffix is not in P,
//            in0(y) iff no x has y's prefix as its suffix.  S is cut into
//            chunks of whole nodes; for each first symbol a, the entries
//            a.s with s in the chunk's node range are a contiguous run of S
//            (found by one search per chunk boundary), and each is looked up
//            in the chunk's prefixes held in shared memory.
//   ends     the edges with out0 or in0 (the graph's dead ends, a small
//            fraction of S) go into a small open-addressing hash table with
//            their two flags, which stays in L2.
//   probe    fragments in groups of 32 a warp (a lane per short fragment,
//            its window rolled on; a long fragment by the whole warp, a
//            window a lane): a test of three bits
//            of one word in a blocked Bloom filter of the edges without
//            outdegree (about 8 bits per dead end), and for the few
//            positives a probe of the small table;
//            every window p without outdegree is recorded as a hit (its
//            position and the end of its fragment).
//   walk     thread per hit: step forward to the next solid window q; if
//            q > p+1 and q has no indegree, the windows p+1..q-1 are emitted
//            (canonical keys).  Solidity: a search of the counting spectrum
//            (distinct canonical keys, ascending as mix_key images, so their
//            top bits are evenly spread, with their run lengths) through a
//            bucket index on the top bits of the top word; handles without a
//            mixed spectrum: a hash set of the canonical solid keys.
//   finish   sort + dedup of the candidates, counts looked up in the
//            counting spectrum, both strands, sorted.
#include "mh_internal.cuh"

namespace mh {

template <int NW>
struct Slot {
    uint64_t k[NW];
    uint32_t tag;
    uint32_t flags;
};

__device__ __forceinline__ uint32_t slot_tag(uint64_t h) { return (uint32_t)(h >> 32) | 1u; }

template <int NW>
__host__ __device__ constexpr int deg_chunk() {
    return 2048 / NW;  // entries of S per chunk (16 KB of prefixes in shared memory)
}

// First index in [0, n) with S[i] >= q.
template <int NW>
__device__ __forceinline__ uint64_t lb_key(const uint64_t* __restrict__ S, uint64_t n, const Key<NW>& q) {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (key_less<NW>(load_key<NW>(S, mid), q)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The (k+1)-mer a followed by k symbols A (a in ACGT).
template <int NW>
__device__ __forceinline__ Key<NW> first_symbol_key(uint32_t a, int k) {
    Key<NW> q = key_zero<NW>();
    q.w[0] = a;
    return key_shl<NW>(q, 2 * k);
}

// st[t] (t = 0..n_chunks): start of chunk t, the first node start at or after
// t * chunk (st[n_chunks] = n).  xb[4t + a]: first entry of S that is >= a.P_t
// where P_t is the first node of chunk t (xb[a] = start of the entries with
// first symbol a, xb[4 n_chunks + a] = their end).
template <int NW>
__global__ void degree_bounds_kernel(const uint64_t* __restrict__ S, uint64_t n, int k, uint64_t n_chunks,
                                     uint64_t* __restrict__ st, uint64_t* __restrict__ xb) {
    constexpr int C = deg_chunk<NW>();
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < (n_chunks + 1) * 4;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = g >> 2;
        const uint32_t a = (uint32_t)(g & 3);
        uint64_t s = t == 0 ? 0 : (t == n_chunks ? n : t * C);
        if (t > 0)
            while (s < n && key_eq<NW>(key_shr<NW>(load_key<NW>(S, s), 2), key_shr<NW>(load_key<NW>(S, s - 1), 2)))
                s++;
        if (a == 0) st[t] = s;
        uint64_t b;
        if (t == 0) {
            b = lb_key<NW>(S, n, first_symbol_key<NW>(a, k));
        } else if (s >= n) {
            b = a == 3 ? n : lb_key<NW>(S, n, first_symbol_key<NW>(a + 1, k));
        } else {
            Key<NW> q = first_symbol_key<NW>(a, k);
            const Key<NW> p = key_shr<NW>(load_key<NW>(S, s), 2);
#pragma unroll
            for (int w = 0; w < NW; w++) q.w[w] |= p.w[w];
            b = lb_key<NW>(S, n, q);
        }
        xb[g] = b;
    }
}

// Block per chunk.  fout[j] = 1 iff entry j has no outdegree (for the
// entries whose suffix falls in the chunk's node range); flags[i] = 2 iff
// entry i of the chunk has no indegree, else 0.
template <int NW>
__global__ void __launch_bounds__(256) degree_kernel(const uint64_t* __restrict__ S, int k,
                                                     const uint64_t* __restrict__ st,
                                                     const uint64_t* __restrict__ xb, uint8_t* __restrict__ fout,
                                                     uint8_t* __restrict__ flags, uint32_t* __restrict__ err) {
    constexpr int C = deg_chunk<NW>();
    constexpr int CAP = C + 4;  // a node has at most 4 entries, so a chunk at most C + 3
    __shared__ uint64_t pk[CAP * NW];
    __shared__ uint8_t found[CAP];
    const uint64_t t = blockIdx.x;
    const uint64_t p0 = st[t], p1 = st[t + 1];
    if (p1 - p0 > (uint64_t)CAP) {
        if (threadIdx.x == 0) atomicOr(err, ST_BAD_TABLE);
        return;
    }
    const uint32_t np = (uint32_t)(p1 - p0);
    {
        // all loads of the chunk in flight at once (blockDim.x == 256)
        constexpr int R = (CAP + 255) / 256;
        Key<NW> v[R];
#pragma unroll
        for (int q = 0; q < R; q++) {
            const uint32_t i = threadIdx.x + q * 256;
            if (i < np) v[q] = load_key<NW>(S, p0 + i);
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            const uint32_t i = threadIdx.x + q * 256;
            if (i < np) {
                const Key<NW> p = key_shr<NW>(v[q], 2);
#pragma unroll
                for (int w = 0; w < NW; w++) pk[i * NW + w] = p.w[w];
                found[i] = 0;
            }
        }
    }
    __syncthreads();
    auto pkey = [&](uint32_t i) {
        Key<NW> r;
#pragma unroll
        for (int w = 0; w < NW; w++) r.w[w] = pk[i * NW + w];
        return r;
    };
    for (uint32_t a = 0; a < 4; a++) {
        const uint64_t x0 = xb[t * 4 + a], x1 = xb[(t + 1) * 4 + a];
        for (uint64_t j = x0 + threadIdx.x; j < x1; j += blockDim.x) {
            const Key<NW> sfx = key_low<NW>(load_key<NW>(S, j), 2 * k);
            uint32_t lo = 0, hi = np;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (key_less<NW>(pkey(mid), sfx)) lo = mid + 1; else hi = mid;
            }
            const bool hit = lo < np && key_eq<NW>(pkey(lo), sfx);
            if (hit) found[lo] = 1;
            fout[j] = hit ? 0 : 1;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
        const Key<NW> p = pkey(i);
        uint32_t f = i;
        while (f > 0 && key_eq<NW>(pkey(f - 1), p)) f--;
        flags[p0 + i] = found[f] ? 0 : 2;
    }
}

// flags[i] |= fout[i]; counts the entries with a flag.
__global__ void degree_flags_kernel(const uint8_t* __restrict__ fout, uint8_t* __restrict__ flags, uint64_t n,
                                    unsigned long long* __restrict__ n_ends) {
    uint32_t ends = 0;
    const uint64_t n4 = n / 4;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t f = reinterpret_cast<const uint32_t*>(flags)[i] | reinterpret_cast<const uint32_t*>(fout)[i];
        reinterpret_cast<uint32_t*>(flags)[i] = f;
        ends += ((f & 0xFFu) != 0) + ((f & 0xFF00u) != 0) + ((f & 0xFF0000u) != 0) + ((f >> 24) != 0);
    }
    if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) {
        const uint64_t i = 4 * n4 + threadIdx.x;
        const uint8_t f = flags[i] | fout[i];
        flags[i] = f;
        ends += f != 0;
    }
    for (int off = 16; off; off >>= 1) ends += __shfl_xor_sync(0xFFFFFFFFu, ends, off);
    if ((threadIdx.x & 31) == 0 && ends) atomicAdd(n_ends, (unsigned long long)ends);
}

// Prefilter of the edges without outdegree: a blocked Bloom filter, three
// bits of one 32-bit word per key, so a query is one load; about 5% false
// positives at 8 bits per key.  Its hash is one multiply per key word (the
// filter is probed for every read window; the table keeps key_hash): the
// word comes from the product's top 32 bits, the bit positions from three
// 5-bit fields of its middle bits.
template <int NW>
__device__ __forceinline__ uint64_t filter_hash(const Key<NW>& x) {
    uint64_t h = x.w[0] * 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 1; w < NW; w++) h ^= (x.w[w] + h) * 0xBF58476D1CE4E5B9ull;
    return h;
}
__device__ __forceinline__ uint64_t filter_word(uint64_t h, uint64_t words_mask) { return (h >> 32) & words_mask; }
__device__ __forceinline__ uint32_t filter_bits(uint64_t h) {
    return (1u << ((h >> 17) & 31)) | (1u << ((h >> 22) & 31)) | (1u << ((h >> 27) & 31));
}

// Dead-end edges (oriented) with their flags into the small table; edges
// without outdegree also into the prefilter bitmap.
template <int NW>
__global__ void __launch_bounds__(256) ends_insert_kernel(const uint64_t* __restrict__ S, uint64_t n,
                                                          const uint8_t* __restrict__ flags,
                                                          Slot<NW>* __restrict__ table, uint64_t cap_mask,
                                                          uint32_t* __restrict__ filter, uint64_t filter_mask,
                                                          uint32_t* __restrict__ err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t f = flags[i];
        if (!f) continue;
        Key<NW> x = load_key<NW>(S, i);
        uint64_t h = key_hash<NW>(x);
        if (f & 1u) {
            const uint64_t fh = filter_hash<NW>(x);
            atomicOr(&filter[filter_word(fh, filter_mask)], filter_bits(fh));
        }
        uint32_t tag = slot_tag(h);
        uint64_t s = h & cap_mask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= cap_mask; probe++) {
            if (atomicCAS(&table[s].tag, 0u, tag) == 0u) {
#pragma unroll
                for (int w = 0; w < NW; w++) table[s].k[w] = x.w[w];
                table[s].flags = f;
                placed = true;
                break;
            }
            s = (s + 1) & cap_mask;
        }
        if (!placed) atomicOr(err, ST_TABLE_FULL);
    }
}

// Flags of the oriented key x if it is a dead-end edge, else 0.
template <int NW>
__device__ __forceinline__ uint32_t ends_find(const Slot<NW>* __restrict__ table, uint64_t cap_mask,
                                              const Key<NW>& x) {
    uint64_t h = key_hash<NW>(x);
    uint32_t tag = slot_tag(h);
    uint64_t s = h & cap_mask;
    for (uint64_t probe = 0; probe <= cap_mask; probe++) {
        uint32_t t = table[s].tag;
        if (t == 0u) return 0;
        if (t == tag) {
            bool eq = true;
#pragma unroll
            for (int w = 0; w < NW; w++) eq &= table[s].k[w] == x.w[w];
            if (eq) return table[s].flags;
        }
        s = (s + 1) & cap_mask;
    }
    return 0;
}

// Canonical solid keys into the solidity set.  1-word keys use 8-byte slots
// holding the key itself, empty = all ones (never canonical: the reverse
// complement of T...T is A...A, which is smaller); wider keys use Slot
// (32-bit tag + key).
// Bucket index over the ascending mixed spectrum keys: off[b] = first index
// whose top `bits` bits (of the top word) are >= b, for b = 0..2^bits
// (thread per key; each bucket boundary is written by exactly one thread).
template <int NW>
__global__ void canon_index_kernel(const uint64_t* __restrict__ canon, uint64_t n, int bits,
                                   uint64_t* __restrict__ off) {
    const int sh = 64 - bits;
    const uint64_t nb = 1ull << bits;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = canon[i * NW + NW - 1] >> sh;
        const uint64_t b0 = i == 0 ? 0 : (canon[(i - 1) * NW + NW - 1] >> sh) + 1;
        for (uint64_t x = b0; x <= b; x++) off[x] = i;
        if (i == n - 1)
            for (uint64_t x = b + 1; x <= nb; x++) off[x] = n;
    }
}

// Run length of the mixed key m in the ascending spectrum (bucket index
// off over `bits` top bits of the top word), 0 if absent.
template <int NW>
__device__ __forceinline__ uint32_t spec_find(const uint64_t* __restrict__ spec, const uint32_t* __restrict__ len,
                                              const uint64_t* __restrict__ off, int bits, const Key<NW>& m) {
    const uint64_t b = m.w[NW - 1] >> (64 - bits);
    uint64_t i = off[b];
    const uint64_t e = off[b + 1];
    for (; i < e; i++) {
        const Key<NW> v = load_key<NW>(spec, i);
        if (!key_less<NW>(v, m)) return key_eq<NW>(v, m) ? len[i] : 0u;
    }
    return 0u;
}

template <int NW>
__global__ void __launch_bounds__(256) solid_insert_kernel(const uint64_t* __restrict__ S, uint64_t n, int K1,
                                                           Slot<NW>* __restrict__ table, uint64_t cap_mask,
                                                           uint32_t* __restrict__ err) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        Key<NW> x = load_key<NW>(S, i);
        if (key_less<NW>(key_rc<NW>(x, K1), x)) continue;
        uint64_t h = key_hash<NW>(x);
        uint32_t tag = slot_tag(h);
        uint64_t s = h & cap_mask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= cap_mask; probe++) {
            if (atomicCAS(&table[s].tag, 0u, tag) == 0u) {
#pragma unroll
                for (int w = 0; w < NW; w++) table[s].k[w] = x.w[w];
                placed = true;
                break;
            }
            s = (s + 1) & cap_mask;
        }
        if (!placed) atomicOr(err, ST_TABLE_FULL);
    }
}

template <int NW>
__device__ __forceinline__ bool table_has(const Slot<NW>* __restrict__ table, uint64_t cap_mask, const Key<NW>& x) {
    uint64_t h = key_hash<NW>(x);
    uint32_t tag = slot_tag(h);
    uint64_t s = h & cap_mask;
    for (uint64_t probe = 0; probe <= cap_mask; probe++) {
        uint32_t t = table[s].tag;
        if (t == 0u) return false;
        if (t == tag) {
            bool eq = true;
#pragma unroll
            for (int w = 0; w < NW; w++) eq &= table[s].k[w] == x.w[w];
            if (eq) return true;
        }
        s = (s + 1) & cap_mask;
    }
    return false;
}

// Fragments of at most this many windows are probed by one lane.
constexpr int kProbeLaneWindows = 48;

// Probe every window; record windows without outdegree as (position, end).
// Fragments in groups of 32 a warp: a short fragment is probed by one lane,
// which assembles its first window and rolls it on by one symbol a window
// (the lanes step together to the group's longest short fragment, so that
// the hits of a step are counted by one atomic); longer fragments are then
// probed by the whole warp, a window a lane.
template <int NW>
__global__ void __launch_bounds__(256) mercy_probe_kernel(const uint32_t* __restrict__ packed,
                                                          const uint64_t* __restrict__ frag_offs, uint64_t n_frags,
                                                          int k, const Slot<NW>* __restrict__ ends, uint64_t cap_mask,
                                                          const uint32_t* __restrict__ filter, uint64_t filter_mask,
                                                          ulonglong2* __restrict__ hits, uint64_t hit_cap,
                                                          unsigned long long* __restrict__ n_hits) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int K1 = k + 1;
    auto probe = [&](const Key<NW>& x) {
        const uint64_t h = filter_hash<NW>(x);
        const uint32_t fm = filter_bits(h);
        return (__ldg(&filter[filter_word(h, filter_mask)]) & fm) == fm && (ends_find<NW>(ends, cap_mask, x) & 1u);
    };
    // the hits of one step of the warp, placed by one atomic
    auto record = [&](bool hit, uint64_t p, uint64_t end) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
        if (!m) return;
        uint64_t first = 0;
        if (lane == __ffs(m) - 1) first = atomicAdd(n_hits, (unsigned long long)__popc(m));
        first = __shfl_sync(0xFFFFFFFFu, first, __ffs(m) - 1);
        if (hit) {
            const uint64_t idx = first + __popc(m & ((1u << lane) - 1));
            if (idx < hit_cap) hits[idx] = make_ulonglong2(p, end);
        }
    };
    for (uint64_t g = warp; g * 32 < n_frags; g += n_warps) {
        const uint64_t f = g * 32 + lane;
        uint64_t b = 0, nwin = 0;
        if (f < n_frags) {
            b = frag_offs[f];
            const uint64_t L = frag_offs[f + 1] - b;
            nwin = L > (uint64_t)k ? L - k : 0;
        }
        const bool alone = nwin <= (uint64_t)kProbeLaneWindows;
        const uint64_t mine = alone ? nwin : 0;
        uint64_t most = mine;
        for (int off = 16; off; off >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, most, off);
            most = o > most ? o : most;
        }
        Key<NW> x{};
        if (mine) x = load_window<NW>(packed, b, K1);
        for (uint64_t i = 0; i < most; i++) {
            bool hit = false;
            if (i < mine) {
                if (i) roll_forward<NW>(x, packed_sym(packed, b + i + K1 - 1), K1);
                hit = probe(x);
            }
            record(hit, b + i, b + mine);
        }
        uint32_t big = __ballot_sync(0xFFFFFFFFu, !alone);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint64_t fb = __shfl_sync(0xFFFFFFFFu, b, src);
            const uint64_t fn = __shfl_sync(0xFFFFFFFFu, nwin, src);
            for (uint64_t base = 0; base < fn; base += 32) {
                const uint64_t p = base + lane;
                bool hit = false;
                if (p < fn) hit = probe(load_window<NW>(packed, fb + p, K1));
                record(hit, fb + p, fb + fn);
            }
        }
    }
}

// Walk from each hit to the next solid window; emit the gap if it qualifies.
// MIXED: candidates out as mix_key images; 1-word keys then take solidity
// from the counting spectrum (run length, doubled for a palindrome, >= d)
// through its bucket index, wider keys (and unmixed handles) from the hash
// set `solid`.
template <int NW, bool MIXED>
__global__ void __launch_bounds__(256) mercy_walk_kernel(const uint32_t* __restrict__ packed,
                                                         const ulonglong2* __restrict__ hits, uint64_t n_hits, int k,
                                                         const Slot<NW>* __restrict__ ends, uint64_t ends_mask,
                                                         const Slot<NW>* __restrict__ solid, uint64_t solid_mask,
                                                         const uint64_t* __restrict__ spec,
                                                         const uint32_t* __restrict__ spec_len,
                                                         const uint64_t* __restrict__ spec_off, int spec_bits, int d,
                                                         uint64_t* __restrict__ out, uint64_t out_cap,
                                                         unsigned long long* __restrict__ counter) {
    const int K1 = k + 1;
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n_hits;
         h += (uint64_t)gridDim.x * blockDim.x) {
        const ulonglong2 hp = hits[h];
        const uint64_t p = hp.x, end = hp.y;
        uint64_t q = p + 1;
        Key<NW> y;
        for (; q < end; q++) {
            Key<NW> x = load_window<NW>(packed, q, K1);
            Key<NW> r = key_rc<NW>(x, K1);
            const Key<NW> c = key_less<NW>(r, x) ? r : x;
            bool present;
            if constexpr (MIXED) {
                const uint32_t len = spec_find<NW>(spec, spec_len, spec_off, spec_bits, mix_key<NW>(c));
                present = (uint64_t)len * (key_eq<NW>(r, x) ? 2 : 1) >= (uint64_t)d;
            } else
                present = table_has<NW>(solid, solid_mask, c);
            if (present) {
                y = x;
                break;
            }
        }
        if (q >= end || q == p + 1) continue;
        if (!(ends_find<NW>(ends, ends_mask, y) & 2u)) continue;
        uint64_t idx = atomicAdd(counter, (unsigned long long)(q - p - 1));
        for (uint64_t j = p + 1; j < q; j++, idx++) {
            if (idx >= out_cap) continue;
            Key<NW> z = load_window<NW>(packed, j, K1);
            Key<NW> rz = key_rc<NW>(z, K1);
            Key<NW> c = key_less<NW>(rz, z) ? rz : z;
            if constexpr (MIXED) c = mix_key<NW>(c);
            store_key<NW>(out, idx, c);
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
    Buf<uint8_t> flags(ctx, S ? S : 1);
    Buf<uint64_t> stats(ctx, 2);
    stats.zero();
    if (S) {
        const uint64_t n_chunks = ceil_div(S, deg_chunk<NW>());
        Buf<uint64_t> st(ctx, n_chunks + 1), xb(ctx, 4 * (n_chunks + 1));
        Buf<uint8_t> fout(ctx, S);
        MH_LAUNCH(ctx, "mercy_degree_bounds", grid_for(ctx, 4 * (n_chunks + 1), 256), 256, 0,
                  degree_bounds_kernel<NW>, solid->keys, S, k, n_chunks, st.p, xb.p);
        MH_LAUNCH_B(ctx, "mercy_degree", 2 * S * 8 * NW + 2 * S, (unsigned)n_chunks, 256, 0, degree_kernel<NW>,
                    solid->keys, k, st.p, xb.p, fout.p, flags.p, ctx->d_status);
        MH_LAUNCH(ctx, "mercy_degree_flags", grid_for(ctx, ceil_div(S, 4), 256), 256, 0, degree_flags_kernel, fout.p,
                  flags.p, S, (unsigned long long*)stats.p);
    }
    uint64_t n_ends = 0;
    read_u64(ctx, stats.p, &n_ends, 1);
    const uint64_t cap = next_pow2(std::max<uint64_t>(2 * n_ends, 64));
    Buf<Slot<NW>> table(ctx, cap);
    table.zero();
    // prefilter: about 8 bits per dead end (at least 2^20 bits)
    const uint64_t fbits = next_pow2(std::max<uint64_t>(8 * n_ends, 1u << 20));
    Buf<uint32_t> filter(ctx, fbits / 32);
    filter.zero();
    if (n_ends)
        MH_LAUNCH(ctx, "mercy_ends_insert", grid_for(ctx, S, 256), 256, 0, ends_insert_kernel<NW>, solid->keys, S,
                  flags.p, table.p, cap - 1, filter.p, fbits / 32 - 1, ctx->d_status);
    flags.reset();
    // solidity: the counting handle's ascending mixed spectrum with a bucket
    // index (4 to 8 keys a bucket); without one, a hash set of the canonical
    // solid keys, load <= 1/2 (<= 0.61 if all palindromes)
    const bool mixed = solid->spectrum_mixed;
    Buf<Slot<NW>> sset;
    uint64_t scap = 1;
    Buf<uint64_t> spec_off;
    int spec_bits = 1;
    if (mixed) {
        while (spec_bits < 40 && (2ull << spec_bits) * 4 <= solid->n_spectrum) spec_bits++;
        spec_off = Buf<uint64_t>(ctx, (1ull << spec_bits) + 1);
        spec_off.zero();
        if (solid->n_spectrum)
            MH_LAUNCH(ctx, "mercy_spectrum_index", grid_for(ctx, solid->n_spectrum, 256), 256, 0,
                      canon_index_kernel<NW>, solid->spectrum, solid->n_spectrum, spec_bits, spec_off.p);
    } else {
        scap = next_pow2(std::max<uint64_t>(S + S / 2, 64));
        sset = Buf<Slot<NW>>(ctx, scap);
        sset.zero();
        if (S)
            MH_LAUNCH(ctx, "mercy_solid_insert", grid_for(ctx, S, 256), 256, 0, solid_insert_kernel<NW>, solid->keys,
                      S, k + 1, sset.p, scap - 1, ctx->d_status);
    }
    // windows without outdegree
    uint64_t hit_cap = std::max<uint64_t>(1u << 20, reads->n_packed / 256);
    Buf<ulonglong2> hits;
    uint64_t n_hits = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        hits = Buf<ulonglong2>(ctx, hit_cap);
        MH_CUDA(cudaMemsetAsync(stats.p + 1, 0, sizeof(uint64_t), ctx->stream));
        if (reads->n_frags && n_ends)
            MH_LAUNCH_B(ctx, "mercy_probe", reads->n_packed / 4, grid_for(ctx, reads->n_frags * 32, 256, 8), 256, 0,
                        mercy_probe_kernel<NW>, reads->packed, reads->frag_offs, reads->n_frags, k, table.p, cap - 1,
                        filter.p, fbits / 32 - 1, hits.p, hit_cap, (unsigned long long*)(stats.p + 1));
        read_u64(ctx, stats.p + 1, &n_hits, 1);
        if (n_hits <= hit_cap) break;
        hit_cap = n_hits;
    }
    // the gaps behind the hits
    // candidates in the spectrum's order (mix_key images), so that their
    // sorted spectrum lookups ascend
    uint64_t out_cap = std::max<uint64_t>(1u << 20, 16 * n_hits);
    Buf<uint64_t> cand;
    uint64_t n_cand = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        cand = Buf<uint64_t>(ctx, out_cap * NW);
        MH_CUDA(cudaMemsetAsync(stats.p + 1, 0, sizeof(uint64_t), ctx->stream));
        if (n_hits)
            MH_LAUNCH(ctx, "mercy_walk", grid_for(ctx, n_hits, 256, 8), 256, 0,
                      (mixed ? mercy_walk_kernel<NW, true> : mercy_walk_kernel<NW, false>), reads->packed,
                      hits.p, n_hits, k, table.p, cap - 1, sset.p, scap - 1, solid->spectrum, solid->spectrum_len,
                      spec_off.p, spec_bits, solid->d,
                      cand.p, out_cap, (unsigned long long*)(stats.p + 1));
        read_u64(ctx, stats.p + 1, &n_cand, 1);
        if (n_cand <= out_cap) break;
        out_cap = n_cand;
    }
    hits.reset();
    sset.reset();
    spec_off.reset();
    table.reset();
    Buf<uint64_t> alt(ctx, (n_cand ? n_cand : 1) * NW);
    bool in_alt = mixed ? radix_sort_spread<NW>(ctx, cand.p, alt.p, n_cand)
                        : radix_sort<NW>(ctx, cand.p, alt.p, nullptr, nullptr, n_cand, 0, 2 * (k + 1));
    Buf<uint64_t>& sorted = in_alt ? alt : cand;
    Buf<uint64_t> mk;
    Buf<uint32_t> mc;
    uint64_t M = 0, runs = 0, palins = 0;
    expand_runs<NW>(ctx, sorted.p, n_cand, k, 1, mk, mc, &M, &runs, &palins, solid->spectrum, solid->spectrum_len,
                    solid->n_spectrum, mixed, solid->spectrum_mixed);
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
