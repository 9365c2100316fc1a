// CPU oracle for the SdBG construction hot path of MEGAHIT (Li et al., 2015).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
// baseline of the benchmark may load this code.  The product path (the CUDA
// library) never calls it, shares no code with it, and fails loudly instead of
// falling back to it.
//
// Written for obviousness, not speed: every (k+1)-mer is a std::string over
// "ACGT" (and '$' for padding), sets are std::set / std::map, sorting is
// std::sort.  Results are packed into integer keys only at the very end.
//
// What it computes (paper, Section 2 "Methods"):
//   * counting  (Sec. 2, third paragraph): every (k+1)-mer of the reads on both
//     strands is counted; those seen at least d times are solid.
//   * mercy     (Sec. 2, third paragraph): between a solid x with no outdegree
//     and a solid y with no indegree in the same read, with no solid edge in
//     between, the in-between (k+1)-mers are kept as mercy edges.
//   * SdBG      (Sec. 2, first and second paragraphs): the edges sorted in
//     reverse-lexicographic (colex) order of their k-prefix, encoded as the
//     BOSS arrays W (with the minus flag), last, F, plus the validity
//     bit-vector and the 2kt-bit store of zero-indegree vertices.
//
// Readings where the paper is silent are marked [reading] and match the ones
// listed in the design notes:
//   [reading] a byte outside ACGTacgt splits a read into fragments;
//   [reading] both strands are counted literally, so a palindromic (k+1)-mer
//             gains 2 per occurrence;
//   [reading] counts are exact 32-bit values; larger counts are an error;
//   [reading] mercy uses the degrees of the solid graph, one pass, forward
//             strand of each fragment, then closes the result under reverse
//             complement;
//   [reading] "reverse lexicographical order" = colex: compare node symbols
//             k-1, k-2, ..., 0, then the edge label;
//   [reading] each zero-indegree vertex v gets ONE dummy edge from the node
//             $ v[0..k-2] labelled v[k-1], and v goes to the auxiliary store;
//             each vertex with no outgoing edge gets one edge labelled $.
//
// Key layout of the outputs: a string s[0..n-1] over ACGT (A=0, C=1, G=2, T=3)
// is the integer sum s[i] * 4^(n-1-i), stored as nw little-endian 64-bit words
// (word 0 least significant), nw = the smallest of 1, 2, 4 with 2(k+1) <= 64 nw.

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

int code_of(char c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
    }
    return -1;
}

const char kSym[4] = {'A', 'C', 'G', 'T'};

char complement(char c) { return kSym[3 - code_of(c)]; }

std::string reverse_complement(const std::string& s) {
    std::string r(s.rbegin(), s.rend());
    for (char& c : r) c = complement(c);
    return r;
}

int words_for(int k) { return 2 * (k + 1) <= 64 ? 1 : (2 * (k + 1) <= 128 ? 2 : 4); }

// s -> nw little-endian words holding sum s[i] * 4^(n-1-i).
void encode(const std::string& s, int nw, uint64_t* out) {
    for (int w = 0; w < nw; w++) out[w] = 0;
    for (char c : s) {
        // value = value * 4 + code, across the words
        for (int w = nw - 1; w > 0; w--) out[w] = (out[w] << 2) | (out[w - 1] >> 62);
        out[0] = (out[0] << 2) | (uint64_t)code_of(c);
    }
}

std::string decode(const uint64_t* in, int n) {
    std::string s(n, 'A');
    for (int i = 0; i < n; i++) {
        int bit = 2 * (n - 1 - i);  // symbol i sits at bits [bit, bit+2)
        s[i] = kSym[(in[bit / 64] >> (bit % 64)) & 3];
    }
    return s;
}

// C1: the fragments of every read = its maximal runs of ACGT, upper-cased.
std::vector<std::string> fragments(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads) {
    std::vector<std::string> out;
    for (uint64_t r = 0; r < n_reads; r++) {
        std::string cur;
        for (uint64_t j = offs[r]; j < offs[r + 1]; j++) {
            char c = (char)ascii[j];
            if (c >= 'a' && c <= 'z') c = (char)(c - 'a' + 'A');
            if (code_of(c) >= 0) {
                cur.push_back(c);
            } else if (!cur.empty()) {
                out.push_back(cur);
                cur.clear();
            }
        }
        if (!cur.empty()) out.push_back(cur);
    }
    return out;
}

struct Counted {
    std::vector<std::string> keys;  // distinct (k+1)-mers, ascending
    std::vector<uint64_t> cnt;
    uint64_t n_kmers = 0;
};

// C2 + C3: multiset K of all (k+1)-mers on both strands, sorted and counted.
Counted count_all(const std::vector<std::string>& frags, int k) {
    std::vector<std::string> K;
    for (const std::string& s : frags) {
        if ((int)s.size() < k + 1) continue;
        for (size_t i = 0; i + k < s.size(); i++) {
            std::string e = s.substr(i, k + 1);
            K.push_back(e);
            K.push_back(reverse_complement(e));
        }
    }
    std::sort(K.begin(), K.end());
    Counted c;
    c.n_kmers = K.size();
    for (size_t i = 0; i < K.size();) {
        size_t j = i;
        while (j < K.size() && K[j] == K[i]) j++;
        c.keys.push_back(K[i]);
        c.cnt.push_back(j - i);
        i = j;
    }
    return c;
}

// M1-M3: mercy edges, given the solid set and all counts.
std::vector<std::string> mercy_edges(const std::vector<std::string>& frags, int k,
                                     const std::set<std::string>& solid) {
    std::set<std::string> prefixes, suffixes;  // k-prefixes and k-suffixes of solid edges
    for (const std::string& z : solid) {
        prefixes.insert(z.substr(0, k));
        suffixes.insert(z.substr(1, k));
    }
    // x has no outdegree: no solid z starts with x's k-suffix.
    auto out0 = [&](const std::string& x) { return prefixes.count(x.substr(1, k)) == 0; };
    // y has no indegree: no solid z ends with y's k-prefix.
    auto in0 = [&](const std::string& y) { return suffixes.count(y.substr(0, k)) == 0; };

    std::set<std::string> found;
    for (const std::string& s : frags) {
        if ((int)s.size() < k + 1) continue;
        std::vector<size_t> P;  // positions of solid edges, ascending
        for (size_t i = 0; i + k < s.size(); i++)
            if (solid.count(s.substr(i, k + 1))) P.push_back(i);
        for (size_t a = 0; a + 1 < P.size(); a++) {
            size_t p = P[a], q = P[a + 1];
            if (q > p + 1 && out0(s.substr(p, k + 1)) && in0(s.substr(q, k + 1)))
                for (size_t j = p + 1; j < q; j++) found.insert(s.substr(j, k + 1));
        }
    }
    std::set<std::string> closed(found);
    for (const std::string& e : found) closed.insert(reverse_complement(e));
    return std::vector<std::string>(closed.begin(), closed.end());
}

struct Entry {
    std::string node;  // k symbols; a dummy node starts with '$'
    char label;        // 'A'..'T' or '$'
    bool is_dummy;
    std::string aux;   // the zero-indegree vertex, for dummy entries
    uint32_t mult;
};

// B1: colex order - node symbols k-1 down to 0, then the label ('$' < 'A').
bool colex_less(const Entry& a, const Entry& b) {
    std::string ra(a.node.rbegin(), a.node.rend()), rb(b.node.rbegin(), b.node.rend());
    if (ra != rb) return ra < rb;
    return a.label < b.label;
}

int w_code(char label) { return label == '$' ? 0 : code_of(label) + 1; }

}  // namespace

extern "C" {

typedef struct {
    int status;  // 0 ok, -1 bad argument, -3 count does not fit 32 bits
    int k, nw;
    uint64_t n_kmers, n_distinct;
    uint64_t n_solid;
    uint64_t* solid_keys;
    uint32_t* solid_cnt;
    uint64_t n_mercy;
    uint64_t* mercy_keys;
    uint32_t* mercy_cnt;
} orc_kmer_result;

typedef struct {
    int status;
    int k, nw;
    uint64_t m, t, u, n_nodes;
    uint8_t* W;
    uint8_t* last;
    uint8_t* valid;
    uint8_t* dummy;
    uint32_t* mult;
    uint64_t F[6];
    uint64_t* aux;  // t records of nw words: the zero-indegree vertices
} orc_sdbg_result;

static void put_keys(const std::vector<std::string>& v, int nw, uint64_t** keys) {
    *keys = (uint64_t*)calloc(v.size() * nw + 1, sizeof(uint64_t));
    for (size_t i = 0; i < v.size(); i++) encode(v[i], nw, *keys + i * nw);
}

// C1 alone: the fragments (maximal ACGT runs, upper-cased) of every read,
// concatenated into `bases` (capacity n_bases), with n_frags + 1 offsets into
// it and the read of each fragment.  Returns the number of fragments.
uint64_t orc_fragments(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads, char* bases,
                       uint64_t* frag_offs, uint32_t* frag_read) {
    uint64_t nf = 0, pos = 0;
    frag_offs[0] = 0;
    for (uint64_t r = 0; r < n_reads; r++) {
        std::vector<std::string> fr = fragments(ascii, offs + r, 1);
        for (const std::string& s : fr) {
            std::memcpy(bases + pos, s.data(), s.size());
            pos += s.size();
            frag_read[nf] = (uint32_t)r;
            frag_offs[++nf] = pos;
        }
    }
    return nf;
}

// Counting (C1-C3) and, if do_mercy, mercy (M1-M4).
orc_kmer_result* orc_count(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads, int k,
                           int d, int do_mercy) {
    orc_kmer_result* r = (orc_kmer_result*)calloc(1, sizeof(orc_kmer_result));
    if (k < 2 || k > 127 || d < 1) { r->status = -1; return r; }
    r->k = k;
    r->nw = words_for(k);
    std::vector<std::string> frags = fragments(ascii, offs, n_reads);
    Counted c = count_all(frags, k);
    r->n_kmers = c.n_kmers;
    r->n_distinct = c.keys.size();
    std::map<std::string, uint64_t> count_of;
    std::vector<std::string> solid;
    std::vector<uint32_t> solid_cnt;
    for (size_t i = 0; i < c.keys.size(); i++) {
        if (c.cnt[i] > 0xFFFFFFFFull) { r->status = -3; return r; }
        count_of[c.keys[i]] = c.cnt[i];
        if (c.cnt[i] >= (uint64_t)d) {
            solid.push_back(c.keys[i]);
            solid_cnt.push_back((uint32_t)c.cnt[i]);
        }
    }
    r->n_solid = solid.size();
    put_keys(solid, r->nw, &r->solid_keys);
    r->solid_cnt = (uint32_t*)calloc(solid.size() + 1, sizeof(uint32_t));
    std::copy(solid_cnt.begin(), solid_cnt.end(), r->solid_cnt);
    if (do_mercy) {
        std::set<std::string> solid_set(solid.begin(), solid.end());
        std::vector<std::string> mercy = mercy_edges(frags, k, solid_set);
        r->n_mercy = mercy.size();
        put_keys(mercy, r->nw, &r->mercy_keys);
        r->mercy_cnt = (uint32_t*)calloc(mercy.size() + 1, sizeof(uint32_t));
        for (size_t i = 0; i < mercy.size(); i++) r->mercy_cnt[i] = (uint32_t)count_of[mercy[i]];
    }
    return r;
}

// The same counting and mercy as orc_count, spread over n_threads threads
// (the threaded CPU baseline).  Counting: thread t takes the (k+1)-mers whose
// first 8 symbols (as a number, 4^8 buckets) fall in its range of buckets,
// from both strands of every fragment, and sorts and counts them alone; the
// threads' outputs, in thread order, are the whole sorted table.  Mercy: the
// fragments are split between the threads, each scans its own against the
// shared solid set; the edges found are merged and closed under reverse
// complement.  Same outputs as orc_count.
orc_kmer_result* orc_count_threaded(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads, int k, int d,
                                    int do_mercy, int n_threads) {
    orc_kmer_result* r = (orc_kmer_result*)calloc(1, sizeof(orc_kmer_result));
    if (k < 2 || k > 127 || d < 1) { r->status = -1; return r; }
    if (n_threads < 1) n_threads = 1;
    r->k = k;
    r->nw = words_for(k);
    std::vector<std::string> frags = fragments(ascii, offs, n_reads);
    const int pl = k + 1 < 8 ? k + 1 : 8;  // prefix symbols that pick the bucket
    const uint64_t n_buckets = 1ull << (2 * pl);
    // bucket of the string of symbols f[p..p+pl) read forward, or of the
    // reverse complement of the window ending at p + k (its first pl symbols
    // are the complements of the window's last pl symbols, last first)
    auto fwd_bucket = [&](const std::string& f, size_t p) {
        uint64_t b = 0;
        for (int i = 0; i < pl; i++) b = b * 4 + (uint64_t)code_of(f[p + i]);
        return b;
    };
    auto rc_bucket = [&](const std::string& f, size_t p) {
        uint64_t b = 0;
        for (int i = 0; i < pl; i++) b = b * 4 + (uint64_t)(3 - code_of(f[p + k - i]));
        return b;
    };
    std::vector<Counted> part(n_threads);
    auto count_part = [&](int t) {
        const uint64_t lo = n_buckets * t / n_threads, hi = n_buckets * (t + 1) / n_threads;
        std::vector<std::string> K;
        for (const std::string& f : frags) {
            if ((int)f.size() < k + 1) continue;
            for (size_t i = 0; i + k < f.size(); i++) {
                const uint64_t bf = fwd_bucket(f, i), br = rc_bucket(f, i);
                if (bf >= lo && bf < hi) K.push_back(f.substr(i, k + 1));
                if (br >= lo && br < hi) K.push_back(reverse_complement(f.substr(i, k + 1)));
            }
        }
        std::sort(K.begin(), K.end());
        Counted& c = part[t];
        c.n_kmers = K.size();
        for (size_t i = 0; i < K.size();) {
            size_t j = i;
            while (j < K.size() && K[j] == K[i]) j++;
            c.keys.push_back(K[i]);
            c.cnt.push_back(j - i);
            i = j;
        }
    };
    {
        std::vector<std::thread> th;
        for (int t = 0; t < n_threads; t++) th.emplace_back(count_part, t);
        for (auto& x : th) x.join();
    }
    Counted c;
    for (Counted& p : part) {
        c.n_kmers += p.n_kmers;
        c.keys.insert(c.keys.end(), p.keys.begin(), p.keys.end());
        c.cnt.insert(c.cnt.end(), p.cnt.begin(), p.cnt.end());
    }
    r->n_kmers = c.n_kmers;
    r->n_distinct = c.keys.size();
    std::vector<std::string> solid;
    std::vector<uint32_t> solid_cnt;
    for (size_t i = 0; i < c.keys.size(); i++) {
        if (c.cnt[i] > 0xFFFFFFFFull) { r->status = -3; return r; }
        if (c.cnt[i] >= (uint64_t)d) {
            solid.push_back(c.keys[i]);
            solid_cnt.push_back((uint32_t)c.cnt[i]);
        }
    }
    r->n_solid = solid.size();
    put_keys(solid, r->nw, &r->solid_keys);
    r->solid_cnt = (uint32_t*)calloc(solid.size() + 1, sizeof(uint32_t));
    std::copy(solid_cnt.begin(), solid_cnt.end(), r->solid_cnt);
    if (do_mercy) {
        std::set<std::string> solid_set(solid.begin(), solid.end());
        std::vector<std::vector<std::string>> found(n_threads);
        auto mercy_part = [&](int t) {
            const size_t f0 = frags.size() * t / n_threads, f1 = frags.size() * (t + 1) / n_threads;
            std::vector<std::string> mine(frags.begin() + f0, frags.begin() + f1);
            found[t] = mercy_edges(mine, k, solid_set);
        };
        std::vector<std::thread> th;
        for (int t = 0; t < n_threads; t++) th.emplace_back(mercy_part, t);
        for (auto& x : th) x.join();
        std::set<std::string> all;
        for (auto& v : found) all.insert(v.begin(), v.end());
        std::vector<std::string> mercy(all.begin(), all.end());
        r->n_mercy = mercy.size();
        put_keys(mercy, r->nw, &r->mercy_keys);
        r->mercy_cnt = (uint32_t*)calloc(mercy.size() + 1, sizeof(uint32_t));
        for (size_t i = 0; i < mercy.size(); i++) {
            const size_t j = std::lower_bound(c.keys.begin(), c.keys.end(), mercy[i]) - c.keys.begin();
            r->mercy_cnt[i] = (uint32_t)c.cnt[j];
        }
    }
    return r;
}

void orc_free_kmer_result(orc_kmer_result* r) {
    if (!r) return;
    free(r->solid_keys);
    free(r->solid_cnt);
    free(r->mercy_keys);
    free(r->mercy_cnt);
    free(r);
}

// SdBG construction (B1-B6) from edge keys (solid, then optional mercy).
orc_sdbg_result* orc_build_sdbg(int k, const uint64_t* solid_keys, const uint32_t* solid_cnt,
                                uint64_t n_solid, const uint64_t* mercy_keys,
                                const uint32_t* mercy_cnt, uint64_t n_mercy) {
    orc_sdbg_result* r = (orc_sdbg_result*)calloc(1, sizeof(orc_sdbg_result));
    if (k < 2 || k > 127) { r->status = -1; return r; }
    const int nw = words_for(k);
    r->k = k;
    r->nw = nw;
    std::map<std::string, uint32_t> E;  // edge -> multiplicity
    for (uint64_t i = 0; i < n_solid; i++) E[decode(solid_keys + i * nw, k + 1)] = solid_cnt ? solid_cnt[i] : 0;
    for (uint64_t i = 0; i < n_mercy; i++) E[decode(mercy_keys + i * nw, k + 1)] = mercy_cnt ? mercy_cnt[i] : 0;

    std::set<std::string> sources, targets;
    for (const auto& kv : E) {
        sources.insert(kv.first.substr(0, k));
        targets.insert(kv.first.substr(1, k));
    }
    std::vector<Entry> entries;
    for (const auto& kv : E) entries.push_back({kv.first.substr(0, k), kv.first[k], false, "", kv.second});
    // B2: a zero-indegree vertex v (a source nobody points to) gets one dummy
    // edge from the node $ v[0..k-2], labelled v[k-1].
    for (const std::string& v : sources)
        if (!targets.count(v)) entries.push_back({"$" + v.substr(0, k - 1), v[k - 1], true, v, 0});
    // B3: a vertex with no outgoing edge gets one edge labelled $.
    for (const std::string& v : targets)
        if (!sources.count(v)) entries.push_back({v, '$', false, "", 0});
    std::sort(entries.begin(), entries.end(), colex_less);

    const uint64_t m = entries.size();
    r->m = m;
    r->W = (uint8_t*)calloc(m + 1, 1);
    r->last = (uint8_t*)calloc(m + 1, 1);
    r->valid = (uint8_t*)calloc(m + 1, 1);
    r->dummy = (uint8_t*)calloc(m + 1, 1);
    r->mult = (uint32_t*)calloc(m + 1, sizeof(uint32_t));
    std::vector<std::string> aux;
    std::set<std::pair<std::string, char>> seen;  // (node symbols 1..k-1, label) met so far
    for (uint64_t i = 0; i < m; i++) {
        const Entry& e = entries[i];
        // B4: last marks the final entry of each node.
        r->last[i] = (i + 1 == m || entries[i + 1].node != e.node) ? 1 : 0;
        if (r->last[i]) r->n_nodes++;
        r->valid[i] = 1;
        r->dummy[i] = e.is_dummy ? 1 : 0;
        r->mult[i] = e.mult;
        // B5: minus flag on every later edge into a target already entered.
        int w = w_code(e.label);
        if (e.label != '$') {
            std::pair<std::string, char> key(e.node.substr(1), e.label);
            if (seen.count(key)) w += 4;
            seen.insert(key);
        }
        r->W[i] = (uint8_t)w;
        if (e.is_dummy) aux.push_back(e.aux);
        if (e.label == '$') r->u++;
    }
    r->t = aux.size();
    put_keys(aux, nw, &r->aux);  // k symbols each, in nw words like the edges
    // B6: F[c] = entries whose node ends with a symbol below c, c in $ A C G T.
    const char order[5] = {'$', 'A', 'C', 'G', 'T'};
    for (int c = 0; c < 5; c++) {
        uint64_t n = 0;
        for (const Entry& e : entries)
            if (e.node[k - 1] < order[c]) n++;
        r->F[c] = n;
    }
    r->F[5] = m;
    return r;
}

void orc_free_sdbg_result(orc_sdbg_result* r) {
    if (!r) return;
    free(r->W);
    free(r->last);
    free(r->valid);
    free(r->dummy);
    free(r->mult);
    free(r->aux);
    free(r);
}

// Sampled check at sizes the string oracle cannot hold: the multiplicity in K
// (both strands, C2) of each query (k+1)-mer, found by scanning every fragment
// of every read.  Here a window is a 256-bit packed value updated as the scan
// moves one base to the right (forward: shift in the new symbol at the low
// end; reverse complement: shift right and put the complement of the new
// symbol at the top), which is the same value encode() gives the substring.
// Queries are packed keys (nw words each).  Threads split the reads; their
// counts are summed.  Returns 0, or -1 on a bad argument.
struct Wide {
    uint64_t w[4];
    bool operator==(const Wide& o) const {
        return w[0] == o.w[0] && w[1] == o.w[1] && w[2] == o.w[2] && w[3] == o.w[3];
    }
};
struct WideHash {
    size_t operator()(const Wide& x) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (int i = 0; i < 4; i++) h = (h ^ x.w[i]) * 0xBF58476D1CE4E5B9ull + (h >> 29);
        return (size_t)h;
    }
};

int orc_count_queries(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads, int k,
                      const uint64_t* queries, uint64_t n_queries, uint64_t* counts,
                      int n_threads) {
    if (k < 2 || k > 127) return -1;
    const int nw = words_for(k);
    const int bits = 2 * (k + 1);
    std::unordered_map<Wide, uint64_t, WideHash> index;
    for (uint64_t q = 0; q < n_queries; q++) {
        Wide x = {{0, 0, 0, 0}};
        for (int w = 0; w < nw; w++) x.w[w] = queries[q * nw + w];
        index[x] = q;
    }
    if (n_threads < 1) n_threads = 1;
    std::vector<std::vector<uint64_t>> part(n_threads, std::vector<uint64_t>(n_queries, 0));
    auto work = [&](int t) {
        uint64_t r0 = n_reads * t / n_threads, r1 = n_reads * (t + 1) / n_threads;
        for (uint64_t r = r0; r < r1; r++) {
            Wide fwd = {{0, 0, 0, 0}}, rev = {{0, 0, 0, 0}};
            int run = 0;  // length of the current fragment so far
            for (uint64_t j = offs[r]; j < offs[r + 1]; j++) {
                char ch = (char)ascii[j];
                if (ch >= 'a' && ch <= 'z') ch = (char)(ch - 'a' + 'A');
                int c = code_of(ch);
                if (c < 0) { run = 0; continue; }
                // forward: value = value * 4 + c, keeping the low 2(k+1) bits
                for (int w = 3; w > 0; w--) fwd.w[w] = (fwd.w[w] << 2) | (fwd.w[w - 1] >> 62);
                fwd.w[0] = (fwd.w[0] << 2) | (uint64_t)c;
                for (int w = 0; w < 4; w++) {
                    int lo = 64 * w;
                    if (bits <= lo) fwd.w[w] = 0;
                    else if (bits < lo + 64) fwd.w[w] &= (1ull << (bits - lo)) - 1;
                }
                // reverse complement: value = value / 4 + (3 - c) * 4^k
                for (int w = 0; w < 3; w++) rev.w[w] = (rev.w[w] >> 2) | (rev.w[w + 1] << 62);
                rev.w[3] >>= 2;
                int top = bits - 2;
                rev.w[top / 64] |= (uint64_t)(3 - c) << (top % 64);
                run++;
                if (run >= k + 1) {
                    auto it = index.find(fwd);
                    if (it != index.end()) part[t][it->second]++;
                    it = index.find(rev);
                    if (it != index.end()) part[t][it->second]++;
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; t++) th.emplace_back(work, t);
    for (auto& x : th) x.join();
    for (uint64_t q = 0; q < n_queries; q++) {
        counts[q] = 0;
        for (int t = 0; t < n_threads; t++) counts[q] += part[t][q];
    }
    return 0;
}

// Every occurrence of the query keys as a forward (k+1)-mer window of a
// fragment (no invalid byte inside it): (query index, read index, position
// of the window's first base in the read).  For tracing a (k+1)-mer back to
// the reads that contain it (the mercy rule of Sec. 2, third paragraph, is a
// statement about a read and its windows).  At most `cap` hits are stored,
// sorted by (query, read, position); returns the number of hits found, or -1
// on a bad argument.
int64_t orc_find_windows(const uint8_t* ascii, const uint64_t* offs, uint64_t n_reads, int k,
                         const uint64_t* queries, uint64_t n_queries, uint64_t cap, uint64_t* hit_q,
                         uint64_t* hit_read, uint64_t* hit_pos, int n_threads) {
    if (k < 2 || k > 127) return -1;
    const int nw = words_for(k);
    const int bits = 2 * (k + 1);
    std::unordered_map<Wide, uint64_t, WideHash> index;
    for (uint64_t q = 0; q < n_queries; q++) {
        Wide x = {{0, 0, 0, 0}};
        for (int w = 0; w < nw; w++) x.w[w] = queries[q * nw + w];
        index[x] = q;
    }
    if (n_threads < 1) n_threads = 1;
    struct Hit {
        uint64_t q, r, p;
    };
    std::vector<std::vector<Hit>> part(n_threads);
    auto work = [&](int t) {
        uint64_t r0 = n_reads * t / n_threads, r1 = n_reads * (t + 1) / n_threads;
        for (uint64_t r = r0; r < r1; r++) {
            Wide fwd = {{0, 0, 0, 0}};
            int run = 0;
            for (uint64_t j = offs[r]; j < offs[r + 1]; j++) {
                char ch = (char)ascii[j];
                if (ch >= 'a' && ch <= 'z') ch = (char)(ch - 'a' + 'A');
                int c = code_of(ch);
                if (c < 0) { run = 0; continue; }
                for (int w = 3; w > 0; w--) fwd.w[w] = (fwd.w[w] << 2) | (fwd.w[w - 1] >> 62);
                fwd.w[0] = (fwd.w[0] << 2) | (uint64_t)c;
                for (int w = 0; w < 4; w++) {
                    int lo = 64 * w;
                    if (bits <= lo) fwd.w[w] = 0;
                    else if (bits < lo + 64) fwd.w[w] &= (1ull << (bits - lo)) - 1;
                }
                run++;
                if (run >= k + 1) {
                    auto it = index.find(fwd);
                    if (it != index.end()) part[t].push_back({it->second, r, j - offs[r] - (uint64_t)k});
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; t++) th.emplace_back(work, t);
    for (auto& x : th) x.join();
    std::vector<Hit> all;
    for (auto& v : part) all.insert(all.end(), v.begin(), v.end());
    std::sort(all.begin(), all.end(), [](const Hit& a, const Hit& b) {
        if (a.q != b.q) return a.q < b.q;
        if (a.r != b.r) return a.r < b.r;
        return a.p < b.p;
    });
    for (uint64_t i = 0; i < all.size() && i < cap; i++) {
        hit_q[i] = all[i].q;
        hit_read[i] = all[i].r;
        hit_pos[i] = all[i].p;
    }
    return (int64_t)all.size();
}

}  // extern "C"
