// C ABI entry points, context, allocator, profiling and error handling.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>

#include "mh_internal.cuh"

namespace mh {

void pack_reads(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs,
                uint64_t n_reads, mh_reads* out);
template <int NW>
void count_kmers(mh_ctx* ctx, const mh_reads* reads, int k, int d, mh_kmers* out);
template <int NW>
void mercy_kmers(mh_ctx* ctx, const mh_reads* reads, const mh_kmers* solid, mh_kmers* out);
template <int NW>
void build_sdbg(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, mh_sdbg* out);

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    int code = (e == cudaErrorMemoryAllocation) ? MH_ENOMEM : MH_EDEVICE;
    fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

// Host-side fault injection for tests: MH_FAULT=alloc:N makes the N-th
// device allocation of the process (counted from 1, over all contexts) fail
// as if the device were out of memory; the ones after it succeed.
static bool injected_alloc_failure() {
    static const long target = [] {
        const char* e = std::getenv("MH_FAULT");
        if (!e || std::strncmp(e, "alloc:", 6) != 0) return 0L;
        return std::strtol(e + 6, nullptr, 10);
    }();
    static std::atomic<long> count{0};
    return target > 0 && count.fetch_add(1) + 1 == target;
}

void* ctx_alloc(mh_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 1;
    bytes = (bytes + 255) & ~size_t(255);
    std::lock_guard<std::mutex> lock(ctx->alloc_mu);
    if (injected_alloc_failure()) fail(MH_ENOMEM, "injected allocation failure (MH_FAULT)");
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        fail(MH_ENOMEM, "HBM budget exceeded: " + std::to_string(ctx->in_use) + " + " + std::to_string(bytes) +
                            " > " + std::to_string(ctx->budget) + " bytes");
    void* p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, ctx->stream, ctx->alloc_user);
        if (!p) fail(MH_ENOMEM, "allocator callback failed for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(MH_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                cudaGetErrorString(e));
        }
    }
    ctx->sizes[p] = bytes;
    ctx->in_use += bytes;
    ctx->peak = std::max(ctx->peak, ctx->in_use);
    return p;
}

void ctx_free(mh_ctx* ctx, void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(ctx->alloc_mu);
    auto it = ctx->sizes.find(p);
    size_t bytes = it == ctx->sizes.end() ? 0 : it->second;
    if (it != ctx->sizes.end()) ctx->sizes.erase(it);
    ctx->in_use -= bytes;
    if (ctx->free_fn)
        ctx->free_fn(p, bytes, ctx->stream, ctx->alloc_user);
    else
        cudaFreeAsync(p, ctx->stream);
}

int grid_for(mh_ctx* ctx, uint64_t work_items, int per_block, int blocks_per_sm) {
    uint64_t need = ceil_div(work_items ? work_items : 1, (uint64_t)per_block);
    uint64_t cap = (uint64_t)ctx->num_sms * blocks_per_sm;
    return (int)std::max<uint64_t>(1, std::min(need, cap));
}

static cudaEvent_t take_event(mh_ctx* ctx) {
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    MH_CUDA(cudaEventCreate(&e));
    return e;
}

// Fold finished event pairs into the per-kernel statistics.
static void drain_events(mh_ctx* ctx, bool wait) {
    size_t keep = 0;
    for (size_t i = 0; i < ctx->pending.size(); i++) {
        auto& p = ctx->pending[i];
        if (wait) cudaEventSynchronize(p.b);
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            ctx->pending[keep++] = p;
            continue;
        }
        if (e == cudaSuccess) {
            ctx->stats[p.name].launches++;
            ctx->stats[p.name].total_ms += ms;
            ctx->stats[p.name].bytes += p.bytes;
        } else {
            cudaGetLastError();
        }
        ctx->ev_free.push_back(p.a);
        ctx->ev_free.push_back(p.b);
    }
    ctx->pending.resize(keep);
}

Prof::Prof(mh_ctx* c, const char* name, uint64_t algo_bytes) : range(name), ctx(c), bytes(algo_bytes) {
    if (!ctx->profile) return;
    auto it = ctx->name_id.find(name);
    if (it == ctx->name_id.end()) {
        id = (int)ctx->names.size();
        ctx->name_id[name] = id;
        ctx->names.push_back(name);
        ctx->stats.emplace_back();
    } else {
        id = it->second;
    }
    if (ctx->pending.size() > 4096) drain_events(ctx, true);
    a = take_event(ctx);
    b = take_event(ctx);
    cudaEventRecord(a, ctx->stream);
}

Prof::~Prof() {
    if (id < 0) return;
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({id, a, b, bytes});
}

void sync_and_check(mh_ctx* ctx) {
    MH_CUDA(cudaMemcpyAsync(ctx->h_pinned + 63, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
    MH_CUDA(cudaStreamSynchronize(ctx->stream));
    uint32_t st = (uint32_t)(ctx->h_pinned[63] & 0xFFFFFFFFu);
    if (st) {
        MH_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
        if (st & ST_SPIN_TIMEOUT) fail(MH_ETIMEOUT, "a bounded device wait (radix look-back) ran out");
        if (st & ST_OVERFLOW) fail(MH_EOVERFLOW, "a (k+1)-mer count exceeds 2^32-1");
        if (st & ST_TABLE_FULL) fail(MH_EDEVICE, "hash table probe sequence exhausted");
        if (st & ST_BAD_INPUT) fail(MH_EINVAL, "read offsets are not non-decreasing from 0 to n_bases");
        if (st & ST_BAD_TABLE) fail(MH_EINVAL, "solid table is not a set of distinct sorted (k+1)-mers");
        fail(MH_EDEVICE, "device status " + std::to_string(st));
    }
}

// Add src's kernel statistics to dst's (by kernel name) and clear src's.
void profile_merge(mh_ctx* dst, mh_ctx* src) {
    cudaStreamSynchronize(src->stream);
    drain_events(src, true);
    for (size_t i = 0; i < src->names.size(); i++) {
        KernelStat& s = src->stats[i];
        if (!s.launches) continue;
        auto it = dst->name_id.find(src->names[i]);
        int id;
        if (it == dst->name_id.end()) {
            id = (int)dst->names.size();
            dst->name_id[src->names[i]] = id;
            dst->names.push_back(src->names[i]);
            dst->stats.emplace_back();
        } else {
            id = it->second;
        }
        dst->stats[id].launches += s.launches;
        dst->stats[id].total_ms += s.total_ms;
        dst->stats[id].bytes += s.bytes;
        s = KernelStat();
    }
}

void read_u64(mh_ctx* ctx, const uint64_t* d, uint64_t* h, int count) {
    if (count > 62) fail(MH_EINVAL, "read_u64: too many words");
    MH_CUDA(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(uint64_t) * count, cudaMemcpyDeviceToHost, ctx->stream));
    sync_and_check(ctx);
    std::memcpy(h, ctx->h_pinned, sizeof(uint64_t) * count);
}

}  // namespace mh

using namespace mh;

// Run `body`, turning library errors into return codes.
template <class F>
static int guarded(mh_ctx* ctx, F&& body) {
    try {
        body();
        if (ctx) ctx->last_error.clear();
        return MH_OK;
    } catch (const Error& e) {
        if (ctx) ctx->last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->last_error = "host allocation failed";
        return MH_ENOMEM;
    }
}

extern "C" {

int mh_create(const mh_config* cfg, mh_ctx** out) {
    if (!cfg || !out) return MH_EINVAL;
    *out = nullptr;
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return MH_EINVAL;
    auto ctx = std::make_unique<mh_ctx>();
    int rc = guarded(nullptr, [&] {
        ctx->device = cfg->device;
        MH_CUDA(cudaSetDevice(cfg->device));
        MH_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, cfg->device));
        size_t mem_free = 0, mem_total = 0;
        MH_CUDA(cudaMemGetInfo(&mem_free, &mem_total));
        ctx->device_bytes = mem_total;
        if (cfg->stream) {
            ctx->stream = (cudaStream_t)cfg->stream;
        } else {
            // a blocking stream: ordered with the legacy default stream, as a
            // caller on that stream expects
            MH_CUDA(cudaStreamCreate(&ctx->stream));
            ctx->own_stream = true;
        }
        ctx->alloc = cfg->alloc;
        ctx->free_fn = cfg->free;
        ctx->alloc_user = cfg->alloc_user;
        ctx->budget = cfg->hbm_budget;
        ctx->with_mult = cfg->with_mult;
        ctx->profile = cfg->profile;
        if (!ctx->alloc) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = cfg->device;
            MH_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
            uint64_t thr = UINT64_MAX;
            MH_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr));
        }
        MH_CUDA(cudaMalloc(&ctx->d_status, 256));
        MH_CUDA(cudaMemset(ctx->d_status, 0, 256));
        MH_CUDA(cudaMallocHost(&ctx->h_pinned, 64 * sizeof(uint64_t)));
    });
    if (rc != MH_OK) {
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        return rc;
    }
    *out = ctx.release();
    return MH_OK;
}

void mh_destroy(mh_ctx* ctx) {
    if (!ctx) return;
    for (mh_ctx* w : ctx->workers) mh_destroy(w);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_pinned);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    for (cudaEvent_t e : ctx->pack_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int mh_pack_reads(mh_ctx* ctx, const uint8_t* ascii, uint64_t n_bases, const uint64_t* offs, uint64_t n_reads,
                  int on_device, mh_reads** out) {
    NvtxRange nvtx("mh_pack_reads");
    if (!ctx || !out || !offs || (!ascii && n_bases)) return MH_EINVAL;
    *out = nullptr;
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto r = std::make_unique<mh_reads>();
        r->ctx = ctx;
        if (on_device) {
            pack_reads(ctx, ascii, n_bases, offs, n_reads, r.get());
        } else {
            // monotonicity is checked on the device with the other offset checks
            if (offs[0] != 0 || offs[n_reads] != n_bases) fail(MH_EINVAL, "offs must run from 0 to n_bases");
            pack_reads_host(ctx, ascii, n_bases, offs, n_reads, r.get());
        }
        *out = r.release();
    });
}

int mh_pack_reads_contigs(mh_ctx* ctx, const uint8_t* ascii, uint64_t n_bases, const uint64_t* offs,
                          uint64_t n_reads, const mh_contigs* contigs, int copies, mh_reads** out) {
    NvtxRange nvtx("mh_pack_reads_contigs");
    if (!ctx || !out || !offs || (!ascii && n_bases) || copies < 0) return MH_EINVAL;
    *out = nullptr;
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto r = std::make_unique<mh_reads>();
        r->ctx = ctx;
        pack_with_contigs(ctx, ascii, n_bases, offs, n_reads, contigs, (uint32_t)copies, r.get());
        *out = r.release();
    });
}

int mh_walk_contigs(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, uint64_t n_walks, uint64_t max_len,
                    uint64_t seed, mh_contigs** out) {
    NvtxRange nvtx("mh_walk_contigs");
    if (!ctx || !solid || !out) return MH_EINVAL;
    *out = nullptr;
    if ((mercy && mercy->k != solid->k) || max_len < (uint64_t)solid->k + 1 || max_len >= (1ull << 24) ||
        n_walks >= (1ull << 40)) {
        ctx->last_error = "mh_walk_contigs: need k+1 <= max_len < 2^24, n_walks < 2^40, equal k";
        return MH_EINVAL;
    }
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto c = std::make_unique<mh_contigs>();
        c->ctx = ctx;
        switch (solid->nw) {
            case 1: walk_contigs<1>(ctx, solid, mercy, n_walks, (uint32_t)max_len, seed, c.get()); break;
            case 2: walk_contigs<2>(ctx, solid, mercy, n_walks, (uint32_t)max_len, seed, c.get()); break;
            default: walk_contigs<4>(ctx, solid, mercy, n_walks, (uint32_t)max_len, seed, c.get()); break;
        }
        *out = c.release();
    });
}

int mh_contigs_view_get(const mh_contigs* c, mh_contigs_view* v) {
    if (!c || !v) return MH_EINVAL;
    v->k = c->k;
    v->n = c->n;
    v->n_bases = c->n_bases;
    v->ascii = c->ascii;
    v->offs = c->offs;
    return MH_OK;
}

void mh_free_contigs(mh_contigs* c) {
    if (!c) return;
    ctx_free(c->ctx, c->ascii);
    ctx_free(c->ctx, c->offs);
    delete c;
}

int mh_reads_view_get(const mh_reads* r, mh_reads_view* v) {
    if (!r || !v) return MH_EINVAL;
    v->n_reads = r->n_reads;
    v->n_bases = r->n_bases;
    v->n_frags = r->n_frags;
    v->n_packed = r->n_packed;
    v->packed = r->packed;
    v->frag_offs = r->frag_offs;
    v->frag_read = r->frag_read;
    return MH_OK;
}

void mh_free_reads(mh_reads* r) {
    if (!r) return;
    ctx_free(r->ctx, r->packed);
    ctx_free(r->ctx, r->frag_offs);
    ctx_free(r->ctx, r->frag_read);
    delete r;
}

int mh_count_kmers(mh_ctx* ctx, const mh_reads* reads, int k, int d, mh_kmers** out) {
    NvtxRange nvtx("mh_count_kmers");
    if (!ctx || !reads || !out || k < 2 || k > 127 || d < 1) {
        if (ctx) ctx->last_error = "mh_count_kmers: need ctx, reads, out, 2 <= k <= 127, d >= 1";
        return MH_EINVAL;
    }
    *out = nullptr;
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto s = std::make_unique<mh_kmers>();
        s->ctx = ctx;
        switch (words_for(k)) {
            case 1: count_kmers<1>(ctx, reads, k, d, s.get()); break;
            case 2: count_kmers<2>(ctx, reads, k, d, s.get()); break;
            default: count_kmers<4>(ctx, reads, k, d, s.get()); break;
        }
        *out = s.release();
    });
}

int mh_mercy_kmers(mh_ctx* ctx, const mh_reads* reads, const mh_kmers* solid, mh_kmers** out) {
    NvtxRange nvtx("mh_mercy_kmers");
    if (!ctx || !reads || !solid || !out) return MH_EINVAL;
    *out = nullptr;
    if (!solid->spectrum) {
        ctx->last_error = "mh_mercy_kmers: the solid handle must come from mh_count_kmers";
        return MH_EINVAL;
    }
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto m = std::make_unique<mh_kmers>();
        m->ctx = ctx;
        switch (solid->nw) {
            case 1: mercy_kmers<1>(ctx, reads, solid, m.get()); break;
            case 2: mercy_kmers<2>(ctx, reads, solid, m.get()); break;
            default: mercy_kmers<4>(ctx, reads, solid, m.get()); break;
        }
        *out = m.release();
    });
}

int mh_kmers_view_get(const mh_kmers* s, mh_kmers_view* v) {
    if (!s || !v) return MH_EINVAL;
    v->k = s->k;
    v->nw = s->nw;
    v->n = s->n;
    v->keys = s->keys;
    v->counts = s->counts;
    v->n_kmers = s->n_kmers;
    v->n_distinct = s->n_distinct;
    return MH_OK;
}

void mh_free_kmers(mh_kmers* s) {
    if (!s) return;
    ctx_free(s->ctx, s->keys);
    ctx_free(s->ctx, s->counts);
    ctx_free(s->ctx, s->spectrum);
    ctx_free(s->ctx, s->spectrum_len);
    delete s;
}

int mh_build_sdbg(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, mh_sdbg** out) {
    NvtxRange nvtx("mh_build_sdbg");
    if (!ctx || !solid || !out) return MH_EINVAL;
    *out = nullptr;
    if (mercy && mercy->k != solid->k) {
        ctx->last_error = "mh_build_sdbg: solid and mercy have different k";
        return MH_EINVAL;
    }
    return guarded(ctx, [&] {
        MH_CUDA(cudaSetDevice(ctx->device));
        auto g = std::make_unique<mh_sdbg>();
        g->ctx = ctx;
        switch (solid->nw) {
            case 1: build_sdbg<1>(ctx, solid, mercy, g.get()); break;
            case 2: build_sdbg<2>(ctx, solid, mercy, g.get()); break;
            default: build_sdbg<4>(ctx, solid, mercy, g.get()); break;
        }
        *out = g.release();
    });
}

int mh_sdbg_view_get(const mh_sdbg* g, mh_sdbg_view* v) {
    if (!g || !v) return MH_EINVAL;
    v->k = g->k;
    v->nw = g->nw;
    v->m = g->m;
    v->t = g->t;
    v->u = g->u;
    v->n_nodes = g->n_nodes;
    for (int i = 0; i < 6; i++) v->F[i] = g->F[i];
    v->W = g->W;
    v->last = g->last;
    v->valid = g->valid;
    v->dummy = g->dummy;
    v->aux = g->aux;
    v->mult = g->mult;
    return MH_OK;
}

void mh_free_sdbg(mh_sdbg* g) {
    if (!g) return;
    mh_ctx* c = g->ctx;
    ctx_free(c, g->W);
    ctx_free(c, g->last);
    ctx_free(c, g->valid);
    ctx_free(c, g->dummy);
    ctx_free(c, g->aux);
    ctx_free(c, g->mult);
    delete g;
}

const char* mh_strerror(int code) {
    switch (code) {
        case MH_OK: return "ok";
        case MH_EINVAL: return "invalid argument";
        case MH_ENOMEM: return "out of device memory or over the HBM budget";
        case MH_EOVERFLOW: return "count or size overflow";
        case MH_ETIMEOUT: return "bounded device wait timed out";
        case MH_EDEVICE: return "CUDA error";
        case MH_EUNSUPPORTED: return "unsupported";
    }
    return "unknown error";
}

const char* mh_last_error_message(const mh_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void* mh_stream(const mh_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int mh_trim(mh_ctx* ctx) {
    if (!ctx) return MH_EINVAL;
    return guarded(ctx, [&] {
        if (ctx->pool) {
            MH_CUDA(cudaStreamSynchronize(ctx->stream));
            MH_CUDA(cudaMemPoolTrimTo(ctx->pool, 0));
        }
    });
}

void mh_memory(const mh_ctx* ctx, uint64_t* in_use, uint64_t* peak) {
    if (in_use) *in_use = ctx ? ctx->in_use : 0;
    if (peak) *peak = ctx ? ctx->peak : 0;
}

int mh_profile_count(mh_ctx* ctx) {
    if (!ctx) return 0;
    cudaStreamSynchronize(ctx->stream);
    drain_events(ctx, true);
    return (int)ctx->names.size();
}

int mh_profile_get(mh_ctx* ctx, int i, char* name, int name_cap, uint64_t* launches, double* total_ms,
                   uint64_t* bytes) {
    if (!ctx || i < 0 || i >= (int)ctx->names.size()) return MH_EINVAL;
    drain_events(ctx, true);
    if (name && name_cap > 0) {
        std::strncpy(name, ctx->names[i].c_str(), name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (launches) *launches = ctx->stats[i].launches;
    if (total_ms) *total_ms = ctx->stats[i].total_ms;
    if (bytes) *bytes = ctx->stats[i].bytes;
    return MH_OK;
}

void mh_profile_reset(mh_ctx* ctx) {
    if (!ctx) return;
    drain_events(ctx, true);
    for (auto& s : ctx->stats) s = KernelStat();
}

void mh_set_profile(mh_ctx* ctx, int on) {
    if (ctx) ctx->profile = on;
}

}  // extern "C"
