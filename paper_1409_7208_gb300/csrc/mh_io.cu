// Flat-file SdBG: the BOSS arrays of mh_build_sdbg (Sec. 2: W with the minus
// flag, last, F, the dummy and valid bit-vectors and the auxiliary store of
// the zero-indegree vertices) written to and read from one binary file, so
// that a graph outlives the process that built it.
//
// Layout (little-endian):
//   "MHSDBG01"                                   8 bytes
//   uint32 version (1), int32 k, int32 nw, uint32 flags (bit 0: mult)
//   uint64 m, t, u, n_nodes, F[6]
//   W        m bytes
//   last, valid, dummy   ceil(m / 32) uint32 words each
//   aux      t * nw uint64 words
//   mult     m uint32 (when flagged)
//   uint64   FNV-1a hash of every byte before it
// Arrays move between the device and the file in pieces through one host
// buffer.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mh_internal.cuh"

using namespace mh;

namespace {

constexpr char kMagic[8] = {'M', 'H', 'S', 'D', 'B', 'G', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kPiece = 64u << 20;

struct Fnv {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 0x100000001b3ull;
    }
};

struct Header {
    uint32_t version;
    int32_t k, nw;
    uint32_t flags;
    uint64_t m, t, u, n_nodes, F[6];
};

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

bool put(FILE* f, Fnv& h, const void* p, size_t n) {
    h.add(p, n);
    return fwrite(p, 1, n, f) == n;
}

bool get(FILE* f, Fnv& h, void* p, size_t n) {
    if (fread(p, 1, n, f) != n) return false;
    h.add(p, n);
    return true;
}

// device array -> file, in pieces
bool put_device(mh_ctx* ctx, FILE* f, Fnv& h, const void* d, size_t bytes, std::vector<unsigned char>& buf) {
    for (size_t o = 0; o < bytes; o += kPiece) {
        const size_t n = std::min(kPiece, bytes - o);
        if (cudaMemcpyAsync(buf.data(), static_cast<const unsigned char*>(d) + o, n, cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            throw Error{MH_EDEVICE, "mh_sdbg_save: a device copy failed"};
        if (!put(f, h, buf.data(), n)) return false;
    }
    return true;
}

// file -> device array, in pieces
bool get_device(mh_ctx* ctx, FILE* f, Fnv& h, void* d, size_t bytes, std::vector<unsigned char>& buf) {
    for (size_t o = 0; o < bytes; o += kPiece) {
        const size_t n = std::min(kPiece, bytes - o);
        if (!get(f, h, buf.data(), n)) return false;
        if (cudaMemcpyAsync(static_cast<unsigned char*>(d) + o, buf.data(), n, cudaMemcpyHostToDevice,
                            ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            throw Error{MH_EDEVICE, "mh_sdbg_load: a device copy failed"};
    }
    return true;
}

size_t bit_words(uint64_t m) { return (size_t)((m + 31) / 32); }

}  // namespace

extern "C" {

int mh_sdbg_save(const mh_sdbg* g, const char* path) {
    if (!g || !path || !g->ctx) return MH_EINVAL;
    NvtxRange nvtx("mh_sdbg_save");
    mh_ctx* ctx = g->ctx;
    try {
        if (cudaSetDevice(ctx->device) != cudaSuccess) throw Error{MH_EDEVICE, "cudaSetDevice failed"};
        // every kernel that wrote the graph has finished
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) throw Error{MH_EDEVICE, "stream failed"};
        File file;
        file.f = fopen(path, "wb");
        if (!file.f) throw Error{MH_EINVAL, std::string("mh_sdbg_save: cannot open ") + path};
        Fnv h;
        Header hd{};
        hd.version = kVersion;
        hd.k = g->k;
        hd.nw = g->nw;
        hd.flags = g->mult ? 1u : 0u;
        hd.m = g->m;
        hd.t = g->t;
        hd.u = g->u;
        hd.n_nodes = g->n_nodes;
        for (int i = 0; i < 6; i++) hd.F[i] = g->F[i];
        std::vector<unsigned char> buf(kPiece);
        const size_t bw = bit_words(g->m) * 4;
        bool ok = put(file.f, h, kMagic, 8) && put(file.f, h, &hd, sizeof hd) &&
                  put_device(ctx, file.f, h, g->W, g->m, buf) && put_device(ctx, file.f, h, g->last, bw, buf) &&
                  put_device(ctx, file.f, h, g->valid, bw, buf) && put_device(ctx, file.f, h, g->dummy, bw, buf) &&
                  put_device(ctx, file.f, h, g->aux, g->t * g->nw * 8, buf) &&
                  (!g->mult || put_device(ctx, file.f, h, g->mult, g->m * 4, buf));
        const uint64_t sum = h.h;
        ok = ok && fwrite(&sum, 1, 8, file.f) == 8;
        ok = fclose(file.f) == 0 && ok;
        file.f = nullptr;
        if (!ok) throw Error{MH_EINVAL, std::string("mh_sdbg_save: writing ") + path + " failed"};
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    }
    return MH_OK;
}

int mh_sdbg_load(mh_ctx* ctx, const char* path, mh_sdbg** out) {
    if (!ctx || !path || !out) return MH_EINVAL;
    NvtxRange nvtx("mh_sdbg_load");
    *out = nullptr;
    mh_sdbg* g = nullptr;
    try {
        if (cudaSetDevice(ctx->device) != cudaSuccess) throw Error{MH_EDEVICE, "cudaSetDevice failed"};
        File file;
        file.f = fopen(path, "rb");
        if (!file.f) throw Error{MH_EINVAL, std::string("mh_sdbg_load: cannot open ") + path};
        // the file's size bounds every count before anything is allocated
        if (fseek(file.f, 0, SEEK_END) != 0) throw Error{MH_EINVAL, "mh_sdbg_load: cannot seek"};
        const long size = ftell(file.f);
        rewind(file.f);
        Fnv h;
        char magic[8];
        Header hd{};
        const auto bad = [&](const char* why) { return Error{MH_EINVAL, std::string("mh_sdbg_load: ") + why}; };
        if (!get(file.f, h, magic, 8) || memcmp(magic, kMagic, 8) != 0) throw bad("not an SdBG file");
        if (!get(file.f, h, &hd, sizeof hd)) throw bad("truncated header");
        if (hd.version != kVersion) throw bad("unknown version");
        if (hd.k < 2 || hd.k > 127 || hd.nw != words_for(hd.k) || hd.flags > 1) throw bad("bad header fields");
        const uint64_t bw = bit_words(hd.m) * 4;
        const uint64_t limit = (uint64_t)(size > 0 ? size : 0);
        if (hd.m > limit || hd.t > limit || hd.u > hd.m || hd.t > hd.m || hd.n_nodes > hd.m || hd.F[5] != hd.m)
            throw bad("sizes do not match the file");
        const uint64_t body = 8 + sizeof hd + hd.m + 3 * bw + hd.t * hd.nw * 8 + (hd.flags ? hd.m * 4 : 0) + 8;
        if (body != limit) throw bad("sizes do not match the file");
        g = new mh_sdbg;
        g->ctx = ctx;
        g->k = hd.k;
        g->nw = hd.nw;
        g->m = hd.m;
        g->t = hd.t;
        g->u = hd.u;
        g->n_nodes = hd.n_nodes;
        for (int i = 0; i < 6; i++) g->F[i] = hd.F[i];
        g->W = static_cast<uint8_t*>(ctx_alloc(ctx, hd.m ? hd.m : 1));
        g->last = static_cast<uint32_t*>(ctx_alloc(ctx, bw ? bw : 4));
        g->valid = static_cast<uint32_t*>(ctx_alloc(ctx, bw ? bw : 4));
        g->dummy = static_cast<uint32_t*>(ctx_alloc(ctx, bw ? bw : 4));
        g->aux = static_cast<uint64_t*>(ctx_alloc(ctx, hd.t ? hd.t * hd.nw * 8 : 8));
        if (hd.flags) g->mult = static_cast<uint32_t*>(ctx_alloc(ctx, hd.m ? hd.m * 4 : 4));
        std::vector<unsigned char> buf(kPiece);
        const bool ok = get_device(ctx, file.f, h, g->W, hd.m, buf) &&
                        get_device(ctx, file.f, h, g->last, bw, buf) &&
                        get_device(ctx, file.f, h, g->valid, bw, buf) &&
                        get_device(ctx, file.f, h, g->dummy, bw, buf) &&
                        get_device(ctx, file.f, h, g->aux, hd.t * hd.nw * 8, buf) &&
                        (!hd.flags || get_device(ctx, file.f, h, g->mult, hd.m * 4, buf));
        uint64_t sum = 0;
        if (!ok || fread(&sum, 1, 8, file.f) != 8) throw bad("truncated arrays");
        if (sum != h.h) throw bad("checksum mismatch (the file is damaged)");
    } catch (const Error& e) {
        mh_free_sdbg(g);
        ctx->last_error = e.msg;
        return e.code;
    }
    *out = g;
    return MH_OK;
}

}  // extern "C"
