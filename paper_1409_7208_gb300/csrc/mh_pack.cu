// mh_pack_reads: ASCII reads -> 2-bit packed fragments.
//
// One thread per 16 input bytes: a 16-byte vector load, per-byte code and
// validity with SIMD byte compares, one 32-bit output word (base j at bits
// 31-2(j%16)).  When every byte is a base and no read is empty, fragments are
// the reads and the packed words are the output.  Otherwise the valid bases
// are compacted (scan of per-chunk valid counts) and fragment starts are
// found from the validity masks and the read starts.
#include <cstdlib>

#include "mh_internal.cuh"

namespace mh {

// byte codes: A/a 0, C/c 1, G/g 2, T/t 3 (((c >> 1) ^ (c >> 2)) & 3 on those letters)
__device__ __forceinline__ uint32_t codes4(uint32_t x) { return ((x >> 1) ^ (x >> 2)) & 0x03030303u; }

// 0xFF in each byte lane holding one of ACGTacgt
__device__ __forceinline__ uint32_t valid4(uint32_t x) {
    uint32_t u = x & 0xDFDFDFDFu;
    return __vcmpeq4(u, 0x41414141u) | __vcmpeq4(u, 0x43434343u) | __vcmpeq4(u, 0x47474747u) |
           __vcmpeq4(u, 0x54545454u);
}

// codes of 4 bytes (byte 0 = first base) -> 8 bits, first base most significant
__device__ __forceinline__ uint32_t pack4(uint32_t c) {
    return ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
}

// valid lanes (0xFF bytes) -> 4-bit mask, bit j = byte j
__device__ __forceinline__ uint32_t mask4(uint32_t v) {
    return (v & 1u) | ((v >> 7) & 2u) | ((v >> 14) & 4u) | ((v >> 21) & 8u);
}

// Load the 16 bytes of chunk c as four words (zero past n_bases).
__device__ __forceinline__ void load16(const uint8_t* __restrict__ a, uint64_t n_bases, uint64_t c, bool vec,
                                       uint32_t x[4], uint32_t* present) {
    uint64_t b = c * 16;
    if (vec && b + 16 <= n_bases) {
        uint4 v = reinterpret_cast<const uint4*>(a)[c];
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
        *present = 0xFFFFu;
        return;
    }
    uint32_t pm = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint64_t i = b + 4 * q + j;
            if (i < n_bases) {
                w |= (uint32_t)a[i] << (8 * j);
                pm |= 1u << (4 * q + j);
            }
        }
        x[q] = w;
    }
    *present = pm;
}

// Fast-path pack: code word per chunk; sets *any_invalid if a byte is not a base.
__global__ void pack_chunks_kernel(const uint8_t* __restrict__ ascii, uint64_t n_bases, bool vec,
                                   uint32_t* __restrict__ packed, uint32_t* __restrict__ any_invalid) {
    uint64_t n_chunks = ceil_div(n_bases, 16);
    bool bad = false;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x[4], present;
        load16(ascii, n_bases, c, vec, x, &present);
        uint32_t word = 0, vmask = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            word |= pack4(codes4(x[q])) << (24 - 8 * q);
            vmask |= mask4(valid4(x[q])) << (4 * q);
        }
        packed[c] = word;
        bad |= (vmask & present) != present;
    }
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(any_invalid, 1u);
}

// Validate offsets; flag empty reads.
__global__ void check_offs_kernel(const uint64_t* __restrict__ offs, uint64_t n_reads, uint64_t n_bases,
                                  uint32_t* __restrict__ any_empty, uint32_t* __restrict__ err) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i == 0 && (offs[0] != 0 || offs[n_reads] != n_bases)) atomicOr(err, ST_BAD_INPUT);
    bool empty = false;
    for (; i < n_reads; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = offs[i], b = offs[i + 1];
        if (b < a || b > n_bases) atomicOr(err, ST_BAD_INPUT);
        empty |= a == b;
    }
    if (__any_sync(0xFFFFFFFFu, empty) && (threadIdx.x & 31) == 0) atomicOr(any_empty, 1u);
}

__global__ void iota_u32_kernel(uint32_t* __restrict__ a, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

// --------------------------------------------------------- slow path
// Per chunk: 16-bit validity mask and its popcount.
__global__ void chunk_masks_kernel(const uint8_t* __restrict__ ascii, uint64_t n_bases, bool vec,
                                   uint32_t* __restrict__ mask, uint32_t* __restrict__ cnt) {
    uint64_t n_chunks = ceil_div(n_bases, 16);
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x[4], present;
        load16(ascii, n_bases, c, vec, x, &present);
        uint32_t vmask = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) vmask |= mask4(valid4(x[q])) << (4 * q);
        vmask &= present;
        mask[c] = vmask;
        cnt[c] = __popc(vmask);
    }
}

__global__ void read_starts_kernel(const uint64_t* __restrict__ offs, uint64_t n_reads,
                                   uint32_t* __restrict__ rs_bits) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_reads;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = offs[r];
        if (offs[r + 1] > a) atomicOr(&rs_bits[a >> 5], 1u << (a & 31));
    }
}

// Fragment-start bits of chunk c: valid and (read start or previous base invalid).
__device__ __forceinline__ uint32_t frag_start_bits(const uint32_t* mask, const uint32_t* rs_bits, uint64_t c) {
    uint32_t m = mask[c];
    uint32_t prev_valid_top = c ? (mask[c - 1] >> 15) & 1u : 0u;
    uint32_t prev = (m << 1) | prev_valid_top;  // bit j = validity of base j-1
    uint32_t rs = (rs_bits[(c * 16) >> 5] >> ((c * 16) & 31)) & 0xFFFFu;
    return m & (rs | ~prev) & 0xFFFFu;
}

__global__ void frag_count_kernel(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ rs_bits,
                                  uint64_t n_chunks, uint32_t* __restrict__ fcnt) {
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x)
        fcnt[c] = __popc(frag_start_bits(mask, rs_bits, c));
}

__global__ void frag_write_kernel(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ rs_bits,
                                  const uint64_t* __restrict__ dst, const uint64_t* __restrict__ fidx,
                                  const uint64_t* __restrict__ offs, uint64_t n_reads, uint64_t n_chunks,
                                  uint64_t* __restrict__ frag_offs, uint32_t* __restrict__ frag_read) {
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t fs = frag_start_bits(mask, rs_bits, c);
        uint32_t m = mask[c];
        uint64_t f = fidx[c];
        while (fs) {
            int j = __ffs(fs) - 1;
            fs &= fs - 1;
            frag_offs[f] = dst[c] + __popc(m & ((1u << j) - 1));
            // read holding base c*16+j: last r with offs[r] <= base and a non-empty read
            uint64_t base = c * 16 + j;
            uint64_t lo = 0, hi = n_reads;  // find first r with offs[r] > base, answer r-1
            while (lo < hi) {
                uint64_t mid = (lo + hi) >> 1;
                if (offs[mid] <= base) lo = mid + 1; else hi = mid;
            }
            frag_read[f] = (uint32_t)(lo - 1);
            f++;
        }
    }
}

__global__ void compact_pack_kernel(const uint8_t* __restrict__ ascii, uint64_t n_bases, bool vec,
                                    const uint32_t* __restrict__ mask, const uint64_t* __restrict__ dst,
                                    uint32_t* __restrict__ packed) {
    uint64_t n_chunks = ceil_div(n_bases, 16);
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x[4], present;
        load16(ascii, n_bases, c, vec, x, &present);
        uint32_t m = mask[c];
        if (!m) continue;
        uint64_t pos = dst[c];
        uint64_t w0 = pos >> 4;
        uint32_t acc[2] = {0u, 0u};
#pragma unroll
        for (int j = 0; j < 16; j++) {
            if (m & (1u << j)) {
                uint32_t code = (codes4(x[j >> 2]) >> (8 * (j & 3))) & 3u;
                uint64_t wi = (pos >> 4) - w0;
                acc[wi] |= code << (30 - 2 * (pos & 15));
                pos++;
            }
        }
        if (acc[0]) atomicOr(&packed[w0], acc[0]);
        if (acc[1]) atomicOr(&packed[w0 + 1], acc[1]);
    }
}

void pack_reads(mh_ctx* ctx, const uint8_t* d_ascii, uint64_t n_bases, const uint64_t* d_offs, uint64_t n_reads,
                mh_reads* out) {
    const uint64_t n_chunks = ceil_div(n_bases, 16);
    const bool vec = (reinterpret_cast<uintptr_t>(d_ascii) & 15) == 0;
    out->n_reads = n_reads;
    out->n_bases = n_bases;
    Buf<uint32_t> flags(ctx, 2);  // [0] any invalid byte, [1] any empty read
    flags.zero();
    Buf<uint32_t> packed(ctx, n_chunks + kPackPad);
    MH_CUDA(cudaMemsetAsync(packed.p + n_chunks, 0, kPackPad * sizeof(uint32_t), ctx->stream));
    MH_LAUNCH(ctx, "check_offs", grid_for(ctx, n_reads, 256), 256, 0, check_offs_kernel, d_offs, n_reads, n_bases,
              flags.p + 1, ctx->d_status);
    if (n_chunks)
        MH_LAUNCH(ctx, "pack_chunks", grid_for(ctx, n_chunks, 256), 256, 0, pack_chunks_kernel, d_ascii, n_bases, vec,
                  packed.p, flags.p);
    uint64_t fl[1];
    read_u64(ctx, reinterpret_cast<const uint64_t*>(flags.p), fl, 1);
    const bool any_invalid = (fl[0] & 0xFFFFFFFFull) != 0, any_empty = (fl[0] >> 32) != 0;
    if (!any_invalid && !any_empty) {
        Buf<uint64_t> fo(ctx, n_reads + 1);
        MH_CUDA(cudaMemcpyAsync(fo.p, d_offs, sizeof(uint64_t) * (n_reads + 1), cudaMemcpyDeviceToDevice,
                                ctx->stream));
        Buf<uint32_t> fr(ctx, n_reads);
        if (n_reads) MH_LAUNCH(ctx, "iota", grid_for(ctx, n_reads, 256), 256, 0, iota_u32_kernel, fr.p, n_reads);
        out->n_frags = n_reads;
        out->n_packed = n_bases;
        out->packed = packed.release();
        out->frag_offs = fo.release();
        out->frag_read = fr.release();
        return;
    }
    // compaction of valid bases and fragment discovery
    Buf<uint32_t> mask(ctx, n_chunks), cnt(ctx, n_chunks), fcnt(ctx, n_chunks);
    Buf<uint64_t> dst(ctx, n_chunks + 1), fidx(ctx, n_chunks + 1);
    Buf<uint32_t> rs(ctx, ceil_div(n_bases, 32) + 1);
    rs.zero();
    MH_LAUNCH(ctx, "chunk_masks", grid_for(ctx, n_chunks, 256), 256, 0, chunk_masks_kernel, d_ascii, n_bases, vec,
              mask.p, cnt.p);
    exclusive_scan_u32(ctx, cnt.p, dst.p, n_chunks);
    if (n_reads)
        MH_LAUNCH(ctx, "read_starts", grid_for(ctx, n_reads, 256), 256, 0, read_starts_kernel, d_offs, n_reads, rs.p);
    MH_LAUNCH(ctx, "frag_count", grid_for(ctx, n_chunks, 256), 256, 0, frag_count_kernel, mask.p, rs.p, n_chunks,
              fcnt.p);
    exclusive_scan_u32(ctx, fcnt.p, fidx.p, n_chunks);
    uint64_t tot[2];
    read_u64(ctx, dst.p + n_chunks, &tot[0], 1);
    read_u64(ctx, fidx.p + n_chunks, &tot[1], 1);
    const uint64_t n_packed = tot[0], n_frags = tot[1];
    Buf<uint64_t> fo(ctx, n_frags + 1);
    Buf<uint32_t> fr(ctx, n_frags);
    Buf<uint32_t> cp(ctx, ceil_div(n_packed, 16) + kPackPad);
    cp.zero();
    MH_LAUNCH(ctx, "frag_write", grid_for(ctx, n_chunks, 256), 256, 0, frag_write_kernel, mask.p, rs.p, dst.p, fidx.p,
              d_offs, n_reads, n_chunks, fo.p, fr.p);
    MH_CUDA(cudaMemcpyAsync(fo.p + n_frags, dst.p + n_chunks, sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    MH_LAUNCH(ctx, "compact_pack", grid_for(ctx, n_chunks, 256), 256, 0, compact_pack_kernel, d_ascii, n_bases, vec,
              mask.p, dst.p, cp.p);
    sync_and_check(ctx);
    out->n_frags = n_frags;
    out->n_packed = n_packed;
    out->packed = cp.release();
    out->frag_offs = fo.release();
    out->frag_read = fr.release();
}

// Reads in host memory (pinned for overlap): up to one piece (kPiece bytes)
// is uploaded on the context stream and packed as from the device.  Larger
// inputs stream through two device staging buffers of kPiece bytes on the
// context's copy stream while the context stream packs the piece before
// (piece starts are multiples of 16 bases, so every piece fills whole
// packed words of its own); only the packed stream and the offsets stay on
// the device.  If some byte is not a base or some read is empty, the
// fragments must be found and the bases compacted: the ASCII is then
// uploaded whole and packed as from the device.
constexpr uint64_t kPiece = 256ull << 20;

// staging piece in bytes: kPiece, or MH_PACK_PIECE (a multiple of 16; tests)
static uint64_t piece_bytes() {
    static const uint64_t v = [] {
        const char* e = std::getenv("MH_PACK_PIECE");
        const long long x = e ? std::atoll(e) : 0;
        return x >= 16 ? (uint64_t)x / 16 * 16 : kPiece;
    }();
    return v;
}

static cudaStream_t copy_stream(mh_ctx* ctx) {
    if (!ctx->copy_stream) MH_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    return ctx->copy_stream;
}

void pack_reads_host(mh_ctx* ctx, const uint8_t* h_ascii, uint64_t n_bases, const uint64_t* h_offs, uint64_t n_reads,
                     mh_reads* out) {
    if (n_bases <= piece_bytes()) {
        // one piece: a plain upload on the context stream, then the device path
        Buf<uint8_t> da(ctx, n_bases + 16);
        Buf<uint64_t> doff(ctx, n_reads + 1);
        if (n_bases) MH_CUDA(cudaMemcpyAsync(da.p, h_ascii, n_bases, cudaMemcpyHostToDevice, ctx->stream));
        MH_CUDA(cudaMemcpyAsync(doff.p, h_offs, sizeof(uint64_t) * (n_reads + 1), cudaMemcpyHostToDevice,
                                ctx->stream));
        pack_reads(ctx, da.p, n_bases, doff.p, n_reads, out);
        return;
    }
    cudaStream_t cs = copy_stream(ctx);
    const uint64_t n_chunks = ceil_div(n_bases, 16);
    const uint64_t piece = piece_bytes();
    const uint64_t n_pieces = ceil_div(n_bases, piece);
    Buf<uint64_t> doff(ctx, n_reads + 1);
    Buf<uint32_t> flags(ctx, 2);  // [0] any invalid byte, [1] any empty read
    flags.zero();
    Buf<uint32_t> packed(ctx, n_chunks + kPackPad);
    MH_CUDA(cudaMemsetAsync(packed.p + n_chunks, 0, kPackPad * sizeof(uint32_t), ctx->stream));
    Buf<uint8_t> stage[2] = {Buf<uint8_t>(ctx, piece), Buf<uint8_t>(ctx, piece)};
    cudaEvent_t* ev = ctx->pack_ev;  // created once a context
    for (int i = 0; i < 5; i++)
        if (!ev[i]) MH_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    {
        // the copy stream writes buffers just allocated on the context stream
        MH_CUDA(cudaEventRecord(ev[4], ctx->stream));
        MH_CUDA(cudaStreamWaitEvent(cs, ev[4], 0));
        MH_CUDA(cudaMemcpyAsync(doff.p, h_offs, sizeof(uint64_t) * (n_reads + 1), cudaMemcpyHostToDevice, cs));
        MH_CUDA(cudaEventRecord(ev[4], cs));
        MH_CUDA(cudaStreamWaitEvent(ctx->stream, ev[4], 0));
        MH_LAUNCH(ctx, "check_offs", grid_for(ctx, n_reads, 256), 256, 0, check_offs_kernel, doff.p, n_reads,
                  n_bases, flags.p + 1, ctx->d_status);
        for (uint64_t q = 0; q < n_pieces; q++) {
            const int s = (int)(q & 1);
            const uint64_t b = q * piece, len = n_bases - b < piece ? n_bases - b : piece;
            if (q >= 2) MH_CUDA(cudaStreamWaitEvent(cs, ev[2 + s], 0));  // piece q-2 packed
            MH_CUDA(cudaMemcpyAsync(stage[s].p, h_ascii + b, len, cudaMemcpyHostToDevice, cs));
            MH_CUDA(cudaEventRecord(ev[s], cs));
            MH_CUDA(cudaStreamWaitEvent(ctx->stream, ev[s], 0));
            MH_LAUNCH(ctx, "pack_chunks", grid_for(ctx, ceil_div(len, 16), 256), 256, 0, pack_chunks_kernel,
                      stage[s].p, len, true, packed.p + b / 16, flags.p);
            MH_CUDA(cudaEventRecord(ev[2 + s], ctx->stream));
        }
    }
    stage[0].reset();
    stage[1].reset();
    uint64_t fl[1];
    read_u64(ctx, reinterpret_cast<const uint64_t*>(flags.p), fl, 1);
    if ((fl[0] & 0xFFFFFFFFull) == 0 && (fl[0] >> 32) == 0) {
        Buf<uint32_t> fr(ctx, n_reads);
        if (n_reads) MH_LAUNCH(ctx, "iota", grid_for(ctx, n_reads, 256), 256, 0, iota_u32_kernel, fr.p, n_reads);
        out->n_reads = n_reads;
        out->n_bases = n_bases;
        out->n_frags = n_reads;
        out->n_packed = n_bases;
        out->packed = packed.release();
        out->frag_offs = doff.release();
        out->frag_read = fr.release();
        return;
    }
    packed.reset();
    Buf<uint8_t> da(ctx, n_bases + 16);
    if (n_bases) MH_CUDA(cudaMemcpyAsync(da.p, h_ascii, n_bases, cudaMemcpyHostToDevice, ctx->stream));
    pack_reads(ctx, da.p, n_bases, doff.p, n_reads, out);
}

}  // namespace mh
