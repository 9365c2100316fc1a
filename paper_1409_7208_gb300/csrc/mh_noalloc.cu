// mh_sort_keys_noalloc: the library's LSD radix sort for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc, cudaFree or any allocating routine:
// code that runs inside a host that owns the whole device memory budget (an
// engine that hands out all memory from its own arena and forbids others to
// allocate), latency-critical loops that must never hit the driver's
// allocator, or code that may not synchronise the device the way cudaFree
// does.  This entry point needs nothing from them but their input and output
// buffers: its scratch space (the second buffer of the ping-pong passes, the
// look-back status words, the digit histogram and offsets, the tile counter
// and an error word) lives in one statically sized device array in this file.
//
// That array is a module global: every GPU that loads the library holds it
// (kScratchBytes, about 17 MiB) until the process exits, and every call on
// a device shares the same copy.  Each call clears the parts that must start
// at zero; calls that overlap on the GPU (on different streams, or from
// several threads without ordering) race on the array and must not be made.
//
// In host code the array's name only stands for the device object; its
// device address is looked up with cudaGetSymbolAddress, while that device
// is current, by the first call made on the device, and again only if the
// device's primary context has been torn down and recreated since (a context
// id is kept beside the address, so an address from a dead context is never
// reused).
#include <cuda.h>

#include <mutex>

#include "mh_sort_kernels.cuh"

namespace mh {
namespace {

constexpr uint64_t kMaxKeyWords = 1ull << 21;                  // n * nw limit: 16 MiB of keys
constexpr uint64_t kAltBytes = kMaxKeyWords * 8;               // ping-pong buffer
constexpr uint64_t kMaxTiles = 1ull << 10;                     // >= ceil(limit / tile) for every nw
constexpr uint64_t kStatusBytes = kMaxTiles * 256 * 4;         // look-back status
constexpr int kMaxPasses = 32;                                 // 256-bit keys, 8-bit digits
constexpr uint64_t kHistBytes = kMaxPasses * 256 * 4;
constexpr uint64_t kBaseBytes = kMaxPasses * 256 * 8;
constexpr uint64_t kMiscBytes = 256;                           // tile counter, error word
constexpr uint64_t kAltOff = 0;
constexpr uint64_t kStatusOff = kAltOff + kAltBytes;
constexpr uint64_t kHistOff = kStatusOff + kStatusBytes;
constexpr uint64_t kBaseOff = kHistOff + kHistBytes;
constexpr uint64_t kMiscOff = kBaseOff + kBaseBytes;
constexpr uint64_t kScratchBytes = kMiscOff + kMiscBytes;
static_assert(kMaxTiles * (uint64_t)sort_tile<4>() >= kMaxKeyWords / 4, "status too small for nw = 4");
static_assert(kMaxTiles * (uint64_t)sort_tile<2>() >= kMaxKeyWords / 2, "status too small for nw = 2");
static_assert(kMaxTiles * (uint64_t)sort_tile<1>() >= kMaxKeyWords, "status too small for nw = 1");

constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices];
static unsigned long long g_scratch_ctx[kMaxDevices];  // context id the address belongs to

// Id of the current context (unique for the process's lifetime, unlike the
// context handle), through the driver entry points cudart exposes; 0 if it
// cannot be had.
static unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up on
// the first call per device, and again whenever the device's context is not
// the one the cached address was taken in.
static int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MH_EDEVICE;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long ctx_id = current_context_id();  // 0 before the device's first runtime call
    if (!g_scratch_addr[dev] || ctx_id == 0 || g_scratch_ctx[dev] != ctx_id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the context current
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MH_EDEVICE;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_addr[dev];
    return MH_OK;
}

template <int NW>
static int sort_noalloc(const uint64_t* in, uint64_t* out, uint64_t n, int key_bits, cudaStream_t st,
                        unsigned char* scratch) {
    constexpr int TILE = sort_tile<NW>();
    uint64_t* alt = reinterpret_cast<uint64_t*>(scratch + kAltOff);
    uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kStatusOff);
    uint32_t* hist = reinterpret_cast<uint32_t*>(scratch + kHistOff);
    uint64_t* base = reinterpret_cast<uint64_t*>(scratch + kBaseOff);
    uint32_t* counter = reinterpret_cast<uint32_t*>(scratch + kMiscOff);
    uint32_t* err = counter + 1;
    const int n_passes = (key_bits + 7) / 8;
    const uint64_t tiles = ceil_div(n, TILE);
#define MH_TRY(call)                                    \
    do {                                                \
        if ((call) != cudaSuccess) {                    \
            cudaGetLastError();                         \
            return MH_EDEVICE;                          \
        }                                               \
    } while (0)
    // hist and the error word must start at zero; status and the tile
    // counter are cleared before every pass
    MH_TRY(cudaMemsetAsync(hist, 0, kHistBytes, st));
    MH_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
    int dev = 0, sms = 1;
    MH_TRY(cudaGetDevice(&dev));
    MH_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned hist_grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(n, 256), (uint64_t)sms * 4));
    radix_hist_kernel<NW><<<hist_grid, 256, sizeof(uint32_t) * n_passes * 256, st>>>(in, n, 0, n_passes, hist);
    MH_TRY(cudaGetLastError());
    radix_base_kernel<<<n_passes, 256, 0, st>>>(hist, base, 256);
    MH_TRY(cudaGetLastError());
    constexpr size_t smem = onesweep_smem<NW, false>();
    MH_TRY(cudaFuncSetAttribute(onesweep_kernel<NW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t* src = in;
    for (int p = 0; p < n_passes; p++) {
        // the last pass writes `out`; the ones before alternate so that it does
        uint64_t* dst = ((n_passes - 1 - p) % 2 == 0) ? out : alt;
        MH_TRY(cudaMemsetAsync(status, 0, tiles * 256 * sizeof(uint32_t), st));
        MH_TRY(cudaMemsetAsync(counter, 0, sizeof(uint32_t), st));
        onesweep_kernel<NW, false><<<(unsigned)tiles, kSortThreads, smem, st>>>(
            src, dst, nullptr, nullptr, n, 8 * p, base + (uint64_t)p * 256, nullptr, status, counter, err,
            kSpinLimit, 0, SegIn{});
        MH_TRY(cudaGetLastError());
        src = dst;
    }
    uint32_t h_err = 0;
    MH_TRY(cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    MH_TRY(cudaStreamSynchronize(st));
#undef MH_TRY
    return h_err ? MH_ETIMEOUT : MH_OK;
}

}  // namespace mh

extern "C" int mh_sort_keys_noalloc(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n, int nw, int key_bits,
                                    void* stream) {
    using namespace mh;
    if ((nw != 1 && nw != 2 && nw != 4) || key_bits < 1 || key_bits > 64 * nw) return MH_EINVAL;
    if (n > 0 && (!keys_in || !keys_out || keys_in == keys_out)) return MH_EINVAL;
    // keys move as 8-byte words (one word) or 16-byte vectors (two or four)
    const uintptr_t align = nw == 1 ? 7u : 15u;
    if (n > 0 && (((uintptr_t)keys_in | (uintptr_t)keys_out) & align)) return MH_EINVAL;
    if (n > kMaxKeyWords / (uint64_t)nw) return MH_EOVERFLOW;
    if (n == 0) return MH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 1) {
        if (cudaMemcpyAsync(keys_out, keys_in, 8 * (size_t)nw, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return MH_EDEVICE;
        }
        return MH_OK;
    }
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != MH_OK) return rc;
    unsigned char* s = static_cast<unsigned char*>(scratch);
    switch (nw) {
        case 1: return sort_noalloc<1>(keys_in, keys_out, n, key_bits, st, s);
        case 2: return sort_noalloc<2>(keys_in, keys_out, n, key_bits, st, s);
        default: return sort_noalloc<4>(keys_in, keys_out, n, key_bits, st, s);
    }
}
