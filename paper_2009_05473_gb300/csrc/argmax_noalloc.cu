// sfw_argmax_noalloc: the arg-maximum / top-k of sfw_argmax for callers that
// must not allocate device memory.
//
// sfw_argmax keeps its key scratch in a buffer it allocates with cudaMalloc on
// first use (and re-allocates when a larger top-k needs more).  Some callers
// cannot let a library do that: applications whose device memory is entirely
// owned by another allocator (a framework's caching pool or a fixed budget
// that already reserved the GPU, so a foreign cudaMalloc fails or steals from
// it), and latency-critical loops in which the cudaFree of a re-allocation
// would synchronise the whole device.  This variant takes its scratch from one
// file-scope static __device__ array instead, so it never calls cudaMalloc,
// cudaFree or any allocating library routine.
//
// The array exists on every GPU that loads this library, from load until
// process exit.  Host code cannot use the array's name as a device address, so
// the first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call on a device
// before any stream capture.  Every call shares the array: two calls whose kernels overlap
// on the GPU (other streams, other host threads) race on it and may return
// wrong results, so order such calls.  The kernels write every scratch slot
// before they read it, so nothing needs clearing between calls.
#include <mutex>

#include "sfw_internal.cuh"

// 2^18 keys of 8 bytes = 2 MiB per device.
static constexpr long long kStaticScratchKeys = 1ll << 18;
static __device__ __align__(256) unsigned long long g_argmax_scratch[kStaticScratchKeys];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
unsigned long long* g_addr[kMaxDevices] = {};

// Device address of g_argmax_scratch on the current device (looked up once per device).
sfw_status static_scratch(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sfw::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return sfw::fail(SFW_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_argmax_scratch);
        if (e != cudaSuccess) return sfw::cuda_fail(e, "cudaGetSymbolAddress(argmax scratch)");
        g_addr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_addr[dev];
    return SFW_OK;
}

}  // namespace

extern "C" sfw_status sfw_argmax_noalloc(const float* values, int64_t count, int topk,
                                         float* val_out, int64_t* idx_out, void* stream) {
    using namespace sfw;
    clear_error();
    if (!values || !val_out || !idx_out) return fail(SFW_ERR_ARG, "pointers must be non-NULL");
    if (count < 1 || count >= 0xffffffffll) return fail(SFW_ERR_ARG, "count must be in [1, 2^32 - 2]");
    if (topk < 1 || topk > 64 || topk > count) return fail(SFW_ERR_ARG, "topk must be in [1, min(64, count)]");
    // top-1 uses at most 1024 keys; top-k needs ceil(count / 4096) * topk keys per half
    const long long blocks = (count + 4095) / 4096;
    if (topk > 1 && blocks * topk > kStaticScratchKeys / 2)
        return fail(SFW_ERR_SHAPE,
                    "count * topk too large for the static scratch: ceil(count/4096)*topk = %lld > %lld",
                    blocks * topk, kStaticScratchKeys / 2);
    unsigned long long* scratch = nullptr;
    SFW_TRY(static_scratch(&scratch));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (topk == 1) {
        int nb = (int)((count + 255) / 256);
        if (nb > 1024) nb = 1024;
        SFW_TRY(launch_argmax_keys(values, count, scratch, nb, st));
        return launch_argmax_final(scratch, nb, val_out, idx_out, st);
    }
    return launch_topk(values, count, topk, scratch, kStaticScratchKeys, val_out, idx_out, st);
}
