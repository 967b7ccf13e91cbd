// noalloc.cu -- wt_node_starts_noalloc: the node-starts stage (leaf histogram
// and exclusive scan) for callers that cannot allocate device memory.
//
// Some processes that use this library cannot call cudaMalloc (or any
// allocator) while they run: a server that hands the whole device to its own
// memory pool at start-up and forbids further device allocations, or a
// latency-critical loop that must not take the allocator's locks or the
// implicit device synchronisation a cudaFree may bring.  For them this entry
// point keeps its scratch -- the per-code counts and an error word -- in one
// fixed array compiled into the library's device image, so a call allocates
// nothing.  The price: that array exists on every GPU that loads the library
// (kNoAllocBytes, about 0.5 MB) until the process exits, the alphabet is
// limited to kNoAllocMaxSigma codes, and all calls share the one array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "wt_internal.cuh"

namespace {

constexpr uint64_t kNoAllocMaxSigma = 1ull << 16;  // largest alphabet this entry point accepts
constexpr size_t kNoAllocHistBytes = kNoAllocMaxSigma * sizeof(uint64_t);
constexpr size_t kNoAllocBytes = kNoAllocHistBytes + 256;  // counts, then the error word

// The scratch itself.  Host code must not pass this name to a kernel: on the
// host it only stands in for the symbol, so its device address is looked up
// once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_node_starts_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up and cached
// on the first call made with that device current).
cudaError_t scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_node_starts_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

}  // namespace

namespace wt {
wt_status record_status(wt_status s);  // abi.cu: sets the calling thread's last status
}

extern "C" wt_status wt_node_starts_noalloc(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t *Hex,
                                            void *stream) {
    using namespace wt;
    if (sym_width != 1 && sym_width != 2 && sym_width != 4) return record_status(WT_ERR_ARG);
    if (sigma == 0 || sigma > kNoAllocMaxSigma) return record_status(WT_ERR_ARG);
    if (sym_width < 4 && sigma > (1ull << (8 * sym_width))) return record_status(WT_ERR_ARG);
    if (!Hex || (n > 0 && S == nullptr) || n >= (1ull << 56)) return record_status(WT_ERR_ARG);
    if (n > 0) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, S) != cudaSuccess) {
            cudaGetLastError();
            return record_status(WT_ERR_ARG);
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return record_status(WT_ERR_ARG);
    }
    unsigned char *scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return record_status(WT_ERR_CUDA);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t *hist = reinterpret_cast<uint64_t *>(scratch);
    uint32_t *err = reinterpret_cast<uint32_t *>(scratch + kNoAllocHistBytes);
    const uint32_t L = levels_of(sigma);
    uint32_t herr = 0;
    wt_status r = WT_OK;
    // The previous call left its counts in the array: clear what this call reads.
    if (cudaMemsetAsync(hist, 0, sigma * sizeof(uint64_t), st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(uint32_t), st) != cudaSuccess ||
        launch_histogram(S, n, sym_width, sigma, hist, err, st) != cudaSuccess ||
        launch_node_starts(hist, sigma, L, n, Hex, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK && (herr & kErrSymbol)) r = WT_ERR_SYMBOL_RANGE;
    return record_status(r);
}
