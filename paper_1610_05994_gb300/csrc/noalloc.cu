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
// on the first call made with that device current).  The cache is kept for
// the life of the process: after cudaDeviceReset the device image, and with
// it the array, is loaded anew, so a process that resets a device must not
// call this entry point on it again.
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
// abi.cu: the argument rules every build shares (width, sigma, S present
// and naturally aligned, n below 2^56).
wt_status check_symbol_args(const void *S, uint64_t n, uint64_t sigma, int width);
}

namespace {

// Whether p is device memory of device dev (or managed memory).
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" wt_status wt_node_starts_noalloc(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t *Hex,
                                            void *stream) {
    using namespace wt;
    // The same rules as every build (so a misaligned S is refused here, on
    // the host, before any launch), plus this entry point's own limit.
    const wt_status ar = check_symbol_args(S, n, sigma, sym_width);
    if (ar != WT_OK) return record_status(ar);
    if (sigma > kNoAllocMaxSigma || !Hex) return record_status(WT_ERR_ARG);
    // S and Hex must live on the current device: the scratch used is the
    // current device's copy of the array.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return record_status(WT_ERR_CUDA);
    }
    if ((n > 0 && !on_device(S, dev)) || !on_device(Hex, dev)) return record_status(WT_ERR_ARG);
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
