// selftest.cu -- wt_wait_selftest: runs the library's bounded device wait on
// an mbarrier that nothing completes, so a test can check that a wait which
// runs out becomes WT_ERR_TIMEOUT on the host while the CUDA context stays
// usable.  No bulk copy is ever in flight on the barrier, nothing traps, and
// the wait ends after the caller's limit (at most one second).
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {
wt_status record_status(wt_status s);  // abi.cu: sets the calling thread's last status
}

namespace {

constexpr uint64_t kSelftestMaxNs = 1000000000ull;

// One thread: initialise a barrier for one arrival; with arrive, arrive on it
// (the wait completes at once); wait with the given limit; a give-up sets
// kErrTimeout in *err.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int arrive, uint32_t *err) {
    __shared__ uint64_t bar;
    wt::mbar_init(&bar, 1);
    wt::fence_mbar_init();
    if (arrive) wt::mbar_arrive(&bar);
    if (!wt::mbar_wait_for(&bar, 0u, limit_ns)) atomicOr(err, wt::kErrTimeout);
}

}  // namespace

extern "C" wt_status wt_wait_selftest(uint64_t limit_ns, int arrive, uint32_t *err_word, void *stream) {
    using namespace wt;
    if (limit_ns == 0 || limit_ns > kSelftestMaxNs || !err_word) return record_status(WT_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t herr = 0;
    wt_status r = WT_OK;
    if (cudaMemsetAsync(err_word, 0, sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return record_status(WT_ERR_CUDA);
    }
    wait_selftest_kernel<<<1, 1, 0, st>>>(limit_ns, arrive, err_word);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&herr, err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK && (herr & kErrTimeout)) r = WT_ERR_TIMEOUT;
    return record_status(r);
}
