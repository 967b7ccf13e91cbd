// remap.cu -- alphabet remapping on the device (Section 3: when the codes
// of Sigma are not contiguous, a bitmap remaps the sequence to a contiguous
// alphabet).
//
// Over the code universe [0, U) the alphabet bitmap A has bit c set exactly
// when c occurs in S; the tree is then built over S'[j] = rank1(A, S[j]),
// codes in [0, sigma') with sigma' = the ones of A.  A is laid out like a
// level bitmap, so the level step's count and scan give it the same rank
// directory and select samples (R, Hy, S1, S0), and queries map codes with
// rank1 and select1 on it (query.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

namespace {

constexpr int kRemapThreads = 256;

// Marks every code of S in A (zeroed); flags codes >= universe.  A word is
// read before the atomic: a code already marked (most of them in a long
// sequence) costs a cached load, not an atomic.
template <typename Sym>
__global__ void __launch_bounds__(kRemapThreads) alpha_mark_kernel(const Sym *__restrict__ S, uint64_t n,
                                                                   uint64_t universe, uint32_t *__restrict__ A,
                                                                   uint32_t *__restrict__ err) {
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint64_t c = S[j];
        if (c >= universe) {
            bad = true;
            continue;
        }
        const uint32_t bit = 1u << (c & 31);
        uint32_t *w = A + (c >> 5);
        if (!(*reinterpret_cast<volatile uint32_t *>(w) & bit)) atomicOr(w, bit);
    }
    if (bad) atomicOr(err, kErrSymbol);
}

// S'[j] = rank1(A, S[j]), written with width OutSym.
template <typename Sym, typename OutSym>
__global__ void __launch_bounds__(kRemapThreads) alpha_map_kernel(const Sym *__restrict__ S, uint64_t n, LevelDesc A,
                                                                  OutSym *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += stride)
        out[j] = (OutSym)rank1(A, (uint64_t)S[j]);
}

unsigned remap_grid(uint64_t n) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const uint64_t want = ceil_div(n ? n : 1, (uint64_t)kRemapThreads * 8);
    const uint64_t cap = (uint64_t)sms * 8;
    return (unsigned)(want < cap ? want : cap);
}

template <typename Sym>
cudaError_t map_t(const void *S, uint64_t n, const LevelDesc &A, void *out, int out_width, cudaStream_t st) {
    const Sym *s = static_cast<const Sym *>(S);
    switch (out_width) {
        case 1: alpha_map_kernel<Sym, uint8_t><<<remap_grid(n), kRemapThreads, 0, st>>>(s, n, A, static_cast<uint8_t *>(out)); break;
        case 2: alpha_map_kernel<Sym, uint16_t><<<remap_grid(n), kRemapThreads, 0, st>>>(s, n, A, static_cast<uint16_t *>(out)); break;
        case 4: alpha_map_kernel<Sym, uint32_t><<<remap_grid(n), kRemapThreads, 0, st>>>(s, n, A, static_cast<uint32_t *>(out)); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_alpha_mark(const void *S, uint64_t n, int width, uint64_t universe, uint32_t *A, uint32_t *err,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    switch (width) {
        case 1: alpha_mark_kernel<uint8_t><<<remap_grid(n), kRemapThreads, 0, st>>>(static_cast<const uint8_t *>(S), n, universe, A, err); break;
        case 2: alpha_mark_kernel<uint16_t><<<remap_grid(n), kRemapThreads, 0, st>>>(static_cast<const uint16_t *>(S), n, universe, A, err); break;
        case 4: alpha_mark_kernel<uint32_t><<<remap_grid(n), kRemapThreads, 0, st>>>(static_cast<const uint32_t *>(S), n, universe, A, err); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_alpha_map(const void *S, uint64_t n, int width, const LevelDesc &A, void *out, int out_width,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    switch (width) {
        case 1: return map_t<uint8_t>(S, n, A, out, out_width, st);
        case 2: return map_t<uint16_t>(S, n, A, out, out_width, st);
        case 4: return map_t<uint32_t>(S, n, A, out, out_width, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace wt
