// matrix.cu -- the wavelet matrix: the level-wise variant the paper names
// for future work (Section 5), as defined by Claude and Navarro (2012).
//
// Level l holds bit L-1-l of every symbol of S_l (S_0 = S), and S_{l+1} is
// all of S_l stably partitioned by that bit, zeros first; Z_l is the number
// of zeros of level l.  This is the tree's level step with one node per
// level: a zero at position p goes to zeros_before(p) and a one to
// Z_l + ones_before(p).  The level step places bit 0 at zeros_before(p) +
// OB_l[v] and bit 1 at ones_before(p) + ZE_l[v] for the symbol's top-l-bit
// key v, so the matrix is built by the same count, scan and pass kernels
// with node tables OB_l[v] = 0 and ZE_l[v] = Z_l for every v (S_l is
// ordered by the bit-reversed top l bits, so each key v is one run of S_l
// and the pass's one-run path applies as on the tree).  Those tables
// come from the leaf starts Hex: the codes whose bit L-1-l is zero form
// 2^l runs of 2^(L-1-l) codes, and Z_l sums their counts.
//
// Queries walk the levels with rank alone (no node ranges): access maps p to
// rank0(p) or Z_l + rank1(p) by the bit it reads; rank_c maps both ends of
// [0, i) by the bits of c; select_c walks down to c's range at the bottom and
// climbs back with select0(pos + 1) or select1(pos - Z_l + 1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kMatrixThreads = 256;
constexpr int kTableThreads = 1024;

// One CTA per level l: Z_l = sum over k < 2^l of the count of the codes
// [k 2^(b+1), k 2^(b+1) + 2^b) with b = L-1-l, then OB_l[v] = 0 and
// ZE_l[v] = Z_l for v < 2^l (the tables of level l start at 2^l - 1).
__global__ void __launch_bounds__(kTableThreads) wm_tables_kernel(const uint64_t *__restrict__ hex, uint32_t L,
                                                                  uint64_t *__restrict__ ob,
                                                                  uint64_t *__restrict__ ze) {
    __shared__ uint64_t part[kTableThreads / 32];
    const uint32_t l = blockIdx.x;
    const uint32_t b = L - 1 - l;
    const uint64_t runs = 1ull << l;
    uint64_t z = 0;
    for (uint64_t k = threadIdx.x; k < runs; k += blockDim.x) {
        const uint64_t c0 = k << (b + 1);
        z += hex[c0 + (1ull << b)] - hex[c0];
    }
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = z;
    __syncthreads();
    if (threadIdx.x < 32) {
        z = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (threadIdx.x == 0) part[0] = z;
    }
    __syncthreads();
    z = part[0];
    uint64_t *o = ob + (runs - 1), *e = ze + (runs - 1);
    for (uint64_t v = threadIdx.x; v < runs; v += blockDim.x) {
        o[v] = 0;
        e[v] = z;
    }
}

__device__ __forceinline__ uint64_t wm_zeros(const TreeDesc &t, uint32_t l) { return t.n - t.lv[l].ones; }

__device__ uint32_t wm_access(const TreeDesc &t, uint64_t i) {
    if (i >= t.n) return UINT32_MAX;
    uint64_t p = i;
    uint32_t sym = 0;
    for (uint32_t l = 0; l < t.L; l++) {
        const LevelDesc &d = t.lv[l];
        const uint32_t bit = bit_at(d, p);
        const uint64_t r1 = rank1(d, p);
        p = bit ? wm_zeros(t, l) + r1 : p - r1;
        sym = (sym << 1) | bit;
    }
    return sym;
}

// c's range on the bottom level of the symbols of [b, e) on level 0.
__device__ __forceinline__ void wm_descend(const TreeDesc &t, uint32_t c, uint64_t &b, uint64_t &e) {
    for (uint32_t l = 0; l < t.L; l++) {
        const LevelDesc &d = t.lv[l];
        const uint64_t rb = rank1(d, b), re = rank1(d, e);
        if ((c >> (t.L - 1 - l)) & 1u) {
            const uint64_t z = wm_zeros(t, l);
            b = z + rb;
            e = z + re;
        } else {
            b -= rb;
            e -= re;
        }
    }
}

__device__ uint64_t wm_rank(const TreeDesc &t, uint32_t c, uint64_t i) {
    if ((uint64_t)c >= t.sigma || i > t.n) return UINT64_MAX;
    uint64_t b = 0, e = i;
    wm_descend(t, c, b, e);
    return e - b;
}

__device__ uint64_t wm_select(const TreeDesc &t, uint32_t c, uint64_t j) {
    if ((uint64_t)c >= t.sigma || j == 0) return UINT64_MAX;
    uint64_t b = 0, e = t.n;
    wm_descend(t, c, b, e);
    if (j > e - b) return UINT64_MAX;
    uint64_t pos = b + j - 1;
    for (uint32_t l = t.L; l-- > 0;) {
        const LevelDesc &d = t.lv[l];
        if ((c >> (t.L - 1 - l)) & 1u)
            pos = select_bit(d, t.n, t.nblocks, 1u, pos - wm_zeros(t, l) + 1);
        else
            pos = select_bit(d, t.n, t.nblocks, 0u, pos + 1);
    }
    return pos;
}

__global__ void __launch_bounds__(kMatrixThreads) wm_access_kernel(const TreeDesc *__restrict__ t,
                                                                   const uint64_t *__restrict__ I, uint64_t m,
                                                                   uint32_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = wm_access(*t, I[q]);
}

__global__ void __launch_bounds__(kMatrixThreads) wm_rank_kernel(const TreeDesc *__restrict__ t,
                                                                 const uint32_t *__restrict__ C,
                                                                 const uint64_t *__restrict__ I, uint64_t m,
                                                                 uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = wm_rank(*t, C[q], I[q]);
}

__global__ void __launch_bounds__(kMatrixThreads) wm_select_kernel(const TreeDesc *__restrict__ t,
                                                                   const uint32_t *__restrict__ C,
                                                                   const uint64_t *__restrict__ J, uint64_t m,
                                                                   uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = wm_select(*t, C[q], J[q]);
}

cudaError_t launch_wm_tables(const uint64_t *hex, uint32_t L, uint64_t *ob, uint64_t *ze, cudaStream_t st) {
    if (L == 0) return cudaSuccess;
    wm_tables_kernel<<<L, kTableThreads, 0, st>>>(hex, L, ob, ze);
    note_launches(1);
    return cudaGetLastError();
}

static unsigned query_blocks(uint64_t m) { return (unsigned)ceil_div(m, kMatrixThreads); }

cudaError_t launch_wm_access(const TreeDesc *t, const uint64_t *i, uint64_t m, uint32_t *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    wm_access_kernel<<<query_blocks(m), kMatrixThreads, 0, st>>>(t, i, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_wm_rank(const TreeDesc *t, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                           cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    wm_rank_kernel<<<query_blocks(m), kMatrixThreads, 0, st>>>(t, c, i, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_wm_select(const TreeDesc *t, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                             cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    wm_select_kernel<<<query_blocks(m), kMatrixThreads, 0, st>>>(t, c, j, m, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace wt
