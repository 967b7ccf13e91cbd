// query.cu -- kernel (e): access, rank and select on the level bitmaps.
//
// The pointerless tree is walked top-down with rank on each level's bitmap
// (Section 2.2: the per-node walk of Fig. 2a simulated on the one-pointer-
// per-level layout of Fig. 2b, as in Claude and Navarro 2008).  On level l
// the current node is the range [b, e) of B_l; with z zeros in it,
//   a 0 bit maps p to b + rank0(p) - rank0(b) and the node to [b, b + z),
//   a 1 bit maps p to b + z + rank1(p) - rank1(b) and the node to [b + z, e).
// select walks down the same way, then climbs back with select on each level.
// One thread per query; every query touches O(L) 64-byte blocks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kQueryThreads = 256;

// One level step of the walk: returns the new p and narrows [b, e).
__device__ __forceinline__ void descend(const LevelDesc &d, uint32_t bit, uint64_t &b, uint64_t &e, uint64_t &p) {
    const uint64_t rb = rank1(d, b), re = rank1(d, e), rp = rank1(d, p);
    const uint64_t z = (e - re) - (b - rb);
    if (bit == 0) {
        p = b + (p - rp) - (b - rb);
        e = b + z;
    } else {
        p = b + z + (rp - rb);
        b = b + z;
    }
}

__device__ uint32_t do_access(const TreeDesc &t, uint64_t i) {
    if (i >= t.n) return UINT32_MAX;
    uint64_t b = 0, e = t.n, p = i;
    uint32_t sym = 0;
    for (uint32_t l = 0; l < t.L; l++) {
        const uint32_t bit = bit_at(t.lv[l], p);
        descend(t.lv[l], bit, b, e, p);
        sym = (sym << 1) | bit;
    }
    return sym;
}

__device__ uint64_t do_rank(const TreeDesc &t, uint32_t c, uint64_t i) {
    if ((uint64_t)c >= t.sigma || i > t.n) return UINT64_MAX;
    uint64_t b = 0, e = t.n, p = i;
    for (uint32_t l = 0; l < t.L; l++) descend(t.lv[l], (c >> (t.L - 1 - l)) & 1u, b, e, p);
    return p - b;
}

__device__ uint64_t do_select(const TreeDesc &t, uint32_t c, uint64_t j) {
    if ((uint64_t)c >= t.sigma || j == 0) return UINT64_MAX;
    uint64_t bs[WT_MAX_LEVELS + 1];
    uint64_t b = 0, e = t.n;
    for (uint32_t l = 0; l < t.L; l++) {
        const LevelDesc &d = t.lv[l];
        bs[l] = b;
        const uint64_t rb = rank1(d, b), re = rank1(d, e);
        const uint64_t z = (e - re) - (b - rb);
        if (((c >> (t.L - 1 - l)) & 1u) == 0)
            e = b + z;
        else
            b = b + z;
    }
    bs[t.L] = b;
    if (j > e - b) return UINT64_MAX;
    uint64_t pos = b + j - 1;
    for (uint32_t l = t.L; l-- > 0;) {
        const LevelDesc &d = t.lv[l];
        const uint32_t bit = (c >> (t.L - 1 - l)) & 1u;
        const uint64_t rb = bit ? rank1(d, bs[l]) : bs[l] - rank1(d, bs[l]);
        pos = select_bit(d, t.n, t.nblocks, bit, rb + (pos - bs[l + 1]) + 1);
    }
    return pos;
}

__global__ void __launch_bounds__(kQueryThreads) access_kernel(const TreeDesc *__restrict__ t,
                                                               const uint64_t *__restrict__ I, uint64_t m,
                                                               uint32_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = do_access(*t, I[q]);
}

__global__ void __launch_bounds__(kQueryThreads) rank_kernel(const TreeDesc *__restrict__ t,
                                                             const uint32_t *__restrict__ C,
                                                             const uint64_t *__restrict__ I, uint64_t m,
                                                             uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = do_rank(*t, C[q], I[q]);
}

__global__ void __launch_bounds__(kQueryThreads) select_kernel(const TreeDesc *__restrict__ t,
                                                               const uint32_t *__restrict__ C,
                                                               const uint64_t *__restrict__ J, uint64_t m,
                                                               uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q < m) out[q] = do_select(*t, C[q], J[q]);
}

__global__ void __launch_bounds__(kQueryThreads) multi_kernel(const TreeDesc *const *__restrict__ trees,
                                                              const uint32_t *__restrict__ tidx,
                                                              const uint8_t *__restrict__ op,
                                                              const uint32_t *__restrict__ C,
                                                              const uint64_t *__restrict__ A, uint64_t m,
                                                              uint32_t ntrees, uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const uint32_t ti = tidx[q];
    if (ti >= ntrees) {  // a tree index outside the table: the sentinel, no read
        out[q] = UINT64_MAX;
        return;
    }
    const TreeDesc &t = *trees[ti];
    uint64_t r;
    switch (op[q]) {
        case WT_OP_ACCESS: {
            const uint32_t s = do_access(t, A[q]);
            r = s == UINT32_MAX ? UINT64_MAX : s;
            break;
        }
        case WT_OP_RANK: r = do_rank(t, C[q], A[q]); break;
        case WT_OP_SELECT: r = do_select(t, C[q], A[q]); break;
        default: r = UINT64_MAX;
    }
    out[q] = r;
}

static unsigned grid_for(uint64_t m) { return (unsigned)ceil_div(m, kQueryThreads); }

cudaError_t launch_access(const TreeDesc *t, const uint64_t *i, uint64_t m, uint32_t *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    access_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, i, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rank(const TreeDesc *t, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                        cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    rank_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, c, i, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_select(const TreeDesc *t, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                          cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    select_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, c, j, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_query_multi(const TreeDesc *const *trees, uint32_t ntrees, const uint32_t *tree_idx,
                               const uint8_t *op,
                               const uint32_t *c, const uint64_t *arg, uint64_t m, uint64_t *out,
                               cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    multi_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(trees, tree_idx, op, c, arg, m, ntrees, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace wt

namespace wt {

// ------------------------------------------------ remapped alphabets
// A tree built over the remapped codes (remap.cu): the alphabet bitmap A
// over the universe [0, U) marks the codes that occur; code c is tree symbol
// rank1(A, c).  access maps the tree's answer r back to select1(A, r + 1);
// rank and select map c to rank1(A, c) when A[c] = 1.  A code < U that does
// not occur has rank 0 (for i <= n) and no select; a code >= U gives the
// sentinel.

__device__ __forceinline__ bool alpha_has(const LevelDesc &A, uint64_t universe, uint64_t c) {
    return c < universe && bit_at(A, c);
}

__global__ void __launch_bounds__(kQueryThreads) access_remap_kernel(const TreeDesc *__restrict__ t, LevelDesc A,
                                                                     uint64_t universe, uint64_t ablocks,
                                                                     const uint64_t *__restrict__ I, uint64_t m,
                                                                     uint32_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const uint32_t r = do_access(*t, I[q]);
    out[q] = r == UINT32_MAX ? UINT32_MAX : (uint32_t)select_bit(A, universe, ablocks, 1u, (uint64_t)r + 1);
}

__global__ void __launch_bounds__(kQueryThreads) rank_remap_kernel(const TreeDesc *__restrict__ t, LevelDesc A,
                                                                   uint64_t universe, const uint32_t *__restrict__ C,
                                                                   const uint64_t *__restrict__ I, uint64_t m,
                                                                   uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const uint64_t c = C[q], i = I[q];
    uint64_t r;
    if (c >= universe || i > t->n)
        r = UINT64_MAX;
    else if (!bit_at(A, c))
        r = 0;
    else
        r = do_rank(*t, (uint32_t)rank1(A, c), i);
    out[q] = r;
}

__global__ void __launch_bounds__(kQueryThreads) select_remap_kernel(const TreeDesc *__restrict__ t, LevelDesc A,
                                                                     uint64_t universe,
                                                                     const uint32_t *__restrict__ C,
                                                                     const uint64_t *__restrict__ J, uint64_t m,
                                                                     uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const uint64_t c = C[q];
    out[q] = alpha_has(A, universe, c) ? do_select(*t, (uint32_t)rank1(A, c), J[q]) : UINT64_MAX;
}

cudaError_t launch_access_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint64_t *i,
                                uint64_t m, uint32_t *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    access_remap_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, A, universe, ceil_div(universe, kBlockBits), i, m,
                                                                out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rank_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint32_t *c,
                              const uint64_t *i, uint64_t m, uint64_t *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    rank_remap_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, A, universe, c, i, m, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_select_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint32_t *c,
                                const uint64_t *j, uint64_t m, uint64_t *out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    select_remap_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(t, A, universe, c, j, m, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace wt
