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

__device__ __forceinline__ uint32_t bit_at(const LevelDesc &d, uint64_t p) {
    return (__ldg(d.words + (p >> 5)) >> (p & 31)) & 1u;
}

// Position of the r-th (1-based) set bit of x; x holds at least r set bits.
__device__ __forceinline__ uint32_t select_in_word(uint32_t x, uint32_t r) {
    for (uint32_t k = 1; k < r; k++) x &= x - 1;
    return __ffs(x) - 1;
}

// Position of the k-th (1-based) bit equal to `bit` on a level of n bits;
// 1 <= k <= count of such bits below n.  The select sample of k bounds the
// block from below, the next sample (if any) from above; a binary search on
// the block directory and a scan of the block's 16 words finish it.
__device__ uint64_t select_bit(const LevelDesc &d, uint64_t n, uint64_t nblocks, uint32_t bit, uint64_t k) {
    const uint32_t *samples = bit ? d.S1 : d.S0;
    const uint64_t count = bit ? d.ones : n - d.ones;
    const uint64_t s = (k - 1) / kSample;
    uint64_t lo = samples[s];
    uint64_t hi = nblocks - 1;
    if ((s + 1) * kSample < count) {
        const uint64_t nx = samples[s + 1];
        if (nx < hi) hi = nx;
    }
    // Largest block b in [lo, hi] with (bits equal to `bit` before b) < k.
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        const uint64_t ob = ones_before_block(d, mid);
        const uint64_t before = bit ? ob : (mid << 9) - ob;
        if (before < k)
            lo = mid;
        else
            hi = mid - 1;
    }
    const uint64_t ob = ones_before_block(d, lo);
    uint64_t need = k - (bit ? ob : (lo << 9) - ob);
    const uint32_t *w = d.words + lo * 16;
    for (uint32_t q = 0; q < 16; q++) {
        const uint32_t x = bit ? __ldg(w + q) : ~__ldg(w + q);
        const uint32_t c = __popc(x);
        if (need <= c) return (lo << 9) + q * 32 + select_in_word(x, (uint32_t)need);
        need -= c;
    }
    return UINT64_MAX;  // unreachable for valid k
}

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
                                                              uint64_t *__restrict__ out) {
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const TreeDesc &t = *trees[tidx[q]];
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

cudaError_t launch_query_multi(const TreeDesc *const *trees, const uint32_t *tree_idx, const uint8_t *op,
                               const uint32_t *c, const uint64_t *arg, uint64_t m, uint64_t *out,
                               cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    multi_kernel<<<grid_for(m), kQueryThreads, 0, st>>>(trees, tree_idx, op, c, arg, m, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace wt
