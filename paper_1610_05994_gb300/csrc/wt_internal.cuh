// wt_internal.cuh -- shared device structures and helpers of the CUDA path.
//
// Terms (arXiv 1610.05994, Section 2.2, Section 3, Proposition 1):
//   L        = ceil(lg sigma) levels; level 0 is the root.
//   key_l(s) = s >> (L - l), the node of symbol s on level l (Proposition 1).
//   bit_l(s) = (s >> (L - 1 - l)) & 1, the bit stored for s on level l.
//   P_l      = the symbols in level-l order: S stably ordered by key_l.
//   Hex[c]   = number of symbols < c (exclusive scan of the leaf histogram);
//              node v of level l starts at Hex[v << (L - l)].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wt.h"

namespace wt {

constexpr uint32_t kBlockBits = 512;          // rank block (64 bytes of bitmap)
constexpr uint32_t kSample = 8192;            // select sample rate
constexpr int kSpanShift = 32;                // hyper span = 2^32 bits
constexpr uint32_t kBlocksPerSpanMask = (1u << (kSpanShift - 9)) - 1;

// Device error word bits (OR-ed by kernels, read by the host after a build).
constexpr uint32_t kErrSymbol = 1u;
constexpr uint32_t kErrTimeout = 2u;

// Bounded spin: a device-side wait gives up after this many polls (each poll
// sleeps ~0.1-1 us), sets kErrTimeout and lets the kernel finish.
constexpr uint32_t kMaxSpins = 1u << 22;

struct LevelDesc {
    uint32_t *words;  // ceil(n/512) * 16
    uint32_t *R;      // ceil(n/512) + 1
    uint64_t *Hy;     // ceil(n/2^32) + 1
    uint32_t *S1;     // up to ceil(n/8192) + 1
    uint32_t *S0;     // up to ceil(n/8192) + 1
    uint64_t ones;    // written by the build
};

// Device-resident descriptor of one tree (queries read it).
struct TreeDesc {
    uint64_t n;
    uint64_t sigma;
    uint64_t nblocks;
    uint32_t L;
    uint32_t width;
    LevelDesc lv[WT_MAX_LEVELS];
};

__host__ __device__ inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__host__ __device__ inline uint32_t levels_of(uint64_t sigma) {
    uint32_t L = 0;
    while (L < 63 && (1ull << L) < sigma) L++;
    return L;
}

// Relaxed 64-bit global accesses for the look-back status words (values only;
// no data is published through them).
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Decoupled look-back (Merrill and Garland, 2016) over per-tile counts.
// Status word: top two bits = flag (1 aggregate, 2 inclusive prefix), low 62
// bits = value.  Called by all 32 lanes of one warp; returns the exclusive
// prefix of tile `tile` and publishes its inclusive prefix.  Every wait is
// bounded: on give-up it ORs kErrTimeout into *err and returns what it has.
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t lookback_prefix(uint64_t *status, uint32_t tile, uint64_t agg,
                                                    uint32_t *err) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed(&status[0], kFlagInc | agg);
        return 0;
    }
    if (lane == 0) st_relaxed(&status[tile], kFlagAgg | agg);
    uint64_t excl = 0;
    int64_t pos = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool gave_up = false;
    while (true) {
        const int64_t idx = pos - lane;
        uint64_t s = (idx >= 0) ? ld_relaxed(&status[idx]) : kFlagInc;
        while (!__all_sync(0xffffffffu, (s >> 62) != 0)) {
            if (++spins > kMaxSpins) {
                gave_up = true;
                break;
            }
            __nanosleep(64);
            s = (idx >= 0) ? ld_relaxed(&status[idx]) : kFlagInc;
        }
        if (gave_up) break;
        const uint32_t inc_mask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        if (inc_mask) {
            const int first = __ffs(inc_mask) - 1;
            excl += warp_sum_u64(lane <= first ? (s & kValMask) : 0);
            break;
        }
        excl += warp_sum_u64(s & kValMask);
        pos -= 32;
    }
    if (gave_up && lane == 0) atomicOr(err, kErrTimeout);
    if (lane == 0) st_relaxed(&status[tile], kFlagInc | (excl + agg));
    return excl;
}

// ------------------------------------------------------------ launchers
// (defined in build.cu / query.cu, called from abi.cu)

struct BuildScratch {
    uint64_t *hist;       // sigma
    uint64_t *hex;        // 2^L + 1
    uint64_t *ob;         // 2^L - 1 : ones before each node's start
    uint64_t *ze;         // 2^L - 1 : zeros up to each node's end
    uint64_t *status;     // L * ntiles look-back words
    uint32_t *tickets;    // L tile tickets
    void *ping;           // n * width
    void *pong;           // n * width
};

// Kernel (a): histogram of S into hist (zeroed by the caller) and the symbol
// range check; then the exclusive scan into hex.
cudaError_t launch_histogram(const void *S, uint64_t n, int width, uint64_t sigma, uint64_t *hist,
                             uint32_t *err, cudaStream_t st);
cudaError_t launch_node_starts(const uint64_t *hist, uint64_t sigma, uint32_t L, uint64_t n,
                               uint64_t *hex, cudaStream_t st);
// Per-level node tables ob/ze from hex.
cudaError_t launch_node_tables(const uint64_t *hex, uint32_t L, uint64_t *ob, uint64_t *ze,
                               cudaStream_t st);

// Kernels (b)+(c): one level pass.  status/tickets must be zeroed.
uint32_t lw_tile_elems();
cudaError_t launch_level_pass(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l,
                              const uint64_t *ob, const uint64_t *ze, LevelDesc lv, uint64_t *ones_out,
                              uint64_t *status, uint32_t *ticket, uint32_t *err, cudaStream_t st);

// Kernel (d): dd-direct build of all levels for small sigma.
bool dd_supported(uint64_t sigma, int width);
size_t dd_scratch_bytes(uint64_t n, uint64_t sigma, int width);
cudaError_t launch_dd_build(const void *S, uint64_t n, int width, uint64_t sigma, uint32_t L,
                            const uint64_t *hex, TreeDesc *d_desc, const TreeDesc &h_desc, void *scratch,
                            uint32_t *err, cudaStream_t st);

// Kernel (e): queries.
cudaError_t launch_access(const TreeDesc *t, const uint64_t *i, uint64_t m, uint32_t *out, cudaStream_t st);
cudaError_t launch_rank(const TreeDesc *t, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                        cudaStream_t st);
cudaError_t launch_select(const TreeDesc *t, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                          cudaStream_t st);
cudaError_t launch_query_multi(const TreeDesc *const *trees, const uint32_t *tree_idx, const uint8_t *op,
                               const uint32_t *c, const uint64_t *arg, uint64_t m, uint64_t *out,
                               cudaStream_t st);

}  // namespace wt
