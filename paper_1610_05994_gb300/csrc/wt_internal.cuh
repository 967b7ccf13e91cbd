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

// Publishes a tile's own count: the inclusive prefix for tile 0, else the
// aggregate.  One lane.
__device__ __forceinline__ void publish_aggregate(uint64_t *status, uint32_t tile, uint64_t agg) {
    st_relaxed(&status[tile], (tile == 0 ? kFlagInc : kFlagAgg) | agg);
}

// Decoupled look-back with a 128-tile window, for a tile whose aggregate is
// already published (publish_aggregate): each lane inspects four
// predecessors per round, so the chain of inclusive prefixes advances 128
// tiles per round trip to L2 instead of 32.  Returns the exclusive prefix and
// publishes the inclusive one; bounded like lookback_prefix.
__device__ __forceinline__ uint64_t lookback_published(uint64_t *status, uint32_t tile, uint64_t agg, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) return 0;
    uint64_t excl = 0;
    int64_t pos = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool gave_up = false;
    while (true) {
        uint64_t s[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t idx = pos - (4 * lane + j);
            s[j] = idx >= 0 ? ld_relaxed(&status[idx]) : kFlagInc;
        }
        while (true) {
            bool ready = true;
#pragma unroll
            for (int j = 0; j < 4; j++) ready &= (s[j] >> 62) != 0;
            if (__all_sync(0xffffffffu, ready)) break;
            // Give up after kMaxSpins polls, or at once when another CTA has
            // already given up (its tiles may never be published).
            if (++spins > kMaxSpins || ((spins & 255u) == 0 && (*(volatile uint32_t *)err & kErrTimeout))) {
                gave_up = true;
                break;
            }
            __nanosleep(32);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t idx = pos - (4 * lane + j);
                if ((s[j] >> 62) == 0) s[j] = ld_relaxed(&status[idx]);
            }
        }
        if (gave_up) break;
        int jfirst = 4;
#pragma unroll
        for (int j = 3; j >= 0; j--)
            if ((s[j] >> 62) == 2) jfirst = j;
        const uint32_t inc_lanes = __ballot_sync(0xffffffffu, jfirst < 4);
        if (inc_lanes) {
            const int L = __ffs(inc_lanes) - 1;
            const int jl = __shfl_sync(0xffffffffu, jfirst, L);
            uint64_t v = 0;
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (lane < L || (lane == L && j <= jl)) v += s[j] & kValMask;
            excl += warp_sum_u64(v);
            break;
        }
        uint64_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) v += s[j] & kValMask;
        excl += warp_sum_u64(v);
        pos -= 128;
    }
    if (gave_up && lane == 0) atomicOr(err, kErrTimeout);
    if (lane == 0) st_relaxed(&status[tile], kFlagInc | (excl + agg));
    return excl;
}

// ------------------------------------------------------- TMA + mbarrier
// One-dimensional bulk copies global -> shared (cp.async.bulk) completing on
// an mbarrier.  Every wait is bounded by kMaxSpins polls.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory
// before later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arms the barrier for `bytes` of transaction and issues the copy (bytes and
// both addresses must be multiples of 16).
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Plain arrival (no transaction), for a phase with nothing to copy.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// A device-side wait gives up after this long (nanoseconds of %globaltimer).
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// Waits for the barrier phase with parity `phase`; false if it gave up
// (after kWaitLimitNs).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
    const uint32_t addr = smem_u32(bar);
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; i++) {
        if ((i & 1023u) == 1023u && global_ns() - t0 > kWaitLimitNs) return false;
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------ launchers
// (defined in build.cu / query.cu, called from abi.cu)

struct BuildScratch {
    uint64_t *hist;       // sigma
    uint64_t *hex;        // 2^L + 1
    uint64_t *ob;         // 2^L - 1 : ones before each node's start
    uint64_t *ze;         // 2^L - 1 : zeros up to each node's end
    uint64_t *scan_tmp;   // scan_tmp_bytes(L)
    void *job_slot;       // level_job_slot_bytes()
    uint64_t *status;     // L * ntiles look-back words
    uint32_t *tickets;    // L tile tickets
    void *ping;           // n * width
    void *pong;           // n * width
};

// Kernel (a): histogram of S into hist (zeroed by the caller) and the symbol
// range check; then the exclusive scan into hex.
cudaError_t launch_histogram(const void *S, uint64_t n, int width, uint64_t sigma, uint64_t *hist,
                             uint32_t *err, cudaStream_t st);
// Large alphabets with n < 2^32: hist_replicas(n, sigma) replicas (0 = use
// launch_histogram instead) of sigma u32 counters, zeroed by the caller.
uint32_t hist_replicas(uint64_t n, uint64_t sigma);
cudaError_t launch_histogram_replicated(const void *S, uint64_t n, int width, uint64_t sigma, uint32_t *rep,
                                        uint32_t R, uint32_t *err, cudaStream_t st);
cudaError_t launch_node_starts_replicated(const uint32_t *rep, uint32_t R, uint64_t sigma, uint32_t L,
                                          uint64_t *hex, cudaStream_t st, uint64_t *tmp);
// tmp (scan_tmp_bytes(L) bytes) lets large alphabets scan with many CTAs;
// with tmp == nullptr one CTA scans everything.
cudaError_t launch_node_starts(const uint64_t *hist, uint64_t sigma, uint32_t L, uint64_t n,
                               uint64_t *hex, cudaStream_t st, uint64_t *tmp = nullptr);
// Per-level node tables ob/ze from hex (tmp as above).
cudaError_t launch_node_tables(const uint64_t *hex, uint32_t L, uint64_t *ob, uint64_t *ze,
                               cudaStream_t st, uint64_t *tmp = nullptr);
size_t scan_tmp_bytes(uint32_t L);

// Kernels (b)+(c): one level pass (level.cu).  status/tickets must be
// zeroed.  job_slot: level_job_slot_bytes() of device memory.
uint32_t lw_tile_elems(int width);
size_t level_job_slot_bytes();
cudaError_t launch_level_pass(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l,
                              const uint64_t *ob, const uint64_t *ze, LevelDesc lv, uint64_t *ones_out,
                              uint64_t *status, uint32_t *ticket, uint32_t *err, void *job_slot, cudaStream_t st);
// A batch: one launch runs level l of many sequences of one width (level.cu).
// One sequence's share of a level launch (a batch launches many at once).
struct LevelJob {
    const void *cur;
    void *nxt;                 // nullptr on the sequence's last level
    uint64_t n, nblocks, nspans;
    uint32_t L;                // the sequence's number of levels
    uint32_t ntiles;           // its tiles at this width
    LevelDesc lv;              // its level-l arrays
    uint64_t *ones_out;
    const uint64_t *ob, *ze;   // its level-l node tables
    uint64_t *status;          // ntiles look-back words
};

LevelJob make_level_job(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l, const uint64_t *ob,
                        const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint64_t *status);
size_t level_job_bytes();
cudaError_t launch_level_jobs(int width, uint32_t l, const LevelJob *jobs, const uint32_t *tile_start, uint32_t njobs,
                              uint32_t total_tiles, uint32_t *ticket, uint32_t *err, cudaStream_t st);

// Kernel (d): dd-direct build of all levels for small sigma (dd.cu).
struct DdScratch {
    uint32_t *cnt;   // [tiles][sigma] per-tile leaf counts
    uint32_t *off;   // [tiles][sigma] symbols of earlier tiles per leaf
    uint32_t *csum;  // column-scan chunk sums
    uint64_t *H;     // leaf histogram
};
bool dd_supported(uint64_t n, uint64_t sigma, int width);
uint64_t dd_tiles(uint64_t n);
size_t dd_scratch_bytes(uint64_t n, uint64_t sigma);
DdScratch dd_carve(void *scratch, uint64_t n, uint64_t sigma);
cudaError_t launch_dd_count(const void *S, uint64_t n, uint64_t sigma, const DdScratch &d, uint32_t *err,
                            cudaStream_t st);
cudaError_t launch_dd_scan(uint64_t n, uint64_t sigma, const DdScratch &d, cudaStream_t st);
// The caller zeroes every level's bitmap words first (runs are OR-ed in).
cudaError_t launch_dd_write(const void *S, uint64_t n, uint64_t sigma, uint32_t L, const TreeDesc &h_desc,
                            TreeDesc *d_desc, const DdScratch &d, const uint64_t *hex, const uint64_t *ob,
                            uint32_t *err, cudaStream_t st);

// Batches (batch.cu): per-sequence parameters of the batched kernels (a), (a').
struct SeqJob {
    const void *S;
    uint64_t n, sigma;
    uint32_t L, width;
    uint64_t *hist;   // sigma u64, zeroed
    uint64_t *hex;    // 2^L + 1
    uint64_t *ob, *ze;  // 2^L each
    uint32_t *err;    // the tree's error word
};
uint32_t batch_hist_tiles(uint64_t n);
cudaError_t launch_batch_prepare(const SeqJob *jobs, uint32_t nseq, const uint32_t *hist_tile_start,
                                 uint32_t hist_tiles, const uint32_t *lvl_start, uint32_t total_levels,
                                 cudaStream_t st);

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
