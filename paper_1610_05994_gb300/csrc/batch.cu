// batch.cu -- kernels (a) and (a') for a batch of sequences in single
// launches: every CTA (or CTA group) finds its sequence in a prefix table,
// so thousands of sequences of different length, alphabet and width share
// one histogram launch, one node-starts launch and one node-tables launch.
// The level passes of a batch reuse level.cu's kernel with one job per
// sequence.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kBatchThreads = 512;
constexpr uint32_t kBatchHistTile = 16384;   // symbols per histogram CTA
constexpr uint32_t kBatchSmemBins = 8192;    // alphabets up to this use a shared-memory histogram

constexpr uint64_t kBatchSlab = 1ull << 20;   // symbols per packed-histogram CTA

static bool packed_class(uint64_t sigma) { return sigma > kBatchSmemBins && sigma <= kPackedMaxSigma; }
uint32_t batch_hist_tiles(uint64_t n, uint64_t sigma) {
    return packed_class(sigma) ? 0u : (uint32_t)ceil_div(n, kBatchHistTile);
}
uint32_t batch_hist_slabs(uint64_t n, uint64_t sigma) {
    return packed_class(sigma) ? (uint32_t)ceil_div(n, kBatchSlab) : 0u;
}

// Index of the largest start[k] <= x among k < count (start nondecreasing, start[0] = 0).
__device__ __forceinline__ uint32_t find_seq(const uint32_t *start, uint32_t count, uint32_t x) {
    uint32_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (start[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t load_sym(const void *S, int width, uint64_t j) {
    if (width == 1) return static_cast<const uint8_t *>(S)[j];
    if (width == 2) return static_cast<const uint16_t *>(S)[j];
    return static_cast<const uint32_t *>(S)[j];
}

// Zeroes every sequence's error word (they live in the trees' memory).
__global__ void batch_clear_err_kernel(const SeqJob *__restrict__ jobs, uint32_t nseq) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nseq) *jobs[k].err = 0;
}

// Leaf histogram of the sequences with small (or very large) alphabets:
// CTA b takes one tile of one sequence.
__global__ void __launch_bounds__(kBatchThreads) batch_hist_kernel(const SeqJob *__restrict__ jobs,
                                                                   const uint32_t *__restrict__ tile_start,
                                                                   uint32_t nseq) {
    __shared__ uint32_t bins[kBatchSmemBins];
    const uint32_t k = find_seq(tile_start, nseq, blockIdx.x);
    const SeqJob &J = jobs[k];
    const uint64_t base = (uint64_t)(blockIdx.x - tile_start[k]) * kBatchHistTile;
    if (base >= J.n) return;
    const uint32_t m = (uint32_t)((J.n - base) < kBatchHistTile ? (J.n - base) : kBatchHistTile);
    const bool shared_bins = J.sigma <= kBatchSmemBins;
    // Small alphabets: one private copy of the bins per warp (up to all
    // warps), so the warps of a CTA do not queue on the same few words.
    const uint32_t sig = (uint32_t)J.sigma;
    uint32_t copies = shared_bins ? kBatchSmemBins / sig : 1;
    if (copies > kBatchThreads / 32) copies = kBatchThreads / 32;
    uint32_t *mine = bins + ((threadIdx.x >> 5) % copies) * sig;
    if (shared_bins)
        for (uint32_t c = threadIdx.x; c < sig * copies; c += blockDim.x) bins[c] = 0;
    __syncthreads();
    bool bad = false;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
        const uint32_t s = load_sym(J.S, J.width, base + i);
        if ((uint64_t)s >= J.sigma)
            bad = true;
        else if (shared_bins)
            atomicAdd(&mine[s], 1u);
        else
            atomicAdd(reinterpret_cast<unsigned long long *>(&J.hist[s]), 1ull);
    }
    if (bad) atomicOr(J.err, kErrSymbol);
    if (shared_bins) {
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < sig; c += blockDim.x) {
            uint32_t sum = 0;
            for (uint32_t q = 0; q < copies; q++) sum += bins[q * sig + c];
            if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(&J.hist[c]), (unsigned long long)sum);
        }
    }
}

// Leaf histogram of the sequences with mid-size alphabets (packed 16-bit
// shared bins): CTA b takes one slab of kBatchSlab symbols of one sequence.
__global__ void __launch_bounds__(kPackedThreads) batch_hist_packed_kernel(const SeqJob *__restrict__ jobs,
                                                                          const uint32_t *__restrict__ slab_start,
                                                                          uint32_t nseq) {
    extern __shared__ uint32_t w[];
    const uint32_t k = find_seq(slab_start, nseq, blockIdx.x);
    const SeqJob &J = jobs[k];
    const uint32_t sigma = (uint32_t)J.sigma;
    for (uint32_t j = threadIdx.x; j < (sigma + 1) / 2; j += blockDim.x) w[j] = 0;
    __syncthreads();
    const uint64_t begin = (uint64_t)(blockIdx.x - slab_start[k]) * kBatchSlab;
    const uint64_t end = begin + kBatchSlab < J.n ? begin + kBatchSlab : J.n;
    bool bad = false;
    if (J.width == 2)
        packed_count<uint16_t>(static_cast<const uint16_t *>(J.S), begin, end, sigma, w, J.hist, bad);
    else
        packed_count<uint32_t>(static_cast<const uint32_t *>(J.S), begin, end, sigma, w, J.hist, bad);
    if (bad) atomicOr(J.err, kErrSymbol);
}

// Exclusive scan of one CTA's per-thread values.
__device__ __forceinline__ uint64_t batch_block_scan(uint64_t v, uint64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        const uint64_t w = lane < nw ? s_warp[lane] : 0;
        uint64_t winc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, winc, d);
            if (lane >= d) winc += y;
        }
        if (lane < nw) s_warp[lane] = winc - w;
    }
    __syncthreads();
    const uint64_t r = s_warp[warp] + inc - v;
    __syncthreads();
    return r;
}

// Node starts of every sequence: CTA k scans sequence k's histogram into Hex
// (2^L + 1 entries, bins at and above sigma count 0).
__global__ void __launch_bounds__(kBatchThreads) batch_starts_kernel(const SeqJob *__restrict__ jobs) {
    __shared__ uint64_t s_warp[32];
    const SeqJob &J = jobs[blockIdx.x];
    if (J.L == 0) return;
    const uint64_t entries = (1ull << J.L) + 1;
    const uint64_t chunk = ceil_div(entries, blockDim.x);
    const uint64_t lo = threadIdx.x * chunk < entries ? threadIdx.x * chunk : entries;
    const uint64_t hi = lo + chunk < entries ? lo + chunk : entries;
    uint64_t sum = 0;
    for (uint64_t c = lo; c < hi; c++) sum += c < J.sigma ? J.hist[c] : 0;
    uint64_t run = batch_block_scan(sum, s_warp);
    for (uint64_t c = lo; c < hi; c++) {
        J.hex[c] = run;
        run += c < J.sigma ? J.hist[c] : 0;
    }
}

// Node tables of every (sequence, level): CTA b takes one pair, found in the
// prefix lvl_start of the sequences' level counts.  Same formulas as the
// single-sequence node_tables_kernel.
__global__ void __launch_bounds__(kBatchThreads) batch_tables_kernel(const SeqJob *__restrict__ jobs,
                                                                     const uint32_t *__restrict__ lvl_start,
                                                                     uint32_t nseq) {
    __shared__ uint64_t s_warp[32];
    const uint32_t k = find_seq(lvl_start, nseq, blockIdx.x);
    const SeqJob &J = jobs[k];
    const uint32_t l = blockIdx.x - lvl_start[k];
    if (l >= J.L) return;
    const uint64_t nodes = 1ull << l;
    const uint32_t sh = J.L - l;  // >= 1
    const uint64_t *hex = J.hex;
    const uint64_t chunk = ceil_div(nodes, blockDim.x);
    const uint64_t lo = threadIdx.x * chunk < nodes ? threadIdx.x * chunk : nodes;
    const uint64_t hi = lo + chunk < nodes ? lo + chunk : nodes;
    uint64_t sum = 0;
    for (uint64_t v = lo; v < hi; v++) sum += hex[(2 * v + 1) << (sh - 1)] - hex[(2 * v) << (sh - 1)];
    uint64_t zb = batch_block_scan(sum, s_warp);
    uint64_t *obl = J.ob + (nodes - 1), *zel = J.ze + (nodes - 1);
    for (uint64_t v = lo; v < hi; v++) {
        const uint64_t z = hex[(2 * v + 1) << (sh - 1)] - hex[(2 * v) << (sh - 1)];
        obl[v] = hex[v << sh] - zb;
        zel[v] = zb + z;
        zb += z;
    }
}

cudaError_t launch_batch_prepare(const SeqJob *jobs, uint32_t nseq, const uint32_t *hist_tile_start,
                                 uint32_t hist_tiles, const uint32_t *slab_start, uint32_t slabs,
                                 const uint32_t *lvl_start, uint32_t total_levels, cudaStream_t st) {
    if (nseq == 0) return cudaSuccess;
    batch_clear_err_kernel<<<(nseq + 255) / 256, 256, 0, st>>>(jobs, nseq);
    note_launches(1);
    if (hist_tiles) {
        batch_hist_kernel<<<hist_tiles, kBatchThreads, 0, st>>>(jobs, hist_tile_start, nseq);
        note_launches(1);
    }
    if (slabs) {
        const size_t smem = (kPackedMaxSigma / 2) * sizeof(uint32_t);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(batch_hist_packed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        batch_hist_packed_kernel<<<slabs, kPackedThreads, smem, st>>>(jobs, slab_start, nseq);
        note_launches(1);
    }
    batch_starts_kernel<<<nseq, kBatchThreads, 0, st>>>(jobs);
    note_launches(1);
    if (total_levels) {
        batch_tables_kernel<<<total_levels, kBatchThreads, 0, st>>>(jobs, lvl_start, nseq);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace wt
