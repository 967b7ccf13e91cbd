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

// Zeroes every sequence's error word (they live in the trees' memory).
__global__ void batch_clear_err_kernel(const SeqJob *__restrict__ jobs, uint32_t nseq) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nseq) *jobs[k].err = 0;
}

// One symbol into the bins: the CTA's shared bins (`mine`: this warp's
// copy), or, for alphabets above the shared bins, a 64-bit atomic on the
// sequence's histogram.
__device__ __forceinline__ void batch_add(uint32_t s, uint64_t sigma, uint32_t *mine, uint64_t *hist,
                                          bool shared_bins, bool &bad) {
    if ((uint64_t)s >= sigma)
        bad = true;
    else if (shared_bins)
        atomicAdd(&mine[s], 1u);
    else
        atomicAdd(reinterpret_cast<unsigned long long *>(&hist[s]), 1ull);
}

template <typename Sym>
__device__ __forceinline__ void batch_add_vec(const uint4 q, uint64_t sigma, uint32_t *mine, uint64_t *hist,
                                              bool shared_bins, bool &bad) {
    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (sizeof(Sym) == 1) {
#pragma unroll
            for (int j = 0; j < 4; j++) batch_add((w4[k] >> (8 * j)) & 0xffu, sigma, mine, hist, shared_bins, bad);
        } else if (sizeof(Sym) == 2) {
            batch_add(w4[k] & 0xffffu, sigma, mine, hist, shared_bins, bad);
            batch_add(w4[k] >> 16, sigma, mine, hist, shared_bins, bad);
        } else {
            batch_add(w4[k], sigma, mine, hist, shared_bins, bad);
        }
    }
}

// Symbols [b, e) of one sequence into the bins: whole 16-byte vectors, four
// in flight per thread, single symbols at the ends.
template <typename Sym>
__device__ __forceinline__ void batch_count_range(const SeqJob &J, uint64_t b, uint64_t e, uint32_t *mine,
                                                  bool shared_bins, bool &bad) {
    constexpr uint32_t kPer = 16 / sizeof(Sym);
    const Sym *S = static_cast<const Sym *>(J.S);
    const uint64_t sigma = J.sigma;
    uint64_t *hist = J.hist;
    const uint64_t head = ((16 - (reinterpret_cast<uintptr_t>(S + b) & 15)) & 15) / sizeof(Sym);
    const uint64_t a = b + head < e ? b + head : e;
    const uint64_t nvec = (e - a) / kPer;
    const uint4 *V = reinterpret_cast<const uint4 *>(S + a);
    const uint32_t T = blockDim.x;
    uint64_t r = threadIdx.x;
    for (; r + 3 * T < nvec; r += 4 * T) {
        const uint4 q0 = __ldcs(V + r), q1 = __ldcs(V + r + T), q2 = __ldcs(V + r + 2 * T), q3 = __ldcs(V + r + 3 * T);
        batch_add_vec<Sym>(q0, sigma, mine, hist, shared_bins, bad);
        batch_add_vec<Sym>(q1, sigma, mine, hist, shared_bins, bad);
        batch_add_vec<Sym>(q2, sigma, mine, hist, shared_bins, bad);
        batch_add_vec<Sym>(q3, sigma, mine, hist, shared_bins, bad);
    }
    for (; r < nvec; r += T) batch_add_vec<Sym>(__ldcs(V + r), sigma, mine, hist, shared_bins, bad);
    for (uint64_t i = b + threadIdx.x; i < a; i += T) batch_add((uint32_t)S[i], sigma, mine, hist, shared_bins, bad);
    for (uint64_t i = a + nvec * kPer + threadIdx.x; i < e; i += T)
        batch_add((uint32_t)S[i], sigma, mine, hist, shared_bins, bad);
}

// Leaf histogram of the sequences with small (or very large) alphabets.
// Persistent: CTA b takes a contiguous range of the launch's tiles
// (tile_start: each sequence's first tile, total at [nseq]), so it finds its
// first sequence once, walks forward, and zeroes and flushes its shared bins
// once per sequence of its range.
__global__ void __launch_bounds__(kBatchThreads) batch_hist_kernel(const SeqJob *__restrict__ jobs,
                                                                   const uint32_t *__restrict__ tile_start,
                                                                   uint32_t nseq) {
    __shared__ uint32_t bins[kBatchSmemBins];
    const uint32_t total = tile_start[nseq];
    const uint32_t per = (total + gridDim.x - 1) / gridDim.x;
    uint32_t t0 = min(blockIdx.x * per, total);
    const uint32_t t1 = min(t0 + per, total);
    if (t0 >= t1) return;
    uint32_t k = find_seq(tile_start, nseq, t0);
    while (t0 < t1) {
        const SeqJob &J = jobs[k];
        const uint32_t ks = tile_start[k];
        const uint32_t te = min(t1, tile_start[k + 1]);
        const uint64_t b = (uint64_t)(t0 - ks) * kBatchHistTile;
        const uint64_t e = min(J.n, (uint64_t)(te - ks) * kBatchHistTile);
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
        if (J.width == 1)
            batch_count_range<uint8_t>(J, b, e, mine, shared_bins, bad);
        else if (J.width == 2)
            batch_count_range<uint16_t>(J, b, e, mine, shared_bins, bad);
        else
            batch_count_range<uint32_t>(J, b, e, mine, shared_bins, bad);
        if (bad) atomicOr(J.err, kErrSymbol);
        __syncthreads();
        if (shared_bins)
            for (uint32_t c = threadIdx.x; c < sig; c += blockDim.x) {
                uint32_t sum = 0;
                for (uint32_t q = 0; q < copies; q++) sum += bins[q * sig + c];
                if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(&J.hist[c]), (unsigned long long)sum);
            }
        __syncthreads();  // the bins are zeroed again for the next sequence
        t0 = te;
        while (k + 1 < nseq && tile_start[k + 1] <= t0) k++;
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
    const bool sole = slab_start[k + 1] - slab_start[k] == 1;  // the sequence's only slab owns its histogram
    bool bad = false;
    if (J.width == 2)
        packed_count<uint16_t>(static_cast<const uint16_t *>(J.S), begin, end, sigma, w, J.hist, bad, sole);
    else
        packed_count<uint32_t>(static_cast<const uint32_t *>(J.S), begin, end, sigma, w, J.hist, bad, sole);
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

// Exclusive scan of `count` values (value(i) gives value i) into out(i, x),
// by one CTA, in segments of kSeg values staged in shared memory so that
// loads and stores are coalesced and each thread scans kPer consecutive
// values.
constexpr uint32_t kSegPer = 8;
constexpr uint32_t kSeg = kBatchThreads * kSegPer;

template <typename Val, typename Out>
__device__ __forceinline__ void cta_scan(uint64_t count, Val value, Out out, uint64_t *seg, uint64_t *s_warp) {
    uint64_t carry = 0;
    for (uint64_t s0 = 0; s0 < count; s0 += kSeg) {
#pragma unroll
        for (uint32_t i = 0; i < kSegPer; i++) {
            const uint64_t e = s0 + i * kBatchThreads + threadIdx.x;
            seg[i * kBatchThreads + threadIdx.x] = e < count ? value(e) : 0;
        }
        __syncthreads();
        uint64_t mine[kSegPer], sum = 0;
#pragma unroll
        for (uint32_t i = 0; i < kSegPer; i++) {
            mine[i] = seg[threadIdx.x * kSegPer + i];
            sum += mine[i];
        }
        uint64_t run = carry + batch_block_scan(sum, s_warp);
#pragma unroll
        for (uint32_t i = 0; i < kSegPer; i++) {
            seg[threadIdx.x * kSegPer + i] = run;
            run += mine[i];
        }
        if (threadIdx.x == kBatchThreads - 1) s_warp[32] = run;  // carry into the next segment
        __syncthreads();
#pragma unroll
        for (uint32_t i = 0; i < kSegPer; i++) {
            const uint64_t e = s0 + i * kBatchThreads + threadIdx.x;
            if (e < count) out(e, seg[i * kBatchThreads + threadIdx.x]);
        }
        carry = s_warp[32];
        __syncthreads();
    }
}

// Node starts of the sequences with large alphabets: CTA b scans sequence
// seqs[b]'s histogram into Hex (2^L + 1 entries, bins at and above sigma
// count 0).
__global__ void __launch_bounds__(kBatchThreads) batch_starts_kernel(const SeqJob *__restrict__ jobs,
                                                                     const uint32_t *__restrict__ seqs) {
    __shared__ uint64_t s_warp[33];
    __shared__ uint64_t seg[kSeg];
    const SeqJob &J = jobs[seqs[blockIdx.x]];
    if (J.L == 0) return;
    const uint64_t *hist = J.hist;
    const uint64_t sigma = J.sigma;
    uint64_t *hex = J.hex;
    cta_scan((1ull << J.L) + 1, [&](uint64_t c) { return c < sigma ? hist[c] : 0ull; },
             [&](uint64_t c, uint64_t v) { hex[c] = v; }, seg, s_warp);
}

// Exclusive scan over a warp of one value per lane; `total` gets the sum.
__device__ __forceinline__ uint64_t warp_scan_u64(uint64_t v, uint64_t &total) {
    const int lane = threadIdx.x & 31;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// Node tables of level l of one sequence by one warp (each lane a
// contiguous block of nodes, a warp scan between the blocks).  The node
// tables follow the single-sequence node_tables_kernel: the zeros of node v
// are the symbols of its left child, OB = ones before the node's start,
// ZE = zeros up to its end.  Hex is read through L2 (the same warp may just
// have written it).
__device__ __forceinline__ void warp_tables(const SeqJob &J, uint32_t l) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nodes = 1u << l, sh = J.L - l;
    const uint64_t *hex = J.hex;
    uint64_t *obl = J.ob + (nodes - 1), *zel = J.ze + (nodes - 1);
    const uint32_t m = (nodes + 31) / 32;
    const uint32_t v0 = min(lane * m, nodes), v1 = min(v0 + m, nodes);
    uint64_t sum = 0;
    for (uint32_t v = v0; v < v1; v++)
        sum += __ldcg(hex + ((2 * (uint64_t)v + 1) << (sh - 1))) - __ldcg(hex + ((uint64_t)v << sh));
    uint64_t total;
    uint64_t zb = warp_scan_u64(sum, total);
    for (uint32_t v = v0; v < v1; v++) {
        const uint64_t h0 = __ldcg(hex + ((uint64_t)v << sh)), h1 = __ldcg(hex + ((2 * (uint64_t)v + 1) << (sh - 1)));
        obl[v] = h0 - zb;
        zel[v] = zb + (h1 - h0);
        zb += h1 - h0;
    }
}

// Node tables of the sequences with large alphabets, pairs p = sequence << 5
// | level: CTAs [0, nbig) take one deep level each (big_pairs, the CTA scans
// the level's nodes); the CTAs after them take kBatchThreads / 32 shallow
// levels each, one per warp (small_pairs).
__global__ void __launch_bounds__(kBatchThreads) batch_tables_kernel(const SeqJob *__restrict__ jobs,
                                                                     const uint32_t *__restrict__ big_pairs,
                                                                     uint32_t nbig,
                                                                     const uint32_t *__restrict__ small_pairs,
                                                                     uint32_t nsmall) {
    __shared__ uint64_t s_warp[33];
    __shared__ uint64_t seg[kSeg];
    if (blockIdx.x >= nbig) {
        const uint32_t w = (blockIdx.x - nbig) * (kBatchThreads / 32) + (threadIdx.x >> 5);
        if (w >= nsmall) return;
        const uint32_t pr = small_pairs[w];
        const SeqJob &J = jobs[pr >> 5];
        if ((pr & 31u) < J.L) warp_tables(J, pr & 31u);
        return;
    }
    const uint32_t pr = big_pairs[blockIdx.x];
    const SeqJob &J = jobs[pr >> 5];
    const uint32_t l = pr & 31u;
    if (l >= J.L) return;
    const uint64_t nodes = 1ull << l;
    const uint32_t sh = J.L - l;  // >= 1
    const uint64_t *hex = J.hex;
    uint64_t *obl = J.ob + (nodes - 1), *zel = J.ze + (nodes - 1);
    cta_scan(nodes, [&](uint64_t v) { return hex[(2 * v + 1) << (sh - 1)] - hex[v << sh]; },
             [&](uint64_t v, uint64_t zb) {
                 const uint64_t h0 = hex[v << sh], h1 = hex[(2 * v + 1) << (sh - 1)];
                 obl[v] = h0 - zb;
                 zel[v] = zb + (h1 - h0);
             },
             seg, s_warp);
}

// Node starts and node tables of the sequences with small alphabets
// (2^L <= kBatchWarpLeaves): one warp per sequence seqs[w], each lane a
// contiguous block of leaves, a warp scan between the blocks, then every
// level's tables by the same warp.
__global__ void __launch_bounds__(kBatchThreads) batch_small_kernel(const SeqJob *__restrict__ jobs,
                                                                    const uint32_t *__restrict__ seqs,
                                                                    uint32_t count) {
    const uint32_t w = blockIdx.x * (kBatchThreads / 32) + (threadIdx.x >> 5);
    if (w >= count) return;
    const uint32_t lane = threadIdx.x & 31;
    const SeqJob &J = jobs[seqs[w]];
    const uint32_t L = J.L;
    if (L == 0) return;
    const uint64_t sigma = J.sigma;
    const uint32_t leaves = 1u << L;
    uint64_t *hex = J.hex;
    const uint32_t m = (leaves + 1 + 31) / 32;  // entries per lane
    const uint32_t c0 = lane * m, c1 = min(c0 + m, leaves + 1);
    uint64_t sum = 0;
    for (uint32_t c = c0; c < c1; c++) sum += c < sigma ? J.hist[c] : 0ull;
    uint64_t total;
    uint64_t run = warp_scan_u64(sum, total);
    for (uint32_t c = c0; c < c1; c++) {
        hex[c] = run;
        run += c < sigma ? J.hist[c] : 0ull;
    }
    __syncwarp();
    for (uint32_t l = 0; l < L; l++) warp_tables(J, l);
}

cudaError_t launch_batch_prepare(const SeqJob *jobs, uint32_t nseq, const uint32_t *hist_tile_start,
                                 uint32_t hist_tiles, const uint32_t *slab_start, uint32_t slabs,
                                 const uint32_t *small_seqs, uint32_t nsmall, const uint32_t *big_seqs,
                                 uint32_t nbig, const uint32_t *big_pairs, uint32_t nbig_pairs,
                                 const uint32_t *small_pairs, uint32_t nsmall_pairs, cudaStream_t st) {
    if (nseq == 0) return cudaSuccess;
    batch_clear_err_kernel<<<(nseq + 255) / 256, 256, 0, st>>>(jobs, nseq);
    note_launches(1);
    if (hist_tiles) {
        // Persistent: every resident CTA slot.
        static uint32_t slots = 0;
        if (!slots) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_hist_kernel, kBatchThreads, 0) !=
                    cudaSuccess ||
                per_sm < 1) {
                cudaGetLastError();
                per_sm = 1;
            }
            slots = (uint32_t)(sms > 0 ? sms : 1) * (uint32_t)per_sm;
        }
        batch_hist_kernel<<<hist_tiles < slots ? hist_tiles : slots, kBatchThreads, 0, st>>>(jobs, hist_tile_start,
                                                                                             nseq);
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
    if (nsmall) {
        constexpr uint32_t kWarps = kBatchThreads / 32;
        batch_small_kernel<<<(nsmall + kWarps - 1) / kWarps, kBatchThreads, 0, st>>>(jobs, small_seqs, nsmall);
        note_launches(1);
    }
    if (nbig) {
        batch_starts_kernel<<<nbig, kBatchThreads, 0, st>>>(jobs, big_seqs);
        note_launches(1);
    }
    if (nbig_pairs + nsmall_pairs) {
        constexpr uint32_t kWarps = kBatchThreads / 32;
        batch_tables_kernel<<<nbig_pairs + (nsmall_pairs + kWarps - 1) / kWarps, kBatchThreads, 0, st>>>(
            jobs, big_pairs, nbig_pairs, small_pairs, nsmall_pairs);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace wt
