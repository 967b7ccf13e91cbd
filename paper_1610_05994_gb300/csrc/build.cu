// build.cu -- construction kernels of the level-wise path.
//
// (a)  histogram of the leaf codes + exclusive scan  -> Hex (node starts of
//      every level at once: node v of level l starts at Hex[v << (L - l)]),
//      replacing the per-level "count" and parPrefixSum steps of Algorithm 1.
//      For 1-byte symbols the histogram's read of S also does level 0's
//      count pass (level 0's bitmap and unit counts).
// (a') per-level node tables OB / ZE from Hex.
// The level step (b + c) is in level.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.cuh"
#include "wt_internal.cuh"

namespace wt {

// ------------------------------------------------------------------ (a)

constexpr int kHistThreads = 512;
constexpr uint32_t kHistSmemBins = 48 * 1024;  // u32 bins per CTA for the shared-memory path

template <typename Sym>
__device__ __forceinline__ void hist_add_shared(uint32_t *bins, uint32_t sigma, uint32_t s, bool &bad) {
    if (s < sigma)
        atomicAdd(&bins[s], 1u);
    else
        bad = true;
}

// The bits at shift bsh of the 16 bytes of q, packed: bit k = byte k (one
// multiply gathers the four top bits of a word into a nibble).
__device__ __forceinline__ uint32_t byte_bits16(const uint4 q, uint32_t bsh) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
    uint32_t h = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) h |= ((((w[i] << (7 - bsh)) & 0x80808080u) * 0x00204081u) >> 28) << (4 * i);
    return h;
}

// Level 0's count pass for vector k of S (16 symbols; the 32 lanes of a warp
// hold the 32 vectors of one 512-symbol unit, all active together).
// With z.plane (a pair step at level 0) also bit bsh - 1 of the symbols and
// the unit counts of groups 01 and 11 (bits (L-1, L-2) of the symbol).
__device__ __forceinline__ void level0_vector(const Level0Fuse &z, uint64_t k, const uint4 q) {
    const uint32_t hb = byte_bits16(q, z.bsh);
    reinterpret_cast<uint16_t *>(z.words)[k] = (uint16_t)hb;
    if (z.next) reinterpret_cast<uint16_t *>(z.next)[k] = 0;
    const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(hb));
    if ((threadIdx.x & 31) == 0) z.cnt[k / 32] = c;
    if (z.plane) {
        const uint32_t hp = byte_bits16(q, z.bsh - 1);
        reinterpret_cast<uint16_t *>(z.plane)[k] = (uint16_t)hp;
        if (z.next2) reinterpret_cast<uint16_t *>(z.next2)[k] = 0;
        if (z.plane3) reinterpret_cast<uint16_t *>(z.plane3)[k] = 0;
        const uint32_t c01 = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(~hb & hp));
        const uint32_t c11 = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(hb & hp));
        if ((threadIdx.x & 31) == 0) {
            z.cnt01[k / 32] = c01;
            z.cnt11[k / 32] = c11;
        }
    }
}

// Whole tiles only: the level step's scan reads every unit count of every
// tile, and the histogram writes the counts of the units it covers.
bool level0_fusable(const void *S, uint64_t n, int width, uint64_t sigma) {
    return width == 1 && sigma >= 2 && n > 0 && n % lw_tile_elems(1) == 0 &&
           (reinterpret_cast<uintptr_t>(S) & 15) == 0;
}

// Shared-memory histogram: `copies` private copies of the sigma bins (warp w
// uses copy w % copies) spread same-bin contention for small alphabets.
template <typename Sym>
__global__ void __launch_bounds__(kHistThreads) hist_shared_kernel(const Sym *__restrict__ S, uint64_t n,
                                                                   uint32_t sigma, uint32_t copies,
                                                                   uint64_t *__restrict__ hist,
                                                                   uint32_t *__restrict__ err, Level0Fuse z) {
    extern __shared__ uint32_t bins[];
    const uint32_t total = sigma * copies;
    for (uint32_t k = threadIdx.x; k < total; k += blockDim.x) bins[k] = 0;
    __syncthreads();
    uint32_t *mine = bins + ((threadIdx.x >> 5) % copies) * sigma;
    bool bad = false;
    constexpr int kPer = 16 / sizeof(Sym);
    const bool vec = (reinterpret_cast<uintptr_t>(S) & 15) == 0;
    const uint64_t nvec = vec ? n / kPer : 0;
    const uint4 *V = reinterpret_cast<const uint4 *>(S);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    auto add_vec = [&](const uint4 q) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int t = 0; t < kPer; t++) {
            const uint32_t v = sizeof(Sym) == 4 ? w[t] : (w[t / (4 / sizeof(Sym))] >> (8 * sizeof(Sym) * (t % (4 / sizeof(Sym))))) &
                                                              (sizeof(Sym) == 1 ? 0xffu : 0xffffu);
            hist_add_shared<Sym>(mine, sigma, v, bad);
        }
    };
    uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool fuse = sizeof(Sym) == 1 && z.words != nullptr;
    // Four vectors in flight per thread.
    for (; k + 3 * stride < nvec; k += 4 * stride) {
        const uint4 q0 = __ldcs(V + k), q1 = __ldcs(V + k + stride), q2 = __ldcs(V + k + 2 * stride),
                    q3 = __ldcs(V + k + 3 * stride);
        add_vec(q0);
        add_vec(q1);
        add_vec(q2);
        add_vec(q3);
        if (fuse) {
            level0_vector(z, k, q0);
            level0_vector(z, k + stride, q1);
            level0_vector(z, k + 2 * stride, q2);
            level0_vector(z, k + 3 * stride, q3);
        }
    }
    for (; k < nvec; k += stride) {
        const uint4 q = __ldcs(V + k);
        add_vec(q);
        if (fuse) level0_vector(z, k, q);
    }
    for (uint64_t k = nvec * kPer + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x)
        hist_add_shared<Sym>(mine, sigma, (uint32_t)S[k], bad);
    if (bad) atomicOr(err, kErrSymbol);
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < sigma; c += blockDim.x) {
        uint32_t sum = 0;
        for (uint32_t k = 0; k < copies; k++) sum += bins[k * sigma + c];
        if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(&hist[c]), (unsigned long long)sum);
    }
}

// Alphabets of at most four byte codes (DNA-like): no bins at all.  The two
// low bit planes of four bytes give, by three popcounts, how many of them
// are 1, 2 and 3; the rest are 0.  Any higher bit is a symbol out of range.
// Per-thread counts, one warp sum and four 64-bit atomics per warp.
__global__ void __launch_bounds__(kHistThreads, 2) hist_tiny_kernel(const uint8_t *__restrict__ S, uint64_t n,
                                                                    uint32_t sigma, uint64_t *__restrict__ hist,
                                                                    uint32_t *__restrict__ err, Level0Fuse z) {
    uint32_t c1 = 0, c2 = 0, c3 = 0, total = 0, high = 0;
    auto add_word = [&](uint32_t x) {
        high |= x & 0xfcfcfcfcu;
        const uint32_t lo = x & 0x01010101u, hi = (x >> 1) & 0x01010101u;
        const uint32_t n3 = __popc(lo & hi);
        c3 += n3;
        c1 += __popc(lo) - n3;
        c2 += __popc(hi) - n3;
    };
    const bool vec = (reinterpret_cast<uintptr_t>(S) & 15) == 0;
    const uint64_t nvec = vec ? n / 16 : 0;
    const uint4 *V = reinterpret_cast<const uint4 *>(S);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool fuse = z.words != nullptr;
    for (; k + 3 * stride < nvec; k += 4 * stride) {
        const uint4 q[4] = {__ldcs(V + k), __ldcs(V + k + stride), __ldcs(V + k + 2 * stride),
                            __ldcs(V + k + 3 * stride)};
#pragma unroll
        for (int r = 0; r < 4; r++) {
            add_word(q[r].x);
            add_word(q[r].y);
            add_word(q[r].z);
            add_word(q[r].w);
            if (fuse) level0_vector(z, k + r * stride, q[r]);
        }
        total += 64;
    }
    for (; k < nvec; k += stride) {
        const uint4 q = __ldcs(V + k);
        add_word(q.x);
        add_word(q.y);
        add_word(q.z);
        add_word(q.w);
        if (fuse) level0_vector(z, k, q);
        total += 16;
    }
    for (uint64_t j = nvec * 16 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t s = S[j];
        high |= s & ~3u;
        c1 += s == 1;
        c2 += s == 2;
        c3 += s == 3;
        total += 1;
    }
    c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    c3 = __reduce_add_sync(0xffffffffu, c3);
    total = __reduce_add_sync(0xffffffffu, total);
    high = __reduce_or_sync(0xffffffffu, high);
    if ((threadIdx.x & 31) == 0) {
        const uint32_t c[4] = {total - c1 - c2 - c3, c1, c2, c3};
        bool bad = high != 0;
#pragma unroll
        for (uint32_t v = 0; v < 4; v++) {
            if (v < sigma) {
                if (c[v]) atomicAdd(reinterpret_cast<unsigned long long *>(&hist[v]), (unsigned long long)c[v]);
            } else if (c[v]) {
                bad = true;
            }
        }
        if (bad) atomicOr(err, kErrSymbol);
    }
}

// Large alphabets: global 64-bit atomics, one per group of equal codes in a warp.
template <typename Sym>
__global__ void __launch_bounds__(kHistThreads) hist_global_kernel(const Sym *__restrict__ S, uint64_t n,
                                                                   uint64_t sigma, uint64_t *__restrict__ hist,
                                                                   uint32_t *__restrict__ err) {
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t start = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t rounds = ceil_div(n, stride);
    for (uint64_t r = 0; r < rounds; r++) {
        const uint64_t k = start + r * stride;
        const bool valid = k < n;
        uint32_t s = valid ? (uint32_t)S[k] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, s);
        const int leader = __ffs(peers) - 1;
        if (valid) {
            if ((uint64_t)s >= sigma)
                bad = true;
            else if ((threadIdx.x & 31) == leader)
                atomicAdd(reinterpret_cast<unsigned long long *>(&hist[s]), (unsigned long long)__popc(peers));
        }
    }
    if (bad) atomicOr(err, kErrSymbol);
}

// Large alphabets, n < 2^32: 32-bit counts in R replicas of the sigma bins
// (warp w adds into replica w mod R).  Skewed codes put a large share of all
// additions on a few bins; replicas spread one hot bin over R L2 addresses,
// and equal codes inside a warp still merge into one addition.
template <typename Sym>
__global__ void __launch_bounds__(kHistThreads) hist_replicated_kernel(const Sym *__restrict__ S, uint64_t n,
                                                                       uint64_t sigma, uint32_t *__restrict__ rep,
                                                                       uint32_t R, uint32_t *__restrict__ err) {
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t start = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t rounds = ceil_div(n, stride);
    const uint32_t gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint32_t *mine = rep + (uint64_t)(gwarp % R) * sigma;
    for (uint64_t r = 0; r < rounds; r++) {
        const uint64_t k = start + r * stride;
        const bool valid = k < n;
        const uint32_t s = valid ? (uint32_t)S[k] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, s);
        if (valid) {
            if ((uint64_t)s >= sigma)
                bad = true;
            else if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&mine[s], (uint32_t)__popc(peers));
        }
    }
    if (bad) atomicOr(err, kErrSymbol);
}

// Mid-size alphabets: packed 16-bit shared bins (one CTA per SM, a
// contiguous slab of S each).
template <typename Sym>
__global__ void __launch_bounds__(kPackedThreads) hist_packed_kernel(const Sym *__restrict__ S, uint64_t n,
                                                                    uint32_t sigma, uint64_t slab,
                                                                    uint64_t *__restrict__ hist,
                                                                    uint32_t *__restrict__ err) {
    extern __shared__ uint32_t w[];
    for (uint32_t j = threadIdx.x; j < (sigma + 1) / 2; j += blockDim.x) w[j] = 0;
    __syncthreads();
    const uint64_t begin = blockIdx.x * slab;
    const uint64_t end = begin + slab < n ? begin + slab : n;
    bool bad = false;
    if (begin < end) packed_count<Sym>(S, begin, end, sigma, w, hist, bad);
    if (bad) atomicOr(err, kErrSymbol);
}

uint32_t hist_replicas(uint64_t n, uint64_t sigma) {
    if (sigma <= kPackedMaxSigma || n >= (1ull << 32)) return 0;  // not this path
    uint64_t R = (64ull << 20) / (sigma * 4);                     // at most 64 MB of counters
    if (R > 16) R = 16;
    return R < 1 ? 1 : (uint32_t)R;
}

template <typename Sym>
static cudaError_t histogram_rep_t(const void *S, uint64_t n, uint64_t sigma, uint32_t *rep, uint32_t R,
                                   uint32_t *err, cudaStream_t st);

cudaError_t launch_histogram_replicated(const void *S, uint64_t n, int width, uint64_t sigma, uint32_t *rep,
                                        uint32_t R, uint32_t *err, cudaStream_t st) {
    switch (width) {
        case 1: return histogram_rep_t<uint8_t>(S, n, sigma, rep, R, err, st);
        case 2: return histogram_rep_t<uint16_t>(S, n, sigma, rep, R, err, st);
        case 4: return histogram_rep_t<uint32_t>(S, n, sigma, rep, R, err, st);
    }
    return cudaErrorInvalidValue;
}

static int sm_count() {
    static int count = 0;
    if (!count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 1;
    }
    return count;
}

template <typename Sym>
static cudaError_t histogram_t(const void *S, uint64_t n, uint64_t sigma, uint64_t *hist, uint32_t *err,
                               cudaStream_t st, const Level0Fuse *fuse) {
    Level0Fuse z{};
    if (fuse && sizeof(Sym) == 1 && level0_fusable(S, n, 1, sigma) && sigma <= kHistSmemBins) z = *fuse;
    if (n == 0) return cudaSuccess;
    const Sym *s = static_cast<const Sym *>(S);
    const uint64_t per_cta_cap = 1ull << 30;  // keeps every u32 shared bin below 2^32
    uint64_t grid = (uint64_t)sm_count() * 4;
    grid = grid > ceil_div(n, per_cta_cap) ? grid : ceil_div(n, per_cta_cap);
    uint64_t want = ceil_div(n, (uint64_t)kHistThreads * 16);
    if (grid > want) grid = want ? want : 1;
    if (sizeof(Sym) == 1 && sigma <= 4) {
        // Two resident CTAs per SM (52 registers a thread), all of them at once.
        const uint64_t g2 = grid < (uint64_t)sm_count() * 2 ? grid : (uint64_t)sm_count() * 2;
        hist_tiny_kernel<<<(unsigned)g2, kHistThreads, 0, st>>>(reinterpret_cast<const uint8_t *>(S), n,
                                                                (uint32_t)sigma, hist, err, z);
        note_launches(1);
    } else if (sigma <= kHistSmemBins) {
        uint32_t sig = (uint32_t)sigma;
        uint32_t copies = (uint32_t)(kHistSmemBins / sigma);
        const uint32_t warps = kHistThreads / 32;
        if (copies > warps) copies = warps;
        if (copies < 1) copies = 1;
        size_t smem = (size_t)sig * copies * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(hist_shared_kernel<Sym>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        hist_shared_kernel<Sym><<<(unsigned)grid, kHistThreads, smem, st>>>(s, n, sig, copies, hist, err, z);
        note_launches(1);
    } else if (sigma <= kPackedMaxSigma) {
        const size_t smem = (kPackedMaxSigma / 2) * sizeof(uint32_t);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(hist_packed_kernel<Sym>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const uint64_t g = (uint64_t)sm_count();
        const uint64_t slab = ceil_div(n, g);
        hist_packed_kernel<Sym><<<(unsigned)ceil_div(n, slab), kPackedThreads, smem, st>>>(s, n, (uint32_t)sigma, slab,
                                                                                         hist, err);
        note_launches(1);
    } else {
        hist_global_kernel<Sym><<<(unsigned)grid, kHistThreads, 0, st>>>(s, n, sigma, hist, err);
        note_launches(1);
    }
    return cudaGetLastError();
}

template <typename Sym>
static cudaError_t histogram_rep_t(const void *S, uint64_t n, uint64_t sigma, uint32_t *rep, uint32_t R,
                                   uint32_t *err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    uint64_t grid = (uint64_t)sm_count() * 4;
    const uint64_t want = ceil_div(n, (uint64_t)kHistThreads * 4);
    if (grid > want) grid = want ? want : 1;
    hist_replicated_kernel<Sym><<<(unsigned)grid, kHistThreads, 0, st>>>(static_cast<const Sym *>(S), n, sigma, rep,
                                                                        R, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const void *S, uint64_t n, int width, uint64_t sigma, uint64_t *hist, uint32_t *err,
                             cudaStream_t st, const Level0Fuse *fuse) {
    switch (width) {
        case 1: return histogram_t<uint8_t>(S, n, sigma, hist, err, st, fuse);
        case 2: return histogram_t<uint16_t>(S, n, sigma, hist, err, st, nullptr);
        case 4: return histogram_t<uint32_t>(S, n, sigma, hist, err, st, nullptr);
    }
    return cudaErrorInvalidValue;
}

constexpr int kScanThreads = 1024;

// Exclusive scan of the values of one CTA's threads (one value per thread).
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t w = lane < nw ? s_warp[lane] : 0;
        uint64_t winc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, winc, d);
            if (lane >= d) winc += y;
        }
        if (lane < nw) s_warp[lane] = winc - w;
    }
    __syncthreads();
    const uint64_t r = s_warp[warp] + inc - v;
    __syncthreads();
    return r;
}

// ---- exclusive scans over an implicit sequence val(0..count-1).
// Small inputs: one CTA, each thread a contiguous range (node_starts_kernel,
// node_tables_kernel).  Large inputs: reduce-then-scan over 8192-entry chunks
// in three launches (chunk sums, scan of the sums, chunk scan), no waits.

constexpr int kScanItems = 8;
constexpr uint64_t kScanChunk = (uint64_t)kScanThreads * kScanItems;
constexpr uint64_t kSingleCtaMax = 1ull << 16;  // up to this many entries one CTA scans

struct HistVal {  // leaf counts, zero at and above sigma
    const uint64_t *hist;
    uint64_t sigma;
    __device__ __forceinline__ uint64_t operator()(uint64_t c) const { return c < sigma ? hist[c] : 0; }
};
struct HistRepVal {  // leaf counts summed over the replicas, zero at and above sigma
    const uint32_t *rep;
    uint64_t sigma;
    uint32_t R;
    __device__ __forceinline__ uint64_t operator()(uint64_t c) const {
        if (c >= sigma) return 0;
        uint64_t v = 0;
        for (uint32_t r = 0; r < R; r++) v += rep[(uint64_t)r * sigma + c];
        return v;
    }
};
struct HexOut {
    uint64_t *hex;
    __device__ __forceinline__ void operator()(uint64_t c, uint64_t excl, uint64_t) const { hex[c] = excl; }
};
struct ZeroVal {  // Z_l[v]: size of the left child of node v on level l
    const uint64_t *hex;
    uint32_t sh;      // L - l >= 1
    __device__ __forceinline__ uint64_t operator()(uint64_t v) const {
        return hex[(2 * v + 1) << (sh - 1)] - hex[(2 * v) << (sh - 1)];
    }
};
struct TableOut {  // OB_l[v] = node start - zeros before it; ZE_l[v] = zeros through its end
    const uint64_t *hex;
    uint32_t sh;
    uint64_t *ob, *ze;
    __device__ __forceinline__ void operator()(uint64_t v, uint64_t zb, uint64_t z) const {
        ob[v] = hex[v << sh] - zb;
        ze[v] = zb + z;
    }
};

template <class Val>
__global__ void __launch_bounds__(kScanThreads) chunk_sums_kernel(Val val, uint64_t count, uint64_t *__restrict__ sums) {
    __shared__ uint64_t s_warp[32];
    const uint64_t base = blockIdx.x * kScanChunk;
    uint64_t v = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint64_t c = base + (uint64_t)i * kScanThreads + threadIdx.x;
        if (c < count) v += val(c);
    }
    const uint64_t excl = block_exclusive_scan(v, s_warp);
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = excl + v;
}

// In-place exclusive scan of nchunks values by one CTA.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint64_t *__restrict__ sums, uint64_t nchunks) {
    __shared__ uint64_t s_warp[32];
    const uint64_t per = ceil_div(nchunks, blockDim.x);
    const uint64_t lo = threadIdx.x * per < nchunks ? threadIdx.x * per : nchunks;
    const uint64_t hi = lo + per < nchunks ? lo + per : nchunks;
    uint64_t sum = 0;
    for (uint64_t k = lo; k < hi; k++) sum += sums[k];
    uint64_t run = block_exclusive_scan(sum, s_warp);
    for (uint64_t k = lo; k < hi; k++) {
        const uint64_t x = sums[k];
        sums[k] = run;
        run += x;
    }
}

template <class Val, class Out>
__global__ void __launch_bounds__(kScanThreads) chunk_scan_kernel(Val val, Out out, uint64_t count,
                                                                  const uint64_t *__restrict__ sums) {
    __shared__ uint64_t s_warp[32];
    const uint64_t lo = blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = lo + i < count ? val(lo + i) : 0;
        sum += v[i];
    }
    uint64_t run = sums[blockIdx.x] + block_exclusive_scan(sum, s_warp);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (lo + i < count) out(lo + i, run, v[i]);
        run += v[i];
    }
}

template <class Val, class Out>
static cudaError_t scan_large(Val val, Out out, uint64_t count, uint64_t *tmp, cudaStream_t st) {
    const uint64_t nchunks = ceil_div(count, kScanChunk);
    chunk_sums_kernel<Val><<<(unsigned)nchunks, kScanThreads, 0, st>>>(val, count, tmp);
    note_launches(1);
    scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tmp, nchunks);
    note_launches(1);
    chunk_scan_kernel<Val, Out><<<(unsigned)nchunks, kScanThreads, 0, st>>>(val, out, count, tmp);
    note_launches(1);
    return cudaGetLastError();
}

size_t scan_tmp_bytes(uint32_t L) { return ceil_div((1ull << L) + 1, kScanChunk) * sizeof(uint64_t); }

// Hex[c] = sum of hist[c'] over c' < c, c = 0 .. 2^L (bins at c >= sigma count 0).
__global__ void __launch_bounds__(kScanThreads) node_starts_kernel(const uint64_t *__restrict__ hist,
                                                                   uint64_t sigma, uint64_t entries,
                                                                   uint64_t *__restrict__ hex) {
    __shared__ uint64_t s_warp[32];
    const uint64_t chunk = ceil_div(entries, blockDim.x);
    const uint64_t lo = threadIdx.x * chunk < entries ? threadIdx.x * chunk : entries;
    const uint64_t hi = lo + chunk < entries ? lo + chunk : entries;
    uint64_t sum = 0;
    for (uint64_t c = lo; c < hi; c++) sum += c < sigma ? hist[c] : 0;
    uint64_t run = block_exclusive_scan(sum, s_warp);
    for (uint64_t c = lo; c < hi; c++) {
        hex[c] = run;
        run += c < sigma ? hist[c] : 0;
    }
}

cudaError_t launch_node_starts(const uint64_t *hist, uint64_t sigma, uint32_t L, uint64_t n, uint64_t *hex,
                               cudaStream_t st, uint64_t *tmp) {
    (void)n;
    const uint64_t entries = (1ull << L) + 1;
    if (tmp == nullptr || entries <= kSingleCtaMax) {
        node_starts_kernel<<<1, kScanThreads, 0, st>>>(hist, sigma, entries, hex);
        note_launches(1);
        return cudaGetLastError();
    }
    return scan_large(HistVal{hist, sigma}, HexOut{hex}, entries, tmp, st);
}

cudaError_t launch_node_starts_replicated(const uint32_t *rep, uint32_t R, uint64_t sigma, uint32_t L, uint64_t *hex,
                                          cudaStream_t st, uint64_t *tmp) {
    return scan_large(HistRepVal{rep, sigma, R}, HexOut{hex}, (1ull << L) + 1, tmp, st);
}

// One CTA per small level l: Z_l[v] = size of the left child of node v =
// Hex[(2v+1) << (L-l-1)] - Hex[2v << (L-l-1)]; ZB_l = exclusive scan of Z_l;
// OB_l[v] = Hex[v << (L-l)] - ZB_l[v]; ZE_l[v] = ZB_l[v] + Z_l[v].
// Level l's tables start at offset 2^l - 1.
__global__ void __launch_bounds__(kScanThreads) node_tables_kernel(const uint64_t *__restrict__ hex, uint32_t L,
                                                                   uint64_t *__restrict__ ob,
                                                                   uint64_t *__restrict__ ze) {
    __shared__ uint64_t s_warp[32];
    const uint32_t l = blockIdx.x;
    const uint64_t nodes = 1ull << l;
    const uint32_t sh = L - l;  // >= 1
    const uint64_t chunk = ceil_div(nodes, blockDim.x);
    const uint64_t lo = threadIdx.x * chunk < nodes ? threadIdx.x * chunk : nodes;
    const uint64_t hi = lo + chunk < nodes ? lo + chunk : nodes;
    uint64_t sum = 0;
    for (uint64_t v = lo; v < hi; v++) sum += hex[(2 * v + 1) << (sh - 1)] - hex[(2 * v) << (sh - 1)];
    uint64_t zb = block_exclusive_scan(sum, s_warp);
    uint64_t *obl = ob + (nodes - 1), *zel = ze + (nodes - 1);
    for (uint64_t v = lo; v < hi; v++) {
        const uint64_t z = hex[(2 * v + 1) << (sh - 1)] - hex[(2 * v) << (sh - 1)];
        obl[v] = hex[v << sh] - zb;
        zel[v] = zb + z;
        zb += z;
    }
}

cudaError_t launch_node_tables(const uint64_t *hex, uint32_t L, uint64_t *ob, uint64_t *ze, cudaStream_t st,
                               uint64_t *tmp) {
    if (L == 0) return cudaSuccess;
    // Levels with up to kSingleCtaMax nodes: one CTA each, one launch.
    uint32_t small = 0;
    while (small < L && (1ull << small) <= kSingleCtaMax) small++;
    if (tmp == nullptr) small = L;
    node_tables_kernel<<<small, kScanThreads, 0, st>>>(hex, L, ob, ze);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    for (uint32_t l = small; l < L && e == cudaSuccess; l++) {
        const uint64_t nodes = 1ull << l;
        e = scan_large(ZeroVal{hex, L - l}, TableOut{hex, L - l, ob + (nodes - 1), ze + (nodes - 1)}, nodes, tmp, st);
    }
    return e;
}

}  // namespace wt

namespace wt {

// ------------------------------------------------- node starts by rank
// Node tables of level l without a leaf histogram.  Node v of level l spans
// [C_l[v], C_l[v+1]); once level l's bitmap and rank directory exist, the
// ones before each boundary give everything the pass needs:
//   OB_l[v] = rank1_l(C_l[v])                      (ones before the node)
//   ZE_l[v] = C_l[v+1] - rank1_l(C_l[v+1])          (zeros through its end)
// and the children's starts on level l + 1 (Proposition 1: the zeros of
// node v form node 2v, its ones node 2v + 1):
//   C_{l+1}[2v] = C_l[v],  C_{l+1}[2v+1] = C_l[v+1] - rank1_l(C_l[v+1]) + rank1_l(C_l[v]).
// One thread per node.  start_in: 2^l + 1 entries; start_out: 2^(l+1) + 1
// (or nullptr on the last level).
__global__ void __launch_bounds__(256) rank_tables_kernel(LevelDesc lv, uint64_t nodes,
                                                          const uint64_t *__restrict__ start_in,
                                                          uint64_t *__restrict__ ob, uint64_t *__restrict__ ze,
                                                          uint64_t *__restrict__ start_out) {
    griddep_wait();
    const uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (v >= nodes) return;
    const uint64_t c0 = start_in[v], c1 = start_in[v + 1];
    const uint64_t r0 = rank1(lv, c0), r1 = rank1(lv, c1);
    ob[v] = r0;
    ze[v] = c1 - r1;
    if (start_out) {
        start_out[2 * v] = c0;
        start_out[2 * v + 1] = c1 - r1 + r0;
        if (v + 1 == nodes) start_out[2 * nodes] = c1;
    }
}

__global__ void root_starts_kernel(uint64_t n, uint64_t *start) {
    start[0] = 0;
    start[1] = n;
}

cudaError_t launch_root_starts(uint64_t n, uint64_t *start, cudaStream_t st) {
    root_starts_kernel<<<1, 1, 0, st>>>(n, start);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rank_tables(const LevelDesc &lv, uint32_t l, const uint64_t *start_in, uint64_t *ob,
                               uint64_t *ze, uint64_t *start_out, cudaStream_t st) {
    const uint64_t nodes = 1ull << l;
    const cudaError_t e = launch_dependent(rank_tables_kernel, (unsigned)ceil_div(nodes, 256), 256, 0, st, lv, nodes,
                                           start_in, ob, ze, start_out);
    note_launches(1);
    return e;
}

}  // namespace wt
