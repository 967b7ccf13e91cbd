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
constexpr uint32_t kErrBound = 4u;  // a merge found parts whose node starts do not fit their bitmaps

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

// ------------------------------------------------------- rank and select on a level
// (query.cu, merge.cu, matrix.cu)

// ones in B[0, 512 b): hyper entry plus the wrapped 32-bit block entry.
__device__ __forceinline__ uint64_t ones_before_block(const LevelDesc &d, uint64_t b) {
    const uint64_t hy = d.Hy[(b << 9) >> kSpanShift];
    return hy + (uint32_t)(d.R[b] - (uint32_t)hy);
}

// ones in B[0, i), 0 <= i <= n.
__device__ __forceinline__ uint64_t rank1(const LevelDesc &d, uint64_t i) {
    const uint64_t b = i >> 9;
    uint64_t r = ones_before_block(d, b);
    const uint32_t rem = (uint32_t)(i & 511);
    if (rem) {
        const uint4 *blk = reinterpret_cast<const uint4 *>(d.words + b * 16);
        const uint32_t full = rem >> 5, part = rem & 31;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if ((uint32_t)q * 4 > full) break;
            const uint4 x = __ldg(blk + q);
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t idx = q * 4 + k;
                if (idx < full)
                    r += __popc(w[k]);
                else if (idx == full && part)
                    r += __popc(w[k] & ((1u << part) - 1u));
            }
        }
    }
    return r;
}

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
__device__ inline uint64_t select_bit(const LevelDesc &d, uint64_t n, uint64_t nblocks, uint32_t bit, uint64_t k) {
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

// ------------------------------------------------------- TMA + mbarrier
// One-dimensional bulk copies global -> shared (cp.async.bulk) completing on
// an mbarrier.  Every wait is bounded by kWaitLimitNs of %globaltimer.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Programmatic dependent launch.  A kernel launched by launch_dependent may
// become resident while the kernel before it in the stream is still
// running (its launch and any prologue on its own shared memory overlap the
// other kernel's tail); griddep_wait then blocks the thread until that
// kernel has completed and its memory writes are visible.  Every kernel
// launched this way calls griddep_wait before its first global-memory
// access, so the stream's order of effects is unchanged.  (Outside such a
// launch the instruction returns at once.)  The host side is launch.cuh.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// Copy only (the caller arms the barrier once for all copies of a phase).
__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
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
// (after limit_ns of %globaltimer).
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    const uint32_t addr = smem_u32(bar);
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; i++) {
        if ((i & 1023u) == 1023u && global_ns() - t0 > limit_ns) return false;
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

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) { return mbar_wait_for(bar, phase, kWaitLimitNs); }

// ------------------------------------------------------ packed histogram
// Alphabets too large for 32-bit shared bins: 16-bit bins, two per shared
// word.  A bin that reaches 2^15 hands 2^15 to the global histogram at once,
// so a half-word never carries into its neighbour (fewer than 2^15 further
// additions can land before the hand-over, one per thread at most).
constexpr uint32_t kPackedMaxSigma = 96 * 1024;       // 192 KB of shared words
constexpr uint32_t kPackedThreads = 1024;

__device__ __forceinline__ void packed_add(uint32_t *w, uint64_t *hist, uint32_t s) {
    const uint32_t sh = 16 * (s & 1);
    const uint32_t old = atomicAdd(&w[s >> 1], 1u << sh);
    if (((old >> sh) & 0xffffu) == 0x7fffu) {
        atomicSub(&w[s >> 1], 0x8000u << sh);
        atomicAdd(reinterpret_cast<unsigned long long *>(&hist[s]), 0x8000ull);
    }
}

// Counts S[begin, end) (all threads of the CTA) into the shared words w
// (zeroed), then adds them to hist and clears w again.  Returns (in bad)
// whether a symbol was >= sigma.  sole: this CTA is the only one counting
// into hist (which is zero), so the counts are stored, not added; hand-overs
// of 2^15 still add, before the barrier that precedes the stores.
template <typename Sym>
__device__ __forceinline__ void packed_count(const Sym *__restrict__ S, uint64_t begin, uint64_t end, uint32_t sigma,
                                             uint32_t *w, uint64_t *hist, bool &bad, bool sole = false) {
    auto add = [&](uint32_t s) {
        if (s < sigma)
            packed_add(w, hist, s);
        else
            bad = true;
    };
    constexpr uint32_t kPer = 16 / sizeof(Sym);
    const uint64_t vbegin = (begin + kPer - 1) / kPer * kPer, vend = end / kPer * kPer;
    if ((reinterpret_cast<uintptr_t>(S) & 15) == 0 && vbegin < vend) {
        const uint4 *V = reinterpret_cast<const uint4 *>(S);
        for (uint64_t r = vbegin / kPer + threadIdx.x; r < vend / kPer; r += blockDim.x) {
            const uint4 q = __ldcs(V + r);
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (sizeof(Sym) == 2) {
                    add(w4[k] & 0xffffu);
                    add(w4[k] >> 16);
                } else {
                    add(w4[k]);
                }
            }
        }
        for (uint64_t k = begin + threadIdx.x; k < vbegin; k += blockDim.x) add((uint32_t)S[k]);
        for (uint64_t k = vend + threadIdx.x; k < end; k += blockDim.x) add((uint32_t)S[k]);
    } else {
        for (uint64_t k = begin + threadIdx.x; k < end; k += blockDim.x) add((uint32_t)S[k]);
    }
    __syncthreads();
    const uint32_t words = (sigma + 1) / 2;
    for (uint32_t j = threadIdx.x; j < words; j += blockDim.x) {
        const uint32_t v = w[j];
        if (sole) {
            if (v & 0xffffu) hist[2 * j] += v & 0xffffu;
            if (v >> 16) hist[2 * j + 1] += v >> 16;
        } else {
            if (v & 0xffffu)
                atomicAdd(reinterpret_cast<unsigned long long *>(&hist[2 * j]), (unsigned long long)(v & 0xffffu));
            if (v >> 16) atomicAdd(reinterpret_cast<unsigned long long *>(&hist[2 * j + 1]), (unsigned long long)(v >> 16));
        }
        w[j] = 0;
    }
    __syncthreads();
}

// ------------------------------------------------------------ launchers
// Every kernel launch of the library is counted (the profiler reports the
// launches made inside each timed call).
void note_launches(uint32_t k);

// (defined in build.cu / query.cu, called from abi.cu)

struct BuildScratch {
    uint64_t *hist;       // sigma
    uint64_t *hex;        // 2^L + 1
    uint64_t *ob;         // 2^L - 1 : ones before each node's start
    uint64_t *ze;         // 2^L - 1 : zeros up to each node's end
    uint64_t *scan_tmp;   // scan_tmp_bytes(L)
    void *job_slot;       // level_job_slot_bytes()
    uint32_t *cnt;        // tile counts of a level, lw_counts_bytes(n, width)
    uint64_t *pre;        // ones before each tile, lw_prefix_bytes(n, width)
    void *ping;           // n * width
    void *pong;           // n * width
};

// Kernel (a): histogram of S into hist (zeroed by the caller) and the symbol
// range check; then the exclusive scan into hex.
// Level 0's count pass folded into the histogram's read of S (1-byte
// symbols, S 16-byte aligned, n a multiple of the 8192-symbol tile): the level-0 bit (bit
// bsh) of every symbol goes to level 0's bitmap (words), the ones of every
// 512-symbol unit to cnt (the count pass's layout), and level 1's bitmap is
// zeroed (next, when level 0's pass writes it; else nullptr).
// For a pair step at level 0 it also writes bit L - 2 of every symbol to
// plane, the unit counts of ways 1 and 2 to cnt01 and cnt11, and zeroes
// next2 and plane3 (each when not nullptr).
struct Level0Fuse {
    uint32_t *words, *cnt, *next;
    uint32_t bsh;
    uint32_t *plane = nullptr, *cnt01 = nullptr, *cnt11 = nullptr, *next2 = nullptr, *plane3 = nullptr;
};
bool level0_fusable(const void *S, uint64_t n, int width, uint64_t sigma);
cudaError_t launch_histogram(const void *S, uint64_t n, int width, uint64_t sigma, uint64_t *hist,
                             uint32_t *err, cudaStream_t st, const Level0Fuse *fuse = nullptr);
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
// Node tables without a histogram (large alphabets): C_0 = {0, n}; after
// level l's count and scan, level l's tables and C_{l+1} from rank1 of
// level l at the node boundaries C_l (start_out nullptr on the last level).
cudaError_t launch_root_starts(uint64_t n, uint64_t *start, cudaStream_t st);
cudaError_t launch_rank_tables(const LevelDesc &lv, uint32_t l, const uint64_t *start_in, uint64_t *ob,
                               uint64_t *ze, uint64_t *start_out, cudaStream_t st);

// Kernels (b)+(c): the level passes (level.cu).  Each level: a count pass
// stores the level-l ones of every tile of P_l, a scan turns them into each
// tile's prefix, and the pass writes the level and places P_{l+1}.
uint32_t lw_tile_elems(int width);
size_t lw_counts_bytes(uint64_t n, int width);   // tile counts (uint32)
size_t lw_prefix_bytes(uint64_t n, int width);   // tile prefixes (uint64, padded) and scan sums
size_t level_job_slot_bytes();

// One sequence's share of a level launch (a batch launches many at once).
struct __align__(16) LevelJob {
    const void *cur;
    void *nxt;                 // nullptr on the sequence's last level
    uint64_t n, nblocks, nspans;
    uint32_t L;                // the sequence's number of levels
    uint32_t ntiles;           // its tiles at this width
    LevelDesc lv;              // its level-l arrays
    uint64_t *ones_out;
    const uint64_t *ob, *ze;   // its level-l node tables
    uint32_t *cnt;             // lw_counts_bytes: ones of each unit on level l
    uint64_t *pre;             // lw_prefix_bytes: ones before each unit
    uint32_t *next_words;      // level l + 1's bitmap when this pass writes it, else nullptr
};

LevelJob make_level_job(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l, const uint64_t *ob,
                        const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint32_t *cnt, uint64_t *pre,
                        uint32_t *next_words);
size_t level_job_bytes();
// At most how many node boundaries P_l of one sequence has: level l has
// 2^l nodes, at most sigma of them and at most n non-empty.
inline uint64_t level_boundaries(uint64_t n, uint64_t sigma, uint32_t l) {
    uint64_t m = l < 63 ? (1ull << l) : ~0ull;
    if (sigma < m) m = sigma;
    if (n < m) m = n;
    return m ? m - 1 : 0;
}
// Whether the pass of level l writes level l + 1's bitmap (from its split
// copies), so that level l + 1's count pass reads n/8 bytes instead of n w:
// for 1- and 2-byte symbols (for 4-byte symbols the pass's extra reads of
// its split copy cost as much as the count pass saves), and when at most one
// tile in 64 spans a node boundary, so the tiles placed symbol by symbol
// (whose bits go out one atomicOr each) are few.  Otherwise level l + 1's
// count pass writes the bitmap from the symbols.
inline bool pass_writes_next_bits(uint64_t boundaries, uint64_t tiles, int width) {
    return width <= 2 && boundaries * 64 < tiles;
}
// ------------------------------------------------------- two levels per pass
// (pair.cu) A pair step builds levels l and l + 1 with one read of P_l and
// places every symbol straight into P_{l+2}.  Its count pass stores three
// counts per unit of P_l: the level-l ones (way 0), the symbols with bits
// (l, l + 1) = (0, 1) (way 1) and (1, 1) (way 2); the prefix scan turns each
// into unit prefixes.  The ways live in one array each, way w at offset
// w * stride.
constexpr uint32_t kScanSegUnits = 8192;  // units per segment of the prefix scan (8 per thread)
__host__ __device__ inline uint64_t way_cnt_stride(uint64_t units) { return (units + 3) & ~3ull; }
__host__ __device__ inline uint64_t way_pre_stride(uint64_t units) {
    return (units + 2 + ceil_div(units, kScanSegUnits) + 1 + 1) & ~1ull;
}

// One sequence's share of a pair launch.  Bitmaps written here (next1,
// next2, plane3) must be zero where this step does not store whole words:
// the count pass zeroes them.
struct __align__(16) PairJob {
    const void *cur;           // P_l
    void *nxt;                 // P_{l+2}; nullptr when no later pass reads it
    uint64_t n, nblocks;
    uint32_t L, ntiles;
    uint32_t *words;           // level l's bitmap (the count pass writes it when it reads the symbols)
    uint32_t *plane;           // bit l + 1 of P_l, packed like a bitmap
    uint32_t *next1;           // level l + 1's bitmap
    uint32_t *next2;           // level l + 2's bitmap, or nullptr
    uint32_t *plane3;          // bit l + 3 of P_{l+2}, packed like a bitmap, or nullptr
    const uint64_t *ob, *ze;   // level l's node tables
    const uint64_t *T;         // level l's pair table (4 per node), nullptr when l + 2 = L
    uint32_t *cnt;             // unit counts, three ways
    uint64_t *pre;             // unit prefixes, three ways
    uint32_t need_b;           // l + 2 < L: the symbols are split into their P_{l+2} runs
    uint32_t pad;
};
// Pair table of level l: T[4 v + g] = C_{l+2}[4 v + g] - (symbols of group g
// in the nodes before v), for every node v with 2^l <= kPairMaxNodes; a
// symbol of group g at position p of P_l, in node v, goes to
// T[4 v + g] + (symbols of group g in P_l[0, p)).  Level l's table starts at
// entry pair_table_offset(l).
constexpr uint32_t kPairMaxLevel = 16;
inline uint64_t pair_table_offset(uint32_t l) { return 4 * ((1ull << l) - 1); }
inline size_t pair_table_bytes(uint32_t lmax) { return 8 * 4 * ((1ull << (lmax + 1)) - 1); }
// levels: bit l set for every level whose table is wanted (all l + 2 < L).
cudaError_t launch_pair_tables(const uint64_t *hex, uint32_t L, uint32_t levels, uint64_t *T, cudaStream_t st);
size_t pair_job_slot_bytes();
// One pair step of one sequence (job_slot: pair_job_slot_bytes()): the
// count pass (from_bits: from level l's bitmap and plane l + 1, else from
// the symbols; counted: the counts are already in place), the three-way
// prefix scan with level l's directory (lv, ones_out), the pair pass, then
// level l + 1's directory from the bitmap the pass wrote (lv1, ones1_out).
cudaError_t launch_pair_step(const PairJob &j, int width, uint32_t l, LevelDesc lv, uint64_t *ones_out,
                             LevelDesc lv1, uint64_t *ones1_out, bool from_bits, bool counted, uint32_t *cnt1,
                             uint64_t *pre1, uint32_t *err, void *job_slot, cudaStream_t st);

// Level l of every job (all of one width): counts (from the symbols, which
// also writes level l's bitmap, or from_bits: from that bitmap), prefix
// scan with the rank directory, and (do_pass) the pass that places P_{l+1}.
// max_job_tiles: the most tiles of any one job.
// counted: the units' counts (and level l's bitmap) are already in place
// (level 0 folded into the histogram): no count pass.
// rt: compute the level's node tables (and the next level's node starts)
// from its directory between the scan and the pass (launch_rank_tables).
// check_sigma > 0: the count from the symbols flags any symbol >= it.
struct RankTables {
    LevelDesc lv;
    const uint64_t *start_in;
    uint64_t *ob, *ze, *start_out;
};
cudaError_t launch_level_jobs(int width, uint32_t l, const LevelJob *jobs, const uint32_t *tile_start, uint32_t njobs,
                              uint32_t total_tiles, uint32_t max_job_tiles, bool from_bits, bool do_pass,
                              uint32_t *err, cudaStream_t st, bool counted = false, const RankTables *rt = nullptr,
                              uint32_t check_sigma = 0, bool one_node = false, bool bits = false);
// bits: some job of the launch stores no order (the level before its last)
// while handing over the next bitmap (1-byte codes take lw_bits_tile).
// One sequence (job_slot: level_job_slot_bytes() of device memory).
// one_node: every node of level l has the same offsets (the wavelet
// matrix), so every tile is placed as one node whatever its keys.
cudaError_t launch_level_pass(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l,
                              const uint64_t *ob, const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint32_t *cnt,
                              uint64_t *pre, bool from_bits, uint32_t *next_words, uint32_t *err, void *job_slot,
                              cudaStream_t st, bool counted = false, const RankTables *rt = nullptr,
                              uint32_t check_sigma = 0, bool one_node = false);

// The prefix scan alone of level l (ways count arrays, way 0 with the
// directory), over jobs already in device memory.
cudaError_t launch_level_scans(int width, uint32_t l, const LevelJob *jobs, uint32_t njobs, uint32_t max_job_tiles,
                               uint32_t ways, cudaStream_t st);
// The count pass of level l alone, from the symbols cur (writes level l's
// bitmap and unit counts, zeroes next_words when not nullptr, flags symbols
// >= check_sigma when it is > 0); launch_level_pass with counted = true
// then runs the scan and the pass.
cudaError_t launch_level_count(const void *cur, uint64_t n, int width, uint32_t L, uint32_t l, LevelDesc lv,
                               uint32_t *cnt, uint32_t *next_words, uint32_t *err, void *job_slot, cudaStream_t st,
                               uint32_t check_sigma);
// Level l's directory from its bitmap (already written): count from the
// bitmap and the prefix scan, no pass.
cudaError_t launch_level_directory(uint64_t n, int width, uint32_t L, uint32_t l, LevelDesc lv, uint64_t *ones_out,
                                   uint32_t *cnt, uint64_t *pre, uint32_t *err, void *job_slot, cudaStream_t st);

// Merge of partial trees (merge.cu).  parts: device array of k device
// descriptors of trees with the same alphabet.  launch_merge_starts
// recovers every part's node starts into hex (k x (2^L + 1) uint64) and
// their sums into hex_out (2^L + 1); launch_merge_level writes level l of the
// concatenation (n bits, padded to whole 512-bit blocks) into words.
cudaError_t launch_merge_starts(const TreeDesc *const *parts, uint32_t k, uint32_t L, uint64_t *hex,
                                uint64_t *hex_out, uint32_t *err, cudaStream_t st);
cudaError_t launch_merge_level(const TreeDesc *const *parts, uint32_t k, uint32_t L, uint32_t l, const uint64_t *hex,
                               const uint64_t *hex_out, uint64_t n, uint32_t *words, uint32_t *err,
                               cudaStream_t st);

// The wavelet matrix (matrix.cu): node tables OB_l = 0, ZE_l = Z_l for every
// level from the leaf starts hex, and the matrix's queries.
cudaError_t launch_wm_tables(const uint64_t *hex, uint32_t L, uint64_t *ob, uint64_t *ze, cudaStream_t st);
cudaError_t launch_wm_access(const TreeDesc *t, const uint64_t *i, uint64_t m, uint32_t *out, cudaStream_t st);
cudaError_t launch_wm_rank(const TreeDesc *t, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                           cudaStream_t st);
cudaError_t launch_wm_select(const TreeDesc *t, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                             cudaStream_t st);

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
// Histogram work of a sequence: tiles of the shared-bin kernel (small and
// very large alphabets) and slabs of the packed kernel (the rest).
uint32_t batch_hist_tiles(uint64_t n, uint64_t sigma);
uint32_t batch_hist_slabs(uint64_t n, uint64_t sigma);
// Node starts and tables: sequences with 2^L <= kBatchWarpLeaves take one
// warp each (small_seqs); the others one CTA for the starts (big_seqs), one
// CTA per level with more than kBatchWarpLeaves nodes (big_pairs) and one
// warp per other level (small_pairs); a pair is sequence << 5 | level.
constexpr uint32_t kBatchWarpLeaves = 1024;
inline bool batch_small_alphabet(uint32_t L) { return (1ull << L) <= kBatchWarpLeaves; }
cudaError_t launch_batch_prepare(const SeqJob *jobs, uint32_t nseq, const uint32_t *hist_tile_start,
                                 uint32_t hist_tiles, const uint32_t *slab_start, uint32_t slabs,
                                 const uint32_t *small_seqs, uint32_t nsmall, const uint32_t *big_seqs,
                                 uint32_t nbig, const uint32_t *big_pairs, uint32_t nbig_pairs,
                                 const uint32_t *small_pairs, uint32_t nsmall_pairs, cudaStream_t st);

// Alphabet remapping (remap.cu): mark the codes of S in the alphabet
// bitmap A (zeroed; codes >= universe set kErrSymbol in err), and map S to
// S'[j] = rank1(A, S[j]) with out_width bytes per code.
cudaError_t launch_alpha_mark(const void *S, uint64_t n, int width, uint64_t universe, uint32_t *A, uint32_t *err,
                              cudaStream_t st);
cudaError_t launch_alpha_map(const void *S, uint64_t n, int width, const LevelDesc &A, void *out, int out_width,
                             cudaStream_t st);
// Queries on a tree of remapped codes (query.cu); A with its directory and ones.
cudaError_t launch_access_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint64_t *i,
                                uint64_t m, uint32_t *out, cudaStream_t st);
cudaError_t launch_rank_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint32_t *c,
                              const uint64_t *i, uint64_t m, uint64_t *out, cudaStream_t st);
cudaError_t launch_select_remap(const TreeDesc *t, const LevelDesc &A, uint64_t universe, const uint32_t *c,
                                const uint64_t *j, uint64_t m, uint64_t *out, cudaStream_t st);

// Kernel (e): queries.
cudaError_t launch_access(const TreeDesc *t, const uint64_t *i, uint64_t m, uint32_t *out, cudaStream_t st);
cudaError_t launch_rank(const TreeDesc *t, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                        cudaStream_t st);
cudaError_t launch_select(const TreeDesc *t, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                          cudaStream_t st);
cudaError_t launch_query_multi(const TreeDesc *const *trees, uint32_t ntrees, const uint32_t *tree_idx,
                               const uint8_t *op,
                               const uint32_t *c, const uint64_t *arg, uint64_t m, uint64_t *out,
                               cudaStream_t st);

}  // namespace wt
