// level.cu -- kernels (b) + (c): the level step of the level-wise build
// (count pass, prefix scan with the rank directory, and the fused pass).
//
// One pass over P_l (the symbols in level-l order) places, per tile of 8 KB,
// every symbol at its position in P_{l+1}:
//          bit 0:  dst = zeros_before(p) + OB_l[v]
//          bit 1:  dst = ones_before(p)  + ZE_l[v]
// with v = key_l(s), OB_l[v] = ones on level l before node v's start and
// ZE_l[v] = zeros on level l up to node v's end.  This is the stable
// counting-sort placement of Algorithm 1 ("bitmapSetBit at C[node]++",
// Section 3.1) written as a closed form of two prefix counts, so one global
// scan serves every node of the level.
//
// Where the ones before a position come from: a count pass stores the
// level-l ones of every unit (a warp's 1 KB range of a tile, or a 512-symbol
// rank block when that is shorter); a segmented scan turns them into
// prefixes before the pass starts.  The same scan writes the level's rank
// directory (R, Hy) and select samples (S1, S0), since the prefix at a rank
// block's first unit is R itself.  So the tiles of a pass are independent,
// and inside a tile every warp starts from its own prefix: no CTA waits for
// another and no warp for the others' counts.
//
// Where level l's bitmap comes from: for 1- and 2-byte symbols, on levels
// with few node boundaries, the pass of level l - 1 writes it from its
// shared split copy of P_l (every 32 consecutive symbols there are one
// bitmap word), and the count pass only popcounts it; otherwise the count
// pass writes it from the symbols.  The last level therefore needs no pass.
//
// GPU structure of the pass: a persistent CTA of 128 threads takes a
// contiguous range of tiles and keeps two stages: the last warp claims a
// tile one ahead and one thread issues TMA bulk copies (cp.async.bulk) of its
// symbols, its unit prefixes and its slice of level l's bitmap into a
// shared-memory stage while the CTA works on the current one.  Per tile:
//   * a lane owns 8 consecutive bytes of each 256-byte warp step, so its
//     level bits are 8 (4, 2) consecutive bits of the bitmap copy; per-lane
//     counts of three steps share one shuffle scan;
//   * when the whole tile lies in one node (the common case: nodes are far
//     larger than a tile except on the deepest levels of large alphabets),
//     its zeros and ones go to two contiguous runs of P_{l+1}: every symbol
//     is written into a shared-memory split copy of the two runs laid out at
//     the destination's offset within a 32-symbol bitmap word (which also
//     agrees with the destination modulo 16 bytes); for whole tiles of
//     1-byte symbols one byte permutation per 8-byte chunk puts its zeros
//     first and its ones after, so each byte's place is the chunk's first
//     zero or first one plus a constant; otherwise each lane walks its
//     symbols with one running pointer.  The aligned interior of each run
//     leaves with one bulk store, the ragged ends with byte stores.
//     Tiles that span several nodes store every symbol at its own
//     destination.
//   * one CTA barrier per tile: it hands the split copy to the threads that
//     bulk-store it and write the next bitmap's words, and the next stage to
//     every thread.
// The only waits are on the bulk copies, bounded like every wait of the
// library.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.cuh"
#include "level_common.cuh"

namespace wt {

uint32_t lw_tile_elems(int width) { return kLwTileBytes / (uint32_t)width; }
size_t lw_counts_bytes(uint64_t n, int width) {
    return (size_t)ceil_div(n, lw_tile_elems(width)) * lw_units((uint32_t)width) * 4;
}
// A prefix per unit, the total and one spare (the pass copies a tile's units
// + 2), then one sum per scan segment.
size_t lw_prefix_bytes(uint64_t n, int width) {
    const uint64_t nc = ceil_div(n, lw_tile_elems(width)) * lw_units((uint32_t)width);
    return (size_t)(nc + 2 + ceil_div(nc, kScanSeg) + 1) * 8;
}

// ---------------------------------------------------------------- counts

// The level-l ones of every unit of P_l.  One warp per tile (kUnits units),
// the warps of the grid striding over the tiles together; each warp finds a
// tile's job by binary search from its previous one.  Two kinds:
//   kFromBits = false: read the symbols of P_l (four 16-byte loads per lane
//     in flight), count the symbols with bit L - 1 - l set, and write those
//     bits as level l's bitmap;
//   kFromBits = true: level l's bitmap was written by the pass of level
//     l - 1; popcount it (n/8 bytes instead of n w).
// (When this level's pass will write level l + 1's bitmap, J.next_words,
// scan_segs_kernel zeroes that bitmap's padding beyond n; the pass writes
// every bit below n: whole words by plain stores, words shared by runs
// bit-exactly by atomics.)
constexpr int kCountThreads = 256;
constexpr int kCountWarps = kCountThreads / 32;

template <typename Sym, bool kFromBits>
__global__ void __launch_bounds__(kCountThreads, 4) count_kernel(LevelLaunch a) {
    using Cfg = LwCfg<Sym>;
    constexpr uint32_t kU = Cfg::kUnits;
    constexpr uint32_t kUnitSyms = Cfg::kTile / kU;
    constexpr uint32_t kTileWords = Cfg::kTile / 32;  // bitmap words of a tile
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kCountWarps;
    const uint32_t bsh_l = 1 + a.l;
    bool bad = false;  // a symbol >= a.check_sigma (count from the symbols only)
    uint32_t k = 0;
    for (uint32_t g = blockIdx.x * kCountWarps + (threadIdx.x >> 5); g < a.total_tiles; g += nwarps) {
        if (k + 1 < a.njobs && a.tile_start[k + 1] <= g) {
            uint32_t lo = k + 1, hi = a.njobs - 1;  // the last job starting at or before g
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.tile_start[mid] <= g)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            k = lo;
        }
        const LevelJob &J = a.jobs[k];
        const uint32_t tile = g - a.tile_start[k];
        const uint64_t base = (uint64_t)tile * Cfg::kTile;
        const uint64_t w0 = base / 32;            // the tile's first bitmap word
        const uint64_t nwords = J.nblocks * 16;   // bitmap words of the level
        uint32_t c[kU];
#pragma unroll
        for (int j = 0; j < (int)kU; j++) c[j] = 0;
        if (kFromBits) {
            constexpr uint32_t kWU = kUnitSyms / 32;  // words per unit
            const uint32_t *words = J.lv.words;
            if (w0 + kTileWords <= nwords) {
                // A whole tile: 16-byte loads, four lanes to a unit's 16
                // words, the unit's count reduced by two shuffles.
                static_assert(kWU == 16, "four lanes to a unit");
                constexpr int kVR = (int)((kTileWords + 127) / 128);
#pragma unroll
                for (int r = 0; r < kVR; r++) {
                    const uint32_t wo = (uint32_t)r * 128 + 4 * lane;  // the lane's first word in the tile
                    uint32_t pc = 0;
                    if (wo < kTileWords) {
                        const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(words + w0 + wo));
                        pc = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                    }
                    pc += __shfl_xor_sync(0xffffffffu, pc, 1);
                    pc += __shfl_xor_sync(0xffffffffu, pc, 2);
                    if ((lane & 3) == 0 && wo < kTileWords) J.cnt[(size_t)tile * kU + wo / kWU] = pc;
                }
                continue;
            }
            constexpr int kRows = (int)(kTileWords / 32), kSub = (int)(32 / kWU);
            const uint32_t mysub = (uint32_t)lane / kWU;
#pragma unroll
            for (int r = 0; r < kRows; r++) {
                const uint64_t w = w0 + (uint32_t)r * 32 + lane;
                const uint32_t pc = w < nwords ? __popc(__ldcs(words + w)) : 0u;
#pragma unroll
                for (int sub = 0; sub < kSub; sub++) c[r * kSub + sub] += mysub == (uint32_t)sub ? pc : 0u;
            }
        } else {
            constexpr int kVecs = (int)(kLwTileBytes / 512);  // 16-byte loads per lane per tile
            constexpr int kPerUnit = kVecs / (int)kU;
            const Sym *S = static_cast<const Sym *>(J.cur);
            const uint32_t cnt = (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
            const uint32_t bsh = J.L - bsh_l;
            unsigned char *bm = reinterpret_cast<unsigned char *>(J.lv.words);
            if (cnt == Cfg::kTile && (reinterpret_cast<uintptr_t>(S) & 15) == 0) {
                const uint4 *v = reinterpret_cast<const uint4 *>(S + base) + lane;
                // The lane's chunk of load r is 16 (8, 4) consecutive bits of
                // the bitmap, at byte (base + (512 r + 16 lane) / w) / 8.
                unsigned char *bl = bm + base / 8 + (16 * lane / sizeof(Sym)) / 8;
                const BitGather gg = bit_gather<Sym>(bsh);
#pragma unroll
                for (int h = 0; h < kVecs; h += 4) {
                    uint4 w[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) w[r] = __ldcs(v + (h + r) * 32);
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const uint32_t x[4] = {w[r].x, w[r].y, w[r].z, w[r].w};
                        const uint32_t hb = gather_bits<Sym>(x, gg, bsh);
                        if (a.check_sigma) bad |= chunk_out_of_range<Sym>(x, a.check_sigma);
                        c[(h + r) / kPerUnit] += __popc(hb);
                        unsigned char *d = bl + (h + r) * (512 / sizeof(Sym) / 8);
                        if (sizeof(Sym) == 1) *reinterpret_cast<uint16_t *>(d) = (uint16_t)hb;
                        if (sizeof(Sym) == 2) *d = (unsigned char)hb;
                        if (sizeof(Sym) == 4) {
                            const uint32_t nb = __shfl_down_sync(0xffffffffu, hb, 1);
                            if ((lane & 1) == 0) *d = (unsigned char)(hb | (nb << 4));
                        }
                    }
                }
            } else {
                uint32_t *words = J.lv.words;
#pragma unroll
                for (int j = 0; j < (int)kU; j++)
                    for (uint32_t p0 = j * kUnitSyms; p0 < (j + 1) * kUnitSyms; p0 += 32) {
                        const uint32_t p = p0 + lane;
                        const uint32_t sv = p < cnt ? (uint32_t)S[base + p] : 0u;
                        if (a.check_sigma && sv >= a.check_sigma) bad = true;
                        const uint32_t bit = p < cnt ? (sv >> bsh) & 1u : 0u;
                        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
                        c[j] += bit;
                        if (lane == 0 && w0 + p0 / 32 < nwords) words[w0 + p0 / 32] = bal;
                    }
            }
        }
        uint32_t mine = 0;  // lane j < kU stores unit j's count
#pragma unroll
        for (int j = 0; j < (int)kU; j++) {
            const uint32_t t = __reduce_add_sync(0xffffffffu, c[j]);
            if (lane == j) mine = t;
        }
        if (lane < (int)kU) J.cnt[(size_t)tile * kU + lane] = mine;
    }
    if (bad) atomicOr(a.err, kErrSymbol);
}

// Unit prefixes of every job, pre[u] = ones of the job's units before u, in
// two launches over segments of kScanSeg units (CTA x = job * segs + seg):
// the sums of the segments, then each segment's scan from the sums of the
// segments before it.
// With a.ways = 3 (a pair step) blockIdx.y picks the count array; only way 0
// (the level-l ones) writes the directory.
__global__ void __launch_bounds__(1024) scan_sums_kernel(LevelLaunch a) {
    __shared__ uint32_t part[32];
    griddep_wait();
    const uint32_t job = blockIdx.x / a.segs, seg = blockIdx.x % a.segs;
    const LevelJob &J = a.jobs[job];
    const uint32_t nt = J.ntiles * a.units;  // units
    if (seg * kScanSeg >= nt && !(seg == 0 && nt == 0)) return;
    const uint32_t *cnt = J.cnt + blockIdx.y * way_cnt_stride(nt);
    uint64_t *pre = J.pre + blockIdx.y * way_pre_stride(nt);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t c = 0;
#pragma unroll
    for (int r = 0; r < (int)(kScanSeg / 1024); r++) {
        const uint32_t t = seg * kScanSeg + r * 1024 + tid;
        if (t < nt) c += cnt[t];
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) part[warp] = c;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = part[lane];
        v = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0) pre[nt + 2 + seg] = v;
    }
}

constexpr uint32_t kFoldNodes = 4096;

// Level l's node tables by rank at the node boundaries C_l (the work of
// rank_tables_kernel, which states the formulas), done by the last CTA of
// the scan to finish: every CTA fences its directory writes and counts
// itself done; the CTA that completes the count fences again and reads the
// whole directory.  All threads of the CTA call this once.
__device__ __forceinline__ void fold_rank_tables(const LevelLaunch &a) {
    __shared__ uint32_t s_last;
    if (!a.rt_nodes) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.rt_done, 1u) + 1 == gridDim.x * gridDim.y;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const LevelDesc lv = a.jobs[0].lv;
    for (uint32_t v = threadIdx.x; v < a.rt_nodes; v += blockDim.x) {
        const uint64_t c0 = a.rt_start_in[v], c1 = a.rt_start_in[v + 1];
        const uint64_t r0 = rank1(lv, c0), r1 = rank1(lv, c1);
        a.rt_ob[v] = r0;
        a.rt_ze[v] = c1 - r1;
        if (a.rt_start_out) {
            a.rt_start_out[2 * v] = c0;
            a.rt_start_out[2 * v + 1] = c1 - r1 + r0;
            if (v + 1 == a.rt_nodes) a.rt_start_out[2 * a.rt_nodes] = c1;
        }
    }
}

__global__ void __launch_bounds__(1024) scan_segs_kernel(LevelLaunch a) {
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_bpart[32];
    __shared__ uint64_t s_base;
    griddep_wait();
    const uint32_t job = blockIdx.x / a.segs, seg = blockIdx.x % a.segs;
    const LevelJob &J = a.jobs[job];
    const uint32_t nt = J.ntiles * a.units;  // units
    if (seg * kScanSeg >= nt && !(seg == 0 && nt == 0)) {
        fold_rank_tables(a);
        return;
    }
    const uint32_t way = blockIdx.y;
    if (way == 0 && seg == 0 && J.next_words && threadIdx.x < 32) {
        // Level l + 1's padding beyond n (the rest of its last 512-bit
        // block), which the pass leaves alone.
        for (uint64_t w = J.n / 32 + threadIdx.x; w < J.nblocks * 16; w += 32) J.next_words[w] = 0u;
    }
    const uint32_t *cnt = J.cnt + way * way_cnt_stride(nt);
    uint64_t *pre = J.pre + way * way_pre_stride(nt);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // The sums of the segments before this one: one load per thread per 1024
    // segments, in flight with the count loads below and reduced beside the
    // warp totals (no load waits on another).
    uint64_t bsum = 0;
    for (uint32_t s2 = tid; s2 < seg; s2 += 1024) bsum += pre[nt + 2 + s2];
    // kPer consecutive units per thread, read and written 16 bytes at a time
    // where the segment is whole.  A unit holds at most 512 ones, so the
    // sums of a thread, a warp and the CTA fit 32 bits.
    constexpr int kPer = (int)(kScanSeg / 1024);
    const uint32_t t0 = seg * kScanSeg + kPer * tid;
    const bool whole = t0 + kPer <= nt;
    uint32_t c[kPer];
    if (whole) {
#pragma unroll
        for (int h = 0; h < kPer / 4; h++) {
            const uint4 v = reinterpret_cast<const uint4 *>(cnt + t0)[h];
            c[4 * h] = v.x;
            c[4 * h + 1] = v.y;
            c[4 * h + 2] = v.z;
            c[4 * h + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kPer; k++) c[k] = t0 + k < nt ? cnt[t0 + k] : 0u;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) sum += c[k];
    uint32_t inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, d);
    if (lane == 31) s_warp[warp] = inc;
    if (lane == 0) s_bpart[warp] = bsum;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = (uint32_t)s_warp[lane];
        uint32_t winc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, winc, d);
            if (lane >= d) winc += y;
        }
        s_warp[lane] = winc - w;
        uint64_t bb = s_bpart[lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, d);
        if (lane == 0) s_base = bb;
    }
    __syncthreads();
    const uint64_t run0 = s_base + s_warp[warp] + (inc - sum);
    uint64_t pv[kPer];  // pre[t0 + k]
    {
        uint64_t r = run0;
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            pv[k] = r;
            r += c[k];
        }
    }
    if (whole) {
#pragma unroll
        for (int h = 0; h < kPer / 2; h++)
            reinterpret_cast<ulonglong2 *>(pre + t0)[h] = make_ulonglong2(pv[2 * h], pv[2 * h + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < kPer; k++)
            if (t0 + k < nt) pre[t0 + k] = pv[k];
    }
    // The rank directory of level l (Section 2.2's R, Hy and select
    // samples) from the same prefixes: a rank block starts at every upb-th
    // unit; the samples of the ones (zeros) that fall in a block point to it.
    const uint32_t upb = a.upb;
    if (way == 0) {
        const bool vec_r = whole && upb == 1 && t0 + kPer <= J.nblocks &&
                           (reinterpret_cast<uintptr_t>(J.lv.R + t0) & 15) == 0;
        if (vec_r) {
#pragma unroll
            for (int h = 0; h < kPer / 4; h++)
                reinterpret_cast<uint4 *>(J.lv.R + t0)[h] =
                    make_uint4((uint32_t)pv[4 * h], (uint32_t)pv[4 * h + 1], (uint32_t)pv[4 * h + 2],
                               (uint32_t)pv[4 * h + 3]);
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const uint32_t t = t0 + k;
            const uint64_t b = upb == 1 ? t : t / upb;  // every unit is a rank block for all widths
            if (t < nt && (upb == 1 || t % upb == 0) && b < J.nblocks) {
                const uint64_t run = pv[k];
                const uint64_t next = run + c[k] + (upb == 2 && k + 1 < kPer ? c[k + 1] : 0u);
                if (!vec_r) J.lv.R[b] = (uint32_t)run;
                if ((b & kBlocksPerSpanMask) == 0) J.lv.Hy[b >> (kSpanShift - 9)] = run;
                for (uint64_t k2 = ceil_div(run, kSample); k2 * kSample < next; k2++) J.lv.S1[k2] = (uint32_t)b;
                const uint64_t p0 = b * 512, p1 = min(p0 + 512, J.n);
                for (uint64_t k2 = ceil_div(p0 - run, kSample); k2 * kSample < p1 - next; k2++)
                    J.lv.S0[k2] = (uint32_t)b;
            }
        }
    }
    if (t0 < nt && nt <= t0 + kPer) {  // the total, read with the last tile's prefixes
        const uint64_t total = pv[kPer - 1] + c[kPer - 1];
        pre[nt] = total;
        if (way == 0) {
            J.lv.R[J.nblocks] = (uint32_t)total;
            J.lv.Hy[J.nspans] = total;
            *J.ones_out = total;
        }
    }
    fold_rank_tables(a);
}

// ------------------------------------------------------------------ pass

// One input stage: a tile, its sequence, its prefix, and its symbols.
struct __align__(16) LwStage {
    uint64_t pre[kLwMaxUnits + 2];  // pre[u] of the tile's units u and the next tile's first (one copy)
    LevelJob J;
    uint32_t tile;             // kNoTile: this CTA has no more tiles
    uint32_t full;             // a whole tile, 16-byte aligned: its symbols came in by bulk copy
    uint32_t skip;             // the job's last level: nothing to place
    uint32_t bits_bytes;       // bytes of level l's bitmap copied for the tile
};

struct LwShared {
    LwStage st[kLwStages];
    LevelJob job;                          // the job of the claimer's latest tile
    uint64_t bar[kLwStages];               // a stage is in place
    uint32_t lut[256];                     // zeros_first_perm of every chunk's level bits (1-byte symbols)
};

// Claims this CTA's tile g into stage s (the claiming warp, all lanes): the stage
// record (copied by the lanes) and, by bulk copy, the tile's chunk prefixes
// and (whole aligned tiles) the symbols.  k and have_job are the same in every lane.
template <typename Sym>
__device__ __forceinline__ void lw_claim(const LevelLaunch &a, LwShared &sh, unsigned char *in, int s, uint32_t g,
                                         uint32_t g_end, uint32_t &k, bool &have_job) {
    using Cfg = LwCfg<Sym>;
    constexpr int kJobWords = (int)(sizeof(LevelJob) / 8);
    const int lane = threadIdx.x & 31;
    LwStage &S = sh.st[s];
    if (g >= g_end) {
        if (lane == 0) {
            S.tile = kNoTile;
            S.full = 0;
            mbar_arrive(&sh.bar[s]);
        }
        return;
    }
    while (k + 1 < a.njobs && a.tile_start[k + 1] <= g) {
        k++;
        have_job = false;
    }
    if (!have_job) {
        if (lane < kJobWords)
            reinterpret_cast<uint64_t *>(&sh.job)[lane] = reinterpret_cast<const uint64_t *>(a.jobs + k)[lane];
        have_job = true;
        __syncwarp();
    }
    if (lane < kJobWords) reinterpret_cast<uint64_t *>(&S.J)[lane] = reinterpret_cast<const uint64_t *>(&sh.job)[lane];
    __syncwarp();
    if (lane == 0) {
        const uint32_t tile = g - a.tile_start[k];
        const uint64_t base = (uint64_t)tile * Cfg::kTile;
        // Nothing to place on a sequence's last level.  A pass with no next
        // order to store (the next level is the last) still splits its tiles
        // to hand that level its bitmap.
        const bool skip = S.J.nxt == nullptr && S.J.next_words == nullptr;
        const bool full = !skip && S.J.n - base >= Cfg::kTile && (reinterpret_cast<uintptr_t>(S.J.cur) & 15) == 0;
        S.tile = tile;
        S.full = full;
        S.skip = skip;
        fence_proxy_async_smem();
        // Level l's bitmap over the tile (written by the count pass or by
        // the pass of level l - 1), clamped to the bitmap's 512-bit blocks.
        const uint32_t bits_bytes =
            skip ? 0u : (uint32_t)min((uint64_t)(Cfg::kTile / 8), S.J.nblocks * 64 - base / 8);
        S.bits_bytes = bits_bytes;
        mbar_arrive_expect(&sh.bar[s], Cfg::kPreCopy * 8 + (full ? kLwTileBytes : 0) + bits_bytes);
        bulk_copy(S.pre, S.J.pre + (size_t)tile * Cfg::kUnits, Cfg::kPreCopy * 8, &sh.bar[s]);
        if (full)
            bulk_copy(in + s * kLwTileBytes, static_cast<const Sym *>(S.J.cur) + base, kLwTileBytes, &sh.bar[s]);
        if (bits_bytes)
            bulk_copy(in + kLwStages * kLwTileBytes + s * kLwStageBits,
                      reinterpret_cast<const unsigned char *>(S.J.lv.words) + base / 8, bits_bytes, &sh.bar[s]);
    }
}

// What a tile sends out by bulk store once every thread has written the
// split copy: for a one-node tile its two runs.
struct LwOut {
    bool runs;               // one node: a zeros run and a ones run
    bool bits;               // the split copy holds the runs' next-level bit streams, not their symbols
    bool store;              // the runs go out to P_{l+1} (else only their next-level bits)
    uintptr_t gz_b, go_b;    // their destinations
    uint32_t zt, ones;       // their symbols
    uint32_t offz, B1;       // their places in the split copy (bytes)
    uint64_t gz, go;         // their first positions in P_{l+1}
    uint32_t *next_words;    // level l + 1's bitmap, when this pass writes it
    uint32_t bsh_next;       // level l + 1's bit
};

// The byte permutation that puts a chunk's bytes with level bit 0 first and
// those with bit 1 after, each group in order: entry e (the chunk's 8 level
// bits) holds two PRMT selectors, output bytes 0-3 and 4-7.
__device__ __forceinline__ uint32_t zeros_first_perm(uint32_t e) {
    uint32_t sel = 0;
    int k = 0;
    for (uint32_t want = 0; want < 2; want++)
        for (uint32_t i = 0; i < 8; i++)
            if (((e >> i) & 1u) == want) sel |= i << (k < 4 ? 4 * k : 16 + 4 * (k - 4)), k++;
    return sel;
}

constexpr uint32_t kBitsOnesWord = 272;  // first word of the ones' stream in the split copy

// A one-node tile of 1-byte symbols whose pass stores no order (the level
// before the last): only level l + 1's bits of the two runs are needed, so
// they are built as two bit streams in the split copy instead of splitting
// the symbols.  A lane takes 32 consecutive symbols; per 8-symbol chunk a
// byte permutation puts the chunk's zeros first, one multiply gathers the
// permuted bytes' level l + 1 bits, and the zeros' and ones' parts are
// appended to the lane's two bit strings; each string goes into its stream
// at the run's offset within its first word plus the zeros (ones) of the
// tile before the lane, by at most two shared-memory atomics.  The caller
// copies the streams' words out with lw_next_bits.  All threads; one
// barrier inside (after the streams are cleared).
template <bool kWhole>
__device__ __forceinline__ void lw_bits_tile(const uint32_t *lut, const unsigned char *buf,
                                             const unsigned char *sbits, uint32_t *stream, uint32_t cnt,
                                             uint32_t wx, uint32_t gz5, uint32_t go5, uint32_t Zt,
                                             uint32_t tile_ones, uint32_t bsh_next) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwz = Zt ? (gz5 + Zt + 31) / 32 : 0u, nwo = tile_ones ? (go5 + tile_ones + 31) / 32 : 0u;
    for (uint32_t t = tid; t < nwz; t += kLwThreads) stream[t] = 0u;
    for (uint32_t t = tid; t < nwo; t += kLwThreads) stream[kBitsOnesWord + t] = 0u;
    __syncthreads();
    const BitGather gg = bit_gather<uint8_t>(bsh_next);
    uint32_t oc = wx;  // ones of the tile before the warp's round
#pragma unroll
    for (uint32_t r = 0; r < kLwWarpBytes / 1024; r++) {
        const uint32_t p0 = warp * kLwWarpBytes + r * 1024 + 32 * lane;  // the lane's first symbol
        uint32_t vm = ~0u;                                                  // its symbols below cnt
        if (!kWhole) vm = p0 >= cnt ? 0u : (cnt - p0 >= 32 ? ~0u : (1u << (cnt - p0)) - 1u);
        const uint32_t hb = vm ? reinterpret_cast<const uint32_t *>(sbits)[p0 / 32] & vm : 0u;
        uint32_t tot;
        const uint32_t po = oc + warp_excl_scan((uint32_t)__popc(hb), lane, tot);  // ones of the tile before p0
        oc += tot;
        if (!vm) continue;
        const uint4 v0 = *reinterpret_cast<const uint4 *>(buf + p0);
        const uint4 v1 = *reinterpret_cast<const uint4 *>(buf + p0 + 16);
        const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint32_t zacc = 0, oacc = 0, zs = 0, os = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t h8 = (hb >> (8 * j)) & 0xffu;
            const uint32_t sel = lut[h8];
            const uint64_t X = ((uint64_t)__byte_perm(w[2 * j], w[2 * j + 1], sel >> 16) << 32) |
                               __byte_perm(w[2 * j], w[2 * j + 1], sel & 0xffffu);
            const uint32_t g = (uint32_t)(((X & gg.mask) * gg.mul) >> 56);  // next bits, zeros first
            const uint32_t o8 = (uint32_t)__popc(h8);
            const uint32_t zv = (uint32_t)__popc(~h8 & (vm >> (8 * j)) & 0xffu);  // the chunk's zeros below cnt
            zacc |= (g & ((1u << zv) - 1u)) << zs;
            zs += zv;
            oacc |= (g >> (8 - o8)) << os;
            os += o8;
        }
        const uint32_t zoff = gz5 + (p0 - po), ooff = go5 + po;  // the strings' first bits in the streams
        if (zacc) {
            const uint32_t wi = zoff >> 5, sh = zoff & 31;
            atomicOr(stream + wi, zacc << sh);
            if (sh && sh + zs > 32) atomicOr(stream + wi + 1, zacc >> (32 - sh));
        }
        if (oacc) {
            const uint32_t wi = kBitsOnesWord + (ooff >> 5), sh = ooff & 31;
            atomicOr(stream + wi, oacc << sh);
            if (sh && sh + os > 32) atomicOr(stream + wi + 1, oacc >> (32 - sh));
        }
    }
}

// One tile: count and placement into the split copy, which the caller sends
// out with lw_store after its next barrier (all threads).  Each warp works
// from the prefix of its own range, so no counts are exchanged between the
// warps.  Level l's bitmap is already written (by the count pass or by the
// pass of level l - 1); when J.next_words is set, this pass writes level
// l + 1's: one-node tiles through lw_next_bits (the caller, after its
// barrier, from the split copy), multi-node tiles bit by bit here.
// kWhole: the tile holds kTile symbols (no bound checks per symbol).
// kBits: the launch has jobs on the level before the last (lw_bits_tile).
template <typename Sym, bool kWhole, bool kBits>
__device__ __forceinline__ void lw_tile(const LevelLaunch &a, const LwStage &S, const uint32_t *lut,
                                        const unsigned char *buf, const unsigned char *sbits, unsigned char *split,
                                        bool &bad, LwOut &out) {
    using Cfg = LwCfg<Sym>;
    constexpr int kW = Cfg::kW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l = a.l;
    const LevelJob &J = S.J;
    const uint32_t tile = S.tile;
    const uint64_t base = (uint64_t)tile * Cfg::kTile;
    const uint32_t cnt = kWhole ? Cfg::kTile : (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
    const uint64_t P = S.pre[0];                                             // ones before the tile
    const uint32_t wx = (uint32_t)(S.pre[warp * Cfg::kUnitsPerWarp] - P);    // before this warp's range
    const uint32_t tile_ones = (uint32_t)(S.pre[Cfg::kUnits] - P);
    const uint32_t Zt = cnt - tile_ones;
    const uint32_t bsh = J.L - 1 - l;     // the level-l bit
    uint32_t *const next_words = J.next_words;
    const uint32_t shv = J.L - l;  // key_l = s >> shv
    const uint32_t nodes = 1u << l;
    const Sym *sb = reinterpret_cast<const Sym *>(buf);
    const uint32_t kfirst = a.one_node ? 0u : (uint32_t)sb[0] >> shv;
    const uint32_t klast = a.one_node ? 0u : (uint32_t)sb[cnt - 1] >> shv;
    Sym *nxt = static_cast<Sym *>(J.nxt);
    out.bits = false;
    if (kBits && kW == 1 && nxt == nullptr && next_words != nullptr && kfirst == klast && kfirst < nodes) {
        // The level before the last, a one-node tile: only level l + 1's
        // bits of its two runs are needed (lw_bits_tile).
        const uint64_t gz = (base - P) + __ldg(J.ob + kfirst), go = P + __ldg(J.ze + kfirst);
        const bool ok = gz + Zt <= J.n && go + tile_ones <= J.n;  // the same in every thread
        if (ok)
            lw_bits_tile<kWhole>(lut, buf, sbits, reinterpret_cast<uint32_t *>(split), cnt, wx,
                                 (uint32_t)(gz & 31), (uint32_t)(go & 31), Zt, tile_ones, bsh - 1);
        else
            bad = true;
        out.runs = ok;
        out.bits = ok;
        out.store = false;
        out.gz_b = out.go_b = 0;
        out.zt = Zt;
        out.ones = tile_ones;
        out.offz = out.B1 = 0;
        out.gz = gz;
        out.go = go;
        out.next_words = next_words;
        out.bsh_next = bsh - 1;
        return;
    }

    // Count: level bits of the lane's chunks, per-lane and per-warp ones.  A
    // lane takes 8 consecutive bytes of each 256-byte warp step (8, 4 or 2
    // symbols, i.e. that many consecutive bits of the level's bitmap copy):
    // neighbouring lanes' run pointers are then about 4 bytes apart, one
    // shared-memory bank, so the split's byte stores rarely conflict.  The
    // counts of three steps share a word (10 bits each) and one scan.
    constexpr int kSt = (int)(kLwWarpBytes / 256);  // warp steps of 8 bytes a lane
    constexpr int kSpc = 8 / kW;                    // symbols of a lane's chunk
    constexpr int kPk = (kSt + 2) / 3;
    uint32_t h[kSt];
    uint32_t cpk[kPk], lpk[kPk], tpk[kPk];
#pragma unroll
    for (int k2 = 0; k2 < kPk; k2++) cpk[k2] = 0;
#pragma unroll
    for (int st = 0; st < kSt; st++) {
        const uint32_t q = warp * kLwWarpBytes + st * 256 + 8 * lane;  // the chunk's byte in the tile
        const uint32_t bit = q / kW;                                   // its first symbol = bitmap bit
        uint32_t hb = 0;
        if (kWhole || bit / 8 < S.bits_bytes) hb = (sbits[bit / 8] >> (bit & 7)) & ((1u << kSpc) - 1u);
        h[st] = hb;
        cpk[st / 3] += (uint32_t)__popc(hb) << (10 * (st % 3));
    }
#pragma unroll
    for (int k2 = 0; k2 < kPk; k2++) lpk[k2] = warp_excl_scan(cpk[k2], lane, tpk[k2]);

    // Placement.
    bool runs = false;
    uintptr_t gz_b = 0, go_b = 0;
    uint32_t offz = 0, B1 = 0;
    uint64_t gz = 0, go = 0;
    if (kfirst == klast && kfirst < nodes) {
        gz = (base - P) + __ldg(J.ob + kfirst);  // first zero's position in P_{l+1}
        go = P + __ldg(J.ze + kfirst);           // first one's position
        if (gz + Zt > J.n || go + tile_ones > J.n) {
            bad = true;
        } else {
            runs = true;
            gz_b = nxt ? reinterpret_cast<uintptr_t>(nxt + gz) : 0;
            go_b = nxt ? reinterpret_cast<uintptr_t>(nxt + go) : 0;
            // Each run starts at its destination's offset within a 32-symbol
            // word of the next bitmap (which also agrees with the
            // destination modulo 16 bytes, as the bulk stores need).
            offz = (uint32_t)(gz & 31) * kW;
            B1 = ((offz + Zt * kW + 32 * kW - 1) / (32 * kW)) * (32 * kW) + (uint32_t)(go & 31) * kW;
            uint32_t stx = 0;  // ones of earlier steps of this warp
#pragma unroll
            for (int st = 0; st < kSt; st++) {
                const uint32_t q = warp * kLwWarpBytes + st * 256 + 8 * lane;
                const uint32_t sh10 = 10 * (st % 3);
                const uint32_t o = wx + stx + ((lpk[st / 3] >> sh10) & 0x3ffu);  // ones before the chunk
                stx += (tpk[st / 3] >> sh10) & 0x3ffu;
                const uint2 v = *reinterpret_cast<const uint2 *>(buf + q);
                if (kW == 1 && kWhole) {
                    // Bytes: one byte permutation puts the chunk's zeros
                    // first and its ones after, each group in order, so
                    // permuted byte j goes to the chunk's first zero + j
                    // (j < z) or to its first one + (j - z).
                    const uint32_t h8 = h[st];
                    const uint32_t z = 8u - (uint32_t)__popc(h8);
                    const uint32_t sel = lut[h8];
                    const uint32_t xl = __byte_perm(v.x, v.y, sel & 0xffffu);
                    const uint32_t xh = __byte_perm(v.x, v.y, sel >> 16);
                    const uint32_t zp = offz + q - o;  // the chunk's first zero (zeros of the tile before it)
                    const uint32_t opz = B1 + o - z;   // its first one, less z
#pragma unroll
                    for (uint32_t j = 0; j < 8; j++)
                        split[(j < z ? zp : opz) + j] = (unsigned char)((j < 4 ? xl : xh) >> (8 * (j & 3)));
                    continue;
                }
                const uint32_t x[4] = {v.x, v.y, 0u, 0u};
                // A one goes to po; a zero to C + k kW - po (its zeros-before, scaled).
                uint32_t po = B1 + o * kW;
                const uint32_t C = offz + B1 + q;
#pragma unroll
                for (int kk = 0; kk < kSpc; kk++) {
                    if (kWhole || q / kW + kk < cnt) {
                        const bool one = (h[st] >> kk) & 1u;
                        const uint32_t at = one ? po : C + kk * kW - po;
                        const uint32_t sv = sym_at<Sym>(x, kk);
                        if (kW == 1) split[at] = (unsigned char)sv;
                        if (kW == 2) *reinterpret_cast<uint16_t *>(split + at) = (uint16_t)sv;
                        if (kW == 4) *reinterpret_cast<uint32_t *>(split + at) = sv;
                        po += one ? kW : 0;
                    }
                }
            }
        }
    } else {
        // Several nodes: each symbol to its own position (Proposition 1).
        // A warp takes 32 consecutive symbols of its range per round, so
        // one store instruction covers runs of consecutive destinations
        // and the node tables are read once per node; the ones before a
        // symbol come from a ballot over the round.  Level l + 1's bit of
        // a symbol goes to its destination's bitmap word by atomicOr (these
        // tiles are few wherever the pass writes level l + 1's bitmap).
        constexpr uint32_t kWarpSyms = kLwWarpBytes / kW;
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t o = wx;  // ones of the tile before this round
#pragma unroll 4
        for (uint32_t g = 0; g < kWarpSyms; g += 32) {
            const uint32_t p = warp * kWarpSyms + g + lane;  // tile position
            const bool in = kWhole || p < cnt;
            const uint32_t sv = in ? (uint32_t)sb[p] : 0u;
            const uint32_t bit = (sv >> bsh) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, in && bit);
            const uint32_t ob = o + __popc(bal & lt);  // ones of the tile before p
            o += __popc(bal);
            if (in) {
                const uint32_t v = sv >> shv;
                if (v >= nodes) {
                    bad = true;
                } else {
                    const uint64_t dst = bit ? P + ob + __ldg(J.ze + v) : (base + p - P - ob) + __ldg(J.ob + v);
                    if (dst < J.n) {
                        if (nxt) nxt[dst] = (Sym)sv;
                        if (next_words) {  // set or clear the bit: the word is not zeroed beforehand
                            if ((sv >> (bsh - 1)) & 1u)
                                atomicOr(next_words + (dst >> 5), 1u << (dst & 31));
                            else
                                atomicAnd(next_words + (dst >> 5), ~(1u << (dst & 31)));
                        }
                    } else {
                        bad = true;
                    }
                }
            }
        }
    }
    fence_proxy_async_smem();  // the split copy is read by bulk stores
    out.runs = runs;
    out.store = nxt != nullptr;
    out.gz_b = gz_b;
    out.go_b = go_b;
    out.zt = Zt;
    out.ones = tile_ones;
    out.offz = offz;
    out.B1 = B1;
    out.gz = gz;
    out.go = go;
    out.next_words = next_words;
    out.bsh_next = bsh - 1;
}

// The bulk stores of a tile (threads 0..63, after the barrier that follows
// lw_tile): for a one-node tile its two runs.
template <typename Sym>
__device__ __forceinline__ void lw_store(const LwOut &o, const unsigned char *split) {
    constexpr uint32_t kW = sizeof(Sym);
    const int tid = threadIdx.x;
    if (o.runs && o.store) {
        if (tid < 32)
            store_run(o.gz_b, o.zt * kW, split + o.offz, tid);
        else if (tid < 64)
            store_run(o.go_b, o.ones * kW, split + o.B1, tid - 32);
    }
}

// Level l + 1's bitmap words of a one-node tile's two runs, from its split
// copy (all threads, after the barrier that completes the copy).  A run
// starts in the copy at its destination's offset within a 32-symbol word,
// so bitmap word k of a run is the level l + 1 bits of the k-th group of 32
// symbols there: a word inside the run is stored, a word shared with other
// runs (or with the padding) gets its bits by atomics that clear and set
// only the run's own bits.  The two runs have 256 to 258 words; thread
// (tid + 64) mod 128 takes words t, t + 128, ..., so the at most two words
// beyond 256 fall to warp 2, which neither claims stages nor issues the
// bulk stores.
template <typename Sym, bool kBits>
__device__ __forceinline__ void lw_next_bits(const LwOut &o, const unsigned char *split) {
    constexpr uint32_t kW = sizeof(Sym);
    constexpr uint32_t kGroup = 32 * kW;  // bytes of 32 symbols
    if (!o.runs || !o.next_words) return;
    const uint32_t fz = (uint32_t)(o.gz & 31), fo = (uint32_t)(o.go & 31);  // each run's first bit in its word 0
    const uint32_t ez = fz + o.zt, eo = fo + o.ones;                         // and its end, from word 0's first bit
    const uint32_t nwz = o.zt ? (ez + 31) / 32 : 0u;
    const uint32_t nw = nwz + (o.ones ? (eo + 31) / 32 : 0u);
    const uint32_t obase = o.B1 - fo * kW;  // group 0 of the ones' run in the copy
    uint32_t *const zw = o.next_words + (o.gz >> 5), *const ow = o.next_words + (o.go >> 5);
    const BitGather gg = bit_gather<Sym>(o.bsh_next);
    for (uint32_t t = (threadIdx.x + 64) & (kLwThreads - 1); t < nw; t += kLwThreads) {
        const bool zr = t < nwz;
        const uint32_t k = zr ? t : t - nwz;
        uint32_t bits = 0;
        if (kBits && o.bits) {  // the run's word k of its bit stream
            bits = reinterpret_cast<const uint32_t *>(split)[(zr ? 0u : kBitsOnesWord) + k];
        } else {
            const unsigned char *g = split + (zr ? 0u : obase) + k * kGroup;
#pragma unroll
            for (uint32_t c = 0; c < kW * 2; c++) {
                const uint4 v = *reinterpret_cast<const uint4 *>(g + 16 * c);
                const uint32_t x[4] = {v.x, v.y, v.z, v.w};
                bits |= gather_bits<Sym>(x, gg, o.bsh_next) << (c * (16 / kW));
            }
        }
        uint32_t *w = (zr ? zw : ow) + k;
        const uint32_t first = zr ? fz : fo, end = zr ? ez : eo;
        if ((k > 0 || first == 0) && 32 * k + 32 <= end) {
            *w = bits;  // inside the run
        } else {
            // A word shared with other runs (or with the padding, zeroed by
            // the scan): clear this run's zero bits and set its ones; the
            // runs' masks are disjoint, so any order of the other runs'
            // updates leaves every bit right.
            const uint32_t lo = k == 0 ? first : 0u, hi = min(32u, end - 32 * k);
            const uint32_t mask = (hi == 32 ? ~0u : (1u << hi) - 1u) & ~((1u << lo) - 1u);
            if (~bits & mask) atomicAnd(w, ~(~bits & mask));
            if (bits & mask) atomicOr(w, bits & mask);
        }
    }
}

template <typename Sym, bool kBits>
__global__ void __launch_bounds__(kLwThreads, LwCfg<Sym>::kMinCtas) level_pass_kernel(LevelLaunch a) {
    using Cfg = LwCfg<Sym>;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *in = smem;  // kLwStages x kLwTileBytes of symbols, then kLwStages x kLwStageBits of bitmap
    unsigned char *split_base = in + kLwStages * (kLwTileBytes + kLwStageBits);  // 2 x kLwSplitBytes
    LwShared &sh = *reinterpret_cast<LwShared *>(split_base + 2 * kLwSplitBytes);
    const int tid = threadIdx.x;

    // This CTA's tiles: a contiguous range of the launch's global tiles.
    const uint32_t per = (a.total_tiles + gridDim.x - 1) / gridDim.x;
    const uint32_t g_begin = min(blockIdx.x * per, a.total_tiles);
    const uint32_t g_end = min(g_begin + per, a.total_tiles);
    uint32_t k = 0;  // the claimer's job index
    bool have_job = false;
    // The last warp claims the stages (warps 0 and 1 issue the bulk stores),
    // which spreads the per-tile extra work over three warps.
    const bool claimer = (tid >> 5) == kLwWarps - 1;
    if (tid == 0) {
        for (int s = 0; s < kLwStages; s++) mbar_init(&sh.bar[s], 1);
        fence_mbar_init();
    }
    if (sizeof(Sym) == 1)
        for (uint32_t e = tid; e < 256; e += kLwThreads) sh.lut[e] = zeros_first_perm(e);
    __syncthreads();
    // The set-up above touches only this CTA's shared memory.
    griddep_wait();
    if (claimer) {
        if (g_begin < g_end) k = find_job(a, g_begin);
        for (int s = 0; s < kLwStages - 1; s++) lw_claim<Sym>(a, sh, in, s, g_begin + s, g_end, k, have_job);
    }
    __syncthreads();

    bool failed = false, bad = false;
    // One barrier per tile: it publishes tile i's split copy to every thread
    // (for the bulk stores and the next level's bitmap words) and stage
    // i + 1 to every thread.
    if (__syncthreads_or(!mbar_wait(&sh.bar[0], 0u))) failed = true;
    for (uint32_t i = 0; !failed; i++) {
        const int s = (int)(i % kLwStages), par = (int)(i & 1);
        const LwStage &S = sh.st[s];
        if (S.tile == kNoTile) break;  // every thread reads the same record
        // Stage (i + 3) % 4 held tile i - 1, which is done: claim tile i + 3
        // into it while the other warps count this one.
        if (claimer)
            lw_claim<Sym>(a, sh, in, (int)((i + kLwStages - 1) % kLwStages), g_begin + i + kLwStages - 1, g_end, k,
                          have_job);
        unsigned char *buf = in + s * kLwTileBytes;
        unsigned char *split = split_base + par * kLwSplitBytes;
        LwOut out;
        out.runs = false;
        out.bits = false;
        if (!S.skip) {
            const LevelJob &J = S.J;
            const uint32_t tile = S.tile;
            const uint64_t base = (uint64_t)tile * Cfg::kTile;
            const uint32_t cnt = (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
            if (!S.full) {
                // The sequence's last tile, or symbols not 16-byte aligned:
                // plain loads, zero past the end.
                const Sym *src = static_cast<const Sym *>(J.cur);
                Sym *sb = reinterpret_cast<Sym *>(buf);
                for (uint32_t p = tid; p < Cfg::kTile; p += kLwThreads) sb[p] = p < cnt ? src[base + p] : (Sym)0;
                __syncthreads();
            }
            const unsigned char *sbits = in + kLwStages * kLwTileBytes + s * kLwStageBits;
            if (cnt == Cfg::kTile)
                lw_tile<Sym, true, kBits>(a, S, sh.lut, buf, sbits, split, bad, out);
            else
                lw_tile<Sym, false, kBits>(a, S, sh.lut, buf, sbits, split, bad, out);
        }
        // The split copy of the other parity (tile i - 1) is reused by tile
        // i + 1: its bulk stores must have read it before the barrier (its
        // bitmap words were read by every thread before this barrier).
        if (tid == 0 || tid == 32) bulk_wait_read0();
        const uint32_t i1 = i + 1;
        const bool ok = mbar_wait(&sh.bar[i1 % kLwStages], (i1 / kLwStages) & 1u);
        if (__syncthreads_or(!ok)) {  // a give-up is taken by every thread
            failed = true;
            break;
        }
        lw_store<Sym>(out, split);
        if (tid == 0 || tid == 32) bulk_commit();
        lw_next_bits<Sym, kBits>(out, split);
    }
    if (tid == 0 || tid == 32) bulk_wait_all();
    if (failed && tid == 0) atomicOr(a.err, kErrTimeout);
    if (bad) atomicOr(a.err, kErrTimeout);
}

constexpr size_t kLwSmem = kLwStages * (kLwTileBytes + kLwStageBits) + 2 * kLwSplitBytes + sizeof(LwShared);
// Six CTAs per SM: 228 KB of shared memory, 1 KB of it reserved per CTA.
static_assert(LwCfg<uint8_t>::kMinCtas * (kLwSmem + 1024) <= 228 * 1024, "level pass shared memory");

// Resident CTA slots of level_pass_kernel<Sym, kBits> (set up once).
template <typename Sym, bool kBits>
static int lw_slots(int &sms) {
    static int slots = 0, count = 0;
    if (!slots) {
        if (cudaFuncSetAttribute(level_pass_kernel<Sym, kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLwSmem) != cudaSuccess)
            return 0;
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_pass_kernel<Sym, kBits>, kLwThreads,
                                                          kLwSmem) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        slots = count * per_sm;
    }
    sms = count;
    return slots;
}

template <typename Sym>
static cudaError_t launch_lw(const LevelLaunch &a, bool from_bits, bool do_pass, bool counted, cudaStream_t st,
                             const RankTables *rt, bool bits) {
    // Persistent grid: every resident CTA slot, at most one CTA per tile.
    int sms = 0;
    const int slots = bits ? lw_slots<Sym, true>(sms) : lw_slots<Sym, false>(sms);
    if (!slots) return cudaErrorInvalidValue;
    // Counts: a warp per tile, at most eight CTAs per SM.
    const uint32_t cw = (a.total_tiles + kCountWarps - 1) / kCountWarps;
    const uint32_t g0 = cw < (uint32_t)(sms * 8) ? cw : (uint32_t)(sms * 8);
    if (!counted) {
        const cudaError_t e = from_bits ? launch_dependent(count_kernel<Sym, true>, g0, kCountThreads, 0, st, a)
                                        : launch_dependent(count_kernel<Sym, false>, g0, kCountThreads, 0, st, a);
        note_launches(1);
        if (e != cudaSuccess) return e;
    }
    // The level's node tables from its directory (no histogram): folded into
    // the scan for few nodes, else their own launch after it.
    LevelLaunch as = a;
    const bool fold = rt && a.njobs == 1 && a.ways == 1 && (1ull << a.l) <= kFoldNodes;
    if (fold) {
        as.rt_nodes = 1u << a.l;
        as.rt_done = const_cast<uint32_t *>(a.tile_start) + 2;
        as.rt_start_in = rt->start_in;
        as.rt_ob = rt->ob;
        as.rt_ze = rt->ze;
        as.rt_start_out = rt->start_out;
    }
    const dim3 sg(a.njobs * a.segs, a.ways);
    cudaError_t e = launch_dependent(scan_sums_kernel, sg, 1024, 0, st, a);
    if (e == cudaSuccess) e = launch_dependent(scan_segs_kernel, sg, 1024, 0, st, as);
    note_launches(2);
    if (e != cudaSuccess) return e;
    if (rt && !fold) {
        const cudaError_t e = launch_rank_tables(rt->lv, a.l, rt->start_in, rt->ob, rt->ze, rt->start_out, st);
        if (e != cudaSuccess) return e;
    }
    if (do_pass) {
        const int grid = (int)(a.total_tiles < (uint32_t)slots ? a.total_tiles : (uint32_t)slots);
        e = bits ? launch_dependent(level_pass_kernel<Sym, true>, grid, kLwThreads, kLwSmem, st, a)
                 : launch_dependent(level_pass_kernel<Sym, false>, grid, kLwThreads, kLwSmem, st, a);
        note_launches(1);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

LevelJob make_level_job(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l, const uint64_t *ob,
                        const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint32_t *cnt, uint64_t *pre,
                        uint32_t *next_words) {
    LevelJob j;
    j.cur = cur;
    j.nxt = (l + 1 < L) ? nxt : nullptr;
    j.n = n;
    j.nblocks = ceil_div(n, kBlockBits);
    j.nspans = ceil_div(n, 1ull << kSpanShift);
    j.L = L;
    j.ntiles = (uint32_t)ceil_div(n, lw_tile_elems(width));
    j.lv = lv;
    j.ones_out = ones_out;
    j.ob = ob ? ob + ((1ull << l) - 1) : nullptr;
    j.ze = ze ? ze + ((1ull << l) - 1) : nullptr;
    j.cnt = cnt;
    j.pre = pre;
    j.next_words = (l + 1 < L) ? next_words : nullptr;
    return j;
}

cudaError_t launch_level_jobs(int width, uint32_t l, const LevelJob *jobs, const uint32_t *tile_start, uint32_t njobs,
                              uint32_t total_tiles, uint32_t max_job_tiles, bool from_bits, bool do_pass,
                              uint32_t *err, cudaStream_t st, bool counted, const RankTables *rt,
                              uint32_t check_sigma, bool one_node, bool bits) {
    if (njobs == 0 || total_tiles == 0) return cudaSuccess;
    LevelLaunch a{};
    a.jobs = jobs;
    a.tile_start = tile_start;
    a.njobs = njobs;
    a.total_tiles = total_tiles;
    a.l = l;
    a.units = lw_units((uint32_t)width);
    a.upb = 512u * (uint32_t)width / lw_unit_bytes((uint32_t)width);  // units per rank block of 512 symbols
    a.segs = (uint32_t)ceil_div((uint64_t)(max_job_tiles ? max_job_tiles : 1) * a.units, kScanSeg);
    a.err = err;
    a.ways = 1;
    a.check_sigma = check_sigma;
    a.one_node = one_node;
    switch (width) {
        case 1: return launch_lw<uint8_t>(a, from_bits, do_pass, counted, st, rt, bits);
        case 2: return launch_lw<uint16_t>(a, from_bits, do_pass, counted, st, rt, false);
        case 4: return launch_lw<uint32_t>(a, from_bits, do_pass, counted, st, rt, false);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_level_scans(int width, uint32_t l, const LevelJob *jobs, uint32_t njobs, uint32_t max_job_tiles,
                               uint32_t ways, cudaStream_t st) {
    LevelLaunch a{};
    a.jobs = jobs;
    a.njobs = njobs;
    a.l = l;
    a.units = lw_units((uint32_t)width);
    a.upb = 512u * (uint32_t)width / lw_unit_bytes((uint32_t)width);
    a.segs = (uint32_t)ceil_div((uint64_t)(max_job_tiles ? max_job_tiles : 1) * a.units, kScanSeg);
    a.ways = ways;
    const dim3 sg(a.njobs * a.segs, a.ways);
    scan_sums_kernel<<<sg, 1024, 0, st>>>(a);
    scan_segs_kernel<<<sg, 1024, 0, st>>>(a);
    note_launches(2);
    return cudaGetLastError();
}

// Writes one job and its tile range to device memory (kernel parameters
// carry the values, so no host buffer has to outlive the call).
__global__ void put_job_kernel(LevelJob j, LevelJob *dst, uint32_t *tile_start) {
    griddep_wait();  // the slot may still be read by the previous level's kernels
    *dst = j;
    tile_start[0] = 0;
    tile_start[1] = j.ntiles;
    tile_start[2] = 0;  // the scan's count of finished CTAs (fold_rank_tables)
}

size_t level_job_bytes() { return sizeof(LevelJob); }

size_t level_job_slot_bytes() { return (sizeof(LevelJob) + 4 * sizeof(uint32_t) + 255) & ~size_t(255); }

cudaError_t launch_level_count(const void *cur, uint64_t n, int width, uint32_t L, uint32_t l, LevelDesc lv,
                               uint32_t *cnt, uint32_t *next_words, uint32_t *err, void *job_slot, cudaStream_t st,
                               uint32_t check_sigma) {
    if (n == 0) return cudaSuccess;
    LevelJob j = make_level_job(cur, nullptr, n, width, L, l, nullptr, nullptr, lv, nullptr, cnt, nullptr,
                                next_words);
    LevelJob *dj = static_cast<LevelJob *>(job_slot);
    uint32_t *ts = reinterpret_cast<uint32_t *>(dj + 1);
    const cudaError_t pe = launch_dependent(put_job_kernel, 1, 1, 0, st, j, dj, ts);
    note_launches(1);
    if (pe != cudaSuccess) return pe;
    LevelLaunch a{};
    a.jobs = dj;
    a.tile_start = ts;
    a.njobs = 1;
    a.total_tiles = j.ntiles;
    a.l = l;
    a.units = lw_units((uint32_t)width);
    a.upb = 512u * (uint32_t)width / lw_unit_bytes((uint32_t)width);
    a.segs = 1;
    a.err = err;
    a.ways = 1;
    a.check_sigma = check_sigma;
    const uint32_t cw = (j.ntiles + kCountWarps - 1) / kCountWarps;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t g0 = cw < (uint32_t)(sms * 8) ? cw : (uint32_t)(sms * 8);
    cudaError_t e = cudaErrorInvalidValue;
    switch (width) {
        case 1: e = launch_dependent(count_kernel<uint8_t, false>, g0, kCountThreads, 0, st, a); break;
        case 2: e = launch_dependent(count_kernel<uint16_t, false>, g0, kCountThreads, 0, st, a); break;
        case 4: e = launch_dependent(count_kernel<uint32_t, false>, g0, kCountThreads, 0, st, a); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return e;
}

cudaError_t launch_level_directory(uint64_t n, int width, uint32_t L, uint32_t l, LevelDesc lv, uint64_t *ones_out,
                                   uint32_t *cnt, uint64_t *pre, uint32_t *err, void *job_slot, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    LevelJob j = make_level_job(nullptr, nullptr, n, width, L, l, nullptr, nullptr, lv, ones_out, cnt, pre, nullptr);
    j.nxt = nullptr;
    LevelJob *dj = static_cast<LevelJob *>(job_slot);
    uint32_t *ts = reinterpret_cast<uint32_t *>(dj + 1);
    const cudaError_t pe = launch_dependent(put_job_kernel, 1, 1, 0, st, j, dj, ts);
    note_launches(1);
    if (pe != cudaSuccess) return pe;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_level_jobs(width, l, dj, ts, 1, j.ntiles, j.ntiles, true, false, err, st, false);
}

cudaError_t launch_level_pass(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l,
                              const uint64_t *ob, const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint32_t *cnt,
                              uint64_t *pre, bool from_bits, uint32_t *next_words, uint32_t *err, void *job_slot,
                              cudaStream_t st, bool counted, const RankTables *rt, uint32_t check_sigma,
                              bool one_node) {
    if (n == 0) return cudaSuccess;
    const LevelJob j = make_level_job(cur, nxt, n, width, L, l, ob, ze, lv, ones_out, cnt, pre, next_words);
    LevelJob *dj = static_cast<LevelJob *>(job_slot);
    uint32_t *ts = reinterpret_cast<uint32_t *>(dj + 1);
    const cudaError_t pe = launch_dependent(put_job_kernel, 1, 1, 0, st, j, dj, ts);
    note_launches(1);
    if (pe != cudaSuccess) return pe;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_level_jobs(width, l, dj, ts, 1, j.ntiles, j.ntiles, from_bits, l + 1 < L, err, st, counted, rt,
                             check_sigma, one_node, j.nxt == nullptr && j.next_words != nullptr);
}

}  // namespace wt
