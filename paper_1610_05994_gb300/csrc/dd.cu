// dd.cu -- kernel (d): every level built straight from S for small alphabets
// (sigma <= 256, one byte per symbol, n < 2^32).
//
// This is the domain decomposition of Algorithm 2 (Section 3.2) at tile
// granularity, with the partial trees never leaving shared memory:
//   pass 1 (dd_count)   the leaf histogram of every tile of S: cnt[t][c]
//                       (Function createPartialBA's node counts, at the leaves);
//   pass 2 (dd_colscan) for every leaf c an exclusive scan over the tiles,
//                       off[t][c], and the totals H[c]; a node's run offset is
//                       the sum of its leaves' offsets, which gives Algorithm
//                       2's global offsets G in node-major, tile-minor order
//                       (the per-level parPrefixSum over the k local offsets);
//   pass 3 (dd_write)   per tile, the tile's partial tree level by level in
//                       shared memory (the level-l order of the tile is the
//                       stable split of its level-(l-1) order), and each
//                       level's run of every node copied to its global bit
//                       offset: whole words with plain stores, the first and
//                       last word of a run with atomicOr (the thread-safe
//                       concatenation of Function mergeBA), plus the rank and
//                       select entries that fall inside the run.
// S is read twice; nothing of size n*L is written but the tree itself.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kDdThreads = 512;
constexpr int kDdWarps = kDdThreads / 32;
constexpr uint32_t kDdTile = 16384;                 // symbols per tile (one byte each)
constexpr uint32_t kDdWords = kDdTile / 32;         // bitmap words per tile
constexpr uint32_t kDdRange = kDdTile / kDdWarps;   // symbols per warp
constexpr int kDdSteps = (int)(kDdRange / 128);     // 128-symbol warp steps
constexpr uint32_t kDdMaxLeaves = 256;
constexpr uint32_t kColRows = 256;                  // tiles per column-scan chunk

bool dd_supported(uint64_t n, uint64_t sigma, int width) {
    return width == 1 && sigma >= 2 && sigma <= kDdMaxLeaves && n > 0 && n < (1ull << 32);
}

uint64_t dd_tiles(uint64_t n) { return ceil_div(n, kDdTile); }

// ------------------------------------------------------------------ pass 1

__global__ void __launch_bounds__(kDdThreads) dd_count_kernel(const uint8_t *__restrict__ S, uint64_t n,
                                                              uint32_t sigma, uint32_t *__restrict__ cnt,
                                                              uint32_t *__restrict__ err) {
    __shared__ uint32_t bins[kDdWarps][kDdMaxLeaves];
    const int t = threadIdx.x, warp = t >> 5;
    for (uint32_t k = t; k < kDdWarps * kDdMaxLeaves; k += kDdThreads) (&bins[0][0])[k] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kDdTile;
    const uint32_t m = (uint32_t)((n - base) < kDdTile ? (n - base) : kDdTile);
    bool bad = false;
    const bool vec = ((reinterpret_cast<uintptr_t>(S) & 15) == 0) && m == kDdTile;
    if (vec) {
        const uint4 *q = reinterpret_cast<const uint4 *>(S + base);
        for (uint32_t k = t; k < kDdTile / 16; k += kDdThreads) {
            const uint4 v = __ldcs(q + k);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint32_t s = (w[j >> 2] >> (8 * (j & 3))) & 0xffu;
                if (s < sigma)
                    atomicAdd(&bins[warp][s], 1u);
                else
                    bad = true;
            }
        }
    } else {
        for (uint32_t k = t; k < m; k += kDdThreads) {
            const uint32_t s = S[base + k];
            if (s < sigma)
                atomicAdd(&bins[warp][s], 1u);
            else
                bad = true;
        }
    }
    if (bad) atomicOr(err, kErrSymbol);
    __syncthreads();
    for (uint32_t c = t; c < sigma; c += kDdThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kDdWarps; w++) sum += bins[w][c];
        cnt[(uint64_t)blockIdx.x * sigma + c] = sum;
    }
}

// ------------------------------------------------------------------ pass 2
// Column scan of cnt[tiles][sigma] in chunks of kColRows tiles: (A) chunk
// sums, (B) scan of the chunk sums per column plus the column totals H,
// (C) off[t][c] = tiles before t in column c.

__global__ void dd_colsum_kernel(const uint32_t *__restrict__ cnt, uint64_t tiles, uint32_t sigma,
                                 uint32_t *__restrict__ csum) {
    const uint32_t c = threadIdx.x;
    if (c >= sigma) return;
    const uint64_t r0 = (uint64_t)blockIdx.x * kColRows;
    const uint64_t r1 = r0 + kColRows < tiles ? r0 + kColRows : tiles;
    uint32_t sum = 0;
    for (uint64_t r = r0; r < r1; r++) sum += cnt[r * sigma + c];
    csum[(uint64_t)blockIdx.x * sigma + c] = sum;
}

__global__ void dd_chunkscan_kernel(uint32_t *__restrict__ csum, uint64_t chunks, uint32_t sigma,
                                    uint64_t *__restrict__ H) {
    const uint32_t c = threadIdx.x;
    if (c >= sigma) return;
    uint32_t run = 0;
    for (uint64_t k = 0; k < chunks; k++) {
        const uint32_t x = csum[k * sigma + c];
        csum[k * sigma + c] = run;
        run += x;
    }
    H[c] = run;
}

__global__ void dd_offsets_kernel(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ csum, uint64_t tiles,
                                  uint32_t sigma, uint32_t *__restrict__ off) {
    const uint32_t c = threadIdx.x;
    if (c >= sigma) return;
    const uint64_t r0 = (uint64_t)blockIdx.x * kColRows;
    const uint64_t r1 = r0 + kColRows < tiles ? r0 + kColRows : tiles;
    uint32_t run = csum[(uint64_t)blockIdx.x * sigma + c];
    for (uint64_t r = r0; r < r1; r++) {
        off[r * sigma + c] = run;
        run += cnt[r * sigma + c];
    }
}

// ------------------------------------------------------------------ pass 3

struct DdArgs {
    const uint8_t *S;
    uint64_t n;
    uint32_t sigma, L;
    uint64_t nblocks, nspans;
    uint64_t ncap;               // capacity of S1 / S0
    const uint32_t *cnt, *off;   // [tiles][sigma]
    const uint64_t *hex;         // node starts, 2^L + 1
    const uint64_t *ob;          // per level OB_l (offset 2^l - 1)
    LevelDesc lv[8];
    uint32_t *err;
};

constexpr uint32_t kDdMaxNodes = kDdMaxLeaves / 2;   // nodes of the deepest level (L <= 8)

// Per-tile node records: counts and offsets of every node in heap order
// (level l node v at 2^l - 1 + v), and the current level's layout.
struct DdNodes {
    uint32_t cnt[2 * kDdMaxLeaves];   // symbols of the tile in the node
    uint32_t off[2 * kDdMaxLeaves];   // symbols of earlier tiles in the node
    uint32_t ls[kDdMaxNodes];         // local start of the node in the tile's level-l order
    uint32_t obl[kDdMaxNodes];        // local ones before the node's start
    uint32_t zel[kDdMaxNodes];        // local zeros through the node's end
    uint64_t G[kDdMaxNodes];          // global bit offset of the node's run on level l
    uint64_t O[kDdMaxNodes];          // global ones on level l before the run
    uint32_t wpre[kDdMaxNodes + 1];   // exclusive prefix of the runs' output words
    uint32_t bpre[kDdMaxNodes + 1];   // exclusive prefix of the rank blocks starting in the runs
};

// Largest v in [0, nodes) with pre[v] <= f (pre is nondecreasing, pre[0] = 0).
__device__ __forceinline__ uint32_t find_node(const uint32_t *pre, uint32_t nodes, uint32_t f) {
    uint32_t lo = 0, hi = nodes - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= f)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Ones before local bit i of the tile's current level bitmap.
__device__ __forceinline__ uint32_t local_rank(const uint32_t *lbits, const uint32_t *lrank, uint32_t i) {
    const uint32_t w = i >> 5, r = i & 31;
    return lrank[w] + (r ? __popc(lbits[w] & ((1u << r) - 1u)) : 0u);
}

// Local bit index of the local one (zero if !bit) of 0-based rank k; the
// tile holds more than k such bits.
__device__ uint32_t local_select(const uint32_t *lbits, const uint32_t *lrank, uint32_t nwords, uint32_t bit,
                                 uint32_t k) {
    // largest word w with (bits equal to `bit` before w) <= k
    uint32_t lo = 0, hi = nwords - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        const uint32_t before = bit ? lrank[mid] : 32 * mid - lrank[mid];
        if (before <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    uint32_t x = bit ? lbits[lo] : ~lbits[lo];
    uint32_t need = k - (bit ? lrank[lo] : 32 * lo - lrank[lo]);
    if (need > 31) need = 31;  // only on inconsistent input: keep the loop bounded
    for (uint32_t j = 0; j < need; j++) x &= x - 1;
    return 32 * lo + (x ? __ffs(x) - 1 : 31);
}

__global__ void __launch_bounds__(kDdThreads) dd_write_kernel(DdArgs a) {
    __shared__ __align__(16) uint8_t sym[2][kDdTile];
    __shared__ uint32_t lbits[kDdWords + 1];
    __shared__ uint32_t lrank[kDdWords + 1];
    __shared__ uint32_t wtot[kDdWarps];
    __shared__ DdNodes nd;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (*(volatile uint32_t *)a.err & kErrSymbol) return;  // the tables do not describe S
    const uint64_t tile = blockIdx.x;
    const uint64_t base = tile * kDdTile;
    const uint32_t m = (uint32_t)((a.n - base) < kDdTile ? (a.n - base) : kDdTile);
    const uint32_t L = a.L, leaves = 1u << L;

    // Load the tile (its level-0 order is S itself).
    if (((reinterpret_cast<uintptr_t>(a.S) & 15) == 0) && m == kDdTile) {
        const uint4 *q = reinterpret_cast<const uint4 *>(a.S + base);
        for (uint32_t k = t; k < kDdTile / 16; k += kDdThreads) reinterpret_cast<uint4 *>(sym[0])[k] = __ldcs(q + k);
    } else {
        for (uint32_t k = t; k < kDdTile; k += kDdThreads) sym[0][k] = k < m ? a.S[base + k] : 0;
    }
    // Leaf records of this tile, then node sums bottom-up (heap order).
    for (uint32_t c = t; c < leaves; c += kDdThreads) {
        const bool in = c < a.sigma;
        nd.cnt[leaves - 1 + c] = in ? a.cnt[tile * a.sigma + c] : 0;
        nd.off[leaves - 1 + c] = in ? a.off[tile * a.sigma + c] : 0;
    }
    if (t == 0) lbits[kDdWords] = 0;
    __syncthreads();
    for (int l = (int)L - 1; l >= 0; l--) {
        const uint32_t first = (1u << l) - 1;
        for (uint32_t v = t; v < (1u << l); v += kDdThreads) {
            const uint32_t h = first + v, c0 = 2 * h + 1;
            nd.cnt[h] = nd.cnt[c0] + nd.cnt[c0 + 1];
            nd.off[h] = nd.off[c0] + nd.off[c0 + 1];
        }
        __syncthreads();
    }

    int cur = 0;
    for (uint32_t l = 0; l < L; l++) {
        const uint32_t nodes = 1u << l, first = nodes - 1, child_first = 2 * nodes - 1;
        // Local node layout of level l: starts, ones before each start, zeros
        // through each end (one warp scans up to 256 nodes, 8 per lane).
        if (warp == 0) {
            // up to 128 nodes, 4 per lane: local layout, global run offsets,
            // and the number of output words / rank blocks of each run
            uint32_t c_[4], z_[4], o_[4], w_[4], b_[4];
            uint32_t sc = 0, sz = 0, so = 0, sw = 0, sb = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t v = lane * 4 + j;
                c_[j] = z_[j] = o_[j] = w_[j] = b_[j] = 0;
                if (v < nodes) {
                    c_[j] = nd.cnt[first + v];
                    z_[j] = nd.cnt[child_first + 2 * v];
                    o_[j] = nd.cnt[child_first + 2 * v + 1];
                    const uint64_t G = a.hex[(uint64_t)v << (L - l)] + nd.off[first + v];
                    nd.G[v] = G;
                    nd.O[v] = a.ob[first + v] + nd.off[child_first + 2 * v + 1];
                    if (c_[j]) {
                        w_[j] = (uint32_t)(((G + c_[j] - 1) >> 5) - (G >> 5) + 1);
                        const uint64_t b0 = (G + 511) >> 9, b1 = (G + c_[j] - 1) >> 9;
                        b_[j] = b1 >= b0 ? (uint32_t)(b1 - b0 + 1) : 0u;
                    }
                }
                sc += c_[j], sz += z_[j], so += o_[j], sw += w_[j], sb += b_[j];
            }
            uint32_t ic = sc, iz = sz, io = so, iw = sw, ib = sb;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t yc = __shfl_up_sync(0xffffffffu, ic, d), yz = __shfl_up_sync(0xffffffffu, iz, d),
                               yo = __shfl_up_sync(0xffffffffu, io, d), yw = __shfl_up_sync(0xffffffffu, iw, d),
                               yb = __shfl_up_sync(0xffffffffu, ib, d);
                if (lane >= d) ic += yc, iz += yz, io += yo, iw += yw, ib += yb;
            }
            uint32_t rc = ic - sc, rz = iz - sz, ro = io - so, rw = iw - sw, rb = ib - sb;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t v = lane * 4 + j;
                if (v < nodes) {
                    nd.ls[v] = rc;
                    nd.obl[v] = ro;
                    nd.zel[v] = rz + z_[j];
                    nd.wpre[v] = rw;
                    nd.bpre[v] = rb;
                }
                rc += c_[j], rz += z_[j], ro += o_[j], rw += w_[j], rb += b_[j];
            }
            if (lane == 31) {
                nd.wpre[nodes] = rw;
                nd.bpre[nodes] = rb;
            }
        }
        __syncthreads();

        // Phase 1: the level bit of every symbol of the local level-l order;
        // bitmap words into shared memory; per-lane / per-warp counts.
        const uint8_t *src = sym[cur];
        const uint32_t bsh = L - 1 - l;
        const uint32_t wbase = warp * kDdRange;
        uint32_t x4[kDdSteps], nib = 0, cpk[(kDdSteps + 3) / 4];
#pragma unroll
        for (int g = 0; g < (kDdSteps + 3) / 4; g++) cpk[g] = 0;
#pragma unroll
        for (int k = 0; k < kDdSteps; k++) {
            const uint32_t q = wbase + 128u * k + 4u * lane;
            x4[k] = *reinterpret_cast<const uint32_t *>(src + q);
            uint32_t nb = (((x4[k] << (7 - bsh)) & 0x80808080u) * 0x00204081u) >> 28;
            nb &= q < m ? ((m - q >= 4) ? 15u : ((1u << (m - q)) - 1u)) : 0u;
            nib |= nb << (4 * k);
            const uint32_t wv = __reduce_or_sync(0xffu << (lane & 24), nb << (4 * (lane & 7)));
            if ((lane & 7) == 0) lbits[(wbase + 128u * k) / 32 + (lane >> 3)] = wv;
            cpk[k >> 2] += (uint32_t)__popc(nb) << (8 * (k & 3));
        }
        uint32_t lpk[(kDdSteps + 3) / 4], tpk[(kDdSteps + 3) / 4];
#pragma unroll
        for (int g = 0; g < (kDdSteps + 3) / 4; g++) {
            uint32_t inc = cpk[g];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
            lpk[g] = inc - cpk[g];
            tpk[g] = __shfl_sync(0xffffffffu, inc, 31);
        }
        uint32_t wrun = 0;
#pragma unroll
        for (int k = 0; k < kDdSteps; k++) wrun += (tpk[k >> 2] >> (8 * (k & 3))) & 0xffu;
        if (lane == 0) wtot[warp] = wrun;
        __syncthreads();
        uint32_t wexcl = 0, tile_ones = 0;
#pragma unroll
        for (int w = 0; w < kDdWarps; w++) {
            const uint32_t x = wtot[w];
            wexcl += w < warp ? x : 0u;
            tile_ones += x;
        }
        // local rank of every bitmap word: lane holds 4 words per step
        {
            uint32_t run = wexcl;
#pragma unroll
            for (int k = 0; k < kDdSteps; k++) {
                // words of step k: (wbase + 128k)/32 + j, j = 0..3, owned by lanes 8j..8j+7
                if ((lane & 7) == 0) {
                    const uint32_t wi = (wbase + 128u * k) / 32 + (lane >> 3);
                    // ones before this word inside the step = lanes below 8*(lane>>3)
                    lrank[wi] = run + ((lpk[k >> 2] >> (8 * (k & 3))) & 0xffu);
                }
                run += (tpk[k >> 2] >> (8 * (k & 3))) & 0xffu;
            }
            if (t == 0) lrank[kDdWords] = tile_ones;
        }

        // Phase 2: split the local order by the bit (the next level's local
        // order): a symbol of node v goes to ZEloc[v] + ones before it, or to
        // OBloc[v] + zeros before it.
        if (l + 1 < L) {
            uint8_t *dst = sym[cur ^ 1];
            const uint32_t shv = L - l;
            uint32_t crun = wexcl;
#pragma unroll
            for (int k = 0; k < kDdSteps; k++) {
                const uint32_t nb = (nib >> (4 * k)) & 15u;
                const uint32_t q = wbase + 128u * k + 4u * lane;
                const uint32_t ob0 = crun + ((lpk[k >> 2] >> (8 * (k & 3))) & 0xffu);
                crun += (tpk[k >> 2] >> (8 * (k & 3))) & 0xffu;
                uint32_t ones = ob0;  // local ones before the symbol
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    const uint32_t s = (x4[k] >> (8 * x)) & 0xffu;
                    const uint32_t v = s >> shv;
                    const bool bit = (nb >> x) & 1u;
                    const uint32_t d = bit ? nd.zel[v] + ones : nd.obl[v] + (q + x - ones);
                    if (q + x < m) {
                        if (d < kDdTile)  // always, unless the tables were corrupted
                            dst[d] = (uint8_t)s;
                        else
                            atomicOr(a.err, kErrTimeout);
                    }
                    ones += bit;
                }
            }
        }
        __syncthreads();

        // Phase 3: copy every node's run of local bits to its global offset
        // (all threads share the output words of all runs), and write the
        // directory entries that fall inside the runs.
        LevelDesc &lv = a.lv[l];
        const uint32_t total_words = nd.wpre[nodes], total_blocks = nd.bpre[nodes];
        for (uint32_t f = t; f < total_words; f += kDdThreads) {
            const uint32_t v = find_node(nd.wpre, nodes, f);
            const uint32_t c = nd.cnt[first + v], ls = nd.ls[v];
            const uint64_t G = nd.G[v];
            const uint64_t gw = (G >> 5) + (f - nd.wpre[v]);
            // word bits [lo, hi) belong to the run; they are local bits L0 ..
            const uint64_t gbit = gw << 5;
            const uint32_t lo = (uint32_t)(G > gbit ? G - gbit : 0);
            const uint32_t hi = (uint32_t)((G + c - gbit) < 32 ? (G + c - gbit) : 32);
            const uint32_t L0 = ls + (uint32_t)(gbit + lo - G);
            const uint32_t val = __funnelshift_r(lbits[L0 >> 5], lbits[(L0 >> 5) + 1], L0 & 31) << lo;
            const uint32_t mask = (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
            if (gw >= a.nblocks * 16) {  // never for consistent tables: do not write past the level
                atomicOr(a.err, kErrTimeout);
            } else if (mask == 0xffffffffu) {
                lv.words[gw] = val;
            } else if (val & mask) {
                atomicOr(&lv.words[gw], val & mask);
            }
        }
        // rank entries of the blocks that start inside the runs
        for (uint32_t f = t; f < total_blocks; f += kDdThreads) {
            const uint32_t v = find_node(nd.bpre, nodes, f);
            const uint32_t ls = nd.ls[v];
            const uint64_t G = nd.G[v];
            const uint64_t b = ((G + 511) >> 9) + (f - nd.bpre[v]);
            if (b >= a.nblocks) continue;
            const uint64_t before =
                nd.O[v] + (local_rank(lbits, lrank, ls + (uint32_t)((b << 9) - G)) - local_rank(lbits, lrank, ls));
            lv.R[b] = (uint32_t)before;
            if ((b & kBlocksPerSpanMask) == 0) lv.Hy[b >> (kSpanShift - 9)] = before;
        }
        // select samples whose one (zero) lies inside a run (a few per tile)
        for (uint32_t v = t; v < nodes; v += kDdThreads) {
            const uint32_t c = nd.cnt[first + v];
            if (c == 0) continue;
            const uint32_t ls = nd.ls[v];
            const uint64_t G = nd.G[v], O = nd.O[v];
            const uint32_t r0 = local_rank(lbits, lrank, ls);
            const uint32_t ones = local_rank(lbits, lrank, ls + c) - r0;
            for (uint64_t k = ceil_div(O, kSample); k * kSample < O + ones && k < a.ncap; k++) {
                const uint32_t li = local_select(lbits, lrank, kDdWords, 1, r0 + (uint32_t)(k * kSample - O));
                lv.S1[k] = (uint32_t)((G + (li - ls)) >> 9);
            }
            const uint64_t Z = G - O;      // global zeros before the run
            const uint32_t z0 = ls - r0;   // local zeros before ls
            for (uint64_t k = ceil_div(Z, kSample); k * kSample < Z + (c - ones) && k < a.ncap; k++) {
                const uint32_t li = local_select(lbits, lrank, kDdWords, 0, z0 + (uint32_t)(k * kSample - Z));
                lv.S0[k] = (uint32_t)((G + (li - ls)) >> 9);
            }
        }
        __syncthreads();
        cur ^= 1;
    }
}

// Per level: total ones (sum of H over the codes whose level-l bit is 1, from
// the node starts), R[nblocks] and Hy[nspans].
__global__ void dd_finalize_kernel(const uint64_t *__restrict__ hex, uint32_t L, uint64_t nblocks, uint64_t nspans,
                                   TreeDesc *desc, DdArgs a) {
    const uint32_t l = threadIdx.x;
    if (l >= L) return;
    const uint32_t sh = L - l - 1;  // level l+1 nodes are codes >> sh
    uint64_t ones = 0;
    for (uint64_t v = 1; v < (2ull << l); v += 2) ones += hex[(v + 1) << sh] - hex[v << sh];
    a.lv[l].R[nblocks] = (uint32_t)ones;
    a.lv[l].Hy[nspans] = ones;
    desc->lv[l].ones = ones;
}

size_t dd_scratch_bytes(uint64_t n, uint64_t sigma) {
    const uint64_t tiles = dd_tiles(n);
    const uint64_t chunks = ceil_div(tiles, kColRows);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    return al(tiles * sigma * 4) * 2 + al(chunks * sigma * 4) + al(sigma * 8);
}

DdScratch dd_carve(void *scratch, uint64_t n, uint64_t sigma) {
    const uint64_t tiles = dd_tiles(n);
    const uint64_t chunks = ceil_div(tiles, kColRows);
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    char *p = static_cast<char *>(scratch);
    DdScratch d;
    d.cnt = reinterpret_cast<uint32_t *>(p);
    p += al(tiles * sigma * 4);
    d.off = reinterpret_cast<uint32_t *>(p);
    p += al(tiles * sigma * 4);
    d.csum = reinterpret_cast<uint32_t *>(p);
    p += al(chunks * sigma * 4);
    d.H = reinterpret_cast<uint64_t *>(p);
    return d;
}

cudaError_t launch_dd_count(const void *S, uint64_t n, uint64_t sigma, const DdScratch &d, uint32_t *err,
                            cudaStream_t st) {
    dd_count_kernel<<<(unsigned)dd_tiles(n), kDdThreads, 0, st>>>(static_cast<const uint8_t *>(S), n, (uint32_t)sigma,
                                                                  d.cnt, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dd_scan(uint64_t n, uint64_t sigma, const DdScratch &d, cudaStream_t st) {
    const uint64_t tiles = dd_tiles(n);
    const uint64_t chunks = ceil_div(tiles, kColRows);
    const uint32_t sig = (uint32_t)sigma;
    dd_colsum_kernel<<<(unsigned)chunks, 256, 0, st>>>(d.cnt, tiles, sig, d.csum);
    dd_chunkscan_kernel<<<1, 256, 0, st>>>(d.csum, chunks, sig, d.H);
    dd_offsets_kernel<<<(unsigned)chunks, 256, 0, st>>>(d.cnt, d.csum, tiles, sig, d.off);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_dd_write(const void *S, uint64_t n, uint64_t sigma, uint32_t L, const TreeDesc &h_desc,
                            TreeDesc *d_desc, const DdScratch &d, const uint64_t *hex, const uint64_t *ob,
                            uint32_t *err, cudaStream_t st) {
    DdArgs a;
    a.S = static_cast<const uint8_t *>(S);
    a.n = n;
    a.sigma = (uint32_t)sigma;
    a.L = L;
    a.nblocks = ceil_div(n, kBlockBits);
    a.nspans = ceil_div(n, 1ull << kSpanShift);
    a.ncap = n / kSample + 2;
    a.cnt = d.cnt;
    a.off = d.off;
    a.hex = hex;
    a.ob = ob;
    for (uint32_t l = 0; l < 8; l++) a.lv[l] = l < L ? h_desc.lv[l] : LevelDesc{};
    a.err = err;
    dd_write_kernel<<<(unsigned)dd_tiles(n), kDdThreads, 0, st>>>(a);
    dd_finalize_kernel<<<1, 32, 0, st>>>(hex, L, a.nblocks, a.nspans, d_desc, a);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace wt
