// pair.cu -- two levels per pass: levels l and l + 1 of the level-wise build
// with one read of P_l, every symbol placed straight into P_{l+2}.
//
// The multi-level-per-pass variant: a radix digit of two tree bits per pass
// over the symbols.  Algorithm 1 (Section 3.1) places each symbol of level l
// at its node's running counter C[node]++; two levels compose: the symbols
// of node v of level l whose bits (l, l + 1) form the group g in {00, 01, 10,
// 11} are, in their order in P_l, exactly node 4v + g of level l + 2
// (Proposition 1).  So a symbol of group g at position p of P_l goes to
//          T_l[4v + g] + (symbols of group g in P_l[0, p))
// with T_l[4v + g] = C_{l+2}[4v + g] - (symbols of group g in the nodes of
// level l before v), a per-level table from the node starts.  The counts of
// the groups come from three per-unit counts (level-l ones, group 01, group
// 11) and their prefix scan, the same way the one-level step gets its ones.
//
// Level l + 1's bitmap holds, at the positions of P_{l+1}, bit l + 1 of the
// symbols in level-(l+1) order; the pass writes it from a split of each tile
// into its level-(l+1) runs (A).  It then splits A's two runs again, by bit
// l + 1, into the tile's four runs of P_{l+2} (B), which leave by bulk store;
// B also gives level l + 2's bitmap (the hand-over of the one-level step)
// and bit l + 3 of P_{l+2}, so that the next pair step's counts read bits,
// not symbols.
//
// GPU structure: the one-level pass's persistent CTA (128 threads, tiles of
// 8 KB, TMA bulk copies of the symbols, level l's bitmap, bit l + 1 of P_l
// and the unit prefixes into three stages claimed by the last warp).  Per
// tile in one node of level l:
//   1. split by bit l into A (each lane walks its 16-byte chunks, as in the
//      one-level pass); barrier;
//   2. every thread takes a 32-symbol group of A: level l + 1's bitmap word
//      and the group's ones of bit l + 1; a block scan of those; barrier;
//   3. each group splits by bit l + 1 into B; barrier;
//   4. bulk stores of B's four runs; level l + 2's bitmap words and bit
//      l + 3 from B.
// Tiles spanning several nodes of level l place every symbol on its own,
// with atomicOr for the bits of levels l + 1, l + 2 and plane l + 3.
#include <cuda_runtime.h>
#include <stdint.h>

#include "level_common.cuh"

namespace wt {

namespace {

constexpr int kPairStages = 3;
constexpr uint32_t kPairBBytes = kLwTileBytes + 1024;  // four runs at their destinations' offsets in 32-symbol words
// Batches of kLwThreads 32-symbol groups of A a tile can need: the two runs
// of a tile of 8192 bytes span at most 8192 / 32 + 4 groups of 1-byte
// symbols (fewer for wider symbols).
constexpr int kGB = (int)((kLwTileBytes / 32 + 4 + kLwThreads - 1) / kLwThreads);

struct PairLaunch {
    const PairJob *jobs;          // device array of njobs
    const uint32_t *tile_start;   // device, njobs + 1
    uint32_t njobs, total_tiles, l;
    uint32_t need_b;              // every job's need_b (the same in a launch)
    uint32_t *err;
};

__device__ __forceinline__ uint32_t pair_find_job(const PairLaunch &a, uint32_t t) {
    uint32_t lo = 0, hi = a.njobs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.tile_start[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- counts

// Three counts per unit of P_l: level-l ones, group 01 and group 11 (bits
// l and l + 1 of the symbol).  One warp per tile.
//   kFromBits: from level l's bitmap and plane l + 1 (both in P_l order);
//   else from the symbols, writing level l's bitmap and plane l + 1.
// Zeroes the tile's words of next1, next2 and plane3 (the pass ORs its
// boundary words into them).
template <typename Sym, bool kFromBits>
__global__ void __launch_bounds__(256, 4) pair_count_kernel(PairLaunch a) {
    using Cfg = LwCfg<Sym>;
    constexpr uint32_t kU = Cfg::kUnits;
    constexpr uint32_t kUnitSyms = Cfg::kTile / kU;
    constexpr uint32_t kTileWords = Cfg::kTile / 32;
    constexpr int kWarps = 256 / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kWarps;
    const uint32_t bsh0 = a.l + 1;  // level l's bit is L - bsh0
    uint32_t k = 0;
    for (uint32_t g = blockIdx.x * kWarps + (threadIdx.x >> 5); g < a.total_tiles; g += nwarps) {
        if (k + 1 < a.njobs && a.tile_start[k + 1] <= g) {
            uint32_t lo = k + 1, hi = a.njobs - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.tile_start[mid] <= g)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            k = lo;
        }
        const PairJob &J = a.jobs[k];
        const uint32_t tile = g - a.tile_start[k];
        const uint64_t base = (uint64_t)tile * Cfg::kTile;
        const uint64_t w0 = base / 32;
        const uint64_t nwords = J.nblocks * 16;
        const uint64_t units = (uint64_t)J.ntiles * kU;
        uint32_t *c0 = J.cnt + (size_t)tile * kU;
        uint32_t *c1 = c0 + way_cnt_stride(units);
        uint32_t *c2 = c1 + way_cnt_stride(units);
        if (kFromBits) {
            constexpr uint32_t kWU = kUnitSyms / 32;  // words per unit
            constexpr int kRows = (int)(kTileWords / 32);
#pragma unroll
            for (int r = 0; r < kRows; r++) {
                const uint64_t w = w0 + (uint32_t)r * 32 + lane;
                const uint32_t x = w < nwords ? __ldcs(J.words + w) : 0u;
                const uint32_t y = w < nwords ? __ldcs(J.plane + w) : 0u;
                uint32_t v0 = __popc(x), v1 = __popc(~x & y), v2 = __popc(x & y);
#pragma unroll
                for (uint32_t d = kWU / 2; d >= 1; d >>= 1) {
                    v0 += __shfl_xor_sync(0xffffffffu, v0, d);
                    v1 += __shfl_xor_sync(0xffffffffu, v1, d);
                    v2 += __shfl_xor_sync(0xffffffffu, v2, d);
                }
                if (lane % kWU == 0) {
                    const uint32_t u = ((uint32_t)r * 32 + lane) / kWU;
                    c0[u] = v0;
                    c1[u] = v1;
                    c2[u] = v2;
                }
            }
        } else {
            constexpr int kVecs = (int)(kLwTileBytes / 512);  // 16-byte loads per lane per tile
            constexpr int kPerUnit = kVecs / (int)kU;
            const Sym *S = static_cast<const Sym *>(J.cur);
            const uint32_t cnt = (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
            const uint32_t bsh = J.L - bsh0;
            unsigned char *bm = reinterpret_cast<unsigned char *>(J.words);
            unsigned char *pm = reinterpret_cast<unsigned char *>(J.plane);
            if (cnt == Cfg::kTile && (reinterpret_cast<uintptr_t>(S) & 15) == 0) {
                const uint4 *v = reinterpret_cast<const uint4 *>(S + base) + lane;
                const size_t boff = base / 8 + (16 * lane / sizeof(Sym)) / 8;
                const BitGather g0 = bit_gather<Sym>(bsh), g1 = bit_gather<Sym>(bsh - 1);
                uint32_t a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
                for (int h = 0; h < kVecs; h += 4) {
                    uint4 w[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) w[r] = __ldcs(v + (h + r) * 32);
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const uint32_t x[4] = {w[r].x, w[r].y, w[r].z, w[r].w};
                        const uint32_t hb = gather_bits<Sym>(x, g0, bsh);
                        const uint32_t hp = gather_bits<Sym>(x, g1, bsh - 1);
                        a0 += __popc(hb);
                        a1 += __popc(~hb & hp);
                        a2 += __popc(hb & hp);
                        const size_t d = boff + (h + r) * (512 / sizeof(Sym) / 8);
                        if (sizeof(Sym) == 1) {
                            *reinterpret_cast<uint16_t *>(bm + d) = (uint16_t)hb;
                            *reinterpret_cast<uint16_t *>(pm + d) = (uint16_t)hp;
                        }
                        if (sizeof(Sym) == 2) {
                            bm[d] = (unsigned char)hb;
                            pm[d] = (unsigned char)hp;
                        }
                        if (sizeof(Sym) == 4) {
                            const uint32_t nb = __shfl_down_sync(0xffffffffu, hb, 1);
                            const uint32_t np = __shfl_down_sync(0xffffffffu, hp, 1);
                            if ((lane & 1) == 0) {
                                bm[d] = (unsigned char)(hb | (nb << 4));
                                pm[d] = (unsigned char)(hp | (np << 4));
                            }
                        }
                        if ((h + r + 1) % kPerUnit == 0) {
                            const uint32_t t0 = __reduce_add_sync(0xffffffffu, a0);
                            const uint32_t t1 = __reduce_add_sync(0xffffffffu, a1);
                            const uint32_t t2 = __reduce_add_sync(0xffffffffu, a2);
                            if (lane == 0) {
                                const uint32_t u = (uint32_t)(h + r) / kPerUnit;
                                c0[u] = t0;
                                c1[u] = t1;
                                c2[u] = t2;
                            }
                            a0 = a1 = a2 = 0;
                        }
                    }
                }
            } else {
                for (uint32_t j = 0; j < kU; j++) {
                    uint32_t a0 = 0, a1 = 0, a2 = 0;
                    for (uint32_t p0 = j * kUnitSyms; p0 < (j + 1) * kUnitSyms; p0 += 32) {
                        const uint32_t p = p0 + lane;
                        const uint32_t sv = p < cnt ? (uint32_t)S[base + p] : 0u;
                        const uint32_t b0 = p < cnt ? (sv >> bsh) & 1u : 0u;
                        const uint32_t b1 = p < cnt ? (sv >> (bsh - 1)) & 1u : 0u;
                        const uint32_t m0 = __ballot_sync(0xffffffffu, b0);
                        const uint32_t m1 = __ballot_sync(0xffffffffu, b1);
                        a0 += __popc(m0);
                        a1 += __popc(~m0 & m1);
                        a2 += __popc(m0 & m1);
                        if (lane == 0 && w0 + p0 / 32 < nwords) {
                            J.words[w0 + p0 / 32] = m0;
                            J.plane[w0 + p0 / 32] = m1;
                        }
                    }
                    if (lane == 0) {
                        c0[j] = a0;
                        c1[j] = a1;
                        c2[j] = a2;
                    }
                }
            }
        }
        // Zero the words of the bitmaps this step ORs into, over the tile's positions.
        constexpr uint32_t kVec4 = kTileWords / 4;
        uint32_t *const zs[3] = {J.next1, J.next2, J.plane3};
#pragma unroll
        for (int z = 0; z < 3; z++) {
            if (!zs[z]) continue;
            uint4 *nw = reinterpret_cast<uint4 *>(zs[z] + w0);
#pragma unroll
            for (uint32_t r = 0; r < (kVec4 + 31) / 32; r++) {
                const uint32_t i = r * 32 + lane;
                if (i < kVec4 && w0 + 4ull * i < nwords) nw[i] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

// ------------------------------------------------------------------ pass

struct __align__(16) PairStage {
    uint64_t pre[3][kLwMaxUnits + 2];  // unit prefixes of the three counts, and the next tile's first
    PairJob J;
    uint32_t tile;        // kNoTile: this CTA has no more tiles
    uint32_t full;        // a whole tile, 16-byte aligned: its symbols came in by bulk copy
    uint32_t bits_bytes;  // bytes of level l's bitmap (and of plane l + 1) copied for the tile
    uint32_t pad;
};

// What the phases after a tile's first barrier need (written by thread 0 in
// phase 1; the stage itself may be reclaimed before the last phase ends).
struct PairPlan {
    uint64_t d[4];          // first position in P_{l+2} of the tile's runs of groups 00, 01, 10, 11
    uint64_t gz, go;        // first position in P_{l+1} of the tile's zeros and ones of level l
    uint32_t len[4];        // symbols of the four group runs
    uint32_t boff[4];       // their bytes in B (each at its destination's offset in a 32-symbol word)
    uint32_t zt, ot;        // symbols of the two runs of A
    uint32_t b1;            // byte of A's ones run (the zeros run starts at (gz & 31) w)
    uint32_t groups, zgroups;  // 32-symbol groups of A: all, and those of the zeros run
    uint32_t need_b;
    uint32_t *next1, *next2, *plane3;
    void *nxt;
};

struct PairShared {
    PairStage st[kPairStages];
    PairJob job;              // the job of the claimer's latest tile
    PairPlan plan[2];
    uint64_t bar[kPairStages];
    uint32_t wsum[3][kLwWarps];  // per batch of kLwThreads groups, each warp's ones of bit l + 1
};

template <typename Sym>
__device__ __forceinline__ void pair_claim(const PairLaunch &a, PairShared &sh, unsigned char *in, unsigned char *bits,
                                           unsigned char *planes, int s, uint32_t g, uint32_t g_end, uint32_t &k,
                                           bool &have_job) {
    using Cfg = LwCfg<Sym>;
    constexpr int kJobWords = (int)(sizeof(PairJob) / 8);
    static_assert(kJobWords <= 32, "a pair job is copied by one warp");
    const int lane = threadIdx.x & 31;
    PairStage &S = sh.st[s];
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
        const bool full = S.J.n - base >= Cfg::kTile && (reinterpret_cast<uintptr_t>(S.J.cur) & 15) == 0;
        S.tile = tile;
        S.full = full;
        fence_proxy_async_smem();
        const uint32_t bits_bytes = (uint32_t)min((uint64_t)(Cfg::kTile / 8), S.J.nblocks * 64 - base / 8);
        S.bits_bytes = bits_bytes;
        const uint64_t pstride = way_pre_stride((uint64_t)S.J.ntiles * Cfg::kUnits);
        mbar_arrive_expect(&sh.bar[s], 3 * Cfg::kPreCopy * 8 + (full ? kLwTileBytes : 0) + 2 * bits_bytes);
#pragma unroll
        for (int w = 0; w < 3; w++)
            bulk_copy(S.pre[w], S.J.pre + w * pstride + (size_t)tile * Cfg::kUnits, Cfg::kPreCopy * 8, &sh.bar[s]);
        if (full) bulk_copy(in + s * kLwTileBytes, static_cast<const Sym *>(S.J.cur) + base, kLwTileBytes, &sh.bar[s]);
        if (bits_bytes) {
            bulk_copy(bits + s * kLwStageBits, reinterpret_cast<const unsigned char *>(S.J.words) + base / 8,
                      bits_bytes, &sh.bar[s]);
            bulk_copy(planes + s * kLwStageBits, reinterpret_cast<const unsigned char *>(S.J.plane) + base / 8,
                      bits_bytes, &sh.bar[s]);
        }
    }
}

// Phase 1 of a tile (all threads): a tile in one node of level l is split by
// bit l into A (its zeros run at byte (gz & 31) w, its ones run at plan.b1,
// each at its destination's offset in a 32-symbol word of level l + 1's
// bitmap); thread 0 writes the tile's plan.  A tile spanning several nodes
// places each symbol itself.  runs is the same in every thread.
template <typename Sym, bool kWhole>
__device__ __forceinline__ void pair_tile(const PairLaunch &a, const PairStage &S, const unsigned char *buf,
                                          const unsigned char *sbits, unsigned char *A, PairPlan &plan, bool &runs,
                                          bool &bad) {
    using Cfg = LwCfg<Sym>;
    constexpr int kSps = Cfg::kSps;
    constexpr int kW = Cfg::kW;
    constexpr uint32_t kUpw = Cfg::kUnitsPerWarp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l = a.l;
    const PairJob &J = S.J;
    const uint64_t base = (uint64_t)S.tile * Cfg::kTile;
    const uint32_t cnt = kWhole ? Cfg::kTile : (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
    const uint64_t P = S.pre[0][0], P01 = S.pre[1][0], P11 = S.pre[2][0];  // before the tile
    const uint64_t t1 = S.pre[0][Cfg::kUnits] - P;                          // the tile's level-l ones
    const uint64_t t01 = S.pre[1][Cfg::kUnits] - P01, t11 = S.pre[2][Cfg::kUnits] - P11;
    const uint32_t bsh = J.L - 1 - l;  // level l's bit
    const uint32_t shv = J.L - l;      // key_l = s >> shv
    const uint32_t nodes = 1u << l;
    const Sym *sb = reinterpret_cast<const Sym *>(buf);
    const uint32_t kfirst = (uint32_t)sb[0] >> shv, klast = (uint32_t)sb[cnt - 1] >> shv;
    runs = false;
    // The counts must describe a tile of cnt symbols; anything else is an
    // internal inconsistency and places nothing.
    if (t1 > cnt || t01 > cnt - t1 || t11 > t1) {
        bad = true;
        return;
    }
    const uint32_t Zt = cnt - (uint32_t)t1, Ot = (uint32_t)t1;
    if (kfirst == klast && kfirst < nodes) {
        const uint32_t v = kfirst;
        const uint64_t gz = (base - P) + __ldg(J.ob + v);
        const uint64_t go = P + __ldg(J.ze + v);
        uint64_t d[4] = {0, 0, 0, 0};
        uint32_t len[4] = {Zt - (uint32_t)t01, (uint32_t)t01, Ot - (uint32_t)t11, (uint32_t)t11};
        bool ok = gz + Zt <= J.n && go + Ot <= J.n;
        if (J.need_b) {
            const uint64_t pg[4] = {(base - P) - P01, P01, P - P11, P11};
#pragma unroll
            for (int g = 0; g < 4; g++) {
                d[g] = __ldg(J.T + 4 * v + g) + pg[g];
                ok = ok && d[g] + len[g] <= J.n;
            }
        }
        if (!ok) {
            bad = true;
            return;
        }
        runs = true;
        const uint32_t offz = (uint32_t)(gz & 31) * kW;
        const uint32_t B1 = ((offz + Zt * kW + 32 * kW - 1) / (32 * kW)) * (32 * kW) + (uint32_t)(go & 31) * kW;
        // Level bits of the lane's chunks, counts, and the split by bit l.
        constexpr int kPk = (kLwSteps + 1) / 2;  // two steps' counts per word (16 bits each)
        uint32_t h[kLwSteps];
        uint32_t cpk[kPk], lpk[kPk], tpk[kPk];
#pragma unroll
        for (int k2 = 0; k2 < kPk; k2++) cpk[k2] = 0;
#pragma unroll
        for (int st = 0; st < kLwSteps; st++) {
            const uint32_t q = warp * kLwWarpBytes + st * 512 + 16 * lane;
            const uint32_t b0 = q / kW / 8;
            uint32_t hb = 0;
            if (kWhole || b0 < S.bits_bytes) {
                if (kSps == 16) hb = *reinterpret_cast<const uint16_t *>(sbits + b0);
                if (kSps == 8) hb = sbits[b0];
                if (kSps == 4) hb = (sbits[b0] >> (4 * (lane & 1))) & 15u;
            }
            h[st] = hb;
            cpk[st >> 1] += (uint32_t)__popc(hb) << (16 * (st & 1));
        }
        uint32_t wtot = 0;
#pragma unroll
        for (int k2 = 0; k2 < kPk; k2++) {
            lpk[k2] = warp_excl_scan(cpk[k2], lane, tpk[k2]);
            wtot += (tpk[k2] & 0xffffu) + (tpk[k2] >> 16);
        }
        const uint64_t wx64 = S.pre[0][warp * kUpw] - P;  // ones of the tile before this warp's range
        if (wx64 + wtot > t1 || wx64 > (uint64_t)warp * (kLwWarpBytes / kW)) {
            bad = true;  // this warp's prefix disagrees with the tile's count: it places nothing
        } else {
            const uint32_t wx = (uint32_t)wx64;
            uint32_t stx = 0;
#pragma unroll
            for (int st = 0; st < kLwSteps; st++) {
                const uint32_t q = warp * kLwWarpBytes + st * 512 + 16 * lane;
                const uint32_t sh16 = 16 * (st & 1);
                const uint32_t o = wx + stx + ((lpk[st >> 1] >> sh16) & 0xffffu);
                stx += (tpk[st >> 1] >> sh16) & 0xffffu;
                const uint4 vv = *reinterpret_cast<const uint4 *>(buf + q);
                const uint32_t x[4] = {vv.x, vv.y, vv.z, vv.w};
                uint32_t po = B1 + o * kW;
                const uint32_t C = offz + B1 + q;
#pragma unroll
                for (int kk = 0; kk < kSps; kk++) {
                    if (kWhole || q / kW + kk < cnt) {
                        const bool one = (h[st] >> kk) & 1u;
                        const uint32_t at = one ? po : C + kk * kW - po;
                        const uint32_t sv = sym_at<Sym>(x, kk);
                        if (kW == 1) A[at] = (unsigned char)sv;
                        if (kW == 2) *reinterpret_cast<uint16_t *>(A + at) = (uint16_t)sv;
                        if (kW == 4) *reinterpret_cast<uint32_t *>(A + at) = sv;
                        po += one ? kW : 0;
                    }
                }
            }
        }
        if (tid == 0) {
#pragma unroll
            for (int g = 0; g < 4; g++) {
                plan.d[g] = d[g];
                plan.len[g] = len[g];
            }
            uint32_t off = 0;
#pragma unroll
            for (int g = 0; g < 4; g++) {
                off = g ? (off + 32 * kW - 1) / (32 * kW) * (32 * kW) : 0;
                off += (uint32_t)(d[g] & 31) * kW;
                plan.boff[g] = off;
                off += len[g] * kW;
            }
            plan.gz = gz;
            plan.go = go;
            plan.zt = Zt;
            plan.ot = Ot;
            plan.b1 = B1;
            const uint32_t zg = Zt ? ((uint32_t)(gz & 31) + Zt + 31) / 32 : 0u;
            const uint32_t og = Ot ? ((uint32_t)(go & 31) + Ot + 31) / 32 : 0u;
            plan.zgroups = zg;
            plan.groups = zg + og;
            plan.need_b = J.need_b;
            plan.next1 = J.next1;
            plan.next2 = J.next2;
            plan.plane3 = J.plane3;
            plan.nxt = J.nxt;
        }
        return;
    }
    // Several nodes: each symbol to its positions in P_{l+1} and P_{l+2}.
    // A warp takes 32 consecutive symbols per round; the ones of level l and
    // the symbols of groups 01 and 11 before a symbol come from ballots.
    constexpr uint32_t kWarpSyms = kLwWarpBytes / kW;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t o = S.pre[0][warp * kUpw] - P;
    uint64_t q01 = S.pre[1][warp * kUpw] - P01, q11 = S.pre[2][warp * kUpw] - P11;
    Sym *nxt = static_cast<Sym *>(J.nxt);
    for (uint32_t g0 = 0; g0 < kWarpSyms; g0 += 32) {
        const uint32_t p = warp * kWarpSyms + g0 + lane;
        const bool in = kWhole || p < cnt;
        const uint32_t sv = in ? (uint32_t)sb[p] : 0u;
        const uint32_t b0 = (sv >> bsh) & 1u, b1 = (sv >> (bsh - 1)) & 1u;
        const uint32_t m0 = __ballot_sync(0xffffffffu, in && b0);
        const uint32_t m01 = __ballot_sync(0xffffffffu, in && !b0 && b1);
        const uint32_t m11 = __ballot_sync(0xffffffffu, in && b0 && b1);
        const uint64_t P1 = P + o + __popc(m0 & lt);        // level-l ones before this symbol
        const uint64_t c01 = P01 + q01 + __popc(m01 & lt);  // group-01 symbols before it
        const uint64_t c11 = P11 + q11 + __popc(m11 & lt);
        o += __popc(m0);
        q01 += __popc(m01);
        q11 += __popc(m11);
        if (!in) continue;
        const uint32_t v = sv >> shv;
        if (v >= nodes) {
            bad = true;
            continue;
        }
        const uint64_t pos = base + p;
        const uint64_t dst1 = b0 ? P1 + __ldg(J.ze + v) : (pos - P1) + __ldg(J.ob + v);
        if (dst1 >= J.n) {
            bad = true;
            continue;
        }
        if (b1) atomicOr(J.next1 + (dst1 >> 5), 1u << (dst1 & 31));
        if (!J.need_b) continue;
        const uint32_t grp = 2 * b0 + b1;
        const uint64_t pg = grp == 0 ? pos - P1 - c01 : grp == 1 ? c01 : grp == 2 ? P1 - c11 : c11;
        const uint64_t dst2 = __ldg(J.T + 4 * v + grp) + pg;
        if (dst2 >= J.n) {
            bad = true;
            continue;
        }
        if (nxt) nxt[dst2] = (Sym)sv;
        if (J.next2 && ((sv >> (bsh - 2)) & 1u)) atomicOr(J.next2 + (dst2 >> 5), 1u << (dst2 & 31));
        if (J.plane3 && ((sv >> (bsh - 3)) & 1u)) atomicOr(J.plane3 + (dst2 >> 5), 1u << (dst2 & 31));
    }
}

// The bits at shift bsh of a group of 32 symbols at g (32 w bytes, 16-byte
// aligned in shared memory); x receives the group's 16-byte chunks.
template <typename Sym>
__device__ __forceinline__ uint32_t group_bits(const unsigned char *g, uint32_t bsh, const BitGather &gg,
                                               uint4 (&x)[2 * sizeof(Sym)]) {
    constexpr uint32_t kW = sizeof(Sym);
    uint32_t bits = 0;
#pragma unroll
    for (uint32_t c = 0; c < 2 * kW; c++) {
        x[c] = *reinterpret_cast<const uint4 *>(g + 16 * c);
        const uint32_t w[4] = {x[c].x, x[c].y, x[c].z, x[c].w};
        bits |= gather_bits<Sym>(w, gg, bsh) << (c * (16 / kW));
    }
    return bits;
}

// Word k of a run whose first position is `dest` (first bit dest & 31 in
// word 0) and which holds len symbols: the mask of the run's bits.
__device__ __forceinline__ uint32_t run_word_mask(uint64_t dest, uint32_t len, uint32_t k) {
    const uint32_t first = (uint32_t)(dest & 31);
    const uint32_t lo = k == 0 ? first : 0u;
    const uint32_t hi = min(32u, first + len - 32 * k);
    return (hi == 32 ? ~0u : (1u << hi) - 1u) & ~((1u << lo) - 1u);
}

__device__ __forceinline__ void put_bits(uint32_t *w, uint32_t bits, uint32_t mask) {
    if (mask == ~0u)
        *w = bits;
    else if (bits & mask)
        atomicOr(w, bits & mask);
}

template <typename Sym>
__global__ void __launch_bounds__(kLwThreads, 4) pair_pass_kernel(PairLaunch a) {
    using Cfg = LwCfg<Sym>;
    constexpr uint32_t kW = sizeof(Sym);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *in = smem;                                   // kPairStages x kLwTileBytes
    unsigned char *bits = in + kPairStages * kLwTileBytes;      // kPairStages x kLwStageBits (level l)
    unsigned char *planes = bits + kPairStages * kLwStageBits;  // kPairStages x kLwStageBits (bit l + 1)
    unsigned char *A = planes + kPairStages * kLwStageBits;     // kLwSplitBytes
    unsigned char *B = A + kLwSplitBytes;                       // kPairBBytes
    PairShared &sh = *reinterpret_cast<PairShared *>(B + kPairBBytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const uint32_t per = (a.total_tiles + gridDim.x - 1) / gridDim.x;
    const uint32_t g_begin = min(blockIdx.x * per, a.total_tiles);
    const uint32_t g_end = min(g_begin + per, a.total_tiles);
    uint32_t k = 0;
    bool have_job = false;
    const bool claimer = warp == kLwWarps - 1;
    const bool issuer = tid < 128 && lane == 0;  // threads that bulk-store a run of B
    if (tid == 0) {
        for (int s = 0; s < kPairStages; s++) mbar_init(&sh.bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (claimer) {
        if (g_begin < g_end) k = pair_find_job(a, g_begin);
        for (int s = 0; s < kPairStages - 1; s++)
            pair_claim<Sym>(a, sh, in, bits, planes, s, g_begin + s, g_end, k, have_job);
    }
    __syncthreads();

    bool failed = false, bad = false;
    if (__syncthreads_or(!mbar_wait(&sh.bar[0], 0u))) failed = true;
    for (uint32_t i = 0; !failed; i++) {
        const int s = (int)(i % kPairStages), par = (int)(i & 1);
        const PairStage &S = sh.st[s];
        if (S.tile == kNoTile) break;
        if (claimer)
            pair_claim<Sym>(a, sh, in, bits, planes, (int)((i + kPairStages - 1) % kPairStages),
                            g_begin + i + kPairStages - 1, g_end, k, have_job);
        unsigned char *buf = in + s * kLwTileBytes;
        PairPlan &plan = sh.plan[par];
        // Without B (level l + 1 is the last), A alternates with B's memory:
        // no barrier follows the reads of A then, so tile i + 1 must not
        // split into the buffer tile i is still reading.
        unsigned char *Ab = (a.need_b || par == 0) ? A : B;
        const uint32_t L = S.J.L;
        bool runs = false;
        {
            const PairJob &J = S.J;
            const uint64_t base = (uint64_t)S.tile * Cfg::kTile;
            const uint32_t cnt = (uint32_t)min((uint64_t)Cfg::kTile, J.n - base);
            if (!S.full) {
                const Sym *src = static_cast<const Sym *>(J.cur);
                Sym *sb = reinterpret_cast<Sym *>(buf);
                for (uint32_t p = tid; p < Cfg::kTile; p += kLwThreads) sb[p] = p < cnt ? src[base + p] : (Sym)0;
                __syncthreads();
            }
            const unsigned char *sbits = bits + s * kLwStageBits;
            if (cnt == Cfg::kTile)
                pair_tile<Sym, true>(a, S, buf, sbits, Ab, plan, runs, bad);
            else
                pair_tile<Sym, false>(a, S, buf, sbits, Ab, plan, runs, bad);
        }
        // B's bulk stores of the previous tile must have read it before the
        // groups of this tile write it (after the barriers below).
        if (issuer) bulk_wait_read0();
        const uint32_t i1 = i + 1;
        const bool ok = mbar_wait(&sh.bar[i1 % kPairStages], (i1 / kPairStages) & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (!runs) continue;  // the same in every thread
        // Phase 2: A's 32-symbol groups (thread t: groups t, t + kLwThreads, ...).
        const uint32_t lv1 = L - 2 - a.l;  // level l + 1's bit
        const uint32_t G = plan.groups, ZG = plan.zgroups;
        const BitGather g1 = bit_gather<Sym>(lv1);
        uint32_t gb[kGB], gm[kGB], gc[kGB];
#pragma unroll
        for (int r = 0; r < kGB; r++) {
            gb[r] = gm[r] = gc[r] = 0;
            const uint32_t gi = tid + r * kLwThreads;
            if (gi >= G) continue;
            const bool onesrun = gi >= ZG;
            const uint32_t kk = onesrun ? gi - ZG : gi;
            const uint64_t dest = onesrun ? plan.go : plan.gz;
            const uint32_t len = onesrun ? plan.ot : plan.zt;
            const uint32_t abase = onesrun ? plan.b1 - (uint32_t)(dest & 31) * kW : 0u;
            uint4 x[2 * kW];
            const uint32_t gbits = group_bits<Sym>(Ab + abase + kk * 32 * kW, lv1, g1, x);
            const uint32_t mask = run_word_mask(dest, len, kk);
            put_bits(plan.next1 + (dest >> 5) + kk, gbits, mask);
            gb[r] = gbits & mask;
            gm[r] = mask;
            gc[r] = __popc(gbits & mask);
        }
        if (!plan.need_b) continue;  // level l + 1 is the last: no B
        // Block scan of the groups' ones of bit l + 1, in group order: batch
        // r holds groups [r kLwThreads, (r + 1) kLwThreads).
        uint32_t inc[kGB];
#pragma unroll
        for (int r = 0; r < kGB; r++) {
            inc[r] = gc[r];
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc[r], dd);
                if (lane >= dd) inc[r] += y;
            }
            if (lane == 31) sh.wsum[r][warp] = inc[r];
        }
        __syncthreads();
        uint32_t pref[kGB];
        uint32_t done = 0;  // ones of the batches before r
#pragma unroll
        for (int r = 0; r < kGB; r++) {
            uint32_t before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kLwWarps; w++) {
                const uint32_t t = sh.wsum[r][w];
                before += w < warp ? t : 0u;
                total += t;
            }
            pref[r] = done + before + inc[r] - gc[r];
            done += total;
        }
        // Phase 3: each group splits by bit l + 1 into B.
#pragma unroll
        for (int r = 0; r < kGB; r++) {
            const uint32_t gi = tid + r * kLwThreads;
            if (gi >= G) continue;
            const uint32_t onesrun = gi >= ZG ? 1u : 0u;
            const uint32_t kk = onesrun ? gi - ZG : gi;
            const uint64_t dest = onesrun ? plan.go : plan.gz;
            const uint32_t a0 = (uint32_t)(dest & 31);
            const uint32_t abase = onesrun ? plan.b1 - a0 * kW : 0u;
            const uint32_t ones_before = pref[r] - (onesrun ? plan.len[1] : 0u);
            const uint32_t valid_before = kk ? 32 * kk - a0 : 0u;
            const uint32_t lo = kk ? 0u : a0;
            const uint32_t len1 = plan.len[2 * onesrun + 1], len0 = plan.len[2 * onesrun];
            const uint32_t c1 = gc[r], cv = __popc(gm[r]);
            // Counts must fit the group runs (and so B); else this group places nothing.
            if (ones_before > valid_before || ones_before + c1 > len1 ||
                valid_before - ones_before + (cv - c1) > len0 ||
                (!onesrun && kk + 1 == ZG && pref[r] + c1 != plan.len[1])) {
                bad = true;
                continue;
            }
            const uint32_t zeros_before = valid_before - ones_before;
            const uint32_t B0 = plan.boff[2 * onesrun], B1r = plan.boff[2 * onesrun + 1];
            uint32_t po = B1r + ones_before * kW;
            const uint32_t Cz = B0 + zeros_before * kW + B1r + ones_before * kW - lo * kW;
            const unsigned char *g = A + abase + kk * 32 * kW;
            const uint32_t m = gm[r], bb = gb[r];
#pragma unroll
            for (uint32_t c = 0; c < 2 * kW; c++) {
                const uint4 v4 = *reinterpret_cast<const uint4 *>(g + 16 * c);
                const uint32_t xw[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (uint32_t q = 0; q < 16 / kW; q++) {
                    const uint32_t j = c * (16 / kW) + q;
                    if ((m >> j) & 1u) {
                        const bool one = (bb >> j) & 1u;
                        const uint32_t at = one ? po : Cz + j * kW - po;
                        const uint32_t sv = sym_at<Sym>(xw, (int)q);
                        if (kW == 1) B[at] = (unsigned char)sv;
                        if (kW == 2) *reinterpret_cast<uint16_t *>(B + at) = (uint16_t)sv;
                        if (kW == 4) *reinterpret_cast<uint32_t *>(B + at) = sv;
                        po += one ? kW : 0u;
                    }
                }
            }
        }
        fence_proxy_async_smem();  // B is read by bulk stores
        __syncthreads();
        // Phase 4: B's runs go out; level l + 2's bitmap and bit l + 3 from B.
        if (plan.nxt && tid < 128) {
            const uint32_t g = (uint32_t)tid >> 5;
            const uintptr_t g0 = reinterpret_cast<uintptr_t>(static_cast<Sym *>(plan.nxt) + plan.d[g]);
            store_run(g0, plan.len[g] * kW, B + plan.boff[g], lane);
            if (lane == 0) bulk_commit();
        }
        if (plan.next2 || plan.plane3) {
            const uint32_t lv2 = lv1 - 1;  // level l + 2's bit; bit l + 3 is lv2 - 1
            const BitGather g2 = bit_gather<Sym>(lv2);
            const BitGather g3 = bit_gather<Sym>(plan.plane3 ? lv2 - 1 : 0u);
            uint32_t nw[4], tot = 0;
#pragma unroll
            for (int g = 0; g < 4; g++) {
                nw[g] = plan.len[g] ? ((uint32_t)(plan.d[g] & 31) + plan.len[g] + 31) / 32 : 0u;
                tot += nw[g];
            }
            for (uint32_t t = tid; t < tot; t += kLwThreads) {
                // The run of word t and the word's index in it.
                const uint32_t e1 = nw[0], e2 = e1 + nw[1], e3 = e2 + nw[2];
                const uint32_t g = t < e1 ? 0u : t < e2 ? 1u : t < e3 ? 2u : 3u;
                const uint32_t kk = t - (g == 0 ? 0u : g == 1 ? e1 : g == 2 ? e2 : e3);
                const uint64_t dest = plan.d[g];
                const unsigned char *gp = B + plan.boff[g] - (uint32_t)(dest & 31) * kW + kk * 32 * kW;
                uint4 x[2 * kW];
                const uint32_t b2 = group_bits<Sym>(gp, lv2, g2, x);
                const uint32_t mask = run_word_mask(dest, plan.len[g], kk);
                if (plan.next2) put_bits(plan.next2 + (dest >> 5) + kk, b2, mask);
                if (plan.plane3) {
                    uint32_t b3 = 0;
#pragma unroll
                    for (uint32_t c = 0; c < 2 * kW; c++) {
                        const uint32_t w[4] = {x[c].x, x[c].y, x[c].z, x[c].w};
                        b3 |= gather_bits<Sym>(w, g3, lv2 - 1) << (c * (16 / kW));
                    }
                    put_bits(plan.plane3 + (dest >> 5) + kk, b3, mask);
                }
            }
        }
    }
    if (issuer) bulk_wait_all();
    if (failed && tid == 0) atomicOr(a.err, kErrTimeout);
    if (bad) atomicOr(a.err, kErrTimeout);
}

constexpr size_t kPairSmem = kPairStages * (kLwTileBytes + 2 * kLwStageBits) + kLwSplitBytes + kPairBBytes +
                             sizeof(PairShared);
static_assert(4 * (kPairSmem + 1024) <= 228 * 1024, "pair pass shared memory: four CTAs per SM");

template <typename Sym>
cudaError_t launch_pair_t(const PairLaunch &a, bool from_bits, bool counted, const LevelJob *scan_job,
                          uint32_t ntiles, cudaStream_t st) {
    static int slots = 0, sms = 0;
    if (!slots) {
        cudaError_t e =
            cudaFuncSetAttribute(pair_pass_kernel<Sym>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem);
        if (e != cudaSuccess) return e;
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_pass_kernel<Sym>, kLwThreads, kPairSmem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        slots = sms * per_sm;
    }
    if (!counted) {
        const uint32_t cw = (a.total_tiles + 7) / 8;
        const uint32_t g0 = cw < (uint32_t)(sms * 8) ? cw : (uint32_t)(sms * 8);
        if (from_bits)
            pair_count_kernel<Sym, true><<<g0, 256, 0, st>>>(a);
        else
            pair_count_kernel<Sym, false><<<g0, 256, 0, st>>>(a);
        note_launches(1);
    }
    cudaError_t e = launch_level_scans((int)sizeof(Sym), a.l, scan_job, 1, ntiles, 3, st);
    if (e != cudaSuccess) return e;
    const int grid = (int)(a.total_tiles < (uint32_t)slots ? a.total_tiles : (uint32_t)slots);
    pair_pass_kernel<Sym><<<grid, kLwThreads, kPairSmem, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

// Writes the pair job, the scan job of level l and the tile range to device memory.
__global__ void put_pair_job_kernel(PairJob pj, LevelJob lj, PairJob *dp, LevelJob *dl, uint32_t *tile_start) {
    *dp = pj;
    *dl = lj;
    tile_start[0] = 0;
    tile_start[1] = pj.ntiles;
}

// Pair tables of the levels in `levels`: one CTA each (at most 2^16 nodes).
// CTA b takes the b-th set bit l.  Sizes of the four grandchildren of node
// v: C_{l+2}[4v + g + 1] - C_{l+2}[4v + g], C_{l+2}[x] = Hex[x << (L - l - 2)].
constexpr int kTabThreads = 1024;

__device__ __forceinline__ uint64_t tab_block_scan(uint64_t v, uint64_t *s_warp) {
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
        const uint64_t w = s_warp[lane];
        uint64_t winc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, winc, d);
            if (lane >= d) winc += y;
        }
        s_warp[lane] = winc - w;
    }
    __syncthreads();
    const uint64_t r = s_warp[warp] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kTabThreads) pair_tables_kernel(const uint64_t *__restrict__ hex, uint32_t L,
                                                                  uint32_t levels, uint64_t *__restrict__ T) {
    __shared__ uint64_t s_warp[32];
    uint32_t l = 0, b = blockIdx.x;
    for (;; l++)
        if ((levels >> l) & 1u) {
            if (b == 0) break;
            b--;
        }
    const uint64_t nodes = 1ull << l;
    const uint32_t sh = L - l - 2;
    const uint64_t chunk = ceil_div(nodes, kTabThreads);
    const uint64_t lo = min(threadIdx.x * chunk, nodes), hi = min(lo + chunk, nodes);
    uint64_t *Tl = T + 4 * (nodes - 1);
#pragma unroll
    for (int g = 0; g < 4; g++) {
        uint64_t sum = 0;
        for (uint64_t v = lo; v < hi; v++) sum += hex[(4 * v + g + 1) << sh] - hex[(4 * v + g) << sh];
        uint64_t run = tab_block_scan(sum, s_warp);
        for (uint64_t v = lo; v < hi; v++) {
            const uint64_t c0 = hex[(4 * v + g) << sh];
            Tl[4 * v + g] = c0 - run;
            run += hex[(4 * v + g + 1) << sh] - c0;
        }
    }
}

}  // namespace

cudaError_t launch_pair_tables(const uint64_t *hex, uint32_t L, uint32_t levels, uint64_t *T, cudaStream_t st) {
    const int count = __builtin_popcount(levels);
    if (count == 0) return cudaSuccess;
    pair_tables_kernel<<<count, kTabThreads, 0, st>>>(hex, L, levels, T);
    note_launches(1);
    return cudaGetLastError();
}

size_t pair_job_slot_bytes() {
    return ((sizeof(PairJob) + 255) & ~size_t(255)) + ((sizeof(LevelJob) + 255) & ~size_t(255)) + 256 +
           level_job_slot_bytes();
}

cudaError_t launch_pair_step(const PairJob &j, int width, uint32_t l, LevelDesc lv, uint64_t *ones_out, LevelDesc lv1,
                             uint64_t *ones1_out, bool from_bits, bool counted, uint32_t *cnt1, uint64_t *pre1,
                             uint32_t *err, void *job_slot, cudaStream_t st) {
    if (j.n == 0) return cudaSuccess;
    char *p = static_cast<char *>(job_slot);
    PairJob *dp = reinterpret_cast<PairJob *>(p);
    p += (sizeof(PairJob) + 255) & ~size_t(255);
    LevelJob *dl = reinterpret_cast<LevelJob *>(p);
    p += (sizeof(LevelJob) + 255) & ~size_t(255);
    uint32_t *ts = reinterpret_cast<uint32_t *>(p);
    p += 256;
    void *dir_slot = p;
    // The scan job of level l: its units' counts and prefixes (three ways)
    // and its directory.
    LevelJob lj = make_level_job(nullptr, nullptr, j.n, width, j.L, l, nullptr, nullptr, lv, ones_out, j.cnt, j.pre,
                                 nullptr);
    lj.nxt = nullptr;
    put_pair_job_kernel<<<1, 1, 0, st>>>(j, lj, dp, dl, ts);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PairLaunch a;
    a.jobs = dp;
    a.tile_start = ts;
    a.njobs = 1;
    a.total_tiles = j.ntiles;
    a.l = l;
    a.need_b = j.need_b;
    a.err = err;
    switch (width) {
        case 1: e = launch_pair_t<uint8_t>(a, from_bits, counted, dl, j.ntiles, st); break;
        case 2: e = launch_pair_t<uint16_t>(a, from_bits, counted, dl, j.ntiles, st); break;
        case 4: e = launch_pair_t<uint32_t>(a, from_bits, counted, dl, j.ntiles, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    // Level l + 1's directory from the bitmap the pass wrote.
    return launch_level_directory(j.n, width, j.L, l + 1, lv1, ones1_out, cnt1, pre1, err, dir_slot, st);
}

}  // namespace wt
