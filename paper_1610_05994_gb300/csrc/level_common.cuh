// level_common.cuh -- pieces shared by the level passes (level.cu: one
// level per pass; pair.cu: two levels per pass): the tile geometry, the
// launch record, bit extraction from 16-byte chunks of symbols and the bulk
// stores of split runs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kLwThreads = 128;
constexpr int kLwWarps = kLwThreads / 32;
constexpr int kLwSteps = 4;                                        // 512-byte warp steps per warp
constexpr uint32_t kLwWarpBytes = 512 * kLwSteps;                  // a warp's range of the tile
constexpr uint32_t kLwTileBytes = kLwWarpBytes * kLwWarps;         // 8 KB
// Two runs, each starting at its destination's offset in a 32-symbol word
// of the next bitmap, plus the reads of whole 32-symbol groups (4-byte
// symbols: 2048 + 124 symbols at most).
constexpr uint32_t kLwSplitBytes = kLwTileBytes + 512;
constexpr int kLwStages = 2;                                       // input stages: the claimer stays one tile ahead
constexpr uint32_t kLwStageBits = kLwTileBytes / 8;                 // a stage's copy of the level's bitmap (bytes)
constexpr uint32_t kNoTile = 0xffffffffu;
// The counts and prefixes are kept per unit of P_l: a warp's range or a rank
// block of the bitmap, whichever is shorter (kLwWarpBytes or 512 symbols).
// Every warp of the pass then reads the ones before its own range, and the
// prefix scan reads the ones before every rank block, which is the rank
// directory itself.
constexpr uint32_t lw_unit_bytes(uint32_t width) { return 512 * width < kLwWarpBytes ? 512 * width : kLwWarpBytes; }
constexpr uint32_t lw_units(uint32_t width) { return kLwTileBytes / lw_unit_bytes(width); }  // per tile
constexpr uint32_t kLwMaxUnits = lw_units(1);

template <typename Sym>
struct LwCfg {
    static constexpr int kW = (int)sizeof(Sym);
    static constexpr int kSps = 16 / kW;                              // symbols per 16-byte chunk
    static constexpr uint32_t kTile = kLwTileBytes / kW;              // symbols per tile
    static constexpr uint32_t kBlocks = kTile / 512;                  // rank blocks per tile
    static constexpr int kMinCtas = 6;                                // resident CTAs per SM
    static constexpr uint32_t kUnits = lw_units(sizeof(Sym));         // count units per tile
    static constexpr uint32_t kUnitsPerWarp = kLwWarpBytes / lw_unit_bytes(sizeof(Sym));
    static constexpr uint32_t kPreCopy = kUnits + 2;                  // prefixes copied per tile
};

constexpr uint32_t kScanSeg = kScanSegUnits;


struct LevelLaunch {
    const LevelJob *jobs;        // device array of njobs
    const uint32_t *tile_start;  // device, njobs + 1: first global tile of each job
    uint32_t njobs, total_tiles, l;
    uint32_t segs;               // scan segments of the largest job
    uint32_t units, upb;         // count units per tile and per rank block
    uint32_t *err;
    uint32_t ways;               // count arrays the scan turns into prefixes (1, or 3 for a pair step)
    uint32_t check_sigma;        // > 0: the count pass from the symbols flags any symbol >= check_sigma
    uint32_t one_node;           // every node has the same offsets: each tile is placed as node 0
    // Level l's node tables folded into the scan (one job, at most
    // kFoldNodes nodes): the last scan CTA to finish does rank_tables_kernel's
    // work.  rt_nodes = 0: the tables come from their own launch, or none.
    uint32_t rt_nodes;
    uint32_t *rt_done;           // scan CTAs finished, zeroed by put_job_kernel
    const uint64_t *rt_start_in;
    uint64_t *rt_ob, *rt_ze, *rt_start_out;
};

// Whether some symbol of a 16-byte chunk is >= sigma (sigma >= 1).  For bytes
// with sigma <= 128: b >= 128 is out of range, and for b < 128 the byte
// (b | 0x80) - sigma keeps its top bit exactly when b >= sigma, with no
// borrow between bytes; for 128 < sigma < 256 the same test on the low
// seven bits against sigma - 128, for bytes with the top bit set.
template <typename Sym>
__device__ __forceinline__ bool chunk_out_of_range(const uint32_t (&x)[4], uint32_t sigma) {
    if (sizeof(Sym) == 1) {
        if (sigma >= 256) return false;
        uint32_t t = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (sigma <= 128) {
                t |= (x[q] & 0x80808080u) | (((x[q] | 0x80808080u) - sigma * 0x01010101u) & 0x80808080u);
            } else {
                const uint32_t y = (x[q] & 0x7f7f7f7fu) | 0x80808080u;
                t |= x[q] & (y - (sigma - 128u) * 0x01010101u) & 0x80808080u;
            }
        }
        return t != 0;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 16 / (int)sizeof(Sym); k++) {
        const uint32_t v = sizeof(Sym) == 2 ? (x[k >> 1] >> (16 * (k & 1))) & 0xffffu : x[k];
        bad |= v >= sigma;
    }
    return bad;
}

// Job of global tile t: the largest k with tile_start[k] <= t.
__device__ __forceinline__ uint32_t find_job(const LevelLaunch &a, uint32_t t) {
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

// The bits at shift `bsh` of the symbols of one 16-byte chunk, packed: bit k
// = the chunk's symbol k.  Per 32-bit word the bit is first moved to the top
// of each symbol's slot; for bytes one multiply then gathers the four top
// bits into a nibble (its partial products meet only in bits 28..31).
template <typename Sym>
__device__ __forceinline__ uint32_t chunk_bits(const uint32_t (&x)[4], uint32_t bsh) {
    uint32_t h = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (sizeof(Sym) == 1) h |= ((((x[q] << (7 - bsh)) & 0x80808080u) * 0x00204081u) >> 28) << (4 * q);
        if (sizeof(Sym) == 2) {
            const uint32_t m = (x[q] << (15 - bsh)) & 0x80008000u;
            h |= (((m >> 15) | (m >> 30)) & 3u) << (2 * q);
        }
        if (sizeof(Sym) == 4) h |= ((x[q] >> bsh) & 1u) << q;
    }
    return h;
}

// The same bits gathered with one AND and one 64-bit multiply per 8 bytes
// (the multiply runs on the FMA pipe, which the passes leave mostly idle,
// where chunk_bits spends shifts and masks on the ALU pipe).  For bytes the
// AND keeps bit bsh of each byte j at 8 j + bsh; the multiplier (the sum of
// 2^(7 k + 7 - bsh), k = 0..7) moves it to bit 56 + j, every other partial
// product lands on a distinct bit below 56 or beyond 63, so nothing carries
// into the top byte.  For 2-byte symbols the same with 2^(15 k + 15 - bsh),
// k = 0..3, and the top nibble.
struct BitGather {
    uint64_t mask, mul;
};
template <typename Sym>
__device__ __forceinline__ BitGather bit_gather(uint32_t bsh) {
    BitGather g;
    if (sizeof(Sym) == 1) {
        g.mask = 0x0101010101010101ull << bsh;
        g.mul = 0x0102040810204080ull >> bsh;
    } else {
        g.mask = 0x0001000100010001ull << bsh;
        g.mul = ((1ull << 15) | (1ull << 30) | (1ull << 45) | (1ull << 60)) >> bsh;
    }
    return g;
}
template <typename Sym>
__device__ __forceinline__ uint32_t gather_bits(const uint32_t (&x)[4], const BitGather &g, uint32_t bsh) {
    if (sizeof(Sym) == 4) return chunk_bits<Sym>(x, bsh);
    const uint64_t lo = ((uint64_t)x[1] << 32) | x[0], hi = ((uint64_t)x[3] << 32) | x[2];
    constexpr int kTop = sizeof(Sym) == 1 ? 56 : 60, kPer = sizeof(Sym) == 1 ? 8 : 4;
    const uint32_t a = (uint32_t)(((lo & g.mask) * g.mul) >> kTop);
    const uint32_t b = (uint32_t)(((hi & g.mask) * g.mul) >> kTop);
    return a | (b << kPer);
}

template <typename Sym>
__device__ __forceinline__ uint32_t sym_at(const uint32_t (&x)[4], int k) {
    if (sizeof(Sym) == 1) return (x[k >> 2] >> (8 * (k & 3))) & 0xffu;
    if (sizeof(Sym) == 2) return (x[k >> 1] >> (16 * (k & 1))) & 0xffffu;
    return x[k];
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane, uint32_t &total) {
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Writes one run of the split copy to global memory: bytes [g0, g0 + len)
// of the destination, held in shared memory at s (s and g0 agree modulo 16).
// rt == 0 sends the 16-byte-aligned interior with one bulk store; rt in
// [0, 32) (the caller's thread index relative to the run) writes the ragged
// head (< 16 bytes) and tail (< 16 bytes).
__device__ __forceinline__ void store_run(uintptr_t g0, uint32_t len, const unsigned char *s, int rt) {
    if (len == 0) return;
    const uintptr_t g1 = g0 + len;
    const uintptr_t a = (g0 + 15) & ~(uintptr_t)15, b = g1 & ~(uintptr_t)15;
    const uintptr_t head_end = a < g1 ? a : g1;
    if (rt == 0 && b > a) bulk_store(reinterpret_cast<void *>(a), s + (a - g0), (uint32_t)(b - a));
    if (rt < 16) {
        const uintptr_t x = g0 + rt;
        if (x < head_end) *reinterpret_cast<unsigned char *>(x) = s[x - g0];
    } else if (rt < 32) {
        const uintptr_t t0 = b > head_end ? b : head_end;
        const uintptr_t x = t0 + (rt - 16);
        if (x < g1) *reinterpret_cast<unsigned char *>(x) = s[x - g0];
    }
}

}  // namespace wt
