// level.cu -- kernels (b) + (c): the fused per-level pass of the level-wise
// build.
//
// One pass over P_l (the symbols in level-l order) does, per tile of 16 KB:
//   (b) packs the level-l bit of every symbol into the bitmap, counts ones
//       per lane/warp/tile, obtains the ones before the tile with a decoupled
//       look-back, and writes the rank directory (R, Hy) and the select
//       samples (S1, S0) from those prefixes;
//   (c) places every symbol at its position in P_{l+1}:
//          bit 0:  dst = zeros_before(p) + OB_l[v]
//          bit 1:  dst = ones_before(p)  + ZE_l[v]
//       with v = key_l(s), OB_l[v] = ones on level l before node v's start and
//       ZE_l[v] = zeros on level l up to node v's end.  This is the stable
//       counting-sort placement of Algorithm 1 ("bitmapSetBit at C[node]++",
//       Section 3.1) written as a closed form of two prefix counts, so one
//       global scan serves every node of the level.
//
// GPU structure: a persistent, warp-specialised CTA per SM slot.
//   * The producer warp takes tiles from an atomic ticket (two ahead),
//     streams them into a double-buffered shared-memory slot with 1-D TMA
//     bulk copies (cp.async.bulk, mbarrier completion), counts each tile's
//     ones the moment it lands and publishes that aggregate, then runs the
//     decoupled look-back of the oldest tile.
//   * Sixteen compute warps read a slot (four consecutive symbols per lane,
//     128 per warp step), write the bitmap words at once, count, split the
//     tile stably by the bit into a second double-buffered slot (zeros, then
//     ones; lanes write neighbouring bytes, so no bank conflicts), and only
//     then place the previous tile, whose prefix the producer has found
//     meanwhile.  No compute warp ever waits on the look-back chain.
// mbarriers link the two roles; every wait is bounded (kWaitLimitNs) and a
// give-up sets kErrTimeout and drains the CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kCompWarps = 16;
constexpr int kCompThreads = kCompWarps * 32;
constexpr int kLwThreads = kCompThreads + 32;      // + the producer warp
constexpr uint32_t kLwTileBytes = 16384;
constexpr uint32_t kEnd = 0xffffffffu;             // "no more tiles" in a slot

template <typename Sym>
struct LwCfg {
    static constexpr uint32_t kTile = kLwTileBytes / sizeof(Sym);  // symbols per tile
    static constexpr uint32_t kRange = kTile / kCompWarps;         // symbols per compute warp
    static constexpr int kSteps = (int)(kRange / 128);             // 128-symbol warp steps
    static constexpr uint32_t kBlocks = kTile / 512;               // rank blocks per tile
    static constexpr int kWordsPerStep = (int)sizeof(Sym);         // u32 words a lane holds per step
};

uint32_t lw_tile_elems(int width) { return kLwTileBytes / (uint32_t)width; }

struct LevelLaunch {
    const LevelJob *jobs;        // device array of njobs
    const uint32_t *tile_start;  // device, njobs + 1: first global tile of each job
    uint32_t njobs, total_tiles, l;
    uint32_t *ticket;
    uint32_t *err;
};

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

// Per split-slot record of a tile waiting for its placement.
struct TileMeta {
    LevelJob J;                          // the tile's sequence
    uint32_t tile, cnt, ones;            // tile index inside the sequence
    uint32_t wexcl[kCompWarps];          // ones before each warp's range
    uint32_t cpre[kCompWarps][8];        // ones before each step inside the warp's range
};

struct LwShared {
    uint64_t full[2], empty[2], pre[2];
    uint64_t prefix[4];    // ones before tile index i of this CTA, at [i & 3]
    LevelJob job[2];       // sequence of the tile in each input slot
    uint32_t in_tile[2];
    uint32_t wtot[kCompWarps];
    uint32_t abort;
    uint32_t consumed;
    TileMeta meta[2];
};

__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, %0;" ::"n"(kCompThreads) : "memory"); }

// Barrier of the compute warps that also returns the OR of `v` over them, so
// a decision to stop is taken by every compute thread alike.
__device__ __forceinline__ bool bar_compute_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kCompThreads)
        : "memory");
    return r != 0;
}

// Bit `sh` of a lane's 4 consecutive symbols of one step, bit e = symbol e.
template <typename Sym>
__device__ __forceinline__ uint32_t step_bits(const uint32_t *ew, uint32_t sh) {
    if (sizeof(Sym) == 1) {
        // Move bit sh of every byte to bit 7, then gather the four byte-top
        // bits into a nibble with one multiply (the partial products do not
        // overlap below bit 28, so nothing carries into the nibble).
        return (((ew[0] << (7 - sh)) & 0x80808080u) * 0x00204081u) >> 28;
    } else if (sizeof(Sym) == 2) {
        const uint32_t x0 = (ew[0] >> sh) & 0x00010001u, x1 = (ew[1] >> sh) & 0x00010001u;
        return ((x0 | (x0 >> 15)) & 3u) | (((x1 | (x1 >> 15)) & 3u) << 2);
    } else {
        return ((ew[0] >> sh) & 1u) | (((ew[1] >> sh) & 1u) << 1) | (((ew[2] >> sh) & 1u) << 2) |
               (((ew[3] >> sh) & 1u) << 3);
    }
}

template <typename Sym>
__device__ __forceinline__ uint32_t step_sym(const uint32_t *ew, int e) {
    if (sizeof(Sym) == 1) return (ew[0] >> (8 * e)) & 0xffu;
    if (sizeof(Sym) == 2) return (ew[e >> 1] >> (16 * (e & 1))) & 0xffffu;
    return ew[e];
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

// Writes bytes [lo, hi) of the 16-byte value v to A + lo with at most four
// naturally aligned stores (A is 16-byte aligned, 0 <= lo <= hi <= 16).
__device__ __forceinline__ void store_byte_range(unsigned char *A, const uint32_t (&v)[4], uint32_t lo, uint32_t hi) {
    const uint64_t v0 = ((uint64_t)v[1] << 32) | v[0], v1 = ((uint64_t)v[3] << 32) | v[2];
    auto bytes_at = [&](uint32_t p) -> uint64_t {  // bytes p.. of v, p < 16
        if (p == 0) return v0;
        if (p < 8) return (v0 >> (8 * p)) | (v1 << (64 - 8 * p));
        if (p == 8) return v1;
        return v1 >> (8 * (p - 8));
    };
    uint32_t p = lo;
    if ((p & 1) && p < hi) {
        A[p] = (unsigned char)bytes_at(p);
        p += 1;
    }
    if ((p & 2) && p + 2 <= hi) {
        *reinterpret_cast<uint16_t *>(A + p) = (uint16_t)bytes_at(p);
        p += 2;
    }
    if ((p & 4) && p + 4 <= hi) {
        *reinterpret_cast<uint32_t *>(A + p) = (uint32_t)bytes_at(p);
        p += 4;
    }
    if ((p & 8) && p + 8 <= hi) {
        *reinterpret_cast<uint64_t *>(A + p) = bytes_at(p);
        p += 8;
    }
    // What is left lies at the high end of [lo, hi): finish it downwards in
    // aligned pieces (8, 4, 2, 1).
    if (p + 8 <= hi) {
        *reinterpret_cast<uint64_t *>(A + p) = bytes_at(p);
        p += 8;
    }
    if (p + 4 <= hi) {
        *reinterpret_cast<uint32_t *>(A + p) = (uint32_t)bytes_at(p);
        p += 4;
    }
    if (p + 2 <= hi) {
        *reinterpret_cast<uint16_t *>(A + p) = (uint16_t)bytes_at(p);
        p += 2;
    }
    if (p < hi) A[p] = (unsigned char)bytes_at(p);
}

// out = bytes [16 - off, 32 - off) of the 32-byte string V = prev ++ cur
// (off in bytes, 0..15): the 16-byte window that lands on an aligned
// destination when the string cur belongs at a destination `off` bytes past
// an alignment boundary.  kw = off / 4 is uniform across the warp.
__device__ __forceinline__ void realign16(const uint32_t (&prev)[4], const uint32_t (&cur)[4], uint32_t off,
                                          uint32_t (&out)[4]) {
    const uint32_t V[8] = {prev[0], prev[1], prev[2], prev[3], cur[0], cur[1], cur[2], cur[3]};
    const uint32_t r = 8 * (off & 3);
    switch (off >> 2) {
#define WT_REALIGN_CASE(KW)                                                          \
    case KW:                                                                         \
        for (int i = 0; i < 4; i++) out[i] = __funnelshift_l(V[3 + i - KW], V[4 + i - KW], r); \
        break;
        WT_REALIGN_CASE(0)
        WT_REALIGN_CASE(1)
        WT_REALIGN_CASE(2)
        WT_REALIGN_CASE(3)
#undef WT_REALIGN_CASE
    }
}

// Places tile `m` from its split slot: the directory entries that need the
// global prefix, then every symbol to P_{l+1}.  Run by the compute warps.
template <typename Sym>
__device__ void place_tile(const TileMeta &m, uint32_t l, uint64_t prefix, const Sym *__restrict__ split, int ct,
                           bool &bad) {
    const LevelJob &a = m.J;
    using Cfg = LwCfg<Sym>;
    constexpr uint32_t kPerLane = 16 / sizeof(Sym);     // symbols per lane per chunk
    constexpr uint32_t kChunk = 32 * kPerLane;          // symbols per warp chunk (512 bytes)
    const int lane = ct & 31, warp = ct >> 5;
    const uint64_t base = (uint64_t)m.tile * Cfg::kTile;
    const uint32_t cnt = m.cnt, Zt = m.cnt - m.ones;
    // ones before local rank block b (b < kBlocks), and the total after the last one
    auto before = [&](uint32_t b) -> uint32_t {
        if (b >= Cfg::kBlocks) return m.ones;
        const uint32_t pos = b * 512u;
        const uint32_t w = pos / Cfg::kRange, k = (pos % Cfg::kRange) / 128u;
        return m.wexcl[w] + m.cpre[w][k];
    };
    const uint64_t block0 = base >> 9;
    for (uint32_t b = ct; b < Cfg::kBlocks; b += kCompThreads) {
        const uint64_t block = block0 + b;
        if (block < a.nblocks) {
            const uint64_t v = prefix + before(b);
            a.lv.R[block] = (uint32_t)v;
            if ((block & kBlocksPerSpanMask) == 0) a.lv.Hy[block >> (kSpanShift - 9)] = v;
        }
    }
    if (ct == 0) {
        // Select samples that fall in this tile: the block holding the one
        // (zero) of global rank 8192 k.
        for (uint64_t k = ceil_div(prefix, kSample); k * kSample < prefix + m.ones; k++) {
            const uint32_t r = (uint32_t)(k * kSample - prefix);
            uint32_t b = 0;
            while (before(b + 1) <= r) b++;
            a.lv.S1[k] = (uint32_t)(block0 + b);
        }
        const uint64_t zprefix = base - prefix;
        for (uint64_t k = ceil_div(zprefix, kSample); k * kSample < zprefix + Zt; k++) {
            const uint32_t r = (uint32_t)(k * kSample - zprefix);
            uint32_t b = 0;
            while (b + 1 < Cfg::kBlocks && (b + 1) * 512u - before(b + 1) <= r) b++;
            a.lv.S0[k] = (uint32_t)(block0 + b);
        }
        if (m.tile == a.ntiles - 1) {
            const uint64_t total = prefix + m.ones;
            a.lv.R[a.nblocks] = (uint32_t)total;
            a.lv.Hy[a.nspans] = total;
            *a.ones_out = total;
        }
    }
    if (a.nxt == nullptr) return;

    // A warp takes 512 consecutive bytes of the split slot, 16 per lane.
    // When the chunk is one run (one class, one node) its destination is
    // contiguous: lanes shift their bytes into 16-byte aligned windows and
    // store whole vectors; only the two ragged ends use narrower stores.
    Sym *nxt = static_cast<Sym *>(a.nxt);
    const uint64_t zeros_prefix = base - prefix;  // zeros before this tile
    const uint32_t shv = a.L - l;                 // key_l = s >> (L - l)
    const uint32_t nodes = 1u << l;
    for (uint32_t q0 = warp * kChunk; q0 < cnt; q0 += kCompWarps * kChunk) {
        const uint32_t q = q0 + kPerLane * lane;
        const uint4 xv = *reinterpret_cast<const uint4 *>(&split[q]);
        const uint32_t x[4] = {xv.x, xv.y, xv.z, xv.w};
        const uint32_t first = __shfl_sync(0xffffffffu, x[0], 0);
        const uint32_t last = __shfl_sync(0xffffffffu, x[3], 31);
        const uint32_t efirst = sizeof(Sym) == 4 ? first : (first & ((1u << (8 * sizeof(Sym))) - 1u));
        const uint32_t elast = sizeof(Sym) == 4 ? last : (last >> (32 - 8 * sizeof(Sym)));
        const uint32_t nf = efirst >> shv;
        const bool fast = q0 + kChunk - 1 < cnt && (q0 + kChunk - 1 < Zt || q0 >= Zt) && (elast >> shv) == nf &&
                          nf < nodes;
        if (fast) {
            const uint64_t dst0 = q0 < Zt ? zeros_prefix + q0 + __ldg(a.ob + nf) : prefix + (q0 - Zt) + __ldg(a.ze + nf);
            if (dst0 + kChunk > a.n) {
                bad = true;
                continue;
            }
            const uint32_t off = (uint32_t)((dst0 * sizeof(Sym)) & 15);
            unsigned char *A = reinterpret_cast<unsigned char *>(nxt) + (dst0 * sizeof(Sym) - off);
            uint32_t prev[4];
#pragma unroll
            for (int i = 0; i < 4; i++) prev[i] = __shfl_up_sync(0xffffffffu, x[i], 1);
            uint32_t out[4];
            realign16(prev, x, off, out);
            if (lane > 0 || off == 0)
                *reinterpret_cast<uint4 *>(A + 16 * lane) = make_uint4(out[0], out[1], out[2], out[3]);
            else
                store_byte_range(A, out, off, 16);
            if (lane == 31 && off) {
                const uint32_t zero[4] = {0, 0, 0, 0};
                realign16(x, zero, off, out);
                store_byte_range(A + 512, out, 0, off);
            }
        } else {
#pragma unroll
            for (uint32_t k = 0; k < kPerLane; k++) {
                const uint32_t qk = q + k;
                if (qk >= cnt) break;
                const uint32_t e = sizeof(Sym) == 4 ? x[k] : (x[k * sizeof(Sym) / 4] >> (8 * sizeof(Sym) * (k % (4 / sizeof(Sym))))) &
                                                                  ((1u << (8 * sizeof(Sym))) - 1u);
                const uint32_t node = e >> shv;
                if (node >= nodes) {  // only after an earlier fault: never index past the tables
                    bad = true;
                    continue;
                }
                const uint64_t dst = qk < Zt ? zeros_prefix + qk + __ldg(a.ob + node) : prefix + (qk - Zt) + __ldg(a.ze + node);
                if (dst < a.n)
                    nxt[dst] = (Sym)e;
                else
                    bad = true;
            }
        }
    }
}

// Bytes of tile `tile` of job J that a 16-byte-granular bulk copy can bring
// in (0 when the job's symbols are not 16-byte aligned: then every symbol is
// read from global memory directly).
template <typename Sym>
__device__ __forceinline__ uint32_t tile_bytes16(const LevelJob &J, uint32_t tile) {
    if (reinterpret_cast<uintptr_t>(J.cur) & 15) return 0;
    const uint64_t left = (J.n - (uint64_t)tile * LwCfg<Sym>::kTile) * sizeof(Sym);
    return (uint32_t)(left < kLwTileBytes ? left : kLwTileBytes) & ~15u;
}

template <typename Sym>
__global__ void __launch_bounds__(kLwThreads, 2) level_pass_kernel(LevelLaunch a) {
    using Cfg = LwCfg<Sym>;
    constexpr int kSteps = Cfg::kSteps;
    constexpr int kW = Cfg::kWordsPerStep;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *in_buf = smem;                                      // 2 x kLwTileBytes
    Sym *split_buf = reinterpret_cast<Sym *>(smem + 2 * kLwTileBytes);  // 2 x kTile symbols
    LwShared &sh = *reinterpret_cast<LwShared *>(smem + 4 * kLwTileBytes);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l = a.l;
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], kCompWarps);
            mbar_init(&sh.pre[s], 1);
        }
        fence_mbar_init();
        sh.abort = 0;
        sh.consumed = 0;
    }
    __syncthreads();

    if (warp == kCompWarps) {
        // ---------------------------------------------------------- producer
        // Claims tiles two ahead and streams them in; counts each tile's ones
        // as soon as it lands and publishes the aggregate at once, so other
        // CTAs' look-backs never wait on this CTA's compute queue; then looks
        // back for the oldest tile and hands its prefix to the compute warps.
        auto claim = [&](int s) -> uint32_t {  // lane 0: claim a ticket for slot s and stream it in
            const uint32_t t = atomicAdd(a.ticket, 1u);  // claim order: look-back waits only on earlier tiles
            if (t < a.total_tiles) {
                const uint32_t k = find_job(a, t);
                const uint32_t tile = t - a.tile_start[k];
                sh.job[s] = a.jobs[k];
                sh.in_tile[s] = tile;
                const LevelJob &J = sh.job[s];
                fence_proxy_async_smem();
                const uint32_t bytes = tile_bytes16<Sym>(J, tile);
                if (bytes)
                    bulk_load(in_buf + s * kLwTileBytes,
                              reinterpret_cast<const unsigned char *>(J.cur) + (uint64_t)tile * kLwTileBytes, bytes,
                              &sh.full[s]);
                else
                    mbar_arrive(&sh.full[s]);
                return t;
            }
            sh.in_tile[s] = kEnd;
            mbar_arrive(&sh.full[s]);
            return kEnd;
        };
        // Ones of the tile held in slot s (whole warp; tail symbols from global).
        auto count = [&](int s) -> uint32_t {
            const LevelJob &J = sh.job[s];
            const uint32_t tile = sh.in_tile[s];
            const uint32_t bsh = J.L - 1 - l;
            const Sym *cur = static_cast<const Sym *>(J.cur);
            const uint64_t base = (uint64_t)tile * Cfg::kTile;
            const uint32_t cnt = (uint32_t)((J.n - base) < (uint64_t)Cfg::kTile ? (J.n - base) : (uint64_t)Cfg::kTile);
            const uint32_t b16 = tile_bytes16<Sym>(J, tile);
            const uint4 *v = reinterpret_cast<const uint4 *>(in_buf + s * kLwTileBytes);
            uint32_t c = 0;
            for (uint32_t k = lane; k < b16 / 16; k += 32) {
                const uint4 x = v[k];
                const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (sizeof(Sym) == 1) c += __popc((w4[j] << (7 - bsh)) & 0x80808080u);
                    if (sizeof(Sym) == 2) c += __popc((w4[j] >> bsh) & 0x00010001u);
                    if (sizeof(Sym) == 4) c += (w4[j] >> bsh) & 1u;
                }
            }
            for (uint32_t p = b16 / sizeof(Sym) + lane; p < cnt; p += 32) c += ((uint32_t)cur[base + p] >> bsh) & 1u;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
            return c;
        };
        uint32_t t0 = kEnd, t1 = kEnd;
        if (lane == 0) {
            t0 = claim(0);
            if (t0 != kEnd) t1 = claim(1);
        }
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        t1 = __shfl_sync(0xffffffffu, t1, 0);
        uint32_t issued = (t0 != kEnd) + (t1 != kEnd);   // real tiles streamed so far
        bool ended = t0 == kEnd || t1 == kEnd;
        bool ok = true;
        uint32_t agg = 0;
        if (t0 != kEnd) {
            ok = mbar_wait(&sh.full[0], 0);
            agg = count(0);
            if (lane == 0) publish_aggregate(sh.job[0].status, sh.in_tile[0], agg);
        }
        uint32_t tnext = t1;
        for (uint32_t i = 0; ok && i < issued; i++) {
            const int s = i & 1;
            uint32_t agg_next = 0;
            if (tnext != kEnd) {  // tile index i + 1, in the other slot
                ok = mbar_wait(&sh.full[s ^ 1], ((i + 1) >> 1) & 1u);
                agg_next = count(s ^ 1);
                if (lane == 0) publish_aggregate(sh.job[s ^ 1].status, sh.in_tile[s ^ 1], agg_next);
            }
            const uint64_t prefix = lookback_published(sh.job[s].status, sh.in_tile[s], agg, a.err);
            // Hand the prefix over only once the compute warps have read tile
            // i: then they have also taken the previous prefix of this slot,
            // so pre[s] never runs two phases ahead of its waiters.
            ok = ok && mbar_wait(&sh.empty[s], (i >> 1) & 1u);
            if (lane == 0) {
                sh.prefix[i & 3] = prefix;
                mbar_arrive(&sh.pre[s]);
            }
            // Slot s takes tile index i + 2.
            uint32_t tnn = kEnd;
            if (!ended && ok) {
                if (lane == 0) tnn = claim(s);
                tnn = __shfl_sync(0xffffffffu, tnn, 0);
                if (tnn != kEnd) issued++;
                else ended = true;
            }
            if (*(volatile uint32_t *)&sh.abort) ok = false;
            tnext = tnn;
            agg = agg_next;
        }
        if (!ok && lane == 0) {
            atomicOr(&sh.abort, 1u);
            atomicOr(a.err, kErrTimeout);
            // Drain: a bulk copy still filling a slot must land before the CTA exits.
            for (uint32_t i = *(volatile uint32_t *)&sh.consumed; i < issued; i++) mbar_wait(&sh.full[i & 1], (i >> 1) & 1u);
        }
        return;
    }

    // -------------------------------------------------------------- compute
    bool bad = false, failed = false;
    uint32_t i = 0;
    for (;; i++) {
        const int s = i & 1;
        const uint32_t par = (i >> 1) & 1u;
        if (!mbar_wait(&sh.full[s], par)) failed = true;
        const uint32_t tile = sh.in_tile[s];
        // Also the barrier that ends the previous iteration: the split slot
        // and record placed there are free from here on.
        if (bar_compute_any(failed || tile == kEnd || *(volatile uint32_t *)&sh.abort)) break;
        if (tid == 0) sh.consumed = i + 1;
        TileMeta &m = sh.meta[s];
        // The tile's sequence: everything this iteration needs is read before
        // this warp releases the slot (the producer then refills it).
        const LevelJob &Jin = sh.job[s];
        const Sym *cur = static_cast<const Sym *>(Jin.cur);
        const uint64_t jn = Jin.n, jnblocks = Jin.nblocks;
        uint32_t *const jwords = Jin.lv.words;
        const bool has_next = Jin.nxt != nullptr;
        const uint32_t bsh = Jin.L - 1 - l;  // the level-l bit of a symbol
        const uint64_t base = (uint64_t)tile * Cfg::kTile;
        const uint32_t cnt = (uint32_t)((jn - base) < (uint64_t)Cfg::kTile ? (jn - base) : (uint64_t)Cfg::kTile);
        const uint32_t bytes16 = tile_bytes16<Sym>(Jin, tile);
        const unsigned char *src = in_buf + s * kLwTileBytes;
        if (tid == 0) m.J = Jin;

        // Phase 1: read the lane's symbols, write the bitmap words, count.
        // A lane holds 4 consecutive symbols per 128-symbol step; the step's
        // bitmap word of each group of 8 lanes is one redux-or, and the
        // per-lane counts of four steps share one shuffle scan (8-bit fields:
        // a field's warp sum is at most 128, so no field carries).
        constexpr int kGroups = (kSteps + 3) / 4;
        const bool full_tile = cnt == Cfg::kTile && bytes16 == kLwTileBytes;
        const uint32_t wbase = warp * Cfg::kRange;
        const uint32_t gmask = 0xffu << (lane & 24);
        const uint64_t word0 = (base + wbase) / 32 + (lane >> 3);
        uint32_t ew[kSteps * kW];
        uint32_t nib = 0;
        uint32_t cpk[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; g++) cpk[g] = 0;
#pragma unroll
        for (int k = 0; k < kSteps; k++) {
            const uint32_t q = wbase + 128u * k + 4u * lane;  // tile-local position of the lane's first symbol
            uint32_t *e = &ew[k * kW];
            if (full_tile || (q + 4) * sizeof(Sym) <= bytes16) {
                if (sizeof(Sym) == 1) e[0] = *reinterpret_cast<const uint32_t *>(src + q);
                if (sizeof(Sym) == 2) {
                    const uint2 v = *reinterpret_cast<const uint2 *>(src + 2 * q);
                    e[0] = v.x, e[1] = v.y;
                }
                if (sizeof(Sym) == 4) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(src + 4 * q);
                    e[0] = v.x, e[1] = v.y, e[2] = v.z, e[3] = v.w;
                }
            } else {
#pragma unroll
                for (int w = 0; w < kW; w++) e[w] = 0;
#pragma unroll
                for (int x = 0; x < 4; x++) {
                    const uint32_t p = q + x;
                    uint32_t v = 0;
                    if (p < cnt)
                        v = (p * sizeof(Sym) < bytes16) ? (uint32_t)reinterpret_cast<const Sym *>(src)[p]
                                                         : (uint32_t)cur[base + p];
                    if (sizeof(Sym) == 1) e[0] |= v << (8 * x);
                    if (sizeof(Sym) == 2) e[x >> 1] |= v << (16 * (x & 1));
                    if (sizeof(Sym) == 4) e[x] = v;
                }
            }
            uint32_t nb = step_bits<Sym>(e, bsh);
            if (!full_tile) {
                const uint32_t valid = q < cnt ? (cnt - q < 4u ? cnt - q : 4u) : 0u;
                nb &= (1u << valid) - 1u;
            }
            nib |= nb << (4 * k);
            const uint32_t wv = __reduce_or_sync(gmask, nb << (4 * (lane & 7)));
            const uint64_t word = word0 + 4u * k;
            if ((lane & 7) == 0 && word < jnblocks * 16) jwords[word] = wv;
            cpk[k >> 2] += (uint32_t)__popc(nb) << (8 * (k & 3));
        }
        // Exclusive per-lane prefixes (packed) and warp totals of every step.
        uint32_t lpk[kGroups], tpk[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; g++) lpk[g] = warp_excl_scan(cpk[g], lane, tpk[g]);
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < kSteps; k++) {
            if (lane == 0) m.cpre[warp][k] = run;
            run += (tpk[k >> 2] >> (8 * (k & 3))) & 0xffu;
        }
        __syncwarp();
        if (lane == 0) {
            sh.wtot[warp] = run;
            mbar_arrive(&sh.empty[s]);  // the slot's bytes now live in registers
        }
        bar_compute();
        // Per-warp prefix of the 16 warp totals (each warp derives it itself).
        const uint32_t wt = lane < kCompWarps ? sh.wtot[lane] : 0u;
        uint32_t tile_ones;
        const uint32_t wx = warp_excl_scan(wt, lane, tile_ones);
        const uint32_t warp_excl = __shfl_sync(0xffffffffu, wx, warp);
        if (warp == 0 && lane < kCompWarps) m.wexcl[lane] = wx;
        if (tid == 0) {
            m.tile = tile;
            m.cnt = cnt;
            m.ones = tile_ones;
        }
        const uint32_t Zt = cnt - tile_ones;

        // Phase 3: stable split of the tile by the bit into the split slot:
        // zeros to [0, Zt), ones to [Zt, cnt), order kept.  Each symbol's
        // slot follows from the ones before it: in the tile, in the warp's
        // step, in the lane.
        if (has_next) {
            Sym *split = split_buf + s * Cfg::kTile;
            uint32_t crun = warp_excl;
#pragma unroll
            for (int k = 0; k < kSteps; k++) {
                const uint32_t nb = (nib >> (4 * k)) & 15u;
                const uint32_t q = wbase + 128u * k + 4u * lane;
                const uint32_t ob = crun + ((lpk[k >> 2] >> (8 * (k & 3))) & 0xffu);  // ones before q in the tile
                crun += (tpk[k >> 2] >> (8 * (k & 3))) & 0xffu;
                uint32_t po = Zt + ob, pz = q - ob;  // next slot of a one / of a zero
                const uint32_t *e = &ew[k * kW];
                if (full_tile) {
#pragma unroll
                    for (int x = 0; x < 4; x++) {
                        const bool bit = (nb >> x) & 1u;
                        split[bit ? po : pz] = (Sym)step_sym<Sym>(e, x);
                        po += bit;
                        pz += !bit;
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < 4; x++) {
                        const bool bit = (nb >> x) & 1u;
                        if (q + x < cnt) split[bit ? po : pz] = (Sym)step_sym<Sym>(e, x);
                        po += bit;
                        pz += !bit;
                    }
                }
            }
        }

        // Place the previous tile (its prefix arrived while this one was read).
        if (i > 0) {
            const int ps = s ^ 1;
            if (mbar_wait(&sh.pre[ps], ((i - 1) >> 1) & 1u))
                place_tile<Sym>(sh.meta[ps], l, sh.prefix[(i - 1) & 3], split_buf + ps * Cfg::kTile, tid, bad);
            else
                failed = true;
        }
    }
    // The last tile still waits for its placement (unless a wait gave up).
    if (!bar_compute_any(failed || *(volatile uint32_t *)&sh.abort) && i > 0) {
        const int ps = (i - 1) & 1;
        if (mbar_wait(&sh.pre[ps], ((i - 1) >> 1) & 1u))
            place_tile<Sym>(sh.meta[ps], l, sh.prefix[(i - 1) & 3], split_buf + ps * Cfg::kTile, tid, bad);
        else
            failed = true;
    }
    if (failed && tid == 0) atomicOr(&sh.abort, 1u);
    if (bad || failed) atomicOr(a.err, kErrTimeout);
}

constexpr size_t kLwSmem = 4 * kLwTileBytes + sizeof(LwShared);

static int lw_grid(const void *kernel, uint32_t ntiles) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLwThreads, kLwSmem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const uint64_t g = (uint64_t)sms * per_sm;
    return (int)(g < ntiles ? g : ntiles);
}

template <typename Sym>
static cudaError_t launch_lw(const LevelLaunch &a, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(level_pass_kernel<Sym>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kLwSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = lw_grid((const void *)level_pass_kernel<Sym>, a.total_tiles);
    level_pass_kernel<Sym><<<grid, kLwThreads, kLwSmem, st>>>(a);
    return cudaGetLastError();
}

LevelJob make_level_job(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l, const uint64_t *ob,
                        const uint64_t *ze, LevelDesc lv, uint64_t *ones_out, uint64_t *status) {
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
    j.ob = ob + ((1ull << l) - 1);
    j.ze = ze + ((1ull << l) - 1);
    j.status = status;
    return j;
}

cudaError_t launch_level_jobs(int width, uint32_t l, const LevelJob *jobs, const uint32_t *tile_start, uint32_t njobs,
                              uint32_t total_tiles, uint32_t *ticket, uint32_t *err, cudaStream_t st) {
    if (njobs == 0 || total_tiles == 0) return cudaSuccess;
    LevelLaunch a;
    a.jobs = jobs;
    a.tile_start = tile_start;
    a.njobs = njobs;
    a.total_tiles = total_tiles;
    a.l = l;
    a.ticket = ticket;
    a.err = err;
    switch (width) {
        case 1: return launch_lw<uint8_t>(a, st);
        case 2: return launch_lw<uint16_t>(a, st);
        case 4: return launch_lw<uint32_t>(a, st);
    }
    return cudaErrorInvalidValue;
}

// Writes one job and its tile range to device memory (kernel parameters
// carry the values, so no host buffer has to outlive the call).
__global__ void put_job_kernel(LevelJob j, LevelJob *dst, uint32_t *tile_start) {
    *dst = j;
    tile_start[0] = 0;
    tile_start[1] = j.ntiles;
}

size_t level_job_bytes() { return sizeof(LevelJob); }

size_t level_job_slot_bytes() { return (sizeof(LevelJob) + 2 * sizeof(uint32_t) + 255) & ~size_t(255); }

cudaError_t launch_level_pass(const void *cur, void *nxt, uint64_t n, int width, uint32_t L, uint32_t l,
                              const uint64_t *ob, const uint64_t *ze, LevelDesc lv, uint64_t *ones_out,
                              uint64_t *status, uint32_t *ticket, uint32_t *err, void *job_slot, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const LevelJob j = make_level_job(cur, nxt, n, width, L, l, ob, ze, lv, ones_out, status);
    LevelJob *dj = static_cast<LevelJob *>(job_slot);
    uint32_t *ts = reinterpret_cast<uint32_t *>(dj + 1);
    put_job_kernel<<<1, 1, 0, st>>>(j, dj, ts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_level_jobs(width, l, dj, ts, 1, j.ntiles, ticket, err, st);
}

}  // namespace wt
