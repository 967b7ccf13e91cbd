// merge.cu -- the merge of partial trees: the tree of the concatenation
// S_0 S_1 ... S_{k-1} from the trees of its parts (the buffered build of
// Section 5, finished with the global offsets and Function mergeBA of
// Algorithm 2, Section 3.2).
//
// Node starts of the parts.  A tree keeps no node offsets (Section 2.2's
// one-pointer-per-level layout), so each part's leaf-level starts Hex_a
// (node v of level l at Hex_a[v << (L - l)]) are recovered top-down from its
// bitmaps: node [b, e) of level l splits at b + rank0(e) - rank0(b).  One
// launch per level, one thread per (part, node).  The result's starts are
// the sums over the parts, Hex[c] = sum_a Hex_a[c].
//
// Bits.  Level l of the result holds, node by node, the parts' runs of that
// node in part order: Algorithm 2's global offsets, node-major and
// part-minor.  A thread writes groups of 128 consecutive bits of the result,
// one 16-byte store each.  It finds the run (part a of node v) that holds a
// group's first bit by binary search over the result's node starts and a
// walk over that node's parts, and keeps it for its next group, where it
// usually still holds.  A group inside one run is a funnel shift of five
// source words; otherwise the thread copies pieces of at most 32 bits (one or
// two source words each, never crossing an output word) until its 128 bits
// are done, moving to the next part's run and, when a node is exhausted,
// searching again.  Where mergeBA writes each run's boundary words
// atomically, here every output word has exactly one writer: no atomics, and
// the padding bits beyond n are written as zeros by the same stores.
//
// The directory of each merged level (R, Hy, S1, S0 and its ones) comes from
// the level step's count-from-bitmap and scan kernels (createRankSelect).
#include <cuda_runtime.h>
#include <stdint.h>

#include "wt_internal.cuh"

namespace wt {

constexpr int kMergeThreads = 256;

static int merge_sms() {
    static int count = 0;
    if (!count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 1;
    }
    return count;
}

static unsigned merge_grid(uint64_t items, uint32_t per_sm) {
    const uint64_t need = ceil_div(items ? items : 1, kMergeThreads);
    const uint64_t cap = (uint64_t)merge_sms() * per_sm;
    return (unsigned)(need < cap ? need : cap);
}

// Hex_a[0] = 0 and Hex_a[2^L] = n_a for every part a.
__global__ void merge_init_kernel(const TreeDesc *const *__restrict__ parts, uint32_t k, uint32_t L,
                                  uint64_t *__restrict__ hex) {
    const uint64_t stride = (1ull << L) + 1;
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
        hex[a * stride] = 0;
        hex[a * stride + (1ull << L)] = parts[a]->n;
    }
}

// Level l (< L): node v of part a, [b, e) = [Hex_a[v << s], Hex_a[(v + 1) << s])
// with s = L - l, has z zeros on level l; its left child (on level l + 1)
// is [b, b + z), so Hex_a[(2 v + 1) << (s - 1)] = b + z.
__global__ void merge_starts_kernel(const TreeDesc *const *__restrict__ parts, uint32_t k, uint32_t L, uint32_t l,
                                    uint64_t *__restrict__ hex, uint32_t *__restrict__ err) {
    const uint64_t stride = (1ull << L) + 1;
    const uint64_t nodes = 1ull << l;
    const uint32_t s = L - l;
    const uint64_t total = nodes * k;
    bool bad = false;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)(t >> l);
        const uint64_t v = t & (nodes - 1);
        uint64_t *h = hex + a * stride;
        const uint64_t b = h[v << s], e = h[(v + 1) << s];
        uint64_t z = 0;
        if (e < b) {
            bad = true;
        } else if (e > b) {
            const TreeDesc *d = parts[a];
            if (e > d->n) {
                bad = true;
            } else {
                const LevelDesc lv = d->lv[l];
                const uint64_t ones = rank1(lv, e) - rank1(lv, b);
                if (ones > e - b)
                    bad = true;
                else
                    z = (e - b) - ones;
            }
        }
        h[(v << s) + (1ull << (s - 1))] = b + z;
    }
    if (bad) atomicOr(err, kErrBound);
}

// Hex[c] = sum over the parts of Hex_a[c], c = 0 .. 2^L.
__global__ void merge_sum_kernel(const uint64_t *__restrict__ hex, uint32_t k, uint32_t L,
                                 uint64_t *__restrict__ hex_out) {
    const uint64_t stride = (1ull << L) + 1;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < stride;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = 0;
        for (uint32_t a = 0; a < k; a++) x += hex[a * stride + c];
        hex_out[c] = x;
    }
}

struct MergeLevel {
    const TreeDesc *const *parts;
    const uint64_t *hex;    // k x (2^L + 1) part starts
    const uint64_t *hexm;   // 2^L + 1 starts of the result
    uint32_t *words;        // the result's level-l bitmap, nblocks * 16 words
    uint32_t *err;
    uint64_t n;             // the result's length
    uint64_t groups;        // 128-bit groups of the padded level: nblocks * 4
    uint32_t k, L, l;
};

// The part run of node v that holds result bit pos: part a, its source start
// src and length len, and d, where the run starts in the result.  false if
// no run of the node holds pos.
__device__ __forceinline__ bool merge_locate(const MergeLevel &m, uint64_t v, uint32_t s, uint64_t pos, uint32_t &a,
                                             uint64_t &d, uint64_t &src, uint64_t &len) {
    const uint64_t stride = (1ull << m.L) + 1;
    d = m.hexm[v << s];
    for (a = 0; a < m.k; a++) {
        const uint64_t *h = m.hex + a * stride;
        src = h[v << s];
        len = h[(v + 1) << s] - src;
        if (pos < d + len) return true;
        d += len;
    }
    return false;
}

// The node of the result that holds bit pos: the last v with Hex[v << s] <= pos.
__device__ __forceinline__ uint64_t merge_node(const MergeLevel &m, uint32_t s, uint64_t pos) {
    uint64_t lo = 0, hi = (1ull << m.l) - 1;
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (m.hexm[mid << s] <= pos)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// A warp takes kMergeRun consecutive 32-group blocks; lane i writes group i of
// each (so every store instruction covers 512 consecutive bytes) and keeps
// the part run that held its last bit: the next group, 4096 bits on, usually
// lies in the same run, and the node search is taken only where a run ends.
constexpr uint32_t kMergeRun = 8;

__global__ void __launch_bounds__(kMergeThreads) merge_level_kernel(MergeLevel m) {
    const uint32_t s = m.L - m.l;
    const uint64_t stride = (1ull << m.L) + 1;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint64_t blocks = ceil_div(m.groups, 32ull * kMergeRun);  // warp work units
    bool bad = false;
    for (uint64_t u = blockIdx.x * (uint64_t)(blockDim.x / 32) + (threadIdx.x >> 5); u < blocks && !bad;
         u += warps) {
        // The part run (part a of node v) that holds the lane's current bit:
        // result bits [d, d + len) from the part's bits [src, src + len).
        bool have = false;
        uint64_t v = 0, d = 0, src = 0, len = 0, pn = 0;
        uint32_t a = 0;
        const uint32_t *sw = nullptr;
        for (uint32_t j = 0; j < kMergeRun && !bad; j++) {
            const uint64_t g = (u * kMergeRun + j) * 32 + lane;
            if (g >= m.groups) break;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            uint64_t pos = g * 128;
            const uint64_t end = min(pos + 128, m.n);
            while (pos < end) {
                if (!have || pos < d || pos >= d + len) {
                    v = merge_node(m, s, pos);
                    if (!merge_locate(m, v, s, pos, a, d, src, len)) {
                        bad = true;
                        break;
                    }
                    const TreeDesc *P = m.parts[a];
                    sw = P->lv[m.l].words;
                    pn = P->n;
                    have = true;
                }
                if (end - pos == 128 && d + len - pos >= 128) {
                    // The whole group lies in one run: a funnel shift of five
                    // consecutive source words.
                    const uint64_t sp = src + (pos - d);
                    if (sp >= pn || pn - sp < 128) {
                        bad = true;
                        break;
                    }
                    const uint32_t so = (uint32_t)(sp & 31);
                    const uint32_t *q = sw + (sp >> 5);
                    const uint32_t x0 = __ldg(q), x1 = __ldg(q + 1), x2 = __ldg(q + 2), x3 = __ldg(q + 3);
                    const uint32_t x4 = so ? __ldg(q + 4) : 0u;
                    w[0] = __funnelshift_r(x0, x1, so);
                    w[1] = __funnelshift_r(x1, x2, so);
                    w[2] = __funnelshift_r(x2, x3, so);
                    w[3] = __funnelshift_r(x3, x4, so);
                    pos = end;
                    break;
                }
                // Pieces of at most 32 bits (one or two source words each,
                // never crossing an output word) up to the group's or the
                // run's end.
                const uint32_t off = (uint32_t)(pos & 31);
                uint64_t cnt = 32 - off;
                if (d + len - pos < cnt) cnt = d + len - pos;
                if (end - pos < cnt) cnt = end - pos;
                const uint64_t sp = src + (pos - d);  // the piece's first source bit
                if (sp >= pn || pn - sp < cnt) {
                    bad = true;
                    break;
                }
                const uint32_t so = (uint32_t)(sp & 31);
                uint64_t x = __ldg(sw + (sp >> 5));
                if (so + cnt > 32) x |= (uint64_t)__ldg(sw + (sp >> 5) + 1) << 32;
                const uint32_t mask = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
                const uint32_t piece = ((uint32_t)(x >> so) & mask) << off;
                const uint32_t wi = (uint32_t)(pos >> 5) & 3u;
#pragma unroll
                for (int q = 0; q < 4; q++) w[q] |= wi == (uint32_t)q ? piece : 0u;
                pos += cnt;
                if (pos == d + len) {
                    // The next part's run of node v, skipping empty ones; past
                    // the node's last part the next bit is searched again.
                    d += len;
                    len = 0;
                    for (a++; a < m.k; a++) {
                        const uint64_t *h = m.hex + a * stride;
                        src = h[v << s];
                        len = h[(v + 1) << s] - src;
                        if (len) break;
                    }
                    if (a < m.k) {
                        const TreeDesc *P = m.parts[a];
                        sw = P->lv[m.l].words;
                        pn = P->n;
                    } else {
                        have = false;
                    }
                }
            }
            if (bad) break;
            reinterpret_cast<uint4 *>(m.words)[g] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    if (bad) atomicOr(m.err, kErrBound);
}

cudaError_t launch_merge_starts(const TreeDesc *const *parts, uint32_t k, uint32_t L, uint64_t *hex,
                                uint64_t *hex_out, uint32_t *err, cudaStream_t st) {
    merge_init_kernel<<<merge_grid(k, 1), kMergeThreads, 0, st>>>(parts, k, L, hex);
    note_launches(1);
    for (uint32_t l = 0; l < L; l++) {
        merge_starts_kernel<<<merge_grid((1ull << l) * k, 8), kMergeThreads, 0, st>>>(parts, k, L, l, hex, err);
        note_launches(1);
    }
    merge_sum_kernel<<<merge_grid((1ull << L) + 1, 8), kMergeThreads, 0, st>>>(hex, k, L, hex_out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_merge_level(const TreeDesc *const *parts, uint32_t k, uint32_t L, uint32_t l, const uint64_t *hex,
                               const uint64_t *hex_out, uint64_t n, uint32_t *words, uint32_t *err,
                               cudaStream_t st) {
    MergeLevel m;
    m.parts = parts;
    m.hex = hex;
    m.hexm = hex_out;
    m.words = words;
    m.err = err;
    m.n = n;
    m.groups = ceil_div(n, kBlockBits) * (kBlockBits / 128);
    m.k = k;
    m.L = L;
    m.l = l;
    if (m.groups == 0) return cudaSuccess;
    merge_level_kernel<<<merge_grid(ceil_div(m.groups, kMergeRun), 8), kMergeThreads, 0, st>>>(m);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace wt
