// abi.cu -- the C ABI of include/wt.h: argument checks, device memory,
// the build driver (which kernels run in which order) and query dispatch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <atomic>
#include <mutex>
#include <optional>
#include <new>
#include <vector>

#include "wt_internal.cuh"

using namespace wt;

namespace {

thread_local wt_status g_last = WT_OK;

struct Allocator {
    void *(*alloc)(size_t, void *, void *);
    void (*free_)(void *, size_t, void *, void *);
    void *ctx;
};
Allocator g_alloc = {nullptr, nullptr, nullptr};
std::mutex g_alloc_mu;

wt_status set_last(wt_status s) {
    g_last = s;
    return s;
}

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

void *dev_alloc(const Allocator &A, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 256;
    if (A.alloc) return A.alloc(bytes, st, A.ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(const Allocator &A, void *p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (A.free_)
        A.free_(p, bytes, st, A.ctx);
    else
        cudaFreeAsync(p, st);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Algorithmic bytes of one level step of n symbols of w bytes, the byte
// model of the level-wise method: read P_l (n w), write level l's bitmap
// (n/8) and its directory (n/128), write P_{l+1} (n w) on every level but
// the last.  (What the kernels move beyond it, such as the count pass's
// read, shows in the measured DRAM traffic; where the pass of level l - 1
// hands level l its bitmap, the count pass reads n/8 instead of n w and
// the last level needs no pass, so fewer bytes than the model move.)
double level_step_bytes(uint64_t n, int w, bool has_next) {
    const double nw = (double)n * w;
    return nw + n / 8.0 + n / 128.0 + (has_next ? nw : 0.0);
}

// ---------------------------------------------------------------- profiler
// While enabled, every kernel launch of the library is bracketed by two CUDA
// events on its own stream and tagged with the launch's algorithmic bytes
// (what the method must move: reads of the symbols, writes of bitmaps,
// directories and the next level's order).  wt_profile_end reduces them per
// kernel.
enum KernelId {
    K_HIST = 0, K_NODE_STARTS, K_NODE_TABLES, K_LEVEL_PASS, K_DD_COUNT, K_DD_SCAN, K_DD_WRITE,
    K_Q_ACCESS, K_Q_RANK, K_Q_SELECT, K_Q_MULTI, K_MERGE_STARTS, K_MERGE, K_LEVEL0_COUNT, K_COUNT
};
const char *kKernelNames[K_COUNT] = {"histogram",  "node_starts", "node_tables",  "level_pass",   "dd_count",
                                     "dd_scan",    "dd_write",    "query_access", "query_rank",   "query_select",
                                     "query_multi", "merge_starts", "merge",      "level0_count"};

struct ProfRecord {
    int kid;
    double bytes;    // the level-wise byte model of what the launch covers
    double vbytes;   // the bytes the launch's variant must move
    uint64_t units;  // the launches (level steps) the record covers
    cudaEvent_t e0, e1;
    uint64_t k0, k1;  // kernel launch counter at the start and the end of the call
};

std::atomic<uint64_t> g_kernel_launches{0};

struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRecord> recs;
    std::vector<cudaEvent_t> pool;

    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
};
Profiler g_prof;

// Brackets one launch (or, with units = 0 and add(), several consecutive
// launches of one kind, so that no event sits between them in the stream);
// a no-op when profiling is off.
struct ProfScope {
    int idx = -1;
    cudaStream_t st;
    unsigned flags = cudaEventRecordDefault;
    ProfScope(int kid, double bytes, cudaStream_t s) : ProfScope(kid, bytes, bytes, s) {}
    ProfScope(int kid, double bytes, double vbytes, cudaStream_t s, uint64_t units = 1) : st(s) {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        if (!g_prof.on) return;
        ProfRecord r{kid, bytes, vbytes, units, g_prof.take(), g_prof.take(), g_kernel_launches.load(), 0};
        if (!r.e0 || !r.e1) return;
        // Inside a stream capture the records become event nodes of the graph.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cudaGetLastError();
        if (cap == cudaStreamCaptureStatusActive) flags = cudaEventRecordExternal;
        cudaEventRecordWithFlags(r.e0, st, flags);
        idx = (int)g_prof.recs.size();
        g_prof.recs.push_back(r);
    }
    // One more launch covered by this record.
    void add(double bytes, double vbytes) {
        if (idx < 0) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        g_prof.recs[idx].bytes += bytes;
        g_prof.recs[idx].vbytes += vbytes;
        g_prof.recs[idx].units++;
    }
    ~ProfScope() {
        if (idx < 0) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        cudaEventRecordWithFlags(g_prof.recs[idx].e1, st, flags);
        g_prof.recs[idx].k1 = g_kernel_launches.load();
    }
};

bool is_device_pointer(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

wt_status check_args(const void *S, uint64_t n, uint64_t sigma, int width) {
    if (width != 1 && width != 2 && width != 4) return WT_ERR_ARG;
    if (sigma == 0 || sigma > WT_MAX_SIGMA) return WT_ERR_ARG;
    if (width < 4 && sigma > (1ull << (8 * width))) return WT_ERR_ARG;
    if (n > 0 && S == nullptr) return WT_ERR_ARG;
    if (n > 0 && reinterpret_cast<uintptr_t>(S) % (uintptr_t)width != 0) return WT_ERR_ARG;  // natural alignment
    if (n >= (1ull << 56)) return WT_ERR_ARG;
    return WT_OK;
}

// Per-level sizes of the serialised layout.
struct Shape {
    uint64_t n, nblocks, nspans, ncap;
    size_t words, R, Hy, S;
};

Shape shape_of(uint64_t n) {
    Shape s;
    s.n = n;
    s.nblocks = ceil_div(n, kBlockBits);
    s.nspans = ceil_div(n, 1ull << kSpanShift);
    s.ncap = n / kSample + 2;
    s.words = align256(s.nblocks * 64);
    s.R = align256((s.nblocks + 1) * 4);
    s.Hy = align256((s.nspans + 1) * 8);
    s.S = align256(s.ncap * 4);
    return s;
}

}  // namespace

// Device memory shared by the trees of one wt_build_batch call: the block
// is released when the last of its trees is freed.
struct BatchShared {
    Allocator alloc{};
    void *mem = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *d_err = nullptr;  // the batch's level passes (timeouts)
    std::mutex mu;
    bool err_read = false;
    uint32_t h_err = 0;
    ~BatchShared() {
        if (done) cudaEventDestroy(done);
        if (mem) dev_free(alloc, mem, bytes, stream);
    }
};

struct wt_tree {
    std::shared_ptr<BatchShared> batch;  // set for trees built by wt_build_batch
    uint64_t n = 0, sigma = 0;
    uint32_t L = 0;
    int width = 0;
    int variant = WT_VARIANT_LEVELWISE;
    Allocator alloc{};
    void *mem = nullptr;
    size_t mem_bytes = 0;
    TreeDesc *d_desc = nullptr;
    uint32_t *d_err = nullptr;
    TreeDesc h_desc{};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool finalized = false;
    bool matrix = false;  // a wavelet matrix (wt_build_matrix_async)
    wt_status status = WT_OK;
    // A tree over remapped codes (wt_build_remap): the alphabet bitmap over
    // [0, universe) with its directory, in alpha_mem.
    uint64_t universe = 0;
    LevelDesc alpha{};
    void *alpha_mem = nullptr;
    size_t alpha_bytes = 0;
};

namespace {

// Allocates the resident part of a tree: descriptor, error word and every
// level's bitmap and directories, and fills the host descriptor.
wt_status tree_alloc(wt_tree *t, cudaStream_t st) {
    const Shape s = shape_of(t->n);
    const size_t per_level = s.words + s.R + s.Hy + 2 * s.S;
    t->mem_bytes = align256(sizeof(TreeDesc)) + 256 + per_level * t->L;
    t->mem = dev_alloc(t->alloc, t->mem_bytes, st);
    if (!t->mem) return WT_ERR_OOM;
    char *p = static_cast<char *>(t->mem);
    t->d_desc = reinterpret_cast<TreeDesc *>(p);
    p += align256(sizeof(TreeDesc));
    t->d_err = reinterpret_cast<uint32_t *>(p);
    p += 256;
    memset(&t->h_desc, 0, sizeof(TreeDesc));
    t->h_desc.n = t->n;
    t->h_desc.sigma = t->sigma;
    t->h_desc.nblocks = s.nblocks;
    t->h_desc.L = t->L;
    t->h_desc.width = (uint32_t)t->width;
    for (uint32_t l = 0; l < t->L; l++) {
        LevelDesc &d = t->h_desc.lv[l];
        d.words = reinterpret_cast<uint32_t *>(p);
        p += s.words;
        d.R = reinterpret_cast<uint32_t *>(p);
        p += s.R;
        d.Hy = reinterpret_cast<uint64_t *>(p);
        p += s.Hy;
        d.S1 = reinterpret_cast<uint32_t *>(p);
        p += s.S;
        d.S0 = reinterpret_cast<uint32_t *>(p);
        p += s.S;
        d.ones = 0;
    }
    return WT_OK;
}

#define WT_CK(expr)                                  \
    do {                                             \
        if ((expr) != cudaSuccess) {                 \
            cudaGetLastError();                      \
            return WT_ERR_CUDA;                      \
        }                                            \
    } while (0)

// Scratch of one level-wise build.
struct Scratch {
    void *mem = nullptr;
    size_t bytes = 0;
    BuildScratch b{};
    uint32_t *plane[2] = {nullptr, nullptr};  // pair steps: bit l + 1 of P_l, packed like a bitmap
    uint64_t *ptab = nullptr;                 // pair tables
    uint64_t *starts[2] = {nullptr, nullptr}; // node starts of levels l and l + 1 (rank_starts)
};

// Node tables by rank instead of a leaf histogram (launch_rank_tables): the
// level passes need only rank1 of each level at its node boundaries, which
// its own directory gives after its scan.  Level 0's count from the symbols
// then checks the symbol range.  For alphabets beyond the shared-memory
// histogram (more than 48K codes) the histogram needs global atomics (4.6 ms
// for 2^29 word ids over 2^20 codes, against about 0.02 ms per level for the
// rank tables); for small alphabets the histogram's shared atomics cost more
// than level 0's plain count pass.
bool rank_starts(uint64_t sigma, uint32_t L) { return L > 0 && sigma >= 2; }

// Which steps of a level-wise build take two levels in one pass: pair[l]
// for a step covering levels l and l + 1.  A pair step needs 1- or 2-byte
// symbols (its B split and hand-overs are those of the one-level pass's
// byte path), a level l with at most 2^kPairMaxLevel nodes (its table) and,
// like the one-level hand-over, few tiles spanning a node boundary of level
// l (those place symbol by symbol).
std::vector<uint8_t> level_schedule(uint64_t n, uint64_t sigma, uint32_t L, int width, bool pairs) {
    std::vector<uint8_t> pair(L, 0);
    if (!pairs || width > 2) return pair;
    const uint64_t ntiles = ceil_div(n, lw_tile_elems(width));
    for (uint32_t l = 0; l < L;) {
        if (l + 1 < L && l <= kPairMaxLevel && pass_writes_next_bits(level_boundaries(n, sigma, l), ntiles, width)) {
            pair[l] = 1;
            l += 2;
        } else {
            l += 1;
        }
    }
    return pair;
}

// Bytes a pair step must move (the variant's own model): read P_l, write
// two levels' bitmaps and directories, and write P_{l+2} when a later pass
// reads it.
double pair_step_bytes(uint64_t n, int w, bool store) {
    const double nw = (double)n * w;
    return nw + 2 * (n / 8.0 + n / 128.0) + (store ? nw : 0.0);
}

// pair_lmax: the deepest level whose pair step splits into P_{l+2} (needs a
// pair table), or -1 when no step does; pairs: some step is a pair step.
// by_rank: no leaf histogram (node tables by rank, rank_starts); the Hex
// area then holds the two node-start arrays of consecutive levels.
wt_status scratch_alloc(const Allocator &A, Scratch &sc, uint64_t n, uint64_t sigma, uint32_t L, int width,
                        bool need_levels, cudaStream_t st, bool pairs = false, int pair_lmax = -1,
                        bool by_rank = false) {
    const uint64_t ntiles = ceil_div(n, lw_tile_elems(width));
    const uint32_t R = by_rank ? 0u : hist_replicas(n, sigma);
    const size_t hist = by_rank ? 256 : align256(R ? (size_t)R * sigma * 4 : sigma * 8);
    const size_t hex = align256(((1ull << L) + 4) * 8);
    const size_t tab = need_levels ? align256((1ull << L) * 8) : 0;
    // A pair step keeps three count arrays (and their prefixes), way w at w * stride.
    const uint64_t units = lw_counts_bytes(n, width) / 4;
    const size_t counts = need_levels ? align256(pairs ? 3 * way_cnt_stride(units) * 4 : lw_counts_bytes(n, width)) : 0;
    const size_t prefix =
        need_levels ? align256(pairs ? 3 * way_pre_stride(units) * 8 : lw_prefix_bytes(n, width)) : 0;
    const size_t zeroed = hist;
    const size_t buf = align256(n * (uint64_t)width);
    const size_t stmp = align256(scan_tmp_bytes(L));
    const size_t jslot = std::max(level_job_slot_bytes(), pairs ? pair_job_slot_bytes() : (size_t)0);
    const int nbuf = need_levels ? (L >= 3 ? 2 : (L == 2 ? 1 : 0)) : 0;
    // Two bit planes (bit l + 1 of P_l, read and written in turn) and the pair tables.
    const size_t plane = pairs ? align256(ceil_div(n, kBlockBits) * 64) : 0;
    const size_t ptab = pair_lmax >= 0 ? align256(pair_table_bytes((uint32_t)pair_lmax)) : 0;
    sc.bytes = zeroed + counts + prefix + hex + 2 * tab + stmp + jslot + nbuf * buf + 2 * plane + ptab;
    sc.mem = dev_alloc(A, sc.bytes, st);
    if (!sc.mem) return WT_ERR_OOM;
    char *p = static_cast<char *>(sc.mem);
    sc.b.hist = reinterpret_cast<uint64_t *>(p);
    p += hist;
    sc.b.cnt = reinterpret_cast<uint32_t *>(p);
    p += counts;
    sc.b.pre = reinterpret_cast<uint64_t *>(p);
    p += prefix;
    sc.b.hex = reinterpret_cast<uint64_t *>(p);
    p += hex;
    sc.b.ob = reinterpret_cast<uint64_t *>(p);
    p += tab;
    sc.b.ze = reinterpret_cast<uint64_t *>(p);
    p += tab;
    sc.b.scan_tmp = reinterpret_cast<uint64_t *>(p);
    p += stmp;
    sc.b.job_slot = p;
    p += jslot;
    sc.b.ping = nbuf >= 1 ? p : nullptr;
    p += nbuf >= 1 ? buf : 0;
    sc.b.pong = nbuf >= 2 ? p : nullptr;
    p += nbuf >= 2 ? buf : 0;
    sc.plane[0] = plane ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += plane;
    sc.plane[1] = plane ? reinterpret_cast<uint32_t *>(p) : nullptr;
    p += plane;
    sc.ptab = ptab ? reinterpret_cast<uint64_t *>(p) : nullptr;
    sc.starts[0] = sc.b.hex;
    sc.starts[1] = sc.b.hex + (L ? (1ull << (L - 1)) + 2 : 2);
    if (!by_rank) WT_CK(cudaMemsetAsync(sc.mem, 0, zeroed, st));
    return WT_OK;
}

// The level-wise build (kernels a, a', then b + c per level) of a tree whose
// memory is allocated, from device symbols S.  pairs: take two levels per
// pass where the schedule allows (level_schedule).
wt_status enqueue_levelwise(wt_tree *t, const void *S, cudaStream_t st, bool pairs) {
    const std::vector<uint8_t> pair = level_schedule(t->n, t->sigma, t->L, t->width, pairs);
    int pair_lmax = -1;
    uint32_t table_levels = 0;
    bool any_pair = false;
    for (uint32_t l = 0; l < t->L; l++)
        if (pair[l]) {
            any_pair = true;
            if (l + 2 < t->L) {
                pair_lmax = (int)l;
                table_levels |= 1u << l;
            }
        }
    const bool by_rank = !any_pair && rank_starts(t->sigma, t->L);
    Scratch sc;
    wt_status r =
        scratch_alloc(t->alloc, sc, t->n, t->sigma, t->L, t->width, true, st, any_pair, pair_lmax, by_rank);
    if (r != WT_OK) return r;
    const BuildScratch &b = sc.b;
    const double nw = (double)t->n * t->width;
    const uint32_t R = by_rank ? 0u : hist_replicas(t->n, t->sigma);
    const uint64_t ntiles = ceil_div(t->n, lw_tile_elems(t->width));
    const uint64_t units = lw_counts_bytes(t->n, t->width) / 4;
    LevelDesc *lv = t->h_desc.lv;
    // Level 0's count pass rides on the histogram's read of S where it can
    // (1-byte symbols): level 0's bitmap and unit counts, and the bitmaps
    // the first step ORs into zeroed.  For a pair step at level 0 also bit
    // L - 2 of S and the counts of groups 01 and 11.
    const bool fuse0 = !by_rank && !R && t->L > 0 && level0_fusable(S, t->n, t->width, t->sigma);
    const bool pair0 = t->L > 0 && pair[0];
    const bool next0 = t->L > 1 && pass_writes_next_bits(level_boundaries(t->n, t->sigma, 0), ntiles, t->width);
    if (by_rank) {
        // Level 0's count pass from S (level 0's bitmap, unit counts, the
        // symbol range): the level-wise model's read of S for the counts,
        // profiled on its own as the histogram was.
        ProfScope p(K_LEVEL0_COUNT, nw, nw + t->n / 8.0, st);
        WT_CK(launch_root_starts(t->n, sc.starts[0], st));
        const bool nb0 = t->L > 1 && pass_writes_next_bits(level_boundaries(t->n, t->sigma, 0), ntiles, t->width);
        WT_CK(launch_level_count(S, t->n, t->width, t->L, 0, lv[0], b.cnt, nb0 ? lv[1].words : nullptr, t->d_err,
                                 b.job_slot, st, (uint32_t)t->sigma));
    } else {
        ProfScope p(K_HIST, nw, nw, st);
        if (R) {
            WT_CK(launch_histogram_replicated(S, t->n, t->width, t->sigma, reinterpret_cast<uint32_t *>(b.hist), R,
                                              t->d_err, st));
        } else if (fuse0 && pair0) {
            Level0Fuse z{lv[0].words, b.cnt, lv[1].words, t->L - 1};
            z.plane = sc.plane[0];
            z.cnt01 = b.cnt + way_cnt_stride(units);
            z.cnt11 = b.cnt + 2 * way_cnt_stride(units);
            z.next2 = 2 < t->L ? lv[2].words : nullptr;
            z.plane3 = (3 < t->L && pair[2]) ? sc.plane[1] : nullptr;
            WT_CK(launch_histogram(S, t->n, t->width, t->sigma, b.hist, t->d_err, st, &z));
        } else if (fuse0) {
            const Level0Fuse z{lv[0].words, b.cnt, next0 ? lv[1].words : nullptr, t->L - 1};
            WT_CK(launch_histogram(S, t->n, t->width, t->sigma, b.hist, t->d_err, st, &z));
        } else {
            WT_CK(launch_histogram(S, t->n, t->width, t->sigma, b.hist, t->d_err, st));
        }
    }
    if (t->L > 0 && !by_rank) {
        const double leaves = (double)(1ull << t->L);
        {
            ProfScope p(K_NODE_STARTS, 8.0 * (t->sigma + leaves + 1), 8.0 * (t->sigma + leaves + 1), st);
            if (R)
                WT_CK(launch_node_starts_replicated(reinterpret_cast<const uint32_t *>(b.hist), R, t->sigma, t->L,
                                                    b.hex, st, b.scan_tmp));
            else
                WT_CK(launch_node_starts(b.hist, t->sigma, t->L, t->n, b.hex, st, b.scan_tmp));
        }
        {
            ProfScope p(K_NODE_TABLES, 8.0 * 5 * leaves, 8.0 * 5 * leaves, st);
            WT_CK(launch_node_tables(b.hex, t->L, b.ob, b.ze, st, b.scan_tmp));
            WT_CK(launch_pair_tables(b.hex, t->L, table_levels, sc.ptab, st));
        }
    }
    if (t->L > 0) {
        // Without pair steps every level step is timed under one record, so
        // no profiling event separates two level steps in the stream.
        bool any_pair = false;
        for (uint32_t l = 0; l < t->L; l++) any_pair = any_pair || pair[l];
        std::optional<ProfScope> steps;
        if (!any_pair) steps.emplace(K_LEVEL_PASS, 0.0, 0.0, st, 0);
        const void *cur = S;
        void *bufs[2] = {b.ping, b.pong};
        int bi = 0, pi = 0;
        bool from_bits = false;  // level l's bitmap was written by the step before
        bool plane_ok = false;   // and bit l + 1 of P_l is in sc.plane[pi]
        for (uint32_t l = 0; l < t->L;) {
            if (pair[l]) {
                const bool need_b = l + 2 < t->L;
                const bool store = l + 3 < t->L;  // a pass at level l + 2 reads P_{l+2}
                const bool pnext = need_b && pair[l + 2];
                PairJob j{};
                j.cur = cur;
                j.nxt = store ? bufs[bi] : nullptr;
                j.n = t->n;
                j.nblocks = ceil_div(t->n, kBlockBits);
                j.L = t->L;
                j.ntiles = (uint32_t)ntiles;
                j.words = lv[l].words;
                j.plane = sc.plane[pi];
                j.next1 = lv[l + 1].words;
                j.next2 = need_b ? lv[l + 2].words : nullptr;
                j.plane3 = pnext ? sc.plane[pi ^ 1] : nullptr;
                j.ob = b.ob + ((1ull << l) - 1);
                j.ze = b.ze + ((1ull << l) - 1);
                j.T = need_b ? sc.ptab + pair_table_offset(l) : nullptr;
                j.cnt = b.cnt;
                j.pre = b.pre;
                j.need_b = need_b ? 1u : 0u;
                ProfScope p(K_LEVEL_PASS,
                            level_step_bytes(t->n, t->width, true) + level_step_bytes(t->n, t->width, l + 2 < t->L),
                            pair_step_bytes(t->n, t->width, store), st);
                WT_CK(launch_pair_step(j, t->width, l, lv[l], &t->d_desc->lv[l].ones, lv[l + 1],
                                       &t->d_desc->lv[l + 1].ones, from_bits && plane_ok, l == 0 && fuse0, b.cnt,
                                       b.pre, t->d_err, b.job_slot, st));
                from_bits = need_b;
                plane_ok = pnext;
                if (pnext) pi ^= 1;
                if (store) {
                    cur = bufs[bi];
                    bi ^= 1;
                }
                l += 2;
            } else {
                const bool has_next = l + 1 < t->L;
                const bool next_bits =
                    has_next && pass_writes_next_bits(level_boundaries(t->n, t->sigma, l), ntiles, t->width);
                // The last level needs no symbols when its bitmap is handed over.
                const bool store = has_next && !(l + 2 == t->L && next_bits);
                void *nxt = store ? bufs[bi] : nullptr;
                const double vb = nw + t->n / 8.0 + t->n / 128.0 + (store ? nw : 0.0);
                std::optional<ProfScope> p;
                if (any_pair)
                    p.emplace(K_LEVEL_PASS, level_step_bytes(t->n, t->width, has_next), vb, st);
                else
                    steps->add(level_step_bytes(t->n, t->width, has_next), vb);
                // Without a histogram: level l's tables and C_{l+1} from rank at C_l.
                const RankTables rt{lv[l], sc.starts[l & 1], b.ob + ((1ull << l) - 1), b.ze + ((1ull << l) - 1),
                                    has_next ? sc.starts[(l + 1) & 1] : nullptr};
                WT_CK(launch_level_pass(cur, nxt, t->n, t->width, t->L, l, b.ob, b.ze, lv[l],
                                        &t->d_desc->lv[l].ones, b.cnt, b.pre, from_bits,
                                        next_bits ? lv[l + 1].words : nullptr, t->d_err, b.job_slot, st,
                                        l == 0 && (fuse0 || by_rank), by_rank ? &rt : nullptr));
                from_bits = next_bits;
                plane_ok = false;
                if (store) {
                    cur = bufs[bi];
                    bi ^= 1;
                }
                l += 1;
            }
        }
    }
    dev_free(t->alloc, sc.mem, sc.bytes, st);
    return WT_OK;
}

// The wavelet matrix: the level-wise build with one node per level (node
// tables OB_l = 0, ZE_l = Z_l from matrix.cu).  Every node of a level has
// the same offsets, so the pass places every tile as one node whatever its
// keys (one_node), and each level's pass hands the next level its bitmap
// (1- and 2-byte codes; the last level then needs no symbols).
wt_status enqueue_matrix(wt_tree *t, const void *S, cudaStream_t st) {
    Scratch sc;
    wt_status r = scratch_alloc(t->alloc, sc, t->n, t->sigma, t->L, t->width, true, st);
    if (r != WT_OK) return r;
    const BuildScratch &b = sc.b;
    const double nw = (double)t->n * t->width;
    const uint32_t R = hist_replicas(t->n, t->sigma);
    const uint64_t ntiles = ceil_div(t->n, lw_tile_elems(t->width));
    const bool fuse0 = !R && t->L > 0 && level0_fusable(S, t->n, t->width, t->sigma);
    const bool next0 = t->L > 1 && pass_writes_next_bits(0, ntiles, t->width);  // no boundaries: one node
    {
        ProfScope p(K_HIST, nw, st);
        if (R) {
            WT_CK(launch_histogram_replicated(S, t->n, t->width, t->sigma, reinterpret_cast<uint32_t *>(b.hist), R,
                                              t->d_err, st));
        } else if (fuse0) {
            const Level0Fuse z{t->h_desc.lv[0].words, b.cnt, next0 ? t->h_desc.lv[1].words : nullptr, t->L - 1};
            WT_CK(launch_histogram(S, t->n, t->width, t->sigma, b.hist, t->d_err, st, &z));
        } else {
            WT_CK(launch_histogram(S, t->n, t->width, t->sigma, b.hist, t->d_err, st));
        }
    }
    if (t->L > 0) {
        const double leaves = (double)(1ull << t->L);
        {
            ProfScope p(K_NODE_STARTS, 8.0 * (t->sigma + leaves + 1), st);
            if (R)
                WT_CK(launch_node_starts_replicated(reinterpret_cast<const uint32_t *>(b.hist), R, t->sigma, t->L,
                                                    b.hex, st, b.scan_tmp));
            else
                WT_CK(launch_node_starts(b.hist, t->sigma, t->L, t->n, b.hex, st, b.scan_tmp));
        }
        {
            ProfScope p(K_NODE_TABLES, 8.0 * 3 * leaves, st);
            WT_CK(launch_wm_tables(b.hex, t->L, b.ob, b.ze, st));
        }
        const void *cur = S;
        void *bufs[2] = {b.ping, b.pong};
        bool from_bits = false;
        ProfScope steps(K_LEVEL_PASS, 0.0, 0.0, st, 0);  // every level step under one record
        for (uint32_t l = 0; l < t->L; l++) {
            const bool has_next = l + 1 < t->L;
            const bool next_bits = has_next && next0;
            const bool store = has_next && !(l + 2 == t->L && next_bits);
            void *nxt = store ? bufs[l & 1] : nullptr;
            steps.add(level_step_bytes(t->n, t->width, has_next), level_step_bytes(t->n, t->width, has_next));
            WT_CK(launch_level_pass(cur, nxt, t->n, t->width, t->L, l, b.ob, b.ze, t->h_desc.lv[l],
                                    &t->d_desc->lv[l].ones, b.cnt, b.pre, from_bits,
                                    next_bits ? t->h_desc.lv[l + 1].words : nullptr, t->d_err, b.job_slot, st,
                                    l == 0 && fuse0, nullptr, 0, true));
            from_bits = next_bits;
            cur = nxt;
        }
    }
    dev_free(t->alloc, sc.mem, sc.bytes, st);
    return WT_OK;
}

// The dd-direct build (kernel d: per-tile counts, column scan, one write
// pass over all levels) for small alphabets.
wt_status enqueue_dd(wt_tree *t, const void *S, cudaStream_t st) {
    const size_t hex = align256(((1ull << t->L) + 1) * 8);
    const size_t tab = align256((1ull << t->L) * 8);
    const size_t stmp = align256(scan_tmp_bytes(t->L));
    const size_t dds = align256(dd_scratch_bytes(t->n, t->sigma));
    const size_t bytes = 256 + hex + 2 * tab + stmp + dds;
    void *mem = dev_alloc(t->alloc, bytes, st);
    if (!mem) return WT_ERR_OOM;
    char *p = static_cast<char *>(mem) + 256;
    uint64_t *d_hex = reinterpret_cast<uint64_t *>(p);
    p += hex;
    uint64_t *ob = reinterpret_cast<uint64_t *>(p);
    p += tab;
    uint64_t *ze = reinterpret_cast<uint64_t *>(p);
    p += tab;
    uint64_t *scan_tmp = reinterpret_cast<uint64_t *>(p);
    p += stmp;
    const DdScratch d = dd_carve(p, t->n, t->sigma);
    const double nw = (double)t->n * t->width;
    const double table = (double)dd_tiles(t->n) * t->sigma * 4;
    const uint64_t nblocks = ceil_div(t->n, kBlockBits);
    wt_status r = WT_OK;
    {
        // read S, write the per-tile counts
        ProfScope pr(K_DD_COUNT, nw + table, st);
        if (launch_dd_count(S, t->n, t->sigma, d, t->d_err, st) != cudaSuccess) r = WT_ERR_CUDA;
    }
    if (r == WT_OK) {
        // read the counts twice, write the offsets; node starts and tables
        ProfScope pr(K_DD_SCAN, 3 * table + 8.0 * 6 * (1ull << t->L), st);
        if (launch_dd_scan(t->n, t->sigma, d, st) != cudaSuccess ||
            launch_node_starts(d.H, t->sigma, t->L, t->n, d_hex, st, scan_tmp) != cudaSuccess ||
            launch_node_tables(d_hex, t->L, ob, ze, st, scan_tmp) != cudaSuccess)
            r = WT_ERR_CUDA;
    }
    for (uint32_t l = 0; r == WT_OK && l < t->L; l++)
        if (cudaMemsetAsync(t->h_desc.lv[l].words, 0, nblocks * 64, st) != cudaSuccess) r = WT_ERR_CUDA;
    if (r == WT_OK) {
        // read S and the count/offset rows, write every level's bitmap and directory
        ProfScope pr(K_DD_WRITE, nw + 2 * table + t->L * (t->n / 8.0 + t->n / 128.0), st);
        if (launch_dd_write(S, t->n, t->sigma, t->L, t->h_desc, t->d_desc, d, d_hex, ob, t->d_err, st) !=
            cudaSuccess)
            r = WT_ERR_CUDA;
    }
    if (r != WT_OK) cudaGetLastError();
    dev_free(t->alloc, mem, bytes, st);
    return r;
}

// Variant choice (AUTO): the fastest variant measured on GB300 for the
// entry's (symbol width, levels L, n), from `bench.py --workload tune`
// (median build time of each variant over n = 2^12 .. 2^28 for sigma in
// {4, 20, 96, 256} bytes, {1000, 65536} 2-byte and 2^20 4-byte codes).
//  * Small builds are bound by their launches (one level per pass takes four
//    or five launches per level), so dd-direct, three launches in all, wins
//    for 1-byte codes up to kDdMaxLog2N[L] (for example sigma = 96:
//    0.25 ms against 0.39 ms at 2^22), and two levels per pass, half the
//    level steps, wins for 2-byte codes with up to kPairsMaxL levels up to
//    2^kPairsMaxLog2N (sigma = 1000: 0.49 against 0.52 ms at 2^22).
//  * Large builds are bound by the level pass's ALU work, where one level per
//    pass is fastest (sigma = 96 at 2^28: 2.07 ms against 2.60 ms for two
//    levels per pass and 3.95 ms for dd-direct; sigma = 65536: one level per
//    pass at every n).
// n between measured sizes takes the rule of the next measured size above.
constexpr uint8_t kDdMaxLog2N[9] = {0, 20, 20, 24, 24, 24, 24, 24, 24};  // by L, 1-byte codes
constexpr uint32_t kPairsMaxL = 12;
constexpr uint32_t kPairsMaxLog2N = 22;

uint32_t ceil_log2(uint64_t n) {
    uint32_t k = 0;
    while (k < 63 && (1ull << k) < n) k++;
    return k;
}

int choose_variant(uint64_t n, uint64_t sigma, int width) {
    const uint32_t L = levels_of(sigma);
    const uint32_t lg = ceil_log2(n);
    if (width == 1 && L >= 1 && L <= 8 && dd_supported(n, sigma, width) && lg <= kDdMaxLog2N[L])
        return WT_VARIANT_DD;
    if (width == 2 && L >= 2 && L <= kPairsMaxL && lg <= kPairsMaxLog2N) {
        const std::vector<uint8_t> pair = level_schedule(n, sigma, L, width, true);
        for (uint8_t p : pair)
            if (p) return WT_VARIANT_PAIRS;
    }
    return WT_VARIANT_LEVELWISE;
}

wt_status enqueue_build(wt_tree *t, const void *S, int variant, cudaStream_t st) {
    // Descriptor (with level pointers; "ones" is filled by the level passes)
    // and a zero error word.
    WT_CK(cudaMemcpyAsync(t->d_desc, &t->h_desc, sizeof(TreeDesc), cudaMemcpyHostToDevice, st));
    WT_CK(cudaMemsetAsync(t->d_err, 0, sizeof(uint32_t), st));
    if (t->n == 0) {
        // Empty levels: R[0] = Hy[0] = 0, ones = 0.
        for (uint32_t l = 0; l < t->L; l++) {
            WT_CK(cudaMemsetAsync(t->h_desc.lv[l].R, 0, 4, st));
            WT_CK(cudaMemsetAsync(t->h_desc.lv[l].Hy, 0, 8, st));
        }
        return WT_OK;
    }
    if (t->matrix) {
        t->variant = WT_VARIANT_LEVELWISE;
        return enqueue_matrix(t, S, st);
    }
    if (variant == WT_VARIANT_AUTO) variant = choose_variant(t->n, t->sigma, t->width);
    t->variant = variant;
    if (variant == WT_VARIANT_DD) return enqueue_dd(t, S, st);
    return enqueue_levelwise(t, S, st, variant == WT_VARIANT_PAIRS);
}

// Waits for the build, copies the per-level counts back and reads the error word.
wt_status finalize(wt_tree *t) {
    if (t->finalized) return t->status;
    t->finalized = true;
    if (cudaEventSynchronize(t->batch ? t->batch->done : t->done) != cudaSuccess) {
        cudaGetLastError();
        return t->status = WT_ERR_CUDA;
    }
    if (t->batch) {
        std::lock_guard<std::mutex> lk(t->batch->mu);
        if (!t->batch->err_read) {
            if (cudaMemcpy(&t->batch->h_err, t->batch->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return t->status = WT_ERR_CUDA;
            }
            t->batch->err_read = true;
        }
        if (t->batch->h_err & kErrTimeout) t->status = WT_ERR_TIMEOUT;
    }
    uint32_t err = 0;
    TreeDesc d;
    if (cudaMemcpy(&d, t->d_desc, sizeof(TreeDesc), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&err, t->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return t->status = WT_ERR_CUDA;
    }
    for (uint32_t l = 0; l < t->L; l++) t->h_desc.lv[l].ones = d.lv[l].ones;
    if (err & kErrSymbol)
        t->status = WT_ERR_SYMBOL_RANGE;
    else if (err & kErrTimeout)
        t->status = WT_ERR_TIMEOUT;
    else if (err & kErrBound)
        t->status = WT_ERR_ARG;
    return t->status;
}

// Stream-ordered release: the memory returns to the allocator after the work
// already queued on the build stream; the host does not wait.
void tree_destroy(wt_tree *t) {
    if (!t) return;
    if (t->done) cudaEventDestroy(t->done);
    if (t->mem) dev_free(t->alloc, t->mem, t->mem_bytes, t->stream);
    if (t->alpha_mem) dev_free(t->alloc, t->alpha_mem, t->alpha_bytes, t->stream);
    t->batch.reset();  // the batch block goes with its last tree
    delete t;
}

// ------------------------------------------------------------- batches

// Pinned host staging for a batch's tables: two slots used in turn, so the
// host prepares the next batch while the previous one still runs; a slot is
// reused once the build that copied out of it has completed.
struct PinnedSlot {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaEvent_t ready = nullptr;  // the end of the last build that used the slot
};
struct PinnedStaging {
    std::mutex mu;
    PinnedSlot slot[2];
    uint32_t next = 0;
};
PinnedStaging g_pinned;

size_t level_bytes_of(uint64_t n) {
    const Shape s = shape_of(n);
    return s.words + s.R + s.Hy + 2 * s.S;
}

// Fills a tree descriptor's level pointers from a block of level arrays.
void carve_levels(TreeDesc &d, char *p, uint64_t n, uint32_t L) {
    const Shape s = shape_of(n);
    for (uint32_t l = 0; l < L; l++) {
        LevelDesc &v = d.lv[l];
        v.words = reinterpret_cast<uint32_t *>(p);
        p += s.words;
        v.R = reinterpret_cast<uint32_t *>(p);
        p += s.R;
        v.Hy = reinterpret_cast<uint64_t *>(p);
        p += s.Hy;
        v.S1 = reinterpret_cast<uint32_t *>(p);
        p += s.S;
        v.S0 = reinterpret_cast<uint32_t *>(p);
        p += s.S;
        v.ones = 0;
    }
}

// A batch: the trees share one device block; one launch per stage builds
// the histograms, node starts and node tables of all sequences, then one
// launch per (symbol width, level) runs the level pass over every sequence
// that has that level.  The whole sequence of launches is captured into a
// CUDA graph and launched once (unless the stream is already capturing).
wt_status build_batch_impl(const void *const *S, const uint64_t *n, const uint64_t *sigma, const int *width,
                           uint32_t count, wt_handle *out, cudaStream_t st) {
    for (uint32_t k = 0; k < count; k++) out[k] = nullptr;
    if (count >= (1u << 27)) return WT_ERR_ARG;  // (sequence, level) pairs are packed as k << 5 | l
    for (uint32_t k = 0; k < count; k++) {
        wt_status r = check_args(S[k], n[k], sigma[k], width[k]);
        if (r != WT_OK) return r;
        if (n[k] > 0 && !is_device_pointer(S[k])) return WT_ERR_ARG;
        if (n[k] >= (1ull << 40)) return WT_ERR_ARG;
    }
    if (count == 0) return WT_OK;
    const Allocator A = current_allocator();
    auto B = std::make_shared<BatchShared>();
    B->alloc = A;
    B->stream = st;
    if (cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return WT_ERR_CUDA;
    }

    // ---- tree block: batch error word, descriptors, error words, levels
    std::vector<uint32_t> L(count);
    const size_t desc_bytes = align256(sizeof(TreeDesc) * count);
    const size_t errw_bytes = align256(4 * (size_t)count);
    size_t tree_bytes = 256 + desc_bytes + errw_bytes;
    std::vector<size_t> lvl_off(count);
    for (uint32_t k = 0; k < count; k++) {
        L[k] = levels_of(sigma[k]);
        lvl_off[k] = tree_bytes;
        tree_bytes += level_bytes_of(n[k]) * L[k];
    }
    B->bytes = tree_bytes;
    B->mem = dev_alloc(A, tree_bytes, st);
    if (!B->mem) return WT_ERR_OOM;
    char *tb = static_cast<char *>(B->mem);
    B->d_err = reinterpret_cast<uint32_t *>(tb);
    TreeDesc *d_descs = reinterpret_cast<TreeDesc *>(tb + 256);
    uint32_t *d_errs = reinterpret_cast<uint32_t *>(tb + 256 + desc_bytes);

    std::vector<TreeDesc> hdesc(count);
    std::vector<wt_tree *> trees(count, nullptr);
    for (uint32_t k = 0; k < count; k++) {
        TreeDesc &d = hdesc[k];
        memset(&d, 0, sizeof(TreeDesc));
        d.n = n[k];
        d.sigma = sigma[k];
        d.nblocks = ceil_div(n[k], kBlockBits);
        d.L = L[k];
        d.width = (uint32_t)width[k];
        carve_levels(d, tb + lvl_off[k], n[k], L[k]);
    }

    // ---- scratch: per sequence histogram, node starts, node tables, tile
    // counts and prefixes, ping-pong orders; then the batch tables.
    struct Off {
        size_t hist, hex, ob, ze, cnt, pre, ping, pong;
    };
    std::vector<Off> so(count);
    size_t zeroed = 0;
    for (uint32_t k = 0; k < count; k++) {
        so[k].hist = zeroed;
        zeroed += align256(sigma[k] * 8);
    }
    size_t sbytes = zeroed;
    for (uint32_t k = 0; k < count; k++) {
        const bool lv = L[k] > 0 && n[k] > 0;
        so[k].cnt = sbytes;
        sbytes += lv ? align256(lw_counts_bytes(n[k], width[k])) : 0;
        so[k].pre = sbytes;
        sbytes += lv ? align256(lw_prefix_bytes(n[k], width[k])) : 0;
        const size_t leaves = L[k] ? (1ull << L[k]) : 0;
        so[k].hex = sbytes;
        sbytes += align256((leaves + 1) * 8);
        so[k].ob = sbytes;
        sbytes += align256(leaves * 8);
        so[k].ze = sbytes;
        sbytes += align256(leaves * 8);
        const size_t buf = align256(n[k] * (uint64_t)width[k]);
        so[k].ping = sbytes;
        sbytes += L[k] >= 2 ? buf : 0;
        so[k].pong = sbytes;
        sbytes += L[k] >= 3 ? buf : 0;
    }
    // Level jobs per (width class, level).
    uint32_t maxL[3] = {0, 0, 0};
    auto wclass = [](int w) { return w == 1 ? 0 : (w == 2 ? 1 : 2); };
    for (uint32_t k = 0; k < count; k++) maxL[wclass(width[k])] = std::max(maxL[wclass(width[k])], L[k]);
    struct LaunchPlan {
        int width;
        uint32_t l;
        std::vector<uint32_t> seqs;
        size_t jobs_off, ts_off;  // in the staging tables
        uint32_t total, max_tiles;
        bool from_bits;           // level l's bitmaps were written by the passes of level l - 1
        bool next_bits;           // this level's pass writes level l + 1's bitmaps
        bool do_pass;             // some sequence has a level l + 1
        bool bits;                // some sequence stores no order (the level before its last, bitmap handed over)
    };
    std::vector<LaunchPlan> plans;
    for (int c = 0; c < 3; c++)
        for (uint32_t l = 0; l < maxL[c]; l++) {
            LaunchPlan P;
            P.width = c == 0 ? 1 : (c == 1 ? 2 : 4);
            P.l = l;
            for (uint32_t k = 0; k < count; k++)
                if (wclass(width[k]) == c && L[k] > l && n[k] > 0) P.seqs.push_back(k);
            if (!P.seqs.empty()) plans.push_back(std::move(P));
        }

    // Staging layout (same offsets on host and device).
    size_t tbytes = 0;
    const size_t seqjob_off = tbytes;
    tbytes += align256(sizeof(SeqJob) * count);
    const size_t hts_off = tbytes;
    tbytes += align256(4 * ((size_t)count + 1));
    const size_t sls_off = tbytes;
    tbytes += align256(4 * ((size_t)count + 1));
    uint32_t nsmall = 0, nbig = 0, nbig_pairs = 0, nsmall_pairs = 0;
    for (uint32_t k = 0; k < count; k++) {
        if (L[k] == 0) continue;
        if (batch_small_alphabet(L[k])) {
            nsmall++;
        } else {
            nbig++;
            for (uint32_t l = 0; l < L[k]; l++) ((1ull << l) > kBatchWarpLeaves ? nbig_pairs : nsmall_pairs)++;
        }
    }
    const size_t small_off = tbytes;
    tbytes += align256(4 * ((size_t)nsmall + 1));
    const size_t big_off = tbytes;
    tbytes += align256(4 * ((size_t)nbig + 1));
    const size_t bpairs_off = tbytes;
    tbytes += align256(4 * ((size_t)nbig_pairs + 1));
    const size_t spairs_off = tbytes;
    tbytes += align256(4 * ((size_t)nsmall_pairs + 1));
    for (auto &P : plans) {
        P.jobs_off = tbytes;
        tbytes += align256(sizeof(LevelJob) * P.seqs.size());
        P.ts_off = tbytes;
        tbytes += align256(4 * (P.seqs.size() + 1));
    }
    const size_t total_scratch = sbytes + tbytes;
    void *scratch = dev_alloc(A, total_scratch, st);
    if (!scratch) return WT_ERR_OOM;
    char *sc = static_cast<char *>(scratch);
    char *dt = sc + sbytes;  // device tables

    // Host tables, staged in pinned memory.
    std::lock_guard<std::mutex> lk(g_pinned.mu);
    PinnedSlot &ps = g_pinned.slot[g_pinned.next++ & 1];
    const size_t stage_bytes = tbytes + desc_bytes;
    if (ps.ready && cudaEventSynchronize(ps.ready) != cudaSuccess) cudaGetLastError();
    if (ps.bytes < stage_bytes) {
        if (ps.ptr) cudaFreeHost(ps.ptr);
        ps.ptr = nullptr;
        ps.bytes = 0;
        if (cudaMallocHost(&ps.ptr, stage_bytes) != cudaSuccess) {
            cudaGetLastError();
            dev_free(A, scratch, total_scratch, st);
            return WT_ERR_OOM;
        }
        ps.bytes = stage_bytes;
    }
    if (!ps.ready && cudaEventCreateWithFlags(&ps.ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        dev_free(A, scratch, total_scratch, st);
        return WT_ERR_CUDA;
    }
    char *ht = static_cast<char *>(ps.ptr);
    SeqJob *hjobs = reinterpret_cast<SeqJob *>(ht + seqjob_off);
    uint32_t *hts = reinterpret_cast<uint32_t *>(ht + hts_off);
    uint32_t *sls = reinterpret_cast<uint32_t *>(ht + sls_off);
    uint32_t *hsmall = reinterpret_cast<uint32_t *>(ht + small_off);
    uint32_t *hbig = reinterpret_cast<uint32_t *>(ht + big_off);
    uint32_t *hbpairs = reinterpret_cast<uint32_t *>(ht + bpairs_off);
    uint32_t *hspairs = reinterpret_cast<uint32_t *>(ht + spairs_off);
    uint32_t hist_tiles = 0, hist_slabs = 0, ismall = 0, ibig = 0, ibpair = 0, ispair = 0;
    for (uint32_t k = 0; k < count; k++) {
        SeqJob &J = hjobs[k];
        J.S = S[k];
        J.n = n[k];
        J.sigma = sigma[k];
        J.L = L[k];
        J.width = (uint32_t)width[k];
        J.hist = reinterpret_cast<uint64_t *>(sc + so[k].hist);
        J.hex = reinterpret_cast<uint64_t *>(sc + so[k].hex);
        J.ob = reinterpret_cast<uint64_t *>(sc + so[k].ob);
        J.ze = reinterpret_cast<uint64_t *>(sc + so[k].ze);
        J.err = d_errs + k;
        hts[k] = hist_tiles;
        hist_tiles += batch_hist_tiles(n[k], sigma[k]);
        sls[k] = hist_slabs;
        hist_slabs += batch_hist_slabs(n[k], sigma[k]);
        if (L[k] > 0) {
            if (batch_small_alphabet(L[k])) {
                hsmall[ismall++] = k;
            } else {
                hbig[ibig++] = k;
                for (uint32_t l = 0; l < L[k]; l++) {
                    if ((1ull << l) > kBatchWarpLeaves)
                        hbpairs[ibpair++] = k << 5 | l;
                    else
                        hspairs[ispair++] = k << 5 | l;
                }
            }
        }
    }
    hts[count] = hist_tiles;
    sls[count] = hist_slabs;
    bool prev_next_bits[3] = {false, false, false};
    for (auto &P : plans) {
        LevelJob *pj = reinterpret_cast<LevelJob *>(ht + P.jobs_off);
        uint32_t *pts = reinterpret_cast<uint32_t *>(ht + P.ts_off);
        uint32_t tiles = 0;
        P.max_tiles = 0;
        // Whether this level's pass writes the next level's bitmaps: few
        // tiles of the sequences that go on span a node boundary.
        uint64_t bnd = 0, ptiles = 0;
        P.do_pass = false;
        for (uint32_t k : P.seqs)
            if (L[k] > P.l + 1) {
                P.do_pass = true;
                bnd += level_boundaries(n[k], sigma[k], P.l);
                ptiles += ceil_div(n[k], lw_tile_elems(width[k]));
            }
        P.next_bits = P.do_pass && pass_writes_next_bits(bnd, ptiles, P.width);
        P.from_bits = P.l > 0 && prev_next_bits[wclass(P.width)];
        prev_next_bits[wclass(P.width)] = P.next_bits;
        P.bits = false;
        for (size_t q = 0; q < P.seqs.size(); q++) {
            const uint32_t k = P.seqs[q];
            const uint32_t l = P.l;
            const uint64_t ntk = ceil_div(n[k], lw_tile_elems(width[k]));
            const void *cur = l == 0 ? S[k] : sc + ((l & 1) ? so[k].ping : so[k].pong);
            // The last level needs no symbols when its bitmap is handed over.
            const bool no_order = P.next_bits && L[k] == l + 2;
            P.bits = P.bits || no_order;
            void *nxt = no_order ? nullptr : sc + ((l & 1) ? so[k].pong : so[k].ping);
            pj[q] = make_level_job(cur, nxt, n[k], width[k], L[k], l, reinterpret_cast<uint64_t *>(sc + so[k].ob),
                                   reinterpret_cast<uint64_t *>(sc + so[k].ze), hdesc[k].lv[l],
                                   &d_descs[k].lv[l].ones, reinterpret_cast<uint32_t *>(sc + so[k].cnt),
                                   reinterpret_cast<uint64_t *>(sc + so[k].pre),
                                   P.next_bits && l + 1 < L[k] ? hdesc[k].lv[l + 1].words : nullptr);
            pts[q] = tiles;
            tiles += (uint32_t)ntk;
            P.max_tiles = std::max(P.max_tiles, (uint32_t)ntk);
        }
        pts[P.seqs.size()] = tiles;
        P.total = tiles;
    }
    memcpy(ht + tbytes, hdesc.data(), sizeof(TreeDesc) * count);

    // ---- device work (captured into one graph when the stream is idle-capturable)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool use_graph = cap == cudaStreamCaptureStatusNone && st != nullptr;
    cudaGraph_t graph = nullptr;
    wt_status r = WT_OK;
    if (use_graph && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && r == WT_OK) r = WT_ERR_CUDA;
    };
    if (r == WT_OK) {
        if (zeroed) ck(cudaMemsetAsync(sc, 0, zeroed, st));
        ck(cudaMemsetAsync(B->d_err, 0, 4, st));
        ck(cudaMemcpyAsync(dt, ht, tbytes, cudaMemcpyHostToDevice, st));
        ck(cudaMemcpyAsync(d_descs, ht + tbytes, sizeof(TreeDesc) * count, cudaMemcpyHostToDevice, st));

        // empty sequences: R[0] = Hy[0] = 0
        for (uint32_t k = 0; k < count; k++)
            if (n[k] == 0)
                for (uint32_t l = 0; l < L[k]; l++) {
                    ck(cudaMemsetAsync(hdesc[k].lv[l].R, 0, 4, st));
                    ck(cudaMemsetAsync(hdesc[k].lv[l].Hy, 0, 8, st));
                }
        {
            double nw = 0;
            for (uint32_t k = 0; k < count; k++) nw += (double)n[k] * width[k];
            ProfScope p(K_HIST, nw, st);
            ck(launch_batch_prepare(reinterpret_cast<const SeqJob *>(dt + seqjob_off), count,
                                    reinterpret_cast<const uint32_t *>(dt + hts_off), hist_tiles,
                                    reinterpret_cast<const uint32_t *>(dt + sls_off), hist_slabs,
                                    reinterpret_cast<const uint32_t *>(dt + small_off), nsmall,
                                    reinterpret_cast<const uint32_t *>(dt + big_off), nbig,
                                    reinterpret_cast<const uint32_t *>(dt + bpairs_off), nbig_pairs,
                                    reinterpret_cast<const uint32_t *>(dt + spairs_off), nsmall_pairs, st));
        }
        for (size_t q = 0; q < plans.size(); q++) {
            const LaunchPlan &P = plans[q];
            double bytes = 0;
            for (uint32_t k : P.seqs)
                bytes += level_step_bytes(n[k], width[k], P.l + 1 < L[k]);
            ProfScope p(K_LEVEL_PASS, bytes, st);
            ck(launch_level_jobs(P.width, P.l, reinterpret_cast<const LevelJob *>(dt + P.jobs_off),
                                 reinterpret_cast<const uint32_t *>(dt + P.ts_off), (uint32_t)P.seqs.size(), P.total,
                                 P.max_tiles, P.from_bits, P.do_pass, B->d_err, st, false, nullptr, 0, false,
                                 P.bits));
        }
    }
    if (use_graph) {
        if (cudaStreamEndCapture(st, &graph) != cudaSuccess) {
            cudaGetLastError();
            r = WT_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        if (r == WT_OK && (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess || cudaGraphLaunch(exec, st) != cudaSuccess)) {
            cudaGetLastError();
            r = WT_ERR_CUDA;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    ck(cudaEventRecord(ps.ready, st));
    ck(cudaEventRecord(B->done, st));
    dev_free(A, scratch, total_scratch, st);  // stream-ordered, after the batch
    if (r != WT_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        return r;
    }
    for (uint32_t k = 0; k < count; k++) {
        wt_tree *t = new (std::nothrow) wt_tree();
        if (!t) {
            for (uint32_t q = 0; q < k; q++) tree_destroy(trees[q]);
            return WT_ERR_OOM;
        }
        t->batch = B;
        t->n = n[k];
        t->sigma = sigma[k];
        t->L = L[k];
        t->width = width[k];
        t->variant = WT_VARIANT_LEVELWISE;
        t->alloc = A;
        t->stream = st;
        t->d_desc = d_descs + k;
        t->d_err = d_errs + k;
        t->h_desc = hdesc[k];
        t->mem_bytes = level_bytes_of(n[k]) * L[k] + sizeof(TreeDesc) + 4;
        trees[k] = t;
    }
    for (uint32_t k = 0; k < count; k++) out[k] = trees[k];
    return WT_OK;
}

// The library's host-to-device copy stream of the current device (created
// once, non-blocking).
cudaStream_t copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

wt_handle build_async(const void *S, uint64_t n, uint64_t sigma, int width, int variant, cudaStream_t st,
                      bool matrix = false) {
    wt_status r = check_args(S, n, sigma, width);
    if (r != WT_OK) {
        set_last(r);
        return nullptr;
    }
    if (variant < WT_VARIANT_AUTO || variant > WT_VARIANT_PAIRS ||
        (variant == WT_VARIANT_DD && n > 0 && levels_of(sigma) > 0 && !dd_supported(n, sigma, width))) {
        set_last(WT_ERR_ARG);
        return nullptr;
    }
    wt_tree *t = new (std::nothrow) wt_tree();
    if (!t) {
        set_last(WT_ERR_OOM);
        return nullptr;
    }
    t->n = n;
    t->sigma = sigma;
    t->L = levels_of(sigma);
    t->width = width;
    t->stream = st;
    t->alloc = current_allocator();
    t->matrix = matrix;
    if (cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete t;
        set_last(WT_ERR_CUDA);
        return nullptr;
    }
    r = tree_alloc(t, st);
    const void *Sd = S;
    void *staged = nullptr;
    const size_t sbytes = n * (uint64_t)width;
    if (r == WT_OK && n > 0 && !is_device_pointer(S)) {
        // Host symbols are staged on the library's copy stream when the
        // default allocator is in use and st is not being captured: the copy
        // for one call then overlaps the build of the previous call on st,
        // and st waits only for its own copy.  Otherwise the copy goes on st.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cudaGetLastError();
        cudaStream_t cs = (!t->alloc.alloc && cap == cudaStreamCaptureStatusNone) ? copy_stream() : nullptr;
        cudaStream_t on = cs ? cs : st;
        staged = dev_alloc(t->alloc, sbytes, on);
        if (!staged) {
            r = WT_ERR_OOM;
        } else if (cudaMemcpyAsync(staged, S, sbytes, cudaMemcpyHostToDevice, on) != cudaSuccess) {
            cudaGetLastError();
            r = WT_ERR_CUDA;
        } else if (cs) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(ev, cs) != cudaSuccess || cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
                cudaGetLastError();
                r = WT_ERR_CUDA;
            }
            if (ev) cudaEventDestroy(ev);
        }
        Sd = staged;
    }
    if (r == WT_OK) r = enqueue_build(t, Sd, variant, st);
    if (staged) dev_free(t->alloc, staged, sbytes, st);
    if (r == WT_OK && cudaEventRecord(t->done, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r != WT_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        t->finalized = true;
        tree_destroy(t);
        set_last(r);
        return nullptr;
    }
    set_last(WT_OK);
    return t;
}

// ------------------------------------------------------------- merges

// Algorithmic bytes of one merged level of n bits: read the parts' bits,
// write the level and its directory.
double merge_level_bytes(uint64_t n) { return n / 8.0 + n / 8.0 + n / 128.0; }

// Creates the handle of a tree of n symbols (memory allocated, descriptor
// filled, nothing enqueued).
wt_status tree_create(uint64_t n, uint64_t sigma, int width, cudaStream_t st, wt_tree **out) {
    wt_tree *t = new (std::nothrow) wt_tree();
    if (!t) return WT_ERR_OOM;
    t->n = n;
    t->sigma = sigma;
    t->L = levels_of(sigma);
    t->width = width;
    t->stream = st;
    t->alloc = current_allocator();
    if (cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete t;
        return WT_ERR_CUDA;
    }
    const wt_status r = tree_alloc(t, st);
    if (r != WT_OK) {
        t->finalized = true;
        tree_destroy(t);
        return r;
    }
    *out = t;
    return WT_OK;
}

// Enqueues the merge of k finished parts into t (allocated, n = the parts'
// total): every part's node starts, then per level the bits (merge.cu) and
// the directory (the level step's count from the bitmap and its scans).
wt_status enqueue_merge(wt_tree *t, const wt_handle *parts, uint32_t k, cudaStream_t st) {
    WT_CK(cudaMemcpyAsync(t->d_desc, &t->h_desc, sizeof(TreeDesc), cudaMemcpyHostToDevice, st));
    WT_CK(cudaMemsetAsync(t->d_err, 0, sizeof(uint32_t), st));
    if (t->n == 0 || t->L == 0) {
        for (uint32_t l = 0; l < t->L; l++) {
            WT_CK(cudaMemsetAsync(t->h_desc.lv[l].R, 0, 4, st));
            WT_CK(cudaMemsetAsync(t->h_desc.lv[l].Hy, 0, 8, st));
        }
        return WT_OK;
    }
    const uint64_t stride = (1ull << t->L) + 1;
    const size_t ptrs = align256(k * sizeof(TreeDesc *));
    const size_t hex = align256((size_t)k * stride * 8);
    const size_t hexm = align256(stride * 8);
    const size_t counts = align256(lw_counts_bytes(t->n, t->width));
    const size_t prefix = align256(lw_prefix_bytes(t->n, t->width));
    const size_t jslot = level_job_slot_bytes();
    const size_t bytes = ptrs + hex + hexm + counts + prefix + jslot;
    char *mem = static_cast<char *>(dev_alloc(t->alloc, bytes, st));
    if (!mem) return WT_ERR_OOM;
    const TreeDesc **d_parts = reinterpret_cast<const TreeDesc **>(mem);
    uint64_t *d_hex = reinterpret_cast<uint64_t *>(mem + ptrs);
    uint64_t *d_hexm = reinterpret_cast<uint64_t *>(mem + ptrs + hex);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(mem + ptrs + hex + hexm);
    uint64_t *pre = reinterpret_cast<uint64_t *>(mem + ptrs + hex + hexm + counts);
    void *job_slot = mem + ptrs + hex + hexm + counts + prefix;
    std::vector<const TreeDesc *> hp(k);
    for (uint32_t a = 0; a < k; a++) hp[a] = parts[a]->d_desc;
    wt_status r = WT_OK;
    if (cudaMemcpyAsync(d_parts, hp.data(), k * sizeof(TreeDesc *), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK) {
        ProfScope p(K_MERGE_STARTS, 8.0 * (k + 1) * stride, st);
        if (launch_merge_starts(d_parts, k, t->L, d_hex, d_hexm, t->d_err, st) != cudaSuccess) r = WT_ERR_CUDA;
    }
    for (uint32_t l = 0; l < t->L && r == WT_OK; l++) {
        ProfScope p(K_MERGE, merge_level_bytes(t->n), st);
        // With L = l + 1 the level step counts from the bitmap and scans
        // (R, Hy, S1, S0, ones) without a pass; the node tables are unused.
        if (launch_merge_level(d_parts, k, t->L, l, d_hex, d_hexm, t->n, t->h_desc.lv[l].words, t->d_err, st) !=
                cudaSuccess ||
            launch_level_pass(nullptr, nullptr, t->n, t->width, l + 1, l, d_hexm, d_hexm, t->h_desc.lv[l],
                              &t->d_desc->lv[l].ones, cnt, pre, true, nullptr, t->d_err, job_slot, st) !=
                cudaSuccess)
            r = WT_ERR_CUDA;
    }
    if (r != WT_OK) cudaGetLastError();
    dev_free(t->alloc, mem, bytes, st);
    return r;
}

// Largest number of parts of one merge (its scratch holds k (2^L + 1) node
// starts).
constexpr uint32_t kMaxMergeParts = 1u << 16;

wt_handle merge_async(const wt_handle *parts, uint32_t k, cudaStream_t st) {
    if (!parts || k == 0 || k > kMaxMergeParts || !parts[0]) {
        set_last(WT_ERR_ARG);
        return nullptr;
    }
    uint64_t n = 0;
    for (uint32_t a = 0; a < k; a++) {
        if (!parts[a] || parts[a]->sigma != parts[0]->sigma || parts[a]->width != parts[0]->width ||
            parts[a]->matrix || parts[a]->universe) {
            set_last(WT_ERR_ARG);
            return nullptr;
        }
        n += parts[a]->n;
    }
    if (n >= (1ull << 56)) {
        set_last(WT_ERR_ARG);
        return nullptr;
    }
    // The parts' builds must have completed (and succeeded) first.
    for (uint32_t a = 0; a < k; a++) {
        const wt_status ps = finalize(parts[a]);
        if (ps != WT_OK) {
            set_last(ps);
            return nullptr;
        }
    }
    wt_tree *t = nullptr;
    wt_status r = tree_create(n, parts[0]->sigma, parts[0]->width, st, &t);
    if (r != WT_OK) {
        set_last(r);
        return nullptr;
    }
    t->variant = parts[0]->variant;
    r = enqueue_merge(t, parts, k, st);
    if (r == WT_OK && cudaEventRecord(t->done, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r != WT_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        t->finalized = true;
        tree_destroy(t);
        set_last(r);
        return nullptr;
    }
    set_last(WT_OK);
    return t;
}

// The buffered build of Section 5: S in chunks of at most `chunk` symbols,
// each built alone into a partial tree, then one merge.  At most two
// chunks' builds are in flight, so at most two chunks of host symbols are
// staged on the device at a time.
// ------------------------------------------------- alphabet remapping

// The tree of S over a non-contiguous alphabet (Section 3): the alphabet
// bitmap A over [0, universe) marks the codes that occur (remap.cu), the
// level step's count and scan give A its directory, the host reads
// sigma' = the ones of A (the one host wait), then S' = rank1(A, S) is built
// as an ordinary tree over [0, sigma') with the narrowest width that holds
// sigma' codes.  The handle keeps A for the queries.
wt_handle build_remap(const void *S, uint64_t n, uint64_t universe, int width, cudaStream_t st) {
    if (width != 1 && width != 2 && width != 4) return set_last(WT_ERR_ARG), nullptr;
    if (universe == 0 || universe > (1ull << (8 * width)) || (n > 0 && !S) ||
        (n > 0 && reinterpret_cast<uintptr_t>(S) % (uintptr_t)width) || n >= (1ull << 56))
        return set_last(WT_ERR_ARG), nullptr;
    const Allocator A = current_allocator();
    // Device copy of host symbols (in stream order on st).
    const size_t sbytes = n * (uint64_t)width;
    const void *Sd = S;
    void *staged = nullptr;
    if (n > 0 && !is_device_pointer(S)) {
        staged = dev_alloc(A, sbytes, st);
        if (!staged) return set_last(WT_ERR_OOM), nullptr;
        if (cudaMemcpyAsync(staged, S, sbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            dev_free(A, staged, sbytes, st);
            return set_last(WT_ERR_CUDA), nullptr;
        }
        Sd = staged;
    }
    // The alphabet block: A's words and directory, then the count and scan
    // scratch, the error word and the ones count.
    const Shape sa = shape_of(universe);
    const size_t cnt_b = align256(lw_counts_bytes(universe, 1)), pre_b = align256(lw_prefix_bytes(universe, 1));
    const size_t keep = sa.words + sa.R + sa.Hy + 2 * sa.S;
    const size_t abytes = keep + cnt_b + pre_b + level_job_slot_bytes() + 512;
    char *am = static_cast<char *>(dev_alloc(A, abytes, st));
    if (!am) {
        if (staged) dev_free(A, staged, sbytes, st);
        return set_last(WT_ERR_OOM), nullptr;
    }
    LevelDesc ad{};
    char *p = am;
    ad.words = reinterpret_cast<uint32_t *>(p);
    p += sa.words;
    ad.R = reinterpret_cast<uint32_t *>(p);
    p += sa.R;
    ad.Hy = reinterpret_cast<uint64_t *>(p);
    p += sa.Hy;
    ad.S1 = reinterpret_cast<uint32_t *>(p);
    p += sa.S;
    ad.S0 = reinterpret_cast<uint32_t *>(p);
    p += sa.S;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(p);
    p += cnt_b;
    uint64_t *pre = reinterpret_cast<uint64_t *>(p);
    p += pre_b;
    void *slot = p;
    p += level_job_slot_bytes();
    uint32_t *err = reinterpret_cast<uint32_t *>(p);
    uint64_t *ones = reinterpret_cast<uint64_t *>(p + 256);
    uint64_t h_ones = 0;
    uint32_t h_err = 0;
    wt_status r = WT_OK;
    if (cudaMemsetAsync(ad.words, 0, sa.nblocks * 64, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, 4, st) != cudaSuccess || cudaMemsetAsync(ones, 0, 8, st) != cudaSuccess ||
        launch_alpha_mark(Sd, n, width, universe, ad.words, err, st) != cudaSuccess ||
        launch_level_directory(universe, 1, 1, 0, ad, ones, cnt, pre, err, slot, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_ones, ones, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK && (h_err & kErrSymbol)) r = WT_ERR_SYMBOL_RANGE;
    if (r == WT_OK && (h_err & kErrTimeout)) r = WT_ERR_TIMEOUT;
    ad.ones = h_ones;
    const uint64_t sigma_r = h_ones ? h_ones : 1;  // an empty S still has a tree (of no levels)
    const int w_r = sigma_r <= 256 ? 1 : (sigma_r <= 65536 ? 2 : 4);
    wt_tree *t = nullptr;
    void *mapped = nullptr;
    const size_t mbytes = n * (uint64_t)w_r;
    if (r == WT_OK) r = tree_create(n, sigma_r, w_r, st, &t);
    if (r == WT_OK && n > 0) {
        mapped = dev_alloc(A, mbytes, st);
        if (!mapped) r = WT_ERR_OOM;
        else if (launch_alpha_map(Sd, n, width, ad, mapped, w_r, st) != cudaSuccess) r = WT_ERR_CUDA;
    }
    if (r == WT_OK) r = enqueue_build(t, mapped, WT_VARIANT_AUTO, st);
    if (mapped) dev_free(A, mapped, mbytes, st);
    if (staged) dev_free(A, staged, sbytes, st);
    if (r == WT_OK && cudaEventRecord(t->done, st) != cudaSuccess) r = WT_ERR_CUDA;
    if (r != WT_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        dev_free(A, am, abytes, st);
        if (t) {
            t->finalized = true;
            tree_destroy(t);
        }
        return set_last(r), nullptr;
    }
    t->universe = universe;
    t->alpha = ad;
    t->alpha_mem = am;
    t->alpha_bytes = abytes;
    set_last(WT_OK);
    return t;
}

wt_handle build_chunked(const void *S, uint64_t n, uint64_t sigma, int width, uint64_t chunk, cudaStream_t st) {
    wt_status r = check_args(S, n, sigma, width);
    if (r == WT_OK && chunk == 0) r = WT_ERR_ARG;
    const uint64_t k = (r == WT_OK && n) ? ceil_div(n, chunk) : 1;
    if (r == WT_OK && k > kMaxMergeParts) r = WT_ERR_ARG;
    if (r != WT_OK) {
        set_last(r);
        return nullptr;
    }
    if (k == 1) return build_async(S, n, sigma, width, WT_VARIANT_AUTO, st);
    std::vector<wt_handle> parts;
    parts.reserve(k);
    const char *base = static_cast<const char *>(S);
    for (uint64_t a = 0; a < k && r == WT_OK; a++) {
        const uint64_t lo = a * chunk, len = (lo + chunk < n ? chunk : n - lo);
        wt_handle h = build_async(base + lo * (uint64_t)width, len, sigma, width, WT_VARIANT_AUTO, st);
        if (!h) {
            r = g_last;
            break;
        }
        parts.push_back(h);
        if (a >= 2) r = finalize(parts[a - 2]);
    }
    wt_handle out = nullptr;
    if (r == WT_OK) {
        out = merge_async(parts.data(), (uint32_t)k, st);
        if (!out) r = g_last;
    }
    if (r != WT_OK) cudaStreamSynchronize(st);
    // The parts' memory returns in stream order after the merge has read it.
    for (wt_handle h : parts) {
        h->finalized = true;
        tree_destroy(h);
    }
    set_last(r);
    return out;
}

}  // namespace

namespace wt {
void note_launches(uint32_t k) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

wt_status check_symbol_args(const void *S, uint64_t n, uint64_t sigma, int width) {
    return check_args(S, n, sigma, width);
}

// Sets the calling thread's last status (for entry points in other files).
wt_status record_status(wt_status s) { return set_last(s); }
}  // namespace wt

// ====================================================================== ABI

extern "C" {

wt_handle wt_build(const void *S, uint64_t n, uint64_t sigma, int sym_width) {
    wt_handle h = build_async(S, n, sigma, sym_width, WT_VARIANT_AUTO, nullptr);
    if (!h) return nullptr;
    wt_status r = finalize(h);
    if (r != WT_OK) {
        tree_destroy(h);
        set_last(r);
        return nullptr;
    }
    set_last(WT_OK);
    return h;
}

wt_handle wt_build_async(const void *S, uint64_t n, uint64_t sigma, int sym_width, int variant, void *stream) {
    return build_async(S, n, sigma, sym_width, variant, static_cast<cudaStream_t>(stream));
}

wt_status wt_wait(wt_handle h) {
    if (!h) return set_last(WT_ERR_ARG);
    return set_last(finalize(h));
}

wt_status wt_build_batch(const void *const *S, const uint64_t *n, const uint64_t *sigma, const int *sym_width,
                         uint32_t count, wt_handle *out, void *stream) {
    if (count > 0 && (!S || !n || !sigma || !sym_width || !out)) return set_last(WT_ERR_ARG);
    return set_last(build_batch_impl(S, n, sigma, sym_width, count, out, static_cast<cudaStream_t>(stream)));
}

wt_handle wt_build_matrix_async(const void *S, uint64_t n, uint64_t sigma, int sym_width, void *stream) {
    return build_async(S, n, sigma, sym_width, WT_VARIANT_LEVELWISE, static_cast<cudaStream_t>(stream), true);
}

wt_handle wt_build_remap(const void *S, uint64_t n, uint64_t universe, int sym_width, void *stream) {
    return build_remap(S, n, universe, sym_width, static_cast<cudaStream_t>(stream));
}

wt_handle wt_merge_async(const wt_handle *parts, uint32_t k, void *stream) {
    return merge_async(parts, k, static_cast<cudaStream_t>(stream));
}

wt_handle wt_build_chunked(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t chunk, void *stream) {
    return build_chunked(S, n, sigma, sym_width, chunk, static_cast<cudaStream_t>(stream));
}

wt_status wt_access(wt_handle h, const uint64_t *i, uint64_t m, uint32_t *out, void *stream) {
    if (!h || (m && (!i || !out))) return set_last(WT_ERR_ARG);
    ProfScope p(K_Q_ACCESS, 16.0 * m, static_cast<cudaStream_t>(stream));
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = h->matrix      ? launch_wm_access(h->d_desc, i, m, out, st)
                          : h->universe ? launch_access_remap(h->d_desc, h->alpha, h->universe, i, m, out, st)
                                        : launch_access(h->d_desc, i, m, out, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last(WT_ERR_CUDA);
    }
    return set_last(WT_OK);
}

wt_status wt_rank(wt_handle h, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out, void *stream) {
    if (!h || (m && (!c || !i || !out))) return set_last(WT_ERR_ARG);
    ProfScope p(K_Q_RANK, 16.0 * m, static_cast<cudaStream_t>(stream));
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = h->matrix      ? launch_wm_rank(h->d_desc, c, i, m, out, st)
                          : h->universe ? launch_rank_remap(h->d_desc, h->alpha, h->universe, c, i, m, out, st)
                                        : launch_rank(h->d_desc, c, i, m, out, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last(WT_ERR_CUDA);
    }
    return set_last(WT_OK);
}

wt_status wt_select(wt_handle h, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out, void *stream) {
    if (!h || (m && (!c || !j || !out))) return set_last(WT_ERR_ARG);
    ProfScope p(K_Q_SELECT, 16.0 * m, static_cast<cudaStream_t>(stream));
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = h->matrix      ? launch_wm_select(h->d_desc, c, j, m, out, st)
                          : h->universe ? launch_select_remap(h->d_desc, h->alpha, h->universe, c, j, m, out, st)
                                        : launch_select(h->d_desc, c, j, m, out, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last(WT_ERR_CUDA);
    }
    return set_last(WT_OK);
}

wt_status wt_query_multi(const wt_handle *trees, uint32_t ntrees, const uint32_t *tree_idx, const uint8_t *op,
                         const uint32_t *c, const uint64_t *arg, uint64_t m, uint64_t *out, void *stream) {
    if (m == 0) return set_last(WT_OK);
    if (!trees || ntrees == 0 || !tree_idx || !op || !c || !arg || !out) return set_last(WT_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<const TreeDesc *> ptrs(ntrees);
    for (uint32_t k = 0; k < ntrees; k++) {
        if (!trees[k] || trees[k]->matrix || trees[k]->universe) return set_last(WT_ERR_ARG);
        ptrs[k] = trees[k]->d_desc;
    }
    const Allocator A = current_allocator();
    const size_t bytes = ntrees * sizeof(TreeDesc *);
    void *d = dev_alloc(A, bytes, st);
    if (!d) return set_last(WT_ERR_OOM);
    wt_status r = WT_OK;
    ProfScope p(K_Q_MULTI, 25.0 * m, st);
    if (cudaMemcpyAsync(d, ptrs.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        launch_query_multi(static_cast<const TreeDesc *const *>(d), ntrees, tree_idx, op, c, arg, m, out, st) !=
            cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    dev_free(A, d, bytes, st);
    return set_last(r);
}

wt_status wt_free(wt_handle h) {
    if (!h) return set_last(WT_ERR_ARG);
    tree_destroy(h);
    return set_last(WT_OK);
}

wt_status wt_info(wt_handle h, wt_info_t *out) {
    if (!h || !out) return set_last(WT_ERR_ARG);
    finalize(h);
    out->n = h->n;
    out->sigma = h->sigma;
    out->levels = h->L;
    out->sym_width = h->width;
    out->variant = h->variant;
    out->layout = h->matrix ? WT_LAYOUT_MATRIX : WT_LAYOUT_TREE;
    out->device_bytes = h->mem_bytes + h->alpha_bytes;
    out->universe = h->universe;
    return set_last(h->status);
}

wt_status wt_alphabet_view(wt_handle h, wt_level_view_t *out) {
    if (!h || !out || !h->universe) return set_last(WT_ERR_ARG);
    finalize(h);
    const Shape s = shape_of(h->universe);
    const LevelDesc &d = h->alpha;
    out->words = d.words;
    out->R = d.R;
    out->Hy = d.Hy;
    out->S1 = d.S1;
    out->S0 = d.S0;
    out->ones = d.ones;
    out->n_words = s.nblocks * 16;
    out->n_R = s.nblocks + 1;
    out->n_Hy = s.nspans + 1;
    out->n_S1 = ceil_div(d.ones, kSample);
    out->n_S0 = ceil_div(h->universe - d.ones, kSample);
    return set_last(h->status);
}

wt_status wt_level_view(wt_handle h, uint32_t l, wt_level_view_t *out) {
    if (!h || !out || l >= h->L) return set_last(WT_ERR_ARG);
    finalize(h);
    const Shape s = shape_of(h->n);
    const LevelDesc &d = h->h_desc.lv[l];
    out->words = d.words;
    out->R = d.R;
    out->Hy = d.Hy;
    out->S1 = d.S1;
    out->S0 = d.S0;
    out->ones = d.ones;
    out->n_words = s.nblocks * 16;
    out->n_R = s.nblocks + 1;
    out->n_Hy = s.nspans + 1;
    out->n_S1 = ceil_div(d.ones, kSample);
    out->n_S0 = ceil_div(h->n - d.ones, kSample);
    return set_last(h->status);
}

wt_status wt_set_allocator(void *(*alloc)(size_t, void *, void *), void (*free_)(void *, size_t, void *, void *),
                           void *ctx) {
    if ((alloc == nullptr) != (free_ == nullptr)) return set_last(WT_ERR_ARG);
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = {alloc, free_, ctx};
    return set_last(WT_OK);
}

wt_status wt_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto &r : g_prof.recs) {
        g_prof.pool.push_back(r.e0);
        g_prof.pool.push_back(r.e1);
    }
    g_prof.recs.clear();
    g_prof.on = true;
    return set_last(WT_OK);
}

wt_status wt_profile_end(wt_kernel_stat_t *out, uint32_t cap, uint32_t *count) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = false;
    wt_kernel_stat_t acc[K_COUNT];
    memset(acc, 0, sizeof(acc));
    wt_status r = WT_OK;
    for (auto &rec : g_prof.recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(rec.e1) != cudaSuccess || cudaEventElapsedTime(&ms, rec.e0, rec.e1) != cudaSuccess) {
            cudaGetLastError();
            r = WT_ERR_CUDA;
            continue;
        }
        acc[rec.kid].launches += rec.units;
        acc[rec.kid].kernels += rec.k1 - rec.k0;
        acc[rec.kid].total_ms += ms;
        acc[rec.kid].alg_bytes += rec.bytes;
        acc[rec.kid].variant_bytes += rec.vbytes;
        g_prof.pool.push_back(rec.e0);
        g_prof.pool.push_back(rec.e1);
    }
    g_prof.recs.clear();
    uint32_t k = 0;
    for (int id = 0; id < K_COUNT; id++) {
        if (!acc[id].launches) continue;
        if (out && k < cap) {
            out[k] = acc[id];
            strncpy(out[k].name, kKernelNames[id], sizeof(out[k].name) - 1);
        }
        k++;
    }
    if (count) *count = k;
    return set_last(r);
}

wt_status wt_last_status(void) { return g_last; }

const char *wt_status_string(wt_status s) {
    switch (s) {
        case WT_OK: return "ok";
        case WT_ERR_ARG: return "invalid argument";
        case WT_ERR_SYMBOL_RANGE: return "symbol out of range";
        case WT_ERR_OOM: return "out of device memory";
        case WT_ERR_CUDA: return "CUDA error";
        case WT_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

wt_status wt_node_starts(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t *Hex, void *stream) {
    wt_status r = check_args(S, n, sigma, sym_width);
    if (r != WT_OK || !Hex) return set_last(r != WT_OK ? r : WT_ERR_ARG);
    if (n > 0 && !is_device_pointer(S)) return set_last(WT_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Allocator A = current_allocator();
    const uint32_t L = levels_of(sigma);
    const size_t bytes = align256(sigma * 8) + 256;
    void *mem = dev_alloc(A, bytes, st);
    if (!mem) return set_last(WT_ERR_OOM);
    uint64_t *hist = static_cast<uint64_t *>(mem);
    uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<char *>(mem) + align256(sigma * 8));
    uint32_t herr = 0;
    if (cudaMemsetAsync(mem, 0, bytes, st) != cudaSuccess ||
        launch_histogram(S, n, sym_width, sigma, hist, err, st) != cudaSuccess ||
        launch_node_starts(hist, sigma, L, n, Hex, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    dev_free(A, mem, bytes, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK && (herr & kErrSymbol)) r = WT_ERR_SYMBOL_RANGE;
    return set_last(r);
}

wt_status wt_level_step(const void *cur, uint64_t n, uint64_t sigma, int sym_width, uint32_t l, const uint64_t *Hex,
                        uint32_t *words, uint32_t *R, void *nxt, void *stream) {
    wt_status r = check_args(cur, n, sigma, sym_width);
    if (r != WT_OK) return set_last(r);
    const uint32_t L = levels_of(sigma);
    if (l >= L || !Hex || (n > 0 && (!words || !R))) return set_last(WT_ERR_ARG);
    if (nxt && reinterpret_cast<uintptr_t>(nxt) % (uintptr_t)sym_width != 0) return set_last(WT_ERR_ARG);
    if (n == 0) return set_last(WT_OK);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Allocator A = current_allocator();
    const Shape s = shape_of(n);
    // Scratch: error word, tile counts and prefixes, node tables, and the
    // directory parts this entry point does not return (Hy, S1, S0, ones).
    const size_t tab = align256((1ull << L) * 8);
    const size_t counts = align256(lw_counts_bytes(n, sym_width));
    const size_t prefix = align256(lw_prefix_bytes(n, sym_width));
    const size_t zeroed = 256;
    const size_t bytes = zeroed + counts + prefix + 2 * tab + s.Hy + 2 * s.S + 256 + level_job_slot_bytes();
    void *mem = dev_alloc(A, bytes, st);
    if (!mem) return set_last(WT_ERR_OOM);
    char *p = static_cast<char *>(mem);
    uint32_t *err = reinterpret_cast<uint32_t *>(p);
    p += 256;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(p);
    p += counts;
    uint64_t *pre = reinterpret_cast<uint64_t *>(p);
    p += prefix;
    uint64_t *ob = reinterpret_cast<uint64_t *>(p);
    p += tab;
    uint64_t *ze = reinterpret_cast<uint64_t *>(p);
    p += tab;
    LevelDesc lv;
    lv.words = words;
    lv.R = R;
    lv.Hy = reinterpret_cast<uint64_t *>(p);
    p += s.Hy;
    lv.S1 = reinterpret_cast<uint32_t *>(p);
    p += s.S;
    lv.S0 = reinterpret_cast<uint32_t *>(p);
    p += s.S;
    uint64_t *ones = reinterpret_cast<uint64_t *>(p);
    p += 256;
    void *job_slot = p;
    lv.ones = 0;
    uint32_t herr = 0;
    if (cudaMemsetAsync(mem, 0, zeroed, st) != cudaSuccess ||
        launch_node_tables(Hex, L, ob, ze, st) != cudaSuccess ||
        launch_level_pass(cur, (l + 1 < L) ? nxt : nullptr, n, sym_width, L, l, ob, ze, lv, ones, cnt, pre, false,
                          nullptr, err,
                          job_slot, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    dev_free(A, mem, bytes, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        r = WT_ERR_CUDA;
    }
    if (r == WT_OK && (herr & kErrTimeout)) r = WT_ERR_TIMEOUT;
    return set_last(r);
}

}  // extern "C"
