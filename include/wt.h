/*
 * wt.h -- C ABI of the GB300 (sm_103a) builder and query engine for the
 * pointerless, level-wise wavelet tree of "Parallel Construction of Wavelet
 * Trees on Multicore Architectures" (arXiv 1610.05994).
 *
 * The problem (Section 2.3): given S[0..n) over the alphabet [0, sigma),
 * build the wavelet tree with one pointer per level (Section 2.2, Fig. 2b):
 * L = ceil(lg sigma) bitmaps of n bits, level l holding the level-l bit of
 * every symbol with the symbols ordered stably by their top l bits
 * (Proposition 1), plus rank/select directories, and answer access, rank and
 * select (Section 2.2).
 *
 * Conventions shared by every call:
 *   - Symbols are codes in [0, sigma), stored as unsigned integers of
 *     sym_width bytes (1, 2 or 4), little-endian, packed, with the array
 *     aligned to sym_width bytes (else WT_ERR_ARG).
 *   - Level l of node v holds the symbols s with s >> (L - l) == v; a node
 *     splits on the bit (s >> (L - 1 - l)) & 1, so for sigma not a power of
 *     two some nodes are empty.
 *   - rank_c(i) counts c in the half-open prefix [0, i); select_c(j) is the
 *     0-based position of the j-th (1-based) occurrence of c.
 *   - Pointers named "device" must point to device memory of the current
 *     CUDA device; S of a build may be device or host memory.
 *   - A stream argument is a cudaStream_t passed as void*; NULL is the
 *     legacy default stream.  Calls that take a stream are asynchronous on
 *     it unless stated.
 *   - Functions returning wt_status also set the calling thread's last
 *     status (wt_last_status()); functions returning a handle return NULL on
 *     failure and set it.
 *
 * Serialised layout of one level (identical to what the CPU oracle emits):
 *   words: ceil(n/512) * 16 uint32 words; bit p is bit (p & 31) of word
 *          p >> 5 (equivalently byte p >> 3, bit p & 7); bits >= n are 0.
 *   R:     ceil(n/512) + 1 uint32; R[b] = (ones in [0, 512 b)) mod 2^32.
 *   Hy:    ceil(n/2^32) + 1 uint64; Hy[h] = ones in [0, min(n, 2^32 h)).
 *   S1:    ceil(ones/8192) uint32; S1[k] = (position of the one of 0-based
 *          rank 8192 k) >> 9.  S0: the same for zeros at positions < n.
 *   ones:  ones in [0, n).
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque tree handle; owned by the library until wt_free. */
typedef struct wt_tree *wt_handle;

typedef enum {
    WT_OK = 0,
    WT_ERR_ARG = 1,          /* invalid argument (width, sigma, pointer, level) */
    WT_ERR_SYMBOL_RANGE = 2, /* some S[j] >= sigma; found on the device, no trap */
    WT_ERR_OOM = 3,          /* the allocator returned NULL */
    WT_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    WT_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up */
} wt_status;

/* Construction variants.  AUTO picks per (n, sigma, width) from a measured
 * table; LEVELWISE is one level per pass (kernels a + b + c); DD builds every
 * level straight from S with per-tile prefix histograms (kernel d, for small
 * sigma only: it returns WT_ERR_ARG when 2^L - 1 node counters per tile do
 * not fit); PAIRS takes two levels per pass (a radix digit of two tree bits:
 * one read of P_l writes levels l and l + 1 and places every symbol into
 * P_{l+2}) for 1- and 2-byte symbols on levels whose tiles mostly lie in one
 * node, and one level per pass elsewhere.  Every variant builds the same
 * tree, bit for bit. */
typedef enum {
    WT_VARIANT_AUTO = 0,
    WT_VARIANT_LEVELWISE = 1,
    WT_VARIANT_DD = 2,
    WT_VARIANT_PAIRS = 3
} wt_variant;

/* What a handle holds (wt_info_t.layout). */
typedef enum { WT_LAYOUT_TREE = 0, WT_LAYOUT_MATRIX = 1 } wt_layout;

/* Query operation codes for wt_query_multi. */
typedef enum { WT_OP_ACCESS = 0, WT_OP_RANK = 1, WT_OP_SELECT = 2 } wt_op;

/* Largest supported alphabet: 2^28 codes (28 levels; the node tables take
 * 3 * 2^L * 8 bytes during a build). */
#define WT_MAX_SIGMA (1ull << 28)
#define WT_MAX_LEVELS 28

/*
 * Builds the tree of S[0..n) over [0, sigma) (Section 2.3; Algorithm 1 is
 * the sequential statement of what is built).  Synchronous: returns once the
 * tree is resident and checked.  NULL on failure: WT_ERR_ARG for
 * sym_width not in {1, 2, 4}, sigma == 0, sigma > 2^(8 sym_width) or
 * sigma > WT_MAX_SIGMA, or S == NULL with n > 0; WT_ERR_SYMBOL_RANGE if any
 * symbol is >= sigma; WT_ERR_OOM, WT_ERR_CUDA, WT_ERR_TIMEOUT otherwise.
 * S may be host or device memory; the caller keeps ownership.
 */
wt_handle wt_build(const void *S, uint64_t n, uint64_t sigma, int sym_width);

/*
 * As wt_build, but enqueued on stream and returning at once; the handle is
 * valid immediately for further calls on the same stream.  Arguments are
 * checked on the host; device-side faults (symbol range, timeout) are
 * reported by wt_wait.  S must stay valid until the build completes.
 * variant is a wt_variant.  Host symbols are copied to the device first: with
 * the default allocator and a stream that is not being captured, the copy
 * runs on a library-owned stream of the device and `stream` waits for it, so
 * the copy of one call overlaps the builds enqueued before it; otherwise the
 * copy is enqueued on `stream`.
 */
wt_handle wt_build_async(const void *S, uint64_t n, uint64_t sigma, int sym_width, int variant,
                         void *stream);

/*
 * Builds the wavelet matrix of S[0..n) (the level-wise variant Section 5
 * names for future work, as defined by Claude and Navarro 2012): level l
 * holds bit L-1-l of every symbol of S_l, where S_0 = S and S_{l+1} is all
 * of S_l stably partitioned by that bit, zeros first (one node per level).
 * Levels use the layout above (bitmap, R, Hy, S1, S0, ones; Z_l = n - ones
 * of level l).  Arguments, ownership, errors and staging of host symbols as
 * wt_build_async.  wt_access, wt_rank and wt_select answer on the matrix
 * (same conventions and sentinels as on a tree); wt_query_multi and
 * wt_merge_async reject matrices with WT_ERR_ARG.  wt_info reports layout
 * WT_LAYOUT_MATRIX.
 */
wt_handle wt_build_matrix_async(const void *S, uint64_t n, uint64_t sigma, int sym_width, void *stream);

/*
 * The tree of S[0..n) over a non-contiguous alphabet (Section 3: the
 * construction takes the codes of Sigma contiguous; when they are not, a
 * bitmap remaps the sequence to a contiguous alphabet).  Codes are in
 * [0, universe) (universe <= 2^(8 sym_width), else WT_ERR_ARG); the alphabet
 * bitmap A over [0, universe) marks the codes that occur, sigma' = their
 * number, and the tree is built over S'[j] = rank1(A, S[j]) in [0, sigma')
 * with 1, 2 or 4 bytes per code as sigma' needs (wt_info reports sigma =
 * sigma' and the universe).  wt_access returns the original codes;
 * wt_rank and wt_select take original codes: a code < universe that does
 * not occur has rank 0 (i <= n) and no select (UINT64_MAX); a code >=
 * universe gives UINT64_MAX.  wt_level_view shows the levels of the tree of
 * S'; wt_alphabet_view shows A (layout and directory of a level of
 * `universe` bits).  wt_query_multi and wt_merge_async reject such trees.
 * S may be host or device memory.  The call waits once on stream, after A is
 * counted, to size the tree; the build itself is then enqueued on stream and
 * wt_wait completes it.  A symbol >= universe gives WT_ERR_SYMBOL_RANGE (and
 * NULL) from this call.  Device memory: A with its directory (about
 * universe / 7 bytes) for the life of the tree, plus n (sym_width + 1..4)
 * bytes during the build.
 */
wt_handle wt_build_remap(const void *S, uint64_t n, uint64_t universe, int sym_width, void *stream);

/* Waits for a handle's build to finish and returns its device-reported status. */
wt_status wt_wait(wt_handle h);

/*
 * Builds count trees in one batch (the sequences may differ in n, sigma and
 * width): one launch computes every sequence's histogram, a few launches
 * its node starts and node tables, then one launch per (symbol width, level)
 * runs the level pass of Algorithm 1's levels over every sequence that has
 * that level.  On a non-default stream the launches are captured into one
 * CUDA graph and launched together.  The trees share one device block,
 * released when the last of them is freed.  S[k] are device pointers
 * (n[k] < 2^40); count < 2^27.  Any argument error builds nothing: every
 * out[k] is NULL and the error is returned.  Asynchronous on stream; wt_wait on a handle
 * returns that sequence's status (a device-side give-up anywhere in the
 * batch is reported by every handle).
 */
wt_status wt_build_batch(const void *const *S, const uint64_t *n, const uint64_t *sigma,
                         const int *sym_width, uint32_t count, wt_handle *out, void *stream);

/*
 * Merge of partial trees (the buffered build of Section 5, finished with
 * Algorithm 2's global offsets and Function mergeBA, Section 3.2): returns
 * the tree of the concatenation S_0 S_1 ... S_{k-1} of the parts' sequences,
 * in the order of parts[0..k).  parts is a host array of k handles (1 <= k
 * <= 65536) with the same sigma and sym_width and a total length below
 * 2^56; anything else gives WT_ERR_ARG.  The call first waits on the host
 * for every part's build and fails with the first part's error status, if
 * any; then it enqueues the merge on stream and returns (wt_wait completes
 * it).  The parts stay owned by the caller and must stay resident until the
 * merge has completed: free them after wt_wait on the result, or free them
 * in order on the merge's stream.  The trees keep no node offsets
 * (Section 2.2), so each part's node starts are recovered from its bitmaps
 * by rank; parts whose bitmaps and directories are inconsistent give
 * WT_ERR_ARG from wt_wait.  Device scratch: k (2^L + 1) node starts of 8
 * bytes plus the directory scan's per-unit counts.  The result's layout is
 * the one above, bit for bit the tree a single build of the concatenation
 * gives.
 */
wt_handle wt_merge_async(const wt_handle *parts, uint32_t k, void *stream);

/*
 * Buffered build (Section 5): builds S[0..n) in chunks of at most `chunk`
 * symbols, each chunk's tree built alone (as wt_build_async), then merges
 * them (as wt_merge_async); the partial trees are freed in stream order
 * after the merge.  At most two chunks' builds are in flight, so a host S is
 * staged on the device at most two chunks at a time and the level-wise
 * scratch is that of one chunk; the partial trees together take about the
 * size of the final tree.  Arguments as wt_build_async, plus chunk >= 1 and
 * ceil(n / chunk) <= 65536 (else WT_ERR_ARG).  Waits on the host for the
 * chunks' builds and returns with the merge enqueued on stream (wt_wait
 * completes it); a failed chunk (for example WT_ERR_SYMBOL_RANGE) fails the
 * call.  S must stay valid until the call returns.
 */
wt_handle wt_build_chunked(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t chunk,
                           void *stream);

/*
 * access(i) for m device positions i[k] -> out[k] (device, uint32): the
 * top-down walk of Section 2.2 (the worked example access(S, 24) = 't',
 * Fig. 3), simulated on the pointerless levels with rank (Section 2.2, after
 * Claude and Navarro 2008).  i[k] >= n gives UINT32_MAX.  Asynchronous on
 * stream; the caller owns i and out.
 */
wt_status wt_access(wt_handle h, const uint64_t *i, uint64_t m, uint32_t *out, void *stream);

/* rank_c(i) = occurrences of c[k] in [0, i[k]) -> out[k] (device arrays),
 * the operation rank_c(S, i) of Section 2.2 (read as half-open; the paper's
 * inclusive rank on 0-based i is rank_c(i + 1)), by the same walk with the
 * bits of c.  c >= sigma or i > n gives UINT64_MAX.  Asynchronous on stream. */
wt_status wt_rank(wt_handle h, const uint32_t *c, const uint64_t *i, uint64_t m, uint64_t *out,
                  void *stream);

/* select_c(j) = 0-based position of the j[k]-th occurrence of c[k] -> out[k]
 * (device arrays), the operation select_c(S, j) of Section 2.2 (j is
 * 1-based: the j-th appearance), by a descent to c's leaf and an ascent with
 * select on each level's bitmap.  c >= sigma, j == 0 or j > count gives
 * UINT64_MAX.  Asynchronous on stream. */
wt_status wt_select(wt_handle h, const uint32_t *c, const uint64_t *j, uint64_t m, uint64_t *out,
                    void *stream);

/*
 * Mixed queries over several resident trees (the serving path): query k runs
 * op[k] (a wt_op) on trees[tree_idx[k]] with symbol c[k] and argument arg[k]
 * (i for access and rank, j for select); out[k] is the answer widened to
 * uint64 (access sentinel UINT32_MAX becomes UINT64_MAX).  The operations
 * are those of Section 2.2 as for wt_access, wt_rank and wt_select; the
 * paper batches no queries, this call is the serving pattern's.  trees is a
 * host array of ntrees handles (ntrees bounds tree_idx: an index >= ntrees
 * gives UINT64_MAX); the other arrays are device arrays of length m.
 */
wt_status wt_query_multi(const wt_handle *trees, uint32_t ntrees, const uint32_t *tree_idx,
                         const uint8_t *op, const uint32_t *c, const uint64_t *arg, uint64_t m,
                         uint64_t *out, void *stream);

/* Releases a handle (the tree of Section 2.2 and its directories).  The
 * device memory is freed in stream order on the stream the tree was built
 * on, without a host wait; work on other streams that still reads the tree
 * must be complete (or ordered before) first.  NULL gives WT_ERR_ARG. */
wt_status wt_free(wt_handle h);

typedef struct {
    uint64_t n;
    uint64_t sigma;
    uint32_t levels;      /* L */
    int32_t sym_width;
    int32_t variant;      /* the wt_variant that built it */
    int32_t layout;       /* wt_layout: a wavelet tree or a wavelet matrix */
    uint64_t device_bytes; /* resident bytes of the tree (with its alphabet bitmap, if any) */
    uint64_t universe;    /* wt_build_remap: the code universe U (sigma is then the alphabet's size); else 0 */
} wt_info_t;

/* Shape of a built tree (n, sigma, L = ceil(lg sigma) levels of Section
 * 2.2, the variant and layout that built it, its resident bytes); waits for
 * the build.  Returns the build's status. */
wt_status wt_info(wt_handle h, wt_info_t *out);

typedef struct {
    const uint32_t *words;  /* device */
    const uint32_t *R;      /* device */
    const uint64_t *Hy;     /* device */
    const uint32_t *S1;     /* device */
    const uint32_t *S0;     /* device */
    uint64_t ones;
    uint64_t n_words, n_R, n_Hy, n_S1, n_S0;
} wt_level_view_t;

/* Device pointers and sizes of level l (layout above); waits for the build.
 * The pointers stay valid until wt_free. */
wt_status wt_level_view(wt_handle h, uint32_t l, wt_level_view_t *out);

/* The alphabet bitmap of a tree built by wt_build_remap (layout of a level
 * of `universe` bits: words, R, Hy, S1, S0, ones = sigma'); WT_ERR_ARG for
 * other trees.  Waits for the build; pointers valid until wt_free. */
wt_status wt_alphabet_view(wt_handle h, wt_level_view_t *out);

/*
 * Routes every device allocation of the library through alloc/free_ (for
 * example a framework's caching allocator).  alloc(bytes, stream, ctx) must
 * return device memory usable in stream order on stream (or NULL);
 * free_(ptr, bytes, stream, ctx) releases it in stream order.  Passing NULL
 * for both restores cudaMallocAsync / cudaFreeAsync.
 */
wt_status wt_set_allocator(void *(*alloc)(size_t bytes, void *stream, void *ctx),
                           void (*free_)(void *ptr, size_t bytes, void *stream, void *ctx), void *ctx);

/* Last status set by a call of this thread. */
wt_status wt_last_status(void);

/* Static text for a status. */
const char *wt_status_string(wt_status s);

/*
 * Stage entry points: one step of the build each, for tests and tooling.
 *
 * wt_node_starts (Algorithm 1 "count" and parPrefixSum, read as exclusive):
 * Hex[c] = number of symbols < c, for c = 0 .. 2^L (entries at c >= sigma
 * equal n), written to the device array Hex (2^L + 1 uint64).  The start of
 * node v on level l is Hex[v << (L - l)].  S is a device pointer.  Returns
 * WT_ERR_SYMBOL_RANGE (after a stream synchronisation) if a symbol is out of
 * range.
 */
wt_status wt_node_starts(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t *Hex,
                         void *stream);

/*
 * wt_level_step (the bit pass of Algorithm 1 for one level, plus the stable
 * placement that yields the next level's order): given cur = P_l (the
 * level-l order, device, n symbols) and Hex from wt_node_starts, writes the
 * level-l bitmap to words (device, ceil(n/512) * 16 uint32), its block
 * directory to R (device, ceil(n/512) + 1 uint32) and, when nxt is not NULL
 * and l < L - 1, the order P_{l+1} to nxt (device, n symbols).  Synchronous
 * (it waits for its stream).
 */
wt_status wt_level_step(const void *cur, uint64_t n, uint64_t sigma, int sym_width, uint32_t l,
                        const uint64_t *Hex, uint32_t *words, uint32_t *R, void *nxt, void *stream);

/*
 * wt_node_starts_noalloc: the same result as wt_node_starts (Hex, 2^L + 1
 * uint64 node starts written to the device array Hex) for callers that may
 * not allocate device memory while they run -- for example a process that
 * gives the whole device to its own memory pool at start-up, or a loop that
 * must not take the allocator's locks or the synchronisation a free can
 * bring.  The paper has no counterpart; it is a deployment variant.
 *
 * It allocates nothing: its scratch (the per-code counts and an error word)
 * is one fixed array of about 0.5 MB compiled into the library, present on
 * every GPU that loads the library until the process exits.  Limits and
 * behaviour:
 *   - sigma must be at most 65536 (2^16); larger alphabets give WT_ERR_ARG
 *     (use wt_node_starts for them).  S and Hex must be device memory of the
 *     current device (else WT_ERR_ARG); the other argument rules are
 *     wt_build's (a misaligned S gives WT_ERR_ARG before any launch).
 *   - The array's address is cached per device for the life of the
 *     process; after cudaDeviceReset on a device, do not call this entry
 *     point on that device again.
 *   - The first call on a device looks up the array's device address on
 *     that device (with it current); make that first call before any stream
 *     capture.
 *   - Every call shares the one array and clears the part it uses before
 *     use; calls that overlap on the GPU (concurrent streams, threads or
 *     devices sharing a context) race on it and must be serialised by the
 *     caller.
 *   - Synchronous: returns after its stream has finished, with
 *     WT_ERR_SYMBOL_RANGE if some symbol is >= sigma.
 */
wt_status wt_node_starts_noalloc(const void *S, uint64_t n, uint64_t sigma, int sym_width, uint64_t *Hex,
                                 void *stream);

/*
 * Failure detection self test (no counterpart in the paper).  Every wait of
 * the library's kernels is bounded: after its limit the kernel sets a
 * give-up bit in an error word and returns, and the host turns that into
 * WT_ERR_TIMEOUT with the CUDA context still usable.  This call runs that
 * wait on an mbarrier in one thread for at most limit_ns (1 ns .. 1 s, else
 * WT_ERR_ARG): with arrive == 0 nothing completes the barrier, so the wait
 * runs out and the call returns WT_ERR_TIMEOUT; with arrive != 0 the thread
 * arrives first and the call returns WT_OK.  err_word is one device uint32
 * the caller owns (overwritten).  Synchronous on stream.
 */
wt_status wt_wait_selftest(uint64_t limit_ns, int arrive, uint32_t *err_word, void *stream);

/*
 * Per-kernel timing (no counterpart in the paper; it times the hot path).
 * Between wt_profile_begin and wt_profile_end the library's kernel
 * launches are bracketed by CUDA events on the stream they run on.
 * wt_profile_end waits for those events and writes one record per kernel
 * that ran (up to cap records to out; *count receives how many kernels
 * ran): launches (the library calls timed; the level steps of one
 * level-wise build are timed together under one pair of events, so that no
 * event separates them in the stream, and count one launch per level step),
 * the CUDA kernels those calls launched, summed device time and two summed
 * byte counts.  alg_bytes is the
 * level-wise method's byte model of the work the launch covers (per level:
 * symbols read, bitmap and directory written, next-level order written; a
 * step covering two levels counts both).  variant_bytes is what the
 * launch's own variant must move (a two-level step reads the symbols once
 * and writes the order two levels down).
 */
typedef struct {
    char name[24];
    uint64_t launches;
    uint64_t kernels;
    double total_ms;
    double alg_bytes;
    double variant_bytes;
} wt_kernel_stat_t;

wt_status wt_profile_begin(void);
wt_status wt_profile_end(wt_kernel_stat_t *out, uint32_t cap, uint32_t *count);

#ifdef __cplusplus
}
#endif

#endif /* WT_H */
