/*
 * wt_oracle.c -- plain, single-threaded CPU oracle for the pointerless,
 * level-wise wavelet tree studied in "Parallel Construction of Wavelet Trees
 * on Multicore Architectures" (Fuentes-Sepulveda, Elejalde, Ferres, Seco;
 * arXiv 1610.05994).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path.  Everything here is written for a reader checking it against the
 * paper by eye, not for speed.
 *
 * What it computes (Section 2.2, Section 3, Proposition 1, Algorithm 1):
 *   L = ceil(lg sigma) levels (L = 0 when sigma = 1).  Symbols are codes in
 *   [0, sigma).  P_0 = S.  P_{l+1} is P_l with every level-l node (a maximal
 *   run of equal key s >> (L-l), Proposition 1) stably partitioned by the
 *   level-l bit (s >> (L-1-l)) & 1: zeros first, then ones, original order
 *   kept inside each group, nodes kept in increasing key order.  The level-l
 *   bitmap is B_l[p] = (P_l[p] >> (L-1-l)) & 1.  This is the one-pointer-per-
 *   level representation of Section 2.2 (Fig. 2b).
 *
 * Readings of the paper used here (each is also listed in the design notes):
 *   R1 alphabet is [0, sigma) (the worked example in Section 2.2 and
 *      Proposition 1 use 0-based codes; the opening of Section 2.2 writes
 *      [1..sigma]).
 *   R2 nodes split on bits of the code over [0, 2^L), so for sigma not a
 *      power of two some nodes are empty (Proposition 1 and Algorithm 1
 *      split on bits; "first half / second half" in Section 2.2 is read as
 *      the bit split).
 *   R3 the bit test of Algorithm 1 and Function createPartialBA,
 *      "(S[j] & 2^{L-i-1}) == 1", is read as "!= 0" (as printed it is true
 *      only on the last level).
 *   R4 parPrefixSum in Algorithm 1 is an exclusive scan (it yields each
 *      node's starting offset).
 *   R5 rank_c(S, i) counts c in the half-open prefix [0, i); the worked
 *      example's inclusive "rank(B, i) - 1" on 0-based i equals the
 *      half-open rank(i + 1) - 1.  select_c(S, j) is 1-based in j.
 *   R6 out-of-range query arguments give the sentinel UINT64_MAX
 *      (UINT32_MAX for access); the paper does not say.
 *   R7 the serialised layout (bit order, padding, rank/select directory) is
 *      not given by the paper; the one fixed here is documented at
 *      wto_directory().
 *   R8 in Function mergeBA the loop "m = j 2^i to (j+1) 2^i" is read with an
 *      exclusive upper bound, "dest" and "dst" are one variable, m / k is the
 *      node and m mod k the segment; in createPartialBA "n" is the segment
 *      length.
 *   R9 in the buffered extension of Section 5 the per-buffer array L of node
 *      starts is taken as the part's leaf-level node starts Hex (2^L + 1
 *      entries), from which node v of level i starts at Hex[v << (L - i)];
 *      the parts may have any lengths, and the result is the tree of their
 *      concatenation in part order.
 *   R10 the wavelet matrix (named in Section 5, defined by Claude and
 *      Navarro 2012) takes level l to hold bit L-1-l, most significant
 *      first like the tree, with zeros first on the next level, and the
 *      tree's bitmap layout and directory; sigma = 1 gives no levels.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WTO_OK 0
#define WTO_ERR_ARG 1
#define WTO_ERR_SYMBOL 2
#define WTO_ERR_NOMEM 3

#define WTO_BLOCK_BITS 512u           /* rank block: 512 bits = 64 bytes    */
#define WTO_SPAN_BITS (1ull << 32)    /* hyper span for 64-bit rank values */
#define WTO_SAMPLE 8192u              /* select sample rate                 */

/* ---------------------------------------------------------------- helpers */

/* L = ceil(lg sigma); 0 for sigma <= 1 (Section 2.2: ceil(lg sigma) levels). */
uint32_t wto_levels(uint64_t sigma)
{
    uint32_t L = 0;
    while (L < 64 && (1ull << L) < sigma) L++;
    return L;
}

/* Bytes of one padded level bitmap: n bits rounded up to whole 512-bit blocks. */
uint64_t wto_level_bytes(uint64_t n)
{
    return ((n + WTO_BLOCK_BITS - 1) / WTO_BLOCK_BITS) * (WTO_BLOCK_BITS / 8);
}

static uint32_t sym_at(const void *S, int w, uint64_t j)
{
    if (w == 1) return ((const uint8_t *)S)[j];
    if (w == 2) return ((const uint16_t *)S)[j];
    return ((const uint32_t *)S)[j];
}

static int bit_get(const uint8_t *B, uint64_t p) { return (B[p >> 3] >> (p & 7)) & 1; }

static void bit_put(uint8_t *B, uint64_t p, int b)
{
    if (b) B[p >> 3] |= (uint8_t)(1u << (p & 7));
    else B[p >> 3] &= (uint8_t)~(1u << (p & 7));
}

/* Copies S into 32-bit codes and checks every code is below sigma. */
static int load_codes(const void *S, uint64_t n, int w, uint64_t sigma, uint32_t **out)
{
    if (w != 1 && w != 2 && w != 4) return WTO_ERR_ARG;
    if (sigma < 1 || sigma > (1ull << (8 * w))) return WTO_ERR_ARG;
    uint32_t *x = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!x) return WTO_ERR_NOMEM;
    for (uint64_t j = 0; j < n; j++) {
        x[j] = sym_at(S, w, j);
        if ((uint64_t)x[j] >= sigma) { free(x); return WTO_ERR_SYMBOL; }
    }
    *out = x;
    return WTO_OK;
}

/* Node of symbol s at level l (Proposition 1): its top l bits, s >> (L - l). */
static uint64_t node_of(uint32_t s, uint32_t L, uint32_t l)
{
    return (L - l >= 32) ? 0 : (uint64_t)(s >> (L - l));
}

/* Level-l bit of s: bit L-1-l, the most significant bit first. */
static int level_bit(uint32_t s, uint32_t L, uint32_t l) { return (s >> (L - 1 - l)) & 1; }

/*
 * One level step of the definition: stably partition every node of cur by the
 * level-l bit into nxt.  Nodes are the maximal runs of equal key in cur (cur
 * is P_l, so each node's symbols are contiguous and in increasing key order).
 */
static void partition_level(const uint32_t *cur, uint32_t *nxt, uint64_t n, uint32_t L, uint32_t l)
{
    uint64_t start = 0;
    while (start < n) {
        uint64_t v = node_of(cur[start], L, l);
        uint64_t end = start;
        while (end < n && node_of(cur[end], L, l) == v) end++;
        uint64_t out = start;
        for (uint64_t p = start; p < end; p++)          /* zeros, in order */
            if (level_bit(cur[p], L, l) == 0) nxt[out++] = cur[p];
        for (uint64_t p = start; p < end; p++)          /* then ones       */
            if (level_bit(cur[p], L, l) == 1) nxt[out++] = cur[p];
        start = end;
    }
}

/* ------------------------------------------------------ construction */

/*
 * P_l: the order of the symbols on level l (Section 2.2, Fig. 2b), produced
 * by l partition steps starting from P_0 = S.  out holds n codes.
 */
int wto_level_order(const void *S, uint64_t n, int w, uint64_t sigma, uint32_t l, uint32_t *out)
{
    uint32_t *cur = NULL;
    int st = load_codes(S, n, w, sigma, &cur);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    if (l > L) { free(cur); return WTO_ERR_ARG; }
    uint32_t *nxt = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!nxt) { free(cur); return WTO_ERR_NOMEM; }
    for (uint32_t k = 0; k < l; k++) {
        partition_level(cur, nxt, n, L, k);
        uint32_t *t = cur; cur = nxt; nxt = t;
    }
    memcpy(out, cur, n * sizeof(uint32_t));
    free(cur);
    free(nxt);
    return WTO_OK;
}

/*
 * The tree's level bitmaps: L bitmaps, each wto_level_bytes(n) bytes, bit p of
 * level l at byte p >> 3, bit p & 7 (least significant bit first), padding
 * bits zero.  bits must hold L * wto_level_bytes(n) bytes.
 */
int wto_build_bits(const void *S, uint64_t n, int w, uint64_t sigma, uint8_t *bits)
{
    uint32_t *cur = NULL;
    int st = load_codes(S, n, w, sigma, &cur);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    uint64_t lb = wto_level_bytes(n);
    memset(bits, 0, L * lb);
    uint32_t *nxt = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!nxt) { free(cur); return WTO_ERR_NOMEM; }
    for (uint32_t l = 0; l < L; l++) {
        uint8_t *B = bits + l * lb;
        for (uint64_t p = 0; p < n; p++) bit_put(B, p, level_bit(cur[p], L, l));
        if (l + 1 < L) {
            partition_level(cur, nxt, n, L, l);
            uint32_t *t = cur; cur = nxt; nxt = t;
        }
    }
    free(cur);
    free(nxt);
    return WTO_OK;
}

/*
 * Node starts of every level at once: Hex[c] = number of symbols of S below
 * c, for c = 0 .. 2^L (Algorithm 1's "count" step done once on the leaves,
 * then its prefix sum, read as exclusive).  Node v of level l starts at
 * Hex[v << (L - l)] because the node holds exactly the codes
 * [v << (L - l), (v + 1) << (L - l)) (Proposition 1).  out holds 2^L + 1.
 */
int wto_node_starts(const void *S, uint64_t n, int w, uint64_t sigma, uint64_t *out)
{
    uint32_t *x = NULL;
    int st = load_codes(S, n, w, sigma, &x);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    uint64_t leaves = 1ull << L;
    uint64_t *H = (uint64_t *)calloc(leaves, sizeof(uint64_t));
    if (!H) { free(x); return WTO_ERR_NOMEM; }
    for (uint64_t j = 0; j < n; j++) H[x[j]]++;
    uint64_t run = 0;
    for (uint64_t c = 0; c < leaves; c++) { out[c] = run; run += H[c]; }
    out[leaves] = run;
    free(H);
    free(x);
    return WTO_OK;
}

/*
 * Algorithm 1 (pwt) taken literally, run sequentially: for each level i,
 * count the symbols of every node (lines 5-6), take the exclusive prefix sum
 * as node offsets (line 7, reading R4), then scan S once more and set the bit
 * of each symbol at its node's running offset (lines 8-13, reading R3).  It
 * never materialises P_l; the tests use it as a second, independent route to
 * the same bitmaps.
 */
/* One level i of Algorithm 1 over the codes x: counts per node, their
 * exclusive prefix sum, then each symbol's bit at its node's running offset.
 * B (wto_level_bytes(n) bytes) must be zero. */
static int pwt_level(const uint32_t *x, uint64_t n, uint32_t L, uint32_t i, uint8_t *B)
{
    uint64_t nodes = 1ull << i;
    uint64_t *C = (uint64_t *)calloc(nodes, sizeof(uint64_t));
    if (!C) return WTO_ERR_NOMEM;
    for (uint64_t j = 0; j < n; j++) C[node_of(x[j], L, i)]++;
    uint64_t run = 0;                                   /* exclusive prefix sum */
    for (uint64_t v = 0; v < nodes; v++) { uint64_t c = C[v]; C[v] = run; run += c; }
    for (uint64_t j = 0; j < n; j++) {
        uint64_t v = node_of(x[j], L, i);
        bit_put(B, C[v], (x[j] & (1u << (L - i - 1))) != 0);
        C[v]++;
    }
    free(C);
    return WTO_OK;
}

int wto_pwt(const void *S, uint64_t n, int w, uint64_t sigma, uint8_t *bits)
{
    uint32_t *x = NULL;
    int st = load_codes(S, n, w, sigma, &x);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    uint64_t lb = wto_level_bytes(n);
    memset(bits, 0, L * lb);
    for (uint32_t i = 0; i < L && st == WTO_OK; i++) st = pwt_level(x, n, L, i, bits + i * lb);
    free(x);
    return st;
}

/*
 * Level i alone by Algorithm 1 (its per-level body; in Algorithm 1 the
 * levels are independent, which is what pwt parallelises over): B receives
 * wto_level_bytes(n) bytes.  Used to check very long sequences level by
 * level on several host cores.
 */
int wto_pwt_level(const void *S, uint64_t n, int w, uint64_t sigma, uint32_t i, uint8_t *B)
{
    uint32_t L = wto_levels(sigma);
    if (i >= L) return WTO_ERR_ARG;
    uint32_t *x = NULL;
    int st = load_codes(S, n, w, sigma, &x);
    if (st) return st;
    memset(B, 0, wto_level_bytes(n));
    st = pwt_level(x, n, L, i, B);
    free(x);
    return st;
}

/*
 * Algorithm 2 (dd) with k segments, run sequentially: Function createPartialBA
 * builds a partial bitmap per (segment, level) with local node offsets L
 * (exclusive prefix, plus a sentinel equal to the segment length); the
 * per-level prefix sum over the k local offsets gives global offsets G in
 * node-major, segment-minor order; Function mergeBA copies every
 * (segment, node) bit run from its local offset to its global offset
 * (reading R8).  A second independent route to the same bitmaps.
 */
int wto_dd(const void *S, uint64_t n, int w, uint64_t sigma, uint32_t k, uint8_t *bits)
{
    if (k == 0) return WTO_ERR_ARG;
    uint32_t *x = NULL;
    int st = load_codes(S, n, w, sigma, &x);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    uint64_t lb = wto_level_bytes(n);
    memset(bits, 0, L * lb);
    uint64_t seg = (n + k - 1) / k;
    for (uint32_t i = 0; i < L; i++) {
        uint64_t nodes = 1ull << i;
        /* Lo[a][v] local offsets with sentinel, G[a][v] global offsets. */
        uint64_t *Lo = (uint64_t *)calloc((uint64_t)k * (nodes + 1), sizeof(uint64_t));
        uint64_t *G = (uint64_t *)calloc((uint64_t)k * nodes, sizeof(uint64_t));
        uint8_t *pB = (uint8_t *)calloc((uint64_t)k * wto_level_bytes(seg) + 1, 1);
        if (!Lo || !G || !pB) { free(Lo); free(G); free(pB); free(x); return WTO_ERR_NOMEM; }
        /* createPartialBA for every segment a. */
        for (uint32_t a = 0; a < k; a++) {
            uint64_t lo = a * seg < n ? a * seg : n;
            uint64_t hi = (a + 1) * seg < n ? (a + 1) * seg : n;
            uint64_t *La = Lo + (uint64_t)a * (nodes + 1);
            uint64_t *cnt = (uint64_t *)calloc(nodes, sizeof(uint64_t));
            if (!cnt) { free(Lo); free(G); free(pB); free(x); return WTO_ERR_NOMEM; }
            for (uint64_t j = lo; j < hi; j++) cnt[node_of(x[j], L, i)]++;
            uint64_t run = 0;
            for (uint64_t v = 0; v < nodes; v++) { La[v] = run; run += cnt[v]; }
            La[nodes] = hi - lo;
            uint8_t *Ba = pB + (uint64_t)a * wto_level_bytes(seg);
            for (uint64_t v = 0; v < nodes; v++) cnt[v] = La[v];
            for (uint64_t j = lo; j < hi; j++) {
                uint64_t v = node_of(x[j], L, i);
                bit_put(Ba, cnt[v], (x[j] & (1u << (L - i - 1))) != 0);
                cnt[v]++;
            }
            free(cnt);
        }
        /* parPrefixSum over the k local offsets: node-major, segment-minor. */
        uint64_t run = 0;
        for (uint64_t v = 0; v < nodes; v++)
            for (uint32_t a = 0; a < k; a++) {
                uint64_t *La = Lo + (uint64_t)a * (nodes + 1);
                G[(uint64_t)a * nodes + v] = run;
                run += La[v + 1] - La[v];
            }
        /* mergeBA: copy nb bits of (segment m mod k, node m / k). */
        uint8_t *B = bits + i * lb;
        for (uint64_t m = 0; m < (uint64_t)k * nodes; m++) {
            uint32_t a = (uint32_t)(m % k);
            uint64_t v = m / k;
            uint64_t *La = Lo + (uint64_t)a * (nodes + 1);
            uint8_t *src = pB + (uint64_t)a * wto_level_bytes(seg);
            uint64_t go = G[(uint64_t)a * nodes + v], lo = La[v], nb = La[v + 1] - La[v];
            for (uint64_t t = 0; t < nb; t++) bit_put(B, go + t, bit_get(src, lo + t));
        }
        free(Lo);
        free(G);
        free(pB);
    }
    free(x);
    return WTO_OK;
}

/*
 * The merge of partial trees, run sequentially: the extension of Section 5
 * (read S in buffers, build a partial tree per buffer, keep each one's node
 * starts, then merge), whose last two steps are those of Algorithm 2.
 * Inputs: k parts, part a with part_n[a] symbols, its level bitmaps
 * part_bits[a] (L padded levels, the layout of wto_build_bits) and its node
 * starts part_hex[a] (the local offsets: 2^L + 1 entries, as wto_node_starts;
 * node v of level i starts at part_hex[a][v << (L - i)]).  For each level i:
 * the prefix sum over the nodes' sizes, node-major and part-minor (the
 * order of Algorithm 2's global offsets), gives each (part, node) run its
 * offset in the result; Function mergeBA then copies the run's bits there
 * (reading R8).  The result is the tree of the concatenation S_0 S_1 ...
 * S_{k-1}: n = the sum of part_n bits per level.
 */
int wto_merge(const uint8_t *const *part_bits, const uint64_t *part_n, const uint64_t *const *part_hex,
              uint32_t k, uint64_t sigma, uint8_t *bits)
{
    if (k == 0 || sigma < 1) return WTO_ERR_ARG;
    uint32_t L = wto_levels(sigma);
    uint64_t n = 0;
    for (uint32_t a = 0; a < k; a++) {
        if (part_hex[a][0] != 0 || part_hex[a][1ull << L] != part_n[a]) return WTO_ERR_ARG;
        n += part_n[a];
    }
    uint64_t lb = wto_level_bytes(n);
    memset(bits, 0, L * lb);
    for (uint32_t i = 0; i < L; i++) {
        uint64_t nodes = 1ull << i, sh = L - i;
        uint8_t *B = bits + i * lb;
        uint64_t go = 0;  /* the running global offset */
        for (uint64_t v = 0; v < nodes; v++)
            for (uint32_t a = 0; a < k; a++) {
                const uint8_t *src = part_bits[a] + i * wto_level_bytes(part_n[a]);
                uint64_t lo = part_hex[a][v << sh], nb = part_hex[a][(v + 1) << sh] - lo;
                for (uint64_t t = 0; t < nb; t++) bit_put(B, go + t, bit_get(src, lo + t));
                go += nb;
            }
    }
    return WTO_OK;
}

/* ------------------------------------------------------ directories */

/*
 * Rank/select directory of one level bitmap (reading R7; the paper uses the
 * 5%-extra structure of Gonzalez et al. [GGMN05], Section 4, without fixing a
 * layout).  Every entry is a pure function of the bits:
 *   R[b]  = (ones in B[0, 512 b)) mod 2^32,          b = 0 .. ceil(n/512)
 *   Hy[h] = ones in B[0, min(n, 2^32 h)),            h = 0 .. ceil(n/2^32)
 *   S1[k] = (position of the one of 0-based rank 8192 k) >> 9,
 *                                                    k = 0 .. ceil(ones/8192)-1
 *   S0[k] = the same for zeros at positions < n
 *   ones  = ones in B[0, n)
 * Arrays must be sized by the caller; counts of S1/S0 entries are returned.
 */
int wto_directory(const uint8_t *B, uint64_t n, uint32_t *R, uint64_t *Hy, uint32_t *S1,
                  uint32_t *S0, uint64_t *ones_out, uint64_t *n1_out, uint64_t *n0_out)
{
    uint64_t nb = (n + WTO_BLOCK_BITS - 1) / WTO_BLOCK_BITS;
    uint64_t nh = (n + WTO_SPAN_BITS - 1) / WTO_SPAN_BITS;
    uint64_t ones = 0, zeros = 0, n1 = 0, n0 = 0;
    for (uint64_t p = 0; p <= n; p++) {
        if (p % WTO_BLOCK_BITS == 0 && p / WTO_BLOCK_BITS <= nb) R[p / WTO_BLOCK_BITS] = (uint32_t)ones;
        if (p % WTO_SPAN_BITS == 0 && p / WTO_SPAN_BITS <= nh) Hy[p / WTO_SPAN_BITS] = ones;
        if (p == n) break;
        if (bit_get(B, p)) {
            if (ones % WTO_SAMPLE == 0) S1[n1++] = (uint32_t)(p >> 9);
            ones++;
        } else {
            if (zeros % WTO_SAMPLE == 0) S0[n0++] = (uint32_t)(p >> 9);
            zeros++;
        }
    }
    /* Entries whose boundary lies beyond n (the last block or span) hold the total. */
    R[nb] = (uint32_t)ones;
    Hy[nh] = ones;
    *ones_out = ones;
    *n1_out = n1;
    *n0_out = n0;
    return WTO_OK;
}

/* ------------------------------------------------------ queries */

/*
 * Queries on the level bitmaps by the pointerless traversal of Section 2.2
 * (the tree walk simulated with rank on each level's bitmap, [Claude and
 * Navarro 2008]).  The oracle ranks by per-level prefix counts built here by
 * a direct loop, never through the directory it also emits.
 */
typedef struct {
    uint64_t n;
    uint32_t L;
    uint64_t **pre;     /* pre[l][p] = ones in B_l[0, p), p = 0..n */
    const uint8_t *bits;
    uint64_t lb;
} tree_t;

static void tree_free(tree_t *t)
{
    if (t->pre) {
        for (uint32_t l = 0; l < t->L; l++) free(t->pre[l]);
        free(t->pre);
    }
}

static int tree_init(tree_t *t, const uint8_t *bits, uint64_t n, uint32_t L)
{
    t->n = n; t->L = L; t->bits = bits; t->lb = wto_level_bytes(n);
    t->pre = (uint64_t **)calloc(L ? L : 1, sizeof(uint64_t *));
    if (!t->pre) return WTO_ERR_NOMEM;
    for (uint32_t l = 0; l < L; l++) {
        t->pre[l] = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
        if (!t->pre[l]) { tree_free(t); return WTO_ERR_NOMEM; }
        const uint8_t *B = bits + l * t->lb;
        t->pre[l][0] = 0;
        for (uint64_t p = 0; p < n; p++) t->pre[l][p + 1] = t->pre[l][p] + (uint64_t)bit_get(B, p);
    }
    return WTO_OK;
}

static uint64_t rank1(const tree_t *t, uint32_t l, uint64_t i) { return t->pre[l][i]; }
static uint64_t rank0(const tree_t *t, uint32_t l, uint64_t i) { return i - t->pre[l][i]; }
static uint64_t rankb(const tree_t *t, uint32_t l, int b, uint64_t i) { return b ? rank1(t, l, i) : rank0(t, l, i); }

/* Position of the k-th (1-based) bit equal to b on level l: smallest p with rank_b(p + 1) = k. */
static uint64_t selectb(const tree_t *t, uint32_t l, int b, uint64_t k)
{
    uint64_t lo = 0, hi = t->n;  /* answer in [lo, hi) */
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (rankb(t, l, b, mid + 1) >= k) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/*
 * access(i): start with the whole level range [b, e) = [0, n) and p = i; on
 * each level with z zeros in [b, e): a 0 bit maps p to b + (zeros before p
 * inside the node) and keeps the left child [b, b + z); a 1 bit maps p to
 * b + z + (ones before p inside the node) and keeps the right child
 * [b + z, e).  The bits read, most significant first, spell the symbol.
 */
int wto_access(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint64_t *I, uint64_t m, uint32_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t i = I[q];
        if (i >= n) { out[q] = UINT32_MAX; continue; }
        uint64_t b = 0, e = n, p = i;
        uint32_t sym = 0;
        for (uint32_t l = 0; l < L; l++) {
            uint64_t z = rank0(&t, l, e) - rank0(&t, l, b);
            int bit = bit_get(bits + l * t.lb, p);
            if (bit == 0) { p = b + rank0(&t, l, p) - rank0(&t, l, b); e = b + z; }
            else { p = b + z + rank1(&t, l, p) - rank1(&t, l, b); b = b + z; }
            sym = (sym << 1) | (uint32_t)bit;
        }
        out[q] = sym;
    }
    tree_free(&t);
    return WTO_OK;
}

/*
 * access(i) that also reports, after each level, the index of the walked
 * position inside the child node it moves to (p - b after the step).  The
 * worked example of Section 2.2 prints exactly these indices.
 */
int wto_access_trace(const uint8_t *bits, uint64_t n, uint64_t sigma, uint64_t i, uint64_t *trace, uint32_t *out)
{
    uint32_t L = wto_levels(sigma);
    if (i >= n) return WTO_ERR_ARG;
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    uint64_t b = 0, e = n, p = i;
    uint32_t sym = 0;
    for (uint32_t l = 0; l < L; l++) {
        uint64_t z = rank0(&t, l, e) - rank0(&t, l, b);
        int bit = bit_get(bits + l * t.lb, p);
        if (bit == 0) { p = b + rank0(&t, l, p) - rank0(&t, l, b); e = b + z; }
        else { p = b + z + rank1(&t, l, p) - rank1(&t, l, b); b = b + z; }
        sym = (sym << 1) | (uint32_t)bit;
        trace[l] = p - b;
    }
    *out = sym;
    tree_free(&t);
    return WTO_OK;
}

/* rank_c(i): the same walk steered by the bits of c; the answer is p - b at the leaf. */
int wto_rank(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint32_t *C, const uint64_t *I,
             uint64_t m, uint64_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t c = C[q], i = I[q];
        if (c >= sigma || i > n) { out[q] = UINT64_MAX; continue; }
        uint64_t b = 0, e = n, p = i;
        for (uint32_t l = 0; l < L; l++) {
            uint64_t z = rank0(&t, l, e) - rank0(&t, l, b);
            int bit = (int)((c >> (L - 1 - l)) & 1);
            if (bit == 0) { p = b + rank0(&t, l, p) - rank0(&t, l, b); e = b + z; }
            else { p = b + z + rank1(&t, l, p) - rank1(&t, l, b); b = b + z; }
        }
        out[q] = p - b;
    }
    tree_free(&t);
    return WTO_OK;
}

/*
 * select_c(j): walk down by the bits of c recording each level's node start
 * b_l; at the leaf the answer's position is b_L + j - 1 (if the leaf holds at
 * least j symbols); then climb: on level l the position pos in the child
 * (which starts at b_{l+1}) is the (pos - b_{l+1} + 1)-th bit equal to the
 * child's bit after b_l, so pos = select_bit(B_l, rank_bit(b_l) + pos - b_{l+1} + 1).
 */
int wto_select(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint32_t *C, const uint64_t *J,
               uint64_t m, uint64_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    uint64_t bs[66];
    for (uint64_t q = 0; q < m; q++) {
        uint64_t c = C[q], j = J[q];
        if (c >= sigma || j == 0) { out[q] = UINT64_MAX; continue; }
        uint64_t b = 0, e = n;
        for (uint32_t l = 0; l < L; l++) {
            bs[l] = b;
            uint64_t z = rank0(&t, l, e) - rank0(&t, l, b);
            int bit = (int)((c >> (L - 1 - l)) & 1);
            if (bit == 0) e = b + z; else b = b + z;
        }
        bs[L] = b;
        if (j > e - b) { out[q] = UINT64_MAX; continue; }
        uint64_t pos = b + j - 1;
        for (uint32_t l = L; l-- > 0;) {
            int bit = (int)((c >> (L - 1 - l)) & 1);
            pos = selectb(&t, l, bit, rankb(&t, l, bit, bs[l]) + (pos - bs[l + 1]) + 1);
        }
        out[q] = pos;
    }
    tree_free(&t);
    return WTO_OK;
}

/* ------------------------------------------------------ single samples */

/*
 * P_l[p] for one position p, straight from the definition without building
 * any level: count each level-l node's symbols, find the node v whose range
 * [C_l[v], C_l[v+1]) holds p, and return the (p - C_l[v])-th (0-based) symbol
 * of S, in S order, whose key is v (stable order inside a node, Algorithm 1).
 * Used to sample full-size results that are too large to build here.
 */
int wto_level_symbol(const void *S, uint64_t n, int w, uint64_t sigma, uint32_t l, uint64_t p, uint32_t *out)
{
    uint32_t L = wto_levels(sigma);
    if (w != 1 && w != 2 && w != 4) return WTO_ERR_ARG;
    if (l >= L || p >= n) return WTO_ERR_ARG;
    uint64_t nodes = 1ull << l;
    uint64_t *cnt = (uint64_t *)calloc(nodes, sizeof(uint64_t));
    if (!cnt) return WTO_ERR_NOMEM;
    for (uint64_t j = 0; j < n; j++) {
        uint32_t s = sym_at(S, w, j);
        if (s >= sigma) { free(cnt); return WTO_ERR_SYMBOL; }
        cnt[node_of(s, L, l)]++;
    }
    uint64_t start = 0, v = 0;
    while (start + cnt[v] <= p) { start += cnt[v]; v++; }
    uint64_t want = p - start, seen = 0;
    free(cnt);
    for (uint64_t j = 0; j < n; j++) {
        uint32_t s = sym_at(S, w, j);
        if (node_of(s, L, l) == v) {
            if (seen == want) { *out = s; return WTO_OK; }
            seen++;
        }
    }
    return WTO_ERR_ARG;
}

/* ------------------------------------------------------ wavelet matrix */

/*
 * The wavelet matrix, the level-wise variant Section 5 names for future work
 * (Claude and Navarro, SPIRE 2012), written from its definition: S_0 = S;
 * level l stores bit L-1-l of every symbol of S_l (the same bit as the
 * tree's level l); S_{l+1} is the whole of S_l stably partitioned by that
 * bit, zeros first (one node per level, where the tree partitions inside
 * each node).  Z_l = zeros of level l.  The bitmaps use the tree's padded
 * layout, so wto_directory applies unchanged (reading R10).
 */
int wto_wm_build(const void *S, uint64_t n, int w, uint64_t sigma, uint8_t *bits)
{
    uint32_t *x = NULL;
    int st = load_codes(S, n, w, sigma, &x);
    if (st) return st;
    uint32_t L = wto_levels(sigma);
    uint64_t lb = wto_level_bytes(n);
    memset(bits, 0, L * lb);
    uint32_t *nxt = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!nxt) { free(x); return WTO_ERR_NOMEM; }
    for (uint32_t l = 0; l < L; l++) {
        uint8_t *B = bits + l * lb;
        uint64_t k = 0;
        for (uint64_t p = 0; p < n; p++) bit_put(B, p, level_bit(x[p], L, l));
        for (uint64_t p = 0; p < n; p++) if (!level_bit(x[p], L, l)) nxt[k++] = x[p];
        for (uint64_t p = 0; p < n; p++) if (level_bit(x[p], L, l)) nxt[k++] = x[p];
        uint32_t *tmp = x; x = nxt; nxt = tmp;
    }
    free(x);
    free(nxt);
    return WTO_OK;
}

/*
 * access(i) on the matrix: on level l read the bit b at p; a 0 moves p to
 * rank0(p) (its place among the zeros, which come first on level l + 1), a 1
 * to Z_l + rank1(p).  The bits read, most significant first, spell the symbol.
 */
int wto_wm_access(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint64_t *I, uint64_t m, uint32_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t p = I[q];
        if (p >= n) { out[q] = UINT32_MAX; continue; }
        uint32_t sym = 0;
        for (uint32_t l = 0; l < L; l++) {
            int bit = bit_get(bits + l * t.lb, p);
            p = bit ? rank0(&t, l, n) + rank1(&t, l, p) : rank0(&t, l, p);
            sym = (sym << 1) | (uint32_t)bit;
        }
        out[q] = sym;
    }
    tree_free(&t);
    return WTO_OK;
}

/*
 * rank_c(i) on the matrix: the symbols equal to c form one contiguous range
 * of each level; follow the range [b, e) = [0, i) of the prefix: a 0 bit of
 * c maps both ends by rank0, a 1 bit by Z_l + rank1.  The answer is e - b at
 * the bottom.
 */
int wto_wm_rank(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint32_t *C, const uint64_t *I,
                uint64_t m, uint64_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t c = C[q], i = I[q];
        if (c >= sigma || i > n) { out[q] = UINT64_MAX; continue; }
        uint64_t b = 0, e = i;
        for (uint32_t l = 0; l < L; l++) {
            int bit = (int)((c >> (L - 1 - l)) & 1);
            if (bit) { b = rank0(&t, l, n) + rank1(&t, l, b); e = rank0(&t, l, n) + rank1(&t, l, e); }
            else { b = rank0(&t, l, b); e = rank0(&t, l, e); }
        }
        out[q] = e - b;
    }
    tree_free(&t);
    return WTO_OK;
}

/*
 * select_c(j) on the matrix: walk down from b = 0 by the bits of c (as in
 * rank) to the start b_L of c's range at the bottom; the answer's position
 * there is b_L + j - 1 if the range holds j symbols.  Then climb: a position
 * pos on level l + 1 that came from a 0 bit is the (pos + 1)-th zero of
 * level l; one from a 1 bit is the (pos - Z_l + 1)-th one.
 */
int wto_wm_select(const uint8_t *bits, uint64_t n, uint64_t sigma, const uint32_t *C, const uint64_t *J,
                  uint64_t m, uint64_t *out)
{
    uint32_t L = wto_levels(sigma);
    tree_t t;
    int st = tree_init(&t, bits, n, L);
    if (st) return st;
    for (uint64_t q = 0; q < m; q++) {
        uint64_t c = C[q], j = J[q];
        if (c >= sigma || j == 0) { out[q] = UINT64_MAX; continue; }
        uint64_t b = 0, e = n;
        for (uint32_t l = 0; l < L; l++) {
            int bit = (int)((c >> (L - 1 - l)) & 1);
            if (bit) { b = rank0(&t, l, n) + rank1(&t, l, b); e = rank0(&t, l, n) + rank1(&t, l, e); }
            else { b = rank0(&t, l, b); e = rank0(&t, l, e); }
        }
        if (j > e - b) { out[q] = UINT64_MAX; continue; }
        uint64_t pos = b + j - 1;
        for (uint32_t l = L; l-- > 0;) {
            int bit = (int)((c >> (L - 1 - l)) & 1);
            pos = bit ? selectb(&t, l, 1, pos - rank0(&t, l, n) + 1) : selectb(&t, l, 0, pos + 1);
        }
        out[q] = pos;
    }
    tree_free(&t);
    return WTO_OK;
}
